"""Oracle cross approximation of an assembled far block (float64 complex).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 6.5: the compressed operator is built in two steps, local assembly of a
block and then its compression by the "full-cross" approximation of Kurz,
Rain and Rjasanow (2002).  Reading: cross approximation with full (complete)
pivoting over the assembled block.  With E_0 = A, step k takes the entry of
E_k of largest modulus, (i_k, j_k), and removes the cross through it,

    E_{k+1} = E_k - E_k[:, j_k] E_k[i_k, :] / E_k[i_k, j_k],

which zeroes row i_k and column j_k of the residual.  A ~ sum_k u_k v_k^T
with u_k = E_k[:, j_k] and v_k = E_k[i_k, :] / E_k[i_k, j_k] (Gaussian
elimination with complete pivoting, stopped early).  Since the whole residual
is at hand its Frobenius norm is exact, and the iteration stops at the first
k with ||E_k||_F <= eps ||A||_F, the truncation criterion the QR compression
uses.  Ties in |E| go to the smallest column index, then the smallest row.

Pinned by tests/test_oracle_cross.py: a hand-worked 2 x 2 case, exact
termination on rank-r matrices, the skeleton identity
sum_k u_k v_k^T = A[:, J] A[I, J]^-1 A[I, :], interpolation on the pivot
rows and columns, and the Eckart-Young lower bound on the rank.
"""
import numpy as np


def cross_full(A, eps, kmax=None):
    """Cross approximation of A with full pivoting to ||A - U V^T||_F <= eps ||A||_F.

    Returns (U (m x k), V (n x k), pivots [(i_k, j_k)], residual E_k)."""
    E = np.array(A, dtype=complex)
    m, n = E.shape
    target2 = (eps * np.linalg.norm(E)) ** 2
    kmax = min(m, n) if kmax is None else kmax
    us, vs, piv = [], [], []
    while True:
        e2 = float(np.sum(np.abs(E) ** 2))
        if e2 <= target2 or len(us) == min(m, n):
            break
        if len(us) == kmax:
            raise RuntimeError("cross approximation needs a rank above %d" % kmax)
        # column-major scan order: the first maximum has the smallest column, then row
        flat = int(np.argmax(np.abs(E).T))
        j, i = divmod(flat, m)
        p = E[i, j]
        u = E[:, j].copy()
        v = E[i, :] / p
        E -= np.outer(u, v)
        E[i, :] = 0.0
        E[:, j] = 0.0
        us.append(u)
        vs.append(v)
        piv.append((i, j))
    k = len(us)
    U = np.array(us).T.reshape(m, k)
    V = np.array(vs).T.reshape(n, k)
    return U, V, piv, E


def svd_rank(A, eps):
    """Smallest rank r of any approximation with ||A - A_r||_F <= eps ||A||_F (Eckart-Young)."""
    s = np.linalg.svd(np.asarray(A, dtype=complex), compute_uv=False)
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[r] = ||sigma_{r:}||
    target = eps * np.sqrt(np.sum(s ** 2))
    for r in range(len(s)):
        if tail[r] <= target:
            return r
    return len(s)
