"""Oracle QR compression and compressed operator (float64 complex).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 5.2, eq. eq_02: a far block A (m x n) is approximated within a tolerance
eps by Q (m x r) R (r x n) and applied as Q (R x), cost (m + n) r.  The paper
does not state the truncation criterion; reading: per-block relative
Frobenius error, i.e. the smallest r with ||A - Q_r R_r||_F <= eps ||A||_F.
With unpivoted Householder QR the error after r steps is exactly the
Frobenius norm of the not-yet-reduced trailing block, so truncation stops
there (rank-valid, not rank-minimal).

Sec. 5.3, eq. eqn_cgain: G = N_dof^2 / N_QR, N_QR = sum_far (m + n) r + N N_p^2.
"""
import numpy as np

from . import assembly
from .tree import build_tree


def householder_qr_truncated(A, eps):
    """Unpivoted Householder QR of A, stopped at the first r with trailing norm <= eps ||A||_F.

    Returns (Q (m x r) with orthonormal columns, R (r x n), error ||A - QR||_F)."""
    A = np.array(A, dtype=complex)
    m, n = A.shape
    normA = np.linalg.norm(A)
    target = eps * normA
    vs = []
    r = 0
    err = normA
    while r < min(m, n):
        if np.linalg.norm(A[r:, r:]) <= target:
            break
        x = A[r:, r].copy()
        alpha = np.linalg.norm(x)
        if alpha > 0:
            phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
            v = x.copy()
            v[0] += phase * alpha
            v /= np.linalg.norm(v)
            A[r:, r:] -= 2.0 * np.outer(v, v.conj() @ A[r:, r:])
        else:
            v = np.zeros_like(x)
        vs.append(v)
        r += 1
    err = np.linalg.norm(A[r:, r:]) if r < min(m, n) else 0.0
    R = np.triu(A[:r, :])
    Q = np.zeros((m, r), complex)
    Q[:r, :r] = np.eye(r)
    for j in range(r - 1, -1, -1):           # Q = H_0 ... H_{r-1} [I; 0]
        v = vs[j]
        Q[j:, :] -= 2.0 * np.outer(v, v.conj() @ Q[j:, :])
    return Q, R, float(err)


def atom_rows(prob, atoms):
    """Global unknown indices of a list of atoms (concatenated in list order)."""
    return np.concatenate([np.arange(prob.offsets[a], prob.offsets[a + 1]) for a in atoms])


class CompressedOperator:
    """Z_QR = blockdiag(Z_ii) + sum_far rows_b <- Q_b (R_b x[cols_b])."""

    def __init__(self, prob, self_blocks, far):
        self.prob = prob
        self.self_blocks = self_blocks      # {type: N_p x N_p}
        self.far = far                      # list of dicts: level, rows, cols, Q, R

    def apply(self, x):
        """y = Z_QR x in float64 (x: (n,) or (n, s))."""
        p = self.prob
        x = np.asarray(x, complex)
        y = np.zeros_like(x)
        for a in range(p.n_atoms):
            s = slice(p.offsets[a], p.offsets[a + 1])
            y[s] += self.self_blocks[p.types[a]] @ x[s]
        for b in self.far:
            y[b["rows"]] += b["Q"] @ (b["R"] @ x[b["cols"]])
        return y

    def n_qr(self):
        p = self.prob
        near = sum(self.self_blocks[p.types[a]].size for a in range(p.n_atoms))
        far = sum((b["Q"].shape[0] + b["R"].shape[1]) * b["R"].shape[0] for b in self.far)
        return far + near

    def gain(self):
        """Compression gain G = N_dof^2 / N_QR (eq. eqn_cgain)."""
        return self.prob.n ** 2 / self.n_qr()


def compress_dense(prob, Z, eps, self_blocks=None):
    """QR-recursive compression of an assembled dense matrix (small problems)."""
    L, blocks = build_tree(prob.centres)
    if self_blocks is None:
        self_blocks = {}
        for a in range(prob.n_atoms):
            t = prob.types[a]
            if t not in self_blocks:
                s = slice(prob.offsets[a], prob.offsets[a + 1])
                self_blocks[t] = Z[s, s].copy()
    far = []
    for lev, ta, sa in blocks:
        rows = atom_rows(prob, ta)
        cols = atom_rows(prob, sa)
        A = Z[np.ix_(rows, cols)]
        Q, R, err = householder_qr_truncated(A, eps)
        far.append(dict(level=lev, tatoms=ta, satoms=sa, rows=rows, cols=cols, Q=Q, R=R,
                        err=err, norm=float(np.linalg.norm(A))))
    return CompressedOperator(prob, self_blocks, far)


def operator_from_factors(prob, self_blocks, blocks):
    """Compressed operator from externally produced factors.

    blocks: iterable of (tatoms, satoms, Q, R) with Q (m x r), R (r x n)."""
    far = []
    for ta, sa, Q, R in blocks:
        far.append(dict(level=None, tatoms=list(ta), satoms=list(sa), rows=atom_rows(prob, ta),
                        cols=atom_rows(prob, sa), Q=np.asarray(Q, complex), R=np.asarray(R, complex)))
    return CompressedOperator(prob, self_blocks, far)


def product_error(Z, op):
    """eps_prod = ||Z_QR u - Z u|| / ||Z u||, u = (1 + j)[1 ... 1] (Sec. 6.2)."""
    u = (1.0 + 1.0j) * np.ones(Z.shape[0])
    ref = Z @ u
    return float(np.linalg.norm(op.apply(u) - ref) / np.linalg.norm(ref))
