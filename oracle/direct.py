"""Oracle dense direct solve: textbook LU with partial pivoting (float64 complex).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's reference solution J_ref comes from an LU decomposition (Sec. 6.2,
definition of A_s); the same factorisation is used for the block-diagonal
preconditioner (Sec. 4, eq. diagprecond).
"""
import numpy as np


def lu_factor(A):
    """Doolittle LU with row partial pivoting: P A = L U, packed in one array."""
    A = np.array(A, dtype=complex)
    n = A.shape[0]
    piv = np.arange(n)
    for j in range(n):
        p = j + int(np.argmax(np.abs(A[j:, j])))
        if p != j:
            A[[j, p]] = A[[p, j]]
            piv[[j, p]] = piv[[p, j]]
        if A[j, j] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        A[j + 1:, j] /= A[j, j]
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    return A, piv


def lu_solve(LU, piv, b):
    """Solve with the packed factors from :func:`lu_factor` (b: (n,) or (n, s))."""
    x = np.array(b, dtype=complex)[piv]
    n = LU.shape[0]
    for i in range(n):                       # forward: unit lower
        x[i] -= LU[i, :i] @ x[:i]
    for i in range(n - 1, -1, -1):           # backward: upper
        x[i] = (x[i] - LU[i, i + 1:] @ x[i + 1:]) / LU[i, i]
    return x


def solve(A, b):
    LU, piv = lu_factor(A)
    return lu_solve(LU, piv, b)
