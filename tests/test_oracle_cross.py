"""Pins of the oracle's cross approximation with full pivoting (Sec. 6.5 builder)."""
import numpy as np
import pytest

from oracle import cross as X, compress as C


def test_hand_worked_two_by_two():
    # A = [[1, 2], [3, 4]]: the largest entry is A[1, 1] = 4, so u = A[:, 1] = (2, 4),
    # v = A[1, :] / 4 = (3/4, 1) and E_1 = A - u v^T = [[-1/2, 0], [0, 0]];
    # ||A||_F = sqrt(30), so tol 0.1 (0.548) stops at rank 1 and tol 0.05 (0.274)
    # takes the second cross through E_1[0, 0] = -1/2, which leaves zero.
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    U, V, piv, E = X.cross_full(A, 0.1)
    assert piv == [(1, 1)]
    assert np.allclose(U[:, 0], [2.0, 4.0]) and np.allclose(V[:, 0], [0.75, 1.0])
    assert np.allclose(E, [[-0.5, 0.0], [0.0, 0.0]])
    U, V, piv, E = X.cross_full(A, 0.05)
    assert piv == [(1, 1), (0, 0)]
    assert np.allclose(U[:, 1], [-0.5, 0.0]) and np.allclose(V[:, 1], [1.0, 0.0])
    assert np.allclose(U @ V.T, A) and not E.any()


def test_ties_take_the_smallest_column_then_row():
    A = np.array([[1.0, 5.0], [5.0, 5.0]])  # |5| at (1, 0), (0, 1), (1, 1): column 0 first
    _, _, piv, _ = X.cross_full(A, 0.9)
    assert piv[0] == (1, 0)


def test_exact_rank_terminates():
    # Gaussian elimination with complete pivoting leaves a zero Schur complement
    # after r steps of a rank-r matrix
    rng = np.random.default_rng(3)
    for m, n, r in [(40, 30, 5), (17, 60, 1), (25, 25, 12)]:
        A = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ (
            rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
        U, V, piv, E = X.cross_full(A, 1e-10)
        assert U.shape[1] == r and V.shape == (n, r)
        assert np.linalg.norm(A - U @ V.T) <= 1e-11 * np.linalg.norm(A)


def _smooth_kernel(m, n, seed):
    """1 / |x - y| between two separated point clouds: numerically low rank."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (m, 3))
    y = rng.uniform(0, 1, (n, 3)) + np.array([3.0, 0.5, 0.0])
    R = np.linalg.norm(x[:, None, :] - y[None, :, :], axis=2)
    return np.exp(-2j * np.pi * R) / R


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_skeleton_identity_and_interpolation(eps):
    A = _smooth_kernel(70, 50, 5)
    U, V, piv, E = X.cross_full(A, eps)
    I = [p[0] for p in piv]
    J = [p[1] for p in piv]
    k = len(piv)
    assert len(set(I)) == k and len(set(J)) == k
    # the cross approximation is the skeleton A[:, J] A[I, J]^-1 A[I, :]
    S = A[:, J] @ np.linalg.solve(A[np.ix_(I, J)], A[I, :])
    assert np.linalg.norm(U @ V.T - S) <= 1e-9 * np.linalg.norm(A)
    # it reproduces A on the pivot rows and columns
    D = A - U @ V.T
    assert np.abs(D[I, :]).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(D[:, J]).max() <= 1e-12 * np.abs(A).max()
    # the returned residual is A - U V^T and meets the stopping rule
    assert np.linalg.norm(E - D) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(D) <= eps * np.linalg.norm(A)
    # the previous step had not: k is the first rank within the tolerance
    Uk, Vk = U[:, :-1], V[:, :-1]
    assert np.linalg.norm(A - Uk @ Vk.T) > eps * np.linalg.norm(A)


def test_svd_rank_closed_form():
    A = np.diag([3.0, 2.0, 1.0])  # ||A||_F = sqrt(14); tails: sqrt(14), sqrt(5), 1, 0
    assert X.svd_rank(A, 0.3) == 2    # 0.3 sqrt(14) = 1.12 >= 1
    assert X.svd_rank(A, 0.6) == 1    # 2.245 >= sqrt(5) = 2.236
    assert X.svd_rank(A, 0.2) == 3    # 0.748 < 1
    assert X.svd_rank(A, 1.0) == 0


def test_vie_far_blocks_within_tolerance_and_above_the_svd_rank(tiny_dense):
    P, Z, _ = tiny_dense[:3]
    op = C.compress_dense(P, Z, 1e-4)
    for blk in op.far[::9]:
        Ab = Z[np.ix_(blk["rows"], blk["cols"])]
        U, V, piv, E = X.cross_full(Ab, 1e-4)
        assert np.linalg.norm(Ab - U @ V.T) <= 1e-4 * np.linalg.norm(Ab)
        assert U.shape[1] >= X.svd_rank(Ab, 1e-4)
        # the first pivot is the largest entry of A; one elimination step with a
        # complete pivot p at most doubles the largest entry (|e - a b / p| <= 2 |p|)
        p = np.array([abs(U[i, k]) for k, (i, j) in enumerate(piv)])
        assert abs(p[0] - np.abs(Ab).max()) <= 1e-15 * p[0]
        assert np.abs(E).max() <= p[-1] * 2.0
