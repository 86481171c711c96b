"""Pins of the oracle's tree, static map, QR compression, direct solve and GMRES."""
import itertools
import os

import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, tree as T, compress as C
from oracle import krylov as K, direct as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny(tiny_dense):
    return tiny_dense[:3]


# ---------------------------------------------------------------- tree and map
def _coverage(centres):
    L, blocks = T.build_tree(centres)
    N = len(centres)
    cover = np.zeros((N, N), int)
    for _, ta, sa in blocks:
        for a in ta:
            for b in sa:
                cover[a, b] += 1
    return L, blocks, cover


@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 7, 8])
def test_far_blocks_cover_every_distinct_pair_once(ns):
    g = workloads.square_array(ns, 1)
    L, blocks, cover = _coverage(g.centres)
    N = ns * ns
    assert np.array_equal(cover, 1 - np.eye(N, dtype=int))   # Z_N = Z_D at the finest level
    for lev, ta, sa in blocks:
        shift = L - lev
        _, fine = T.atom_box_coords(g.centres)
        tb, sb = fine[ta[0]] >> shift, fine[sa[0]] >> shift
        assert all((fine[a] >> shift == tb).all() for a in ta)
        if lev < L:
            assert np.max(np.abs(tb - sb)) > 1                # far: no shared grid node
        assert np.max(np.abs((tb >> 1) - (sb >> 1))) <= 1     # parents were near


def test_block_counts_per_level():
    # far blocks per level for the 16x16, 32x32 and 64x64 arrays
    expect = {16: [156, 1116, 7488], 32: [156, 1116, 5628, 32832],
              64: [156, 1116, 5628, 25020, 137280]}
    for ns, counts in expect.items():
        g = workloads.square_array(ns, 1)
        L, blocks = T.build_tree(g.centres)
        got = [sum(1 for b in blocks if b[0] == lev) for lev in range(2, L + 1)]
        assert got == counts
        sizes = {lev: {len(b[1]) for b in blocks if b[0] == lev} for lev in range(2, L + 1)}
        assert all(s == {4 ** (L - lev)} for lev, s in sizes.items())


def test_paper_table_par_p():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_par_p.txt")) if l[0] != "#"]
    for N, total, mu, sigma, ratio in rows:
        g = workloads.vogel_spiral(int(N))
        _, blocks = T.build_tree(g.centres)
        tot = sum(len(a) * len(b) for _, a, b in blocks)
        assert tot == int(total)
        _, loads, _ = T.lpt_assign(np.ones(tot), 64)
        assert round(loads.mean()) == int(mu)
        s = loads.std(ddof=1)
        assert abs(s - float(sigma)) < 0.006
        assert abs(s / loads.mean() / float(ratio) - 1) < 0.01


def test_lpt_against_exhaustive_optimum():
    rng = np.random.default_rng(3)
    for _ in range(20):
        w = rng.integers(1, 50, size=7).astype(float)
        m = 3
        owner, loads, _ = T.lpt_assign(w, m)
        assert np.allclose(np.bincount(owner, weights=w, minlength=m), loads)
        best = min(max(np.bincount(np.array(a), weights=w, minlength=m))
                   for a in itertools.product(range(m), repeat=len(w)))
        assert loads.max() <= (4 / 3 - 1 / (3 * m)) * best + 1e-9   # Graham's LPT bound


# -------------------------------------------------------------------- direct
def test_lu_against_library_solve(tiny):
    P, Z, b = tiny
    x = D.solve(Z, b)
    ref = np.linalg.solve(Z, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-12


def test_lu_against_cramer_two_atoms():
    g = workloads.two_cubes(0.5, side=0.2, nv=1)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    b = A.rhs(P, [0, 0, -1.0], [1, 0, 0])
    x = D.solve(Z, b)
    det = np.linalg.det(Z)
    for i in range(P.n):
        Zi = Z.copy()
        Zi[:, i] = b
        assert abs(x[i] - np.linalg.det(Zi) / det) < 1e-10 * np.abs(x).max()


# ---------------------------------------------------------------- compression
def test_householder_qr_bounds(tiny):
    P, Z, _ = tiny
    op = C.compress_dense(P, Z, 1e-4)
    for blk in op.far[::7]:
        Ab = Z[np.ix_(blk["rows"], blk["cols"])]
        Q, R = blk["Q"], blk["R"]
        r = R.shape[0]
        assert np.linalg.norm(Ab - Q @ R) <= 1e-4 * np.linalg.norm(Ab) * (1 + 1e-9)
        assert np.linalg.norm(Q.conj().T @ Q - np.eye(r)) < 1e-12
        s = np.linalg.svd(Ab, compute_uv=False)
        tail = np.sqrt(np.cumsum(s[::-1] ** 2))[::-1]
        svd_rank = int(np.argmax(np.append(tail, 0) <= 1e-4 * np.linalg.norm(Ab)))
        assert r >= svd_rank
        assert np.allclose(np.triu(R), R)


def test_qr_exact_at_zero_tolerance(tiny):
    P, Z, _ = tiny
    op = C.compress_dense(P, Z, 1e-15)
    x = workloads.random_complex(P.n, 7)
    assert np.linalg.norm(op.apply(x) - Z @ x) <= 1e-12 * np.linalg.norm(Z @ x)


def test_product_error_and_gain(tiny):
    P, Z, _ = tiny
    op = C.compress_dense(P, Z, 1e-4)
    assert C.product_error(Z, op) < 1e-4
    # G = N_dof^2 / N_QR with N_QR = sum_far (m+n) r + N N_p^2 (eq. eqn_cgain)
    nqr = sum((b["Q"].shape[0] + b["R"].shape[1]) * b["R"].shape[0] for b in op.far) + 16 * 108 ** 2
    assert op.gain() == pytest.approx(P.n ** 2 / nqr)
    # far entries plus self entries tile the matrix
    assert sum(len(b["rows"]) * len(b["cols"]) for b in op.far) + 16 * 108 ** 2 == P.n ** 2


# -------------------------------------------------------------------- GMRES
def test_gmres_iterate_is_the_krylov_least_squares_minimiser():
    rng = np.random.default_rng(5)
    n = 40
    Am = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n) + 1j * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for k in (1, 3, 6):
        x, info = K.gmres(lambda v: Am @ v, b, tol=0.0, maxiter=k)
        Kr = np.stack([np.linalg.matrix_power(Am, j) @ b for j in range(k)], 1)
        y = np.linalg.lstsq(Am @ Kr, b, rcond=None)[0]
        assert np.linalg.norm(x - Kr @ y) < 1e-9 * np.linalg.norm(x)
        assert info["history"][-1] == pytest.approx(np.linalg.norm(b - Am @ x) / np.linalg.norm(b), rel=1e-8)


def test_gmres_restarted_converges():
    rng = np.random.default_rng(6)
    n = 60
    Am = np.eye(n) * 2 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n).astype(complex)
    x, info = K.gmres(lambda v: Am @ v, b, tol=1e-10, restart=5)
    assert info["converged"]
    assert np.linalg.norm(Am @ x - b) / np.linalg.norm(b) < 1e-9


def test_isolated_atom_converges_in_one_iteration():
    # Sec. 4: the preconditioner is the exact inverse for an isolated meta-atom
    g = workloads.single_cube(0.2, 3)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    M = K.BlockJacobi(P, {0: Z})
    _, info = K.gmres(lambda v: Z @ v, A.rhs(P, [0, 0, -1.0], [1, 0, 0]), M.apply, tol=1e-10)
    assert info["iterations"] == 1


def test_far_apart_atoms_converge_fast():
    g = workloads.two_cubes(20.0, side=0.2, nv=2)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    M = K.BlockJacobi(P, {0: Z[:36, :36]})
    _, info = K.gmres(lambda v: Z @ v, A.rhs(P, [0, 0, -1.0], [1, 0, 0]), M.apply, tol=1e-6)
    assert info["iterations"] <= 3


def test_compressed_solve_matches_dense_direct(tiny):
    P, Z, b = tiny
    op = C.compress_dense(P, Z, 1e-4)
    M = K.BlockJacobi(P, op.self_blocks)
    x, info = K.gmres(op.apply, b, M.apply, tol=1e-6)
    ref = D.solve(Z, b)
    assert info["converged"]
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 5e-4
    _, info0 = K.gmres(lambda v: Z @ v, b, None, tol=1e-6)
    assert info0["iterations"] > info["iterations"]          # the preconditioner helps


# ------------------------------------------------------------------- BiCGStab
def test_bicgstab_matches_library_solve():
    # a well-conditioned complex system: the BiCGStab iterate converges to the
    # LAPACK solution
    rng = np.random.default_rng(21)
    n = 60
    Amat = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = K.bicgstab(lambda v: Amat @ v, b, tol=1e-12)
    assert info["converged"]
    ref = np.linalg.solve(Amat, b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    # the recursively updated residual is the true one (up to rounding)
    assert np.linalg.norm(b - Amat @ x) <= 1e-11 * np.linalg.norm(b)


def test_bicgstab_two_eigenvalues_terminates_in_two_steps():
    # r_k = Q_k(A) P_k(A) r_0 with P_k the BiCG polynomial: for a matrix with two
    # distinct eigenvalues P_2(A) r_0 = 0, so the second iterate is exact
    rng = np.random.default_rng(4)
    d = np.where(np.arange(40) % 2 == 0, 1.0, 3.0 - 0.5j)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)))
    Amat = Q @ np.diag(d) @ Q.conj().T
    b = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    x, info = K.bicgstab(lambda v: Amat @ v, b, tol=1e-12)
    assert info["iterations"] <= 2
    assert np.linalg.norm(Amat @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_bicgstab_identity_one_step():
    b = np.arange(1, 9) * (1 - 0.5j)
    x, info = K.bicgstab(lambda v: v, b, tol=1e-14)
    assert info["iterations"] == 1 and np.allclose(x, b, rtol=0, atol=1e-14)


def test_bicgstab_preconditioned_vie_solve(tiny):
    # the 4x4 array with the block-Jacobi preconditioner: the same solution as
    # the dense direct solve, to the solve tolerance times the conditioning
    P, Z, b = tiny
    sb = {0: Z[:P.offsets[1], :P.offsets[1]]}
    x, info = K.bicgstab(lambda v: Z @ v, b, K.BlockJacobi(P, sb).apply, tol=1e-8)
    assert info["converged"]
    ref = np.linalg.solve(Z, b)
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)
