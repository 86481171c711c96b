"""GPU solves of the aperiodic workload of Sec. 6.1: gold meta-atoms
(eps = -9.428 - 1.513 j under exp(j w t)) on a Vogel spiral, cubes of the
spheres' volume standing in for the spheres.  No two far blocks are translates
of one another, so every block is compressed and stored on its own.  The
currents are compared with the oracle's dense direct solution (Sec. 6.2: the
reference solution is the LU solve) and the cross sections with the oracle's.
"""
import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A
from oracle import fields as OF

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def spiral():
    # 24 atoms, 2^3 voxels each (864 unknowns): a three-level quadtree
    g = workloads.vogel_gold(24, nv=2)
    P = problem_from_geometry(g)
    return g, P, A.dense_matrix(P)


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


def test_vogel_gold_single_rhs_matches_dense(ctx, spiral):
    g, P, Z = spiral
    op = vie.Operator(ctx, g)
    info = op.compress(1e-4, vie.C64)
    assert info["levels"] >= 3
    kh, pol = workloads.normal_incidence()
    I, st, status = op.solve(kh, pol, tol=1e-6, max_iters=3000)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], np.linalg.solve(Z, A.rhs(P, kh[0], pol[0]))) <= 5e-4
    ext, sca = op.sigma(I, kh, pol)[0]
    assert abs(ext - OF.sigma_ext(I[:, 0], A.rhs_v0(P, kh[0], pol[0]))) < 1e-10 * abs(ext)
    assert abs(sca - OF.sigma_sca(P, I[:, 0])) < 1e-10 * abs(sca)
    assert ext > sca * (1 + 1e-2)  # gold absorbs: extinction exceeds scattering
    op.close()


def test_vogel_gold_multi_rhs_bf16x3_matches_dense(ctx, spiral):
    g, P, Z = spiral
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    kh, pol = workloads.angle_sweep(4, 60.0)  # 8 right-hand sides
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=vie.BF16X3, max_iters=3000)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    lu = np.linalg.solve(Z, np.stack([A.rhs(P, kh[c], pol[c]) for c in range(len(kh))], 1))
    for c in range(len(kh)):
        assert rel(I[:, c], lu[:, c]) <= 5e-4, c
    op.close()
