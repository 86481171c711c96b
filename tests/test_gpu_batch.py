"""Several problems in one lockstep solve (the block-diagonal union of their
operators): each problem's result equals its own solve and the oracle's dense
solve, for arrays of different size, wavelength and permittivity."""
import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problems():
    # (array side, eps_r, wavelength, right-hand sides)
    spec = [(3, 12.0, 1.0, 1), (4, 9.0, 0.95, 3), (2, 11.0, 1.05, 2)]
    out = []
    for i, (ns, eps, lam, nr) in enumerate(spec):
        g = workloads.square_array(ns, 3, 0.2, 0.4, eps, lam)
        kh, pol = workloads.random_directions(nr, seed=40 + i)
        out.append((g, kh, pol))
    return out


@pytest.mark.parametrize("precision", [vie.C64, vie.BF16X3])
def test_batch_equals_separate_solves(precision):
    ctx = vie.Context(0)
    probs = _problems()
    ops = []
    for g, _, _ in probs:
        op = vie.Operator(ctx, g)
        op.compress(1e-4, vie.C64)
        ops.append(op)
    Is, stats, status = vie.solve_batch(ops, [(kh, pol) for _, kh, pol in probs], tol=1e-6, precision=precision)
    assert status == vie.VIE_OK
    for p, ((g, kh, pol), op) in enumerate(zip(probs, ops)):
        I1, st1, s1 = op.solve(kh, pol, tol=1e-6, precision=precision)
        assert s1 == vie.VIE_OK
        assert stats[p]["residual"] <= 1e-6
        # the same method on the same operator; the far sums may run in another
        # order (a single right-hand side takes the shared-factor kernel, the
        # batch the multi-column one), so the two converged solutions agree to
        # the solve tolerance rather than to float32 rounding
        assert rel(Is[p], I1) <= 1e-6
        assert abs(stats[p]["iterations"] - st1["iterations"]) <= 2
    # accuracy against the oracle's dense solve for the two smaller problems
    for p in (0, 2):
        g, kh, pol = probs[p]
        P = problem_from_geometry(g)
        Z = A.dense_matrix(P)
        for c in range(len(kh)):
            assert rel(Is[p][:, c], np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))) <= 5e-4
    for op in ops:
        op.close()
    ctx.close()


def test_batch_rejects_mixed_discretisations():
    ctx = vie.Context(0)
    a = vie.Operator(ctx, workloads.square_array(2, 3))
    b = vie.Operator(ctx, workloads.square_array(2, 2))
    a.compress(1e-4, vie.C64)
    b.compress(1e-4, vie.C64)
    kh, pol = workloads.normal_incidence()
    with pytest.raises(vie.VieError) as e:
        vie.solve_batch([a, b], [(kh, pol), (kh, pol)])
    assert e.value.status == vie.VIE_ERR_INVALID_ARG
    a.close()
    b.close()
    ctx.close()
