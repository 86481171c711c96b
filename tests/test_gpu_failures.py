"""Failure paths through the C-ABI, made on the host: a non-finite value in
the incident field (uploaded from the host) is reported as VIE_ERR_NAN by the
solver's device-side finiteness check; a tensor-core kernel whose waits are
given a limit of zero cycles gives up at its first wait, drains what it
started and reports VIE_ERR_TIMEOUT; the context stays usable afterwards."""
import os
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


@pytest.fixture(scope="module")
def op():
    ctx = vie.Context(0)
    o = vie.Operator(ctx, workloads.square_array(3, 2))
    o.compress(1e-4, vie.C64)
    yield o
    o.close()
    ctx.close()


@pytest.mark.parametrize("precision", [vie.C64, vie.BF16X3])
def test_nan_in_incident_field_is_reported(op, precision):
    kh, pol = workloads.angle_sweep(2, 30.0)           # 4 right-hand sides
    bad = pol.copy()
    bad[2, 0] = np.nan                                 # one polarisation component
    with pytest.raises(vie.VieError) as e:
        op.solve(kh, bad, tol=1e-6, precision=precision)
    assert e.value.status == vie.VIE_ERR_NAN
    # the context and operator still work: the same solve with finite input converges
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=precision)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6 and np.all(np.isfinite(I))


def test_infinite_direction_is_reported(op):
    kh, pol = workloads.normal_incidence()
    bad = kh.copy()
    bad[0, 2] = -np.inf
    with pytest.raises(vie.VieError) as e:
        op.solve(bad, pol, tol=1e-6)
    assert e.value.status == vie.VIE_ERR_NAN
    _, st, status = op.solve(kh, pol, tol=1e-6)
    assert status == vie.VIE_OK


def test_tensor_core_wait_timeout_is_reported(op, monkeypatch):
    # the warp-specialised tcgen05 apply (default for 8+ right-hand sides) with
    # a wait limit of 0 cycles: its first wait on a copy or an MMA gives up, the
    # kernel waits for the copies and MMAs it started, frees its tensor memory
    # and sets the error word, which the solve reports at the end of its cycle
    kh, pol = workloads.angle_sweep(4, 30.0)           # 8 right-hand sides
    monkeypatch.setenv("VIE_TEST_WAIT_CYCLES", "0")
    with pytest.raises(vie.VieError) as e:
        op.solve(kh, pol, tol=1e-6, restart=2, max_iters=2, precision=vie.BF16X3)
    assert e.value.status == vie.VIE_ERR_TIMEOUT
    monkeypatch.delenv("VIE_TEST_WAIT_CYCLES")
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=vie.BF16X3)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6 and np.all(np.isfinite(I))
