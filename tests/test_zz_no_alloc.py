"""The allocation-free apply (vie_apply_noalloc) against the regular apply.

vie_apply_noalloc serves callers that cannot obtain device memory with
cudaMalloc once they are running, e.g. because their own pool allocator owns
the device memory or because the device-wide synchronisation of cudaMalloc is
not acceptable in their loop.  It takes its scratch from a fixed device array
of the library.  This file is collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


def rel(a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


def test_noalloc_apply_matches_regular_apply():
    ctx = vie.Context(0)
    g, _, _ = workloads.config("mid")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    n, nrhs = op.n, 3
    xs = [torch.from_numpy(workloads.random_complex(n, seed, cols=nrhs).T.copy().astype(np.complex64)).cuda()
          for seed in (11, 12)]
    y_ref = [torch.empty_like(x) for x in xs]
    y_na = [torch.empty_like(x) for x in xs]
    op.apply_noalloc(xs[0].data_ptr(), y_na[0].data_ptr(), nrhs)   # first call on the device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row: the second must not see the first one's scratch
    for x, y in zip(xs, y_na):
        op.apply_noalloc(x.data_ptr(), y.data_ptr(), nrhs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0   # no device memory taken
    for x, y in zip(xs, y_ref):
        op.apply(x.data_ptr(), y.data_ptr(), nrhs, vie.C64, 0)
    torch.cuda.synchronize()
    for a, b in zip(y_na, y_ref):
        assert rel(a, b) < 1e-5
    # requests beyond the static array are refused before any launch
    big = vie.NOALLOC_SCRATCH_ELEMS // max(1, sum(b["rank"] for b in op.far_blocks(with_factors=False))) + 1
    xb = torch.zeros((big, n), dtype=torch.complex64, device="cuda")
    yb = torch.zeros_like(xb)
    with pytest.raises(vie.VieError):
        op.apply_noalloc(xb.data_ptr(), yb.data_ptr(), big)
    # so are vectors off the 16-byte grid and overlapping vectors (both in bounds)
    for xp, yp in ((xs[0].data_ptr() + 8, y_na[0].data_ptr()), (xs[0].data_ptr(), xs[0].data_ptr() + 16)):
        with pytest.raises(vie.VieError) as e:
            op.apply_noalloc(xp, yp, 1)
        assert e.value.status == vie.VIE_ERR_INVALID_ARG
    op.close()
    ctx.close()
