"""The adjoint apply y = Zs^H x (the Z^H products of Sec. 4), BiCGStab (the
Krylov method Sec. 6 compares GMRES with) and block GMRES (one Krylov space for
all right-hand sides), through the C-ABI, against the oracle: the adjoint of
the compressed operator built from the exported factors, the oracle's BiCGStab
on the same factors, and the dense direct solution."""
import os

import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, compress as OC, krylov as K

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


def _oracle_op(op, P):
    sb = {t: op.export_block(0, t) for t in sorted(set(P.types.tolist()))}
    blocks = op.far_blocks()
    return OC.operator_from_factors(P, sb, [(b["tatoms"], b["satoms"], b["Q"], b["R"]) for b in blocks]), sb


@pytest.mark.parametrize("fprec", [vie.C64, vie.C128])
def test_adjoint_apply_matches_oracle(ctx, fprec):
    g, _, _ = workloads.config("tiny")
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, fprec)
    orc, _ = _oracle_op(op, P)
    Zqr = orc.apply(np.eye(P.n, dtype=complex))          # the compressed operator, densely
    xs = workloads.random_complex(P.n, 17, cols=3)       # n x 3
    ref = Zqr.conj().T @ xs
    cases = [(vie.C64_ACC64, np.complex128, 1e-12), (vie.C64, np.complex64, 1e-5), (vie.BF16X3, np.complex64, 5e-5)]
    if fprec == vie.C128:
        cases = [(vie.C128, np.complex128, 1e-12)]
    for prec, dt, tol in cases:
        X = torch.from_numpy(np.ascontiguousarray(xs.T).astype(dt)).cuda()
        Y = torch.empty_like(X)
        op.apply(X.data_ptr(), Y.data_ptr(), 3, prec, vie.ADJOINT)
        torch.cuda.synchronize()
        assert rel(Y.cpu().numpy().T, ref) < tol, prec
    # the adjoint cannot be fused with the preconditioner
    X = torch.zeros(P.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(vie.VieError):
        op.apply(X.data_ptr(), torch.empty_like(X).data_ptr(), 1, vie.C64, vie.ADJOINT | vie.FUSE_PRECOND)
    op.close()


def test_adjoint_identity_three_levels(ctx):
    # <Zs x, y> = <x, Zs^H y> on the 8x8 array of 4^3 cubes, float64 vectors
    g = workloads.square_array(8, 4)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    x = torch.from_numpy(workloads.random_complex(op.n, 1)).cuda()
    y = torch.from_numpy(workloads.random_complex(op.n, 2)).cuda()
    zx, zhy = torch.empty_like(x), torch.empty_like(y)
    op.apply(x.data_ptr(), zx.data_ptr(), 1, vie.C64_ACC64, 0)
    op.apply(y.data_ptr(), zhy.data_ptr(), 1, vie.C64_ACC64, vie.ADJOINT)
    torch.cuda.synchronize()
    lhs = torch.vdot(y, zx).item()          # y^H Z x
    rhs = torch.vdot(zhy, x).item()         # (Z^H y)^H x
    scale = (torch.linalg.norm(zx) * torch.linalg.norm(y)).item()
    assert abs(lhs - rhs) <= 1e-12 * scale
    op.close()


@pytest.mark.parametrize("precision", [vie.C64, vie.BF16X3])
def test_bicgstab_solve_matches_dense_and_oracle(ctx, tiny_dense, precision):
    P, Z, b, kh, pol = tiny_dense
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    I, st, status = op.solve(kh[None], pol[None], tol=1e-6, precision=precision, method=vie.BICGSTAB)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], np.linalg.solve(Z, b)) <= 5e-4
    assert st["applies"] == 2 * st["iterations"] >= 2
    # the oracle's BiCGStab on the same factors needs about as many iterations
    orc, sb = _oracle_op(op, P)
    _, info = K.bicgstab(orc.apply, b, K.BlockJacobi(P, sb).apply, tol=1e-6)
    assert abs(st["iterations"] - info["iterations"]) <= max(2, 0.15 * info["iterations"])
    op.close()


def test_bicgstab_lockstep_three_levels(ctx):
    # four right-hand sides on the 8x8 array of 3^3 cubes (three-level tree)
    # against the stored dense solutions
    d = np.load(os.path.join(GOLDEN, "mid_8x8_nv3.npz"))
    kh, pol, ref = d["khat"], d["pol"], d["I"]
    op = vie.Operator(ctx, workloads.square_array(8, 3))
    op.compress(1e-4, vie.C64)
    I, st, status = op.solve(kh[1:], pol[1:], tol=1e-6, method=vie.BICGSTAB)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    for c in range(4):
        assert rel(I[:, c], ref[:, c + 1]) <= 5e-4
    with pytest.raises(vie.VieError):
        op.solve(kh, pol, method=7)
    op.close()


@pytest.mark.parametrize("precision", [vie.C64, vie.BF16X3])
def test_block_gmres_matches_dense_and_needs_fewer_steps(ctx, precision):
    # block GMRES (one Krylov space for all right-hand sides) on the 8x8 array:
    # every current within 5e-4 of the stored dense solutions, in fewer block
    # steps than the lockstep GMRES needs Arnoldi steps
    d = np.load(os.path.join(GOLDEN, "mid_8x8_nv3.npz"))
    kh, pol, ref = d["khat"], d["pol"], d["I"]
    op = vie.Operator(ctx, workloads.square_array(8, 3))
    op.compress(1e-4, vie.C64)
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=precision, method=vie.BLOCK_GMRES)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    for c in range(len(kh)):
        assert rel(I[:, c], ref[:, c]) <= 5e-4, c
    _, st_l, _ = op.solve(kh, pol, tol=1e-6, precision=precision)
    assert st["iterations"] < st_l["iterations"]
    op.close()
