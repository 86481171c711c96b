"""GPU tests at the 8x8 and 16x16 (193,536 unknowns) sizes: compression error
bounds on sampled blocks, the product error against the uncompressed operator,
sampled apply parity against the oracle and the converged solve."""
import os

import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, compress as OC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


def test_multibatch_compression_matches_oracle_bound(ctx, monkeypatch):
    # small batches: later batches start from a multi-chunk sketch sized by the
    # level's mean rank, the path the large arrays take
    monkeypatch.setenv("VIE_COMPRESS_MAX_BATCH", "8")
    g, _, _ = workloads.config("mid")
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    blocks = op.far_blocks(with_factors=False)
    key = {(b["level"], int(b["tatoms"][0]), int(b["satoms"][0])): i for i, b in enumerate(blocks)}
    sample = list(range(0, len(blocks), 37))
    for i, blk in zip(sample, op.far_blocks(indices=sample)):
        Ab = np.block([[A.cross_block(P, int(a), int(b)) for b in blk["satoms"]] for a in blk["tatoms"]])
        assert np.linalg.norm(Ab - blk["Q"] @ blk["R"]) <= 1e-4 * np.linalg.norm(Ab)
        if i < key[(blk["level"], int(blk["satoms"][0]), int(blk["tatoms"][0]))]:
            assert np.linalg.norm(blk["Q"].conj().T @ blk["Q"] - np.eye(blk["rank"])) < 1e-4


@pytest.fixture(scope="module")
def scale_op(ctx):
    g, kh, pol = workloads.config("scale")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    return op, g, kh, pol


def test_scale_product_error_against_uncompressed(scale_op):
    # eps_prod with u = (1 + j)[1 ... 1] (Sec. 6.2); the reference is the
    # uncompressed operator with every block regenerated on the device
    op, g, _, _ = scale_op
    u = torch.full((op.n,), 1 + 1j, dtype=torch.complex64, device="cuda")
    yq, yd = torch.empty_like(u), torch.empty_like(u)
    op.apply(u.data_ptr(), yq.data_ptr(), 1, vie.C64, 0)
    op.apply(u.data_ptr(), yd.data_ptr(), 1, vie.C64, vie.DENSE)
    torch.cuda.synchronize()
    eps_prod = (torch.linalg.norm(yq - yd) / torch.linalg.norm(yd)).item()
    assert eps_prod < 1e-4


def _mate(blocks, lev, b):
    return [j for j, c in enumerate(blocks) if c["level"] == lev and
            list(c["tatoms"]) == list(b["satoms"]) and list(c["satoms"]) == list(b["tatoms"])][0]


def test_scale_sampled_blocks_error_bound_against_oracle(scale_op):
    # levels 3 and 4 (3,024^2 and 756^2 blocks): ||A - Q R||_F <= 1e-4 ||A||_F with
    # A assembled by the oracle in float64, on the first, middle and last block
    op, g, _, _ = scale_op
    P = problem_from_geometry(g)
    blocks = op.far_blocks(with_factors=False)
    ids = {}
    for i, b in enumerate(blocks):
        ids.setdefault(b["level"], []).append(i)
    assert sorted(ids) == [2, 3, 4]
    for lev, sample in ((3, (ids[3][0], ids[3][-1])), (4, (ids[4][0], ids[4][len(ids[4]) // 2], ids[4][-1]))):
        for i in sample:
            b = op.far_blocks(indices=[i])[0]
            Ab = np.block([[A.cross_block(P, int(a), int(c)) for c in b["satoms"]] for a in b["tatoms"]])
            err = np.linalg.norm(Ab - b["Q"] @ b["R"]) / np.linalg.norm(Ab)
            assert err <= 1e-4, (lev, i, err)
            if i < _mate(blocks, lev, b):   # compressed block of its mirror pair: orthonormal Q
                assert np.linalg.norm(b["Q"].conj().T @ b["Q"] - np.eye(b["rank"])) < 1e-4


def test_scale_level2_blocks_error_bound(scale_op):
    # level 2 (12,096^2, 256 atom pairs each): A from the device's float64
    # assembly, which equals the oracle's entries to 1e-12 (test_cross_block)
    op, g, _, _ = scale_op
    npp = op.np
    blocks = op.far_blocks(with_factors=False)
    ids = [i for i, b in enumerate(blocks) if b["level"] == 2]
    for i in (ids[0], ids[len(ids) // 2], ids[-1]):
        b = op.far_blocks(indices=[i])[0]
        Ab = torch.zeros((len(b["tatoms"]) * npp, len(b["satoms"]) * npp), dtype=torch.complex128, device="cuda")
        for p, a in enumerate(b["tatoms"]):
            for q, c in enumerate(b["satoms"]):
                blk = op.export_block(1, int(a), int(c), vie.C128)
                Ab[p * npp:(p + 1) * npp, q * npp:(q + 1) * npp] = torch.from_numpy(np.ascontiguousarray(blk)).cuda()
        Q = torch.from_numpy(b["Q"]).cuda()
        R = torch.from_numpy(b["R"]).cuda()
        err = (torch.linalg.norm(Ab - Q @ R) / torch.linalg.norm(Ab)).item()
        assert err <= 1e-4, (i, err)
        if i < _mate(blocks, 2, b):
            eye = torch.eye(b["rank"], dtype=Q.dtype, device="cuda")
            assert torch.linalg.norm(Q.conj().T @ Q - eye).item() < 1e-4


def test_scale_apply_parity_sampled_atoms(scale_op):
    # rows of two atoms: the oracle applies the exported factors of every block
    # whose target box holds the atom (float64) plus the oracle's self block
    op, g, _, _ = scale_op
    P = problem_from_geometry(g)
    npp = op.np
    x = workloads.random_complex(op.n, 1234)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.empty_like(xd)
    op.apply(xd.data_ptr(), yd.data_ptr(), 1, vie.C64, 0)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    meta = op.far_blocks(with_factors=False)
    Zs = A.self_block(P, 0)
    for atom in (0, 137):
        idx = [i for i, b in enumerate(meta) if atom in set(b["tatoms"].tolist())]
        ref = Zs @ x[atom * npp:(atom + 1) * npp]
        for b in op.far_blocks(indices=idx):
            slot = list(b["tatoms"]).index(atom)
            cols = OC.atom_rows(P, b["satoms"])
            ref = ref + b["Q"][slot * npp:(slot + 1) * npp] @ (b["R"] @ x[cols])
        assert rel(y[atom * npp:(atom + 1) * npp], ref) < 1e-5


def test_scale_bf16x3_multi_rhs_apply(scale_op):
    # 64 right-hand sides through the tensor-core (BF16x3) apply at full size:
    # rows of two atoms for three columns against the oracle on the exported
    # factors (float64), every entry against the float32 SIMT apply
    op, g, _, _ = scale_op
    P = problem_from_geometry(g)
    npp, n, k = op.np, op.n, 64
    xs = workloads.random_complex(n, 4321, cols=k)                 # n x k
    X = torch.from_numpy(np.ascontiguousarray(xs.T).astype(np.complex64)).cuda()
    Y, Yr = torch.empty_like(X), torch.empty_like(X)
    for fl in (vie.FUSE_PRECOND, 0):
        op.apply(X.data_ptr(), Y.data_ptr(), k, vie.BF16X3, fl)
        op.apply(X.data_ptr(), Yr.data_ptr(), k, vie.C64, fl)
        torch.cuda.synchronize()
        assert rel(Y.cpu().numpy(), Yr.cpu().numpy()) < 5e-5, fl
    y = Y.cpu().numpy()                                            # k x n, Zs x
    x = xs.astype(np.complex64).astype(np.complex128)
    meta = op.far_blocks(with_factors=False)
    Zs = A.self_block(P, 0)
    cols = [0, 37, 63]
    for atom in (5, 200):
        rows = slice(atom * npp, (atom + 1) * npp)
        idx = [i for i, b in enumerate(meta) if atom in set(b["tatoms"].tolist())]
        ref = Zs @ x[rows][:, cols]
        for b in op.far_blocks(indices=idx):
            slot = list(b["tatoms"]).index(atom)
            src = OC.atom_rows(P, b["satoms"])
            ref = ref + b["Q"][slot * npp:(slot + 1) * npp] @ (b["R"] @ x[src][:, cols])
        assert rel(y[cols][:, rows].T, ref) < 5e-5, atom


def test_scale_solve(scale_op):
    op, g, kh, pol = scale_op
    n = op.n
    xo = torch.empty(n, dtype=torch.complex128, device="cuda")
    _, st, status = op.solve(kh, pol, tol=1e-6, out_ptr=xo.data_ptr())
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert st["true_residual"] < 1e-5
    # residual against the uncompressed operator: bounded by the compression error
    b = torch.empty_like(xo)
    op.rhs(kh, pol, b.data_ptr())
    zx = torch.empty_like(xo)
    op.apply(xo.data_ptr(), zx.data_ptr(), 1, vie.C128, vie.DENSE)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(b - zx) / torch.linalg.norm(b)).item() < 5e-4
