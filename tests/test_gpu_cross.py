"""GPU parity of the cross-approximation builder (vie_compress_cross, Sec. 6.5:
local assembly of each far block, then its cross approximation with full
pivoting) against the CPU oracle: the per-block error bound on the oracle's
float64 blocks, the interpolation of the pivot rows and columns, the rank
against the oracle's own cross approximation and the SVD bound, the apply
against the oracle applying the exported factors, and solves against the
oracle's dense direct solution on two- and three-level trees."""
import os

import numpy as np
import pytest

import workloads
from oracle import assembly as A, compress as C, cross as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cross_ops(ctx):
    g, _, _ = workloads.config("tiny")
    out = {}
    for prec in (vie.C64, vie.C128):
        op = vie.Operator(ctx, g)
        out[prec] = (op, op.compress(TOL, prec, method=vie.COMPRESS_CROSS))
    yield out
    for op, _ in out.values():
        op.close()


def _block(P, Z, blk):
    return Z[np.ix_(C.atom_rows(P, blk["tatoms"]), C.atom_rows(P, blk["satoms"]))]


def test_c128_blocks_bound_interpolation_and_rank(cross_ops, tiny_dense):
    P, Z = tiny_dense[:2]
    op, info = cross_ops[vie.C128]
    assert info["compress_method"] == vie.COMPRESS_CROSS and info["factor_precision"] == vie.C128
    assert info["cross_bytes"] > 0 and info["t_cross_s"] > 0
    blocks = op.far_blocks()
    assert blocks
    for idx, blk in enumerate(blocks):
        Ab = _block(P, Z, blk)
        D = Ab - blk["Q"] @ blk["R"]
        r = blk["rank"]
        # the stopping rule on the formed float64 block (the oracle's entries agree to
        # ~1e-12; translated copies differ from their representative by the rounding
        # of the centres)
        assert np.linalg.norm(D) <= TOL * np.linalg.norm(Ab) * (1 + 1e-6)
        # a cross approximation reproduces its r pivot rows and r pivot columns
        tiny = 1e-9 * np.abs(Ab).max()
        assert (np.abs(D).max(axis=1) <= tiny).sum() >= r
        assert (np.abs(D).max(axis=0) <= tiny).sum() >= r
        assert r >= X.svd_rank(Ab, TOL)
        if idx % 3 == 0:
            # the oracle's cross approximation of the same block; the ranks agree up
            # to the tie-breaking of equal moduli under different rounding
            _, _, piv, _ = X.cross_full(Ab, TOL)
            assert abs(r - len(piv)) <= max(3, 0.1 * len(piv))


def test_c64_blocks_within_bound(cross_ops, tiny_dense):
    P, Z = tiny_dense[:2]
    op, info = cross_ops[vie.C64]
    ranks64 = []
    for blk in op.far_blocks():
        Ab = _block(P, Z, blk)
        # the tolerance on the formed float32 block plus its assembly error (entries of
        # atom-pair blocks within 5e-5 of the oracle's)
        assert np.linalg.norm(Ab - blk["Q"] @ blk["R"]) <= (TOL + 5e-5) * np.linalg.norm(Ab)
        ranks64.append(blk["rank"])
    ranks128 = [b["rank"] for b in cross_ops[vie.C128][0].far_blocks(with_factors=False)]
    assert abs(np.mean(ranks64) - np.mean(ranks128)) <= 0.1 * np.mean(ranks128) + 1


def test_apply_matches_oracle_on_exported_factors(cross_ops, tiny_dense):
    P, Z = tiny_dense[:2]
    sb = {t: A.self_block(P, t) for t in sorted(set(P.types.tolist()))}
    for prec, tol in ((vie.C64, 1e-5), (vie.C128, 1e-12)):
        op = cross_ops[prec][0]
        blocks = op.far_blocks()
        orc = C.operator_from_factors(P, sb, [(b["tatoms"], b["satoms"], b["Q"], b["R"]) for b in blocks])
        xs = workloads.random_complex(P.n, 77, cols=2).T.copy()
        ref = np.stack([orc.apply(x) for x in xs])
        dt = torch.complex64 if prec == vie.C64 else torch.complex128
        xd = torch.from_numpy(xs).to(dt).cuda()
        yd = torch.zeros_like(xd)
        op.apply(xd.data_ptr(), yd.data_ptr(), 2, prec, 0)
        assert rel(yd.cpu().numpy(), ref) < tol


def test_solves_match_dense_direct(cross_ops, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    ref = np.linalg.solve(Z, b)
    op = cross_ops[vie.C64][0]
    I, st, status = op.solve(kh[None], pol[None], tol=1e-6)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], ref) <= 5e-4
    # eight right-hand sides with the far part on the tensor cores (BF16x3)
    khs, pols = workloads.angle_sweep(4, 60.0)
    I8, st8, status8 = op.solve(khs, pols, tol=1e-6, precision=vie.BF16X3)
    assert status8 == vie.VIE_OK and len(khs) == 8
    for c in range(len(khs)):
        assert rel(I8[:, c], np.linalg.solve(Z, A.rhs(P, khs[c], pols[c]))) <= 5e-4


def test_three_level_solve_matches_dense(ctx):
    d = np.load(os.path.join(GOLDEN, "mid_8x8_nv3.npz"))
    kh, pol, ref = d["khat"], d["pol"], d["I"]
    op = vie.Operator(ctx, workloads.square_array(8, 3))
    info = op.compress(TOL, vie.C64, method=vie.COMPRESS_CROSS)
    assert info["levels"] == 3
    I, st, status = op.solve(kh[:1], pol[:1], tol=1e-6)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], ref[:, 0]) <= 5e-4
    op.close()


def test_cross_and_range_finder_operators_agree(ctx, cross_ops):
    g, kh, pol = workloads.config("tiny")
    qr = vie.Operator(ctx, g)
    qr.compress(TOL, vie.C64)
    x = torch.from_numpy(workloads.random_complex(qr.n, 8)).to(torch.complex64).cuda()
    y1, y2 = torch.zeros_like(x), torch.zeros_like(x)
    qr.apply(x.data_ptr(), y1.data_ptr(), 1, vie.C64, 0)
    cross_ops[vie.C64][0].apply(x.data_ptr(), y2.data_ptr(), 1, vie.C64, 0)
    # both within the per-block tolerance of the same matrix
    assert rel(y2.cpu().numpy(), y1.cpu().numpy()) <= 2 * TOL
    qr.close()
