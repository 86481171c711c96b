"""GPU parity tests: the CUDA path (through the C-ABI) against the CPU oracle
on the same seeded inputs."""
import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, tree as T, compress as C, krylov as K
from oracle import fields as OF

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny_op(ctx, tiny_dense):
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    return op


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("nv,side", [(1, 0.2), (2, 0.2), (3, 0.2), (3, 0.05)])
def test_self_block_float64(ctx, nv, side):
    g = workloads.square_array(1, nv, side=side)
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    Zg = op.export_block(0, 0)
    Zo = A.self_block(P, 0)
    assert rel(Zg, Zo) < 1e-12
    inv = op.export_block(2, 0)
    assert np.linalg.norm(inv @ Zo - np.eye(P.n)) < 1e-10


def test_graded_types_self_blocks(ctx):
    g = workloads.graded_array(4, 2, seed=1)
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    for t in sorted(set(g.types.tolist())):
        assert rel(op.export_block(0, t), A.self_block(P, t)) < 1e-12


@pytest.mark.parametrize("pair", [(0, 1), (5, 0), (3, 12), (15, 6)])
def test_cross_block(ctx, tiny_dense, pair):
    P, Z, _, _, _ = tiny_dense
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    a, b = pair
    ref = Z[P.offsets[a]:P.offsets[a + 1], P.offsets[b]:P.offsets[b + 1]]
    assert rel(op.export_block(1, a, b, vie.C128), ref) < 1e-12
    # float64 tables rounded to complex float32: each component within 2^-24 relative
    assert rel(op.export_block(1, a, b, vie.C64), ref) < 1e-7


def test_cross_block_graded_and_large_atoms(ctx):
    g = workloads.graded_array(3, 4, seed=2)
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    for a, b in ((0, 4), (8, 1)):
        ref = A.cross_block(P, a, b)
        assert rel(op.export_block(1, a, b, vie.C128), ref) < 1e-12
        # float32 entries from float64 tables: only their rounding (2^-24 relative)
        assert rel(op.export_block(1, a, b, vie.C64), ref) < 1e-7


def test_rhs(ctx, tiny_dense):
    import torch as th
    P, _, b, _, _ = tiny_dense
    g, kh, pol = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    kh2, pol2 = workloads.angle_sweep(3, 60.0)
    bd = th.zeros((len(kh2), op.n), dtype=th.complex128, device="cuda")
    op.rhs(kh2, pol2, bd.data_ptr())
    bg = bd.cpu().numpy()
    for c in range(len(kh2)):
        assert rel(bg[c], A.rhs(P, kh2[c], pol2[c])) < 1e-12


# ---------------------------------------------------------------------- tree
@pytest.mark.parametrize("ns", [2, 4, 5, 8])
def test_far_block_lists_match_oracle(ctx, ns):
    g = workloads.square_array(ns, 1)
    op = vie.Operator(ctx, g)
    mine = [(b["level"], list(b["tatoms"]), list(b["satoms"])) for b in op.far_blocks(with_factors=False)]
    _, ref = T.build_tree(g.centres)
    assert mine == [(l, list(t), list(s)) for l, t, s in ref]


# ---------------------------------------------------------------- compression
def mirrors(blocks):
    """index of the block (source box, target box) for every block"""
    key = {(b["level"], int(b["tatoms"][0]), int(b["satoms"][0])): i for i, b in enumerate(blocks)}
    return [key[(b["level"], int(b["satoms"][0]), int(b["tatoms"][0]))] for b in blocks]


def check_factors(blocks, ortho_tol):
    """Of each mirror pair the first block is compressed (orthonormal Q); the
    second holds the transposed factors (reciprocity of the rule between atoms)."""
    mir = mirrors(blocks)
    for i, blk in enumerate(blocks):
        j = mir[i]
        assert j != i
        if i < j:
            Q = blk["Q"]
            assert np.linalg.norm(Q.conj().T @ Q - np.eye(blk["rank"])) < ortho_tol
        else:
            p = blocks[j]
            assert blk["rank"] == p["rank"]
            assert np.array_equal(blk["Q"], p["R"].T) and np.array_equal(blk["R"], p["Q"].T)


def test_compression_error_bound(tiny_op, tiny_dense):
    P, Z, _, _, _ = tiny_dense
    blocks = tiny_op.far_blocks()
    for blk in blocks:
        rows = C.atom_rows(P, blk["tatoms"])
        cols = C.atom_rows(P, blk["satoms"])
        Ab = Z[np.ix_(rows, cols)]
        assert np.linalg.norm(Ab - blk["Q"] @ blk["R"]) <= 1e-4 * np.linalg.norm(Ab)
    check_factors(blocks, 1e-4)   # float32 storage


# ---------------------------------------------------------------------- apply
def _oracle_op_from_gpu(op, P, Z):
    blocks = op.far_blocks()
    sb = {t: A.self_block(P, t) for t in sorted(set(P.types.tolist()))}
    return C.operator_from_factors(P, sb, [(b["tatoms"], b["satoms"], b["Q"], b["R"]) for b in blocks]), sb


def test_apply_parity_c64_and_acc64(tiny_op, tiny_dense):
    import torch as th
    P, Z, _, _, _ = tiny_dense
    orc, sb = _oracle_op_from_gpu(tiny_op, P, Z)
    xs = workloads.random_complex(P.n, 1234, cols=3).T.copy()   # 3 RHS, rows contiguous
    ref = np.stack([orc.apply(x) for x in xs])
    x32 = th.from_numpy(xs.astype(np.complex64)).cuda()
    y32 = th.zeros_like(x32)
    tiny_op.apply(x32.data_ptr(), y32.data_ptr(), 3, vie.C64, 0)
    assert rel(y32.cpu().numpy(), ref) < 1e-5
    x64 = th.from_numpy(xs).cuda()
    y64 = th.zeros_like(x64)
    tiny_op.apply(x64.data_ptr(), y64.data_ptr(), 3, vie.C64_ACC64, 0)
    # float32 factors read exactly, float64 arithmetic: rounding-level agreement
    assert rel(y64.cpu().numpy(), ref) < 1e-12


def test_fused_precond_apply(tiny_op, tiny_dense):
    import torch as th
    P, Z, _, _, _ = tiny_dense
    orc, sb = _oracle_op_from_gpu(tiny_op, P, Z)
    M = K.BlockJacobi(P, sb)
    x = workloads.random_complex(P.n, 99)
    ref = M.apply(orc.apply(x))
    xd = th.from_numpy(x.astype(np.complex64)).cuda()
    yd = th.zeros_like(xd)
    tiny_op.apply(xd.data_ptr(), yd.data_ptr(), 1, vie.C64, vie.FUSE_PRECOND)
    assert rel(yd.cpu().numpy(), ref) < 1e-5
    xd = th.from_numpy(x).cuda()
    yd = th.zeros_like(xd)
    tiny_op.precond(xd.data_ptr(), yd.data_ptr(), 1, vie.C128)
    assert rel(yd.cpu().numpy(), M.apply(x)) < 1e-12


def test_c128_factors_apply(ctx, tiny_dense):
    import torch as th
    P, Z, _, _, _ = tiny_dense
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C128)
    orc, _ = _oracle_op_from_gpu(op, P, Z)
    x = workloads.random_complex(P.n, 5)
    xd = th.from_numpy(x).cuda()
    yd = th.zeros_like(xd)
    op.apply(xd.data_ptr(), yd.data_ptr(), 1, vie.C128, 0)
    assert rel(yd.cpu().numpy(), orc.apply(x)) < 1e-12
    blocks = op.far_blocks()
    for blk in blocks:
        rows = C.atom_rows(P, blk["tatoms"])
        cols = C.atom_rows(P, blk["satoms"])
        Ab = Z[np.ix_(rows, cols)]
        assert np.linalg.norm(Ab - blk["Q"] @ blk["R"]) <= 1e-4 * np.linalg.norm(Ab)
    check_factors(blocks, 1e-12)


# ---------------------------------------------------------------------- solve
def test_solve_matches_dense_direct(tiny_op, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    I, st, status = tiny_op.solve(kh[None], pol[None], tol=1e-6)
    assert status == vie.VIE_OK
    ref = np.linalg.solve(Z, b)
    assert rel(I[:, 0], ref) <= 5e-4
    assert st["residual"] <= 1e-6
    # the oracle's GMRES on the GPU's factors needs about as many iterations
    orc, sb = _oracle_op_from_gpu(tiny_op, P, Z)
    _, info = K.gmres(orc.apply, b, K.BlockJacobi(P, sb).apply, tol=1e-6, restart=60)
    assert abs(st["iterations"] - info["iterations"]) <= max(2, 0.1 * info["iterations"])


def test_solve_all_float64(ctx, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C128)
    I, st, status = op.solve(kh[None], pol[None], tol=1e-6, precision=vie.C128)
    assert status == vie.VIE_OK
    assert rel(I[:, 0], np.linalg.solve(Z, b)) <= 5e-4


def test_cross_sections(tiny_op, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    I, _, _ = tiny_op.solve(kh[None], pol[None], tol=1e-8)
    sig = tiny_op.sigma(I, kh[None], pol[None])[0]
    v0 = A.rhs_v0(P, kh, pol)
    assert abs(sig[0] - OF.sigma_ext(I[:, 0], v0)) < 1e-10 * abs(sig[0])
    assert abs(sig[1] - OF.sigma_sca(P, I[:, 0])) < 1e-10 * abs(sig[1])
    assert abs(sig[0] - sig[1]) < 1e-3 * sig[0]   # optical theorem (lossless)


# ------------------------------------------------------------- multi-RHS solve
def test_multi_rhs_solve_matches_dense_and_single(tiny_op, tiny_dense):
    P, Z, _, _, _ = tiny_dense
    kh, pol = workloads.angle_sweep(3, 60.0)          # 6 right-hand sides
    I, st, status = tiny_op.solve(kh, pol, tol=1e-6)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    for c in range(len(kh)):
        ref = np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))
        assert rel(I[:, c], ref) <= 5e-4
        Ic, _, _ = tiny_op.solve(kh[c:c + 1], pol[c:c + 1], tol=1e-6)
        assert rel(I[:, c], Ic[:, 0]) <= 1e-5      # lockstep changes scheduling, not the method
    assert st["applies"] < sum(1 for _ in range(len(kh))) * st["iterations"]


def test_multi_rhs_apply_reads_factors_once(ctx, tiny_op, tiny_dense):
    # 9 right-hand sides (groups of 4 + tail) against one-at-a-time applies
    import torch as th
    P, Z, _, _, _ = tiny_dense
    xs = workloads.random_complex(P.n, 77, cols=9).T.copy()
    X = th.from_numpy(xs.astype(np.complex64)).cuda()
    Y = th.zeros_like(X)
    tiny_op.apply(X.data_ptr(), Y.data_ptr(), 9, vie.C64, vie.FUSE_PRECOND)
    for c in range(9):
        y1 = th.zeros_like(X[c])
        tiny_op.apply(X[c].data_ptr(), y1.data_ptr(), 1, vie.C64, vie.FUSE_PRECOND)
        th.cuda.synchronize()
        assert rel(Y[c].cpu().numpy(), y1.cpu().numpy()) < 1e-6


# ------------------------------------------------- BF16x3 tensor-core far apply
@pytest.mark.parametrize("nrhs", [1, 5, 64, 70])
def test_bf16x3_apply_against_c64(tiny_op, tiny_dense, nrhs):
    # split-precision bf16 (hi.hi + hi.lo + lo.hi, float32 accumulation): the
    # dropped lo.lo term and the bf16 remainders give ~1e-5 relative
    import torch as th
    P, Z, _, _, _ = tiny_dense
    orc, sb = _oracle_op_from_gpu(tiny_op, P, Z)
    xs = workloads.random_complex(P.n, 31, cols=nrhs).T.copy()
    X = th.from_numpy(xs.astype(np.complex64)).cuda()
    Y = th.zeros_like(X)
    tiny_op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.BF16X3, 0)
    th.cuda.synchronize()
    ref = np.stack([orc.apply(x) for x in xs])
    assert rel(Y.cpu().numpy(), ref) < 5e-5


def test_bf16x3_multi_rhs_solve(tiny_op, tiny_dense):
    P, Z, _, _, _ = tiny_dense
    kh, pol = workloads.angle_sweep(4, 60.0)           # 8 right-hand sides
    I, st, status = tiny_op.solve(kh, pol, tol=1e-6, precision=vie.BF16X3)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    for c in range(len(kh)):
        assert rel(I[:, c], np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))) <= 5e-4


# ------------------------------------------------ graph-captured restart cycles
def test_graph_cycle_equals_host_loop(tiny_op, tiny_dense):
    # the same kernels in the same order: one CUDA graph per restart cycle
    # (Arnoldi steps in a conditional while-node) against host-launched steps
    P, Z, _, _, _ = tiny_dense
    kh, pol = workloads.angle_sweep(2, 40.0)           # 4 right-hand sides
    Ig, stg, sg = tiny_op.solve(kh, pol, tol=1e-6, restart=8, launch=0)
    Ih, sth, sh = tiny_op.solve(kh, pol, tol=1e-6, restart=8, launch=1)
    assert sg == sh == vie.VIE_OK
    assert stg["iterations"] == sth["iterations"] > 8 and stg["refinements"] == sth["refinements"] >= 1
    assert np.array_equal(Ig, Ih)
    assert stg["history"] == sth["history"]
    for c in range(len(kh)):
        assert rel(Ig[:, c], np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))) <= 5e-4


def test_solver_history_and_limits(tiny_op, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    I, st, status = tiny_op.solve(kh[None], pol[None], tol=1e-6)
    h = st["history"]
    assert len(h) == st["applies"] and h[-1] <= 1e-6 < h[0]
    # an iteration cap that stops the solve early reports NOT_CONVERGED with the stats written
    I2, st2, status2 = tiny_op.solve(kh[None], pol[None], tol=1e-12, max_iters=3)
    assert status2 == vie.VIE_ERR_NOT_CONVERGED and st2["iterations"] == 3 and st2["residual"] > 1e-12
    with pytest.raises(vie.VieError):
        tiny_op.solve(np.tile(kh, (1025, 1)), np.tile(pol, (1025, 1)))


@pytest.mark.parametrize("nrhs", [3, 16, 64])
def test_bf16x3_apply_4cube_array(ctx, nrhs):
    # 8x8 array of 4^3-voxel cubes (240 unknowns per atom, three tree levels):
    # the tensor-core apply against the float32 SIMT apply of the same factors
    import torch as th
    g = workloads.square_array(8, 4)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    X = th.from_numpy(workloads.random_complex(op.n, 7, cols=nrhs).T.astype(np.complex64).copy()).cuda()
    Y = th.zeros_like(X)
    Yr = th.zeros_like(X)
    for fl in (0, vie.FUSE_PRECOND):
        op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.BF16X3, fl)
        op.apply(X.data_ptr(), Yr.data_ptr(), nrhs, vie.C64, fl)
        th.cuda.synchronize()
        assert rel(Y.cpu().numpy(), Yr.cpu().numpy()) < 5e-5
    op.close()


# ------------------------------------------------------------------- autotuner
def test_autotune_variants_agree(ctx, tiny_dense):
    import torch as th
    P, Z, _, _, _ = tiny_dense
    g, _, _ = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    nrhs = 5
    X = th.from_numpy(workloads.random_complex(P.n, 3, cols=nrhs).T.astype(np.complex64).copy()).cuda()
    res = op.tune(vie.C64, nrhs)
    assert res["variant"] in (vie.VAR_SIMT_R1, vie.VAR_SIMT_R2, vie.VAR_SIMT_R4, vie.VAR_SIMT_R8)
    assert set(res["ms"]) == {vie.VAR_SIMT_R1, vie.VAR_SIMT_R2, vie.VAR_SIMT_R4, vie.VAR_SIMT_R8}
    assert all(t > 0 for t in res["ms"].values())
    out = {}
    for v in (vie.VAR_SIMT_R1, vie.VAR_SIMT_R2, vie.VAR_SIMT_R4, vie.VAR_SIMT_R8):
        op.tune(vie.C64, nrhs, force=v)
        Y = th.zeros_like(X)
        op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.C64, vie.FUSE_PRECOND)
        th.cuda.synchronize()
        out[v] = Y.cpu().numpy()
    # the register tiles keep every column's summation order: bit-identical
    assert np.array_equal(out[vie.VAR_SIMT_R2], out[vie.VAR_SIMT_R4])
    assert np.array_equal(out[vie.VAR_SIMT_R4], out[vie.VAR_SIMT_R8])
    assert rel(out[vie.VAR_SIMT_R1], out[vie.VAR_SIMT_R4]) < 1e-6
    # split-precision variants are admissible for VIE_BF16X3 only
    with pytest.raises(vie.VieError):
        op.tune(vie.C64, nrhs, force=vie.VAR_TCGEN05_BF16X3)
    for v in (vie.VAR_MMA_BF16X3, vie.VAR_TCGEN05_BF16X3, vie.VAR_TCGEN05_PACKED_BF16X3,
              vie.VAR_TCGEN05_WS_BF16X3, vie.VAR_TCGEN05_WS2_BF16X3):
        op.tune(vie.BF16X3, nrhs, force=v)
        Y = th.zeros_like(X)
        op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.BF16X3, vie.FUSE_PRECOND)
        th.cuda.synchronize()
        assert rel(Y.cpu().numpy(), out[vie.VAR_SIMT_R4]) < 5e-5
    res = op.tune(vie.BF16X3, 64)
    assert res["variant"] in range(1, 11) and len(res["ms"]) == 9
    kh, pol = workloads.angle_sweep(2, 30.0)
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=vie.BF16X3, autotune=1)
    assert status == vie.VIE_OK
    for c in range(len(kh)):
        assert rel(I[:, c], np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))) <= 5e-4
    op.close()


def test_shared_factor_apply(ctx, tiny_dense):
    # one right-hand side: the translated copies of a block applied together
    # (each shared factor read once per group of copies, the default when the
    # operator has copies) against the per-block kernel and the oracle
    import torch as th
    P, Z, _, _, _ = tiny_dense
    g, kh, pol = workloads.config("tiny")
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    orc, _ = _oracle_op_from_gpu(op, P, Z)
    xs = workloads.random_complex(P.n, 91, cols=3).T.copy()
    X = th.from_numpy(xs.astype(np.complex64)).cuda()
    res = op.tune(vie.C64, 1)
    assert set(res["ms"]) == {vie.VAR_SIMT_R1, vie.VAR_SIMT_SHARED}
    out = {}
    for v in (vie.VAR_SIMT_R1, vie.VAR_SIMT_SHARED):
        op.tune(vie.C64, 1, force=v)
        op.tune(vie.C64, 3, force=v)
        for fl in (0, vie.FUSE_PRECOND):
            Y = th.zeros_like(X)
            op.apply(X.data_ptr(), Y.data_ptr(), 1, vie.C64, fl)
            Y3 = th.zeros_like(X)
            op.apply(X.data_ptr(), Y3.data_ptr(), 3, vie.C64, fl)   # one column at a time
            th.cuda.synchronize()
            out[v, fl] = Y.cpu().numpy()[0]
            out[v, fl, 3] = Y3.cpu().numpy()
    for fl in (0, vie.FUSE_PRECOND):
        assert rel(out[vie.VAR_SIMT_SHARED, fl], out[vie.VAR_SIMT_R1, fl]) < 1e-6
        assert np.array_equal(out[vie.VAR_SIMT_SHARED, fl, 3][0], out[vie.VAR_SIMT_SHARED, fl])
    ref = np.stack([orc.apply(x) for x in xs])
    assert rel(out[vie.VAR_SIMT_SHARED, 0, 3], ref) < 1e-5
    # deterministic summation order: graph-captured and host-launched solves agree bit for bit
    op.tune(vie.C64, 1, force=vie.VAR_SIMT_SHARED)
    Ig, stg, sg = op.solve(kh, pol, tol=1e-6, restart=8, launch=0)
    Ih, sth, sh = op.solve(kh, pol, tol=1e-6, restart=8, launch=1)
    assert sg == sh == vie.VIE_OK and np.array_equal(Ig, Ih)
    assert rel(Ig[:, 0], np.linalg.solve(Z, A.rhs(P, kh[0], pol[0]))) <= 5e-4
    op.close()


def test_tcgen05_packed_and_warp_specialised_agree_with_unpacked(ctx):
    # the packed variant feeds the tensor core the same bf16 planes in the same
    # MMA order (moved by bulk copies instead of split by the warps):
    # bit-identical; the warp-specialised one forms the same products with four
    # wide MMAs per K step (two accumulator halves added in the epilogue): equal
    # to float32 rounding, and so is the paired-tile one (two row tiles per B
    # tile, 16 K values per stage); fused and unfused, for column counts that
    # fill one 64-column pass, a pass plus a ragged tail, and partial passes
    # (the rings hold 3 to 6 stages by column count)
    import torch as th
    g = workloads.square_array(8, 4)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    for nrhs in (8, 16, 24, 40, 64, 70):
        X = th.from_numpy(workloads.random_complex(op.n, 11, cols=nrhs).T.astype(np.complex64).copy()).cuda()
        for fl in (vie.FUSE_PRECOND, 0):
            out = {}
            for v in (vie.VAR_TCGEN05_BF16X3, vie.VAR_TCGEN05_PACKED_BF16X3, vie.VAR_TCGEN05_WS_BF16X3,
                      vie.VAR_TCGEN05_WS2_BF16X3):
                op.tune(vie.BF16X3, nrhs, force=v)
                Y = th.zeros_like(X)
                op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.BF16X3, fl)
                th.cuda.synchronize()
                out[v] = Y.cpu().numpy()
            assert np.array_equal(out[vie.VAR_TCGEN05_BF16X3], out[vie.VAR_TCGEN05_PACKED_BF16X3]), (nrhs, fl)
            assert rel(out[vie.VAR_TCGEN05_WS_BF16X3], out[vie.VAR_TCGEN05_PACKED_BF16X3]) < 5e-6, (nrhs, fl)
            assert rel(out[vie.VAR_TCGEN05_WS2_BF16X3], out[vie.VAR_TCGEN05_PACKED_BF16X3]) < 5e-6, (nrhs, fl)
    op.close()


# ------------------------------------------------------- translated copies share
def test_translated_blocks_share_factors(ctx, tiny_op, tiny_dense):
    P, Z, b, kh, pol = tiny_dense
    info = tiny_op.info()
    # 4 x 4 array of identical cubes: 240 far blocks, 48 distinct box offsets
    assert info["stored_entries"] * 4 < info["factor_entries"]
    blocks = tiny_op.far_blocks()
    for blk in blocks:  # every block, shared or not, meets its own bound
        rows = C.atom_rows(P, blk["tatoms"])
        cols = C.atom_rows(P, blk["satoms"])
        Ab = Z[np.ix_(rows, cols)]
        assert np.linalg.norm(Ab - blk["Q"] @ blk["R"]) <= 1e-4 * np.linalg.norm(Ab)
    ctx2 = vie.Context(0, no_sharing=1)
    g, _, _ = workloads.config("tiny")
    op2 = vie.Operator(ctx2, g)
    info2 = op2.compress(1e-4, vie.C64)
    assert info2["stored_entries"] == info2["factor_entries"]
    I2, _, s2 = op2.solve(kh[None], pol[None], tol=1e-6)
    I1, _, s1 = tiny_op.solve(kh[None], pol[None], tol=1e-6)
    ref = np.linalg.solve(Z, b)
    assert s1 == s2 == vie.VIE_OK and rel(I1[:, 0], ref) <= 5e-4 and rel(I2[:, 0], ref) <= 5e-4
    op2.close()
    ctx2.close()


def test_graded_array_solve(ctx):
    # three meta-atom types: only blocks with the same types and relative
    # positions share factors
    g = workloads.graded_array(4, 3, seed=0)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    kh, pol = workloads.normal_incidence()
    I, st, status = op.solve(kh, pol, tol=1e-6)
    assert status == vie.VIE_OK
    assert rel(I[:, 0], np.linalg.solve(Z, A.rhs(P, kh[0], pol[0]))) <= 5e-4
    op.close()


# ------------------------------------- other materials, grids and array shapes
@pytest.mark.parametrize("ns,nv,eps", [(4, 3, complex(12.0, -3.0)), (4, 2, 12.0), (3, 4, complex(6.0, -0.5))])
def test_array_solve_against_dense(ctx, ns, nv, eps):
    # a lossy permittivity (Im eps < 0 under exp(j w t), Sec. 2), coarser (36 unknowns per
    # atom) and finer (240) voxel grids, and a 3 x 3 array whose quadtree
    # leaves part of its boxes empty: the GPU solve against a direct solve of
    # the oracle's dense matrix
    g = workloads.square_array(ns, nv, eps=eps)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    kh, pol = workloads.normal_incidence()
    I, st, status = op.solve(kh, pol, tol=1e-6)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], np.linalg.solve(Z, A.rhs(P, kh[0], pol[0]))) <= 5e-4
    ext, sca = op.sigma(I, kh, pol)[0]
    v0 = A.rhs_v0(P, kh[0], pol[0])
    assert abs(ext - OF.sigma_ext(I[:, 0], v0)) < 1e-10 * abs(ext)
    assert abs(sca - OF.sigma_sca(P, I[:, 0])) < 1e-10 * abs(sca)
    if np.imag(eps) != 0:
        assert ext > sca * (1 + 1e-2)             # absorption: extinction exceeds scattering
    else:
        assert abs(ext - sca) < 1e-3 * ext        # optical theorem (lossless)
    op.close()


# ------------------------------------------------------------ C-ABI error paths
def test_apply_rejects_bad_arguments(tiny_op):
    # every case is refused before anything is launched; all pointers stay in bounds
    import torch as th
    n = tiny_op.n
    buf = th.zeros(2 * n + 4, dtype=th.complex64, device="cuda")
    y = th.zeros(2 * n, dtype=th.complex64, device="cuda")
    x128 = th.zeros(n, dtype=th.complex128, device="cuda")
    y128 = th.zeros(n, dtype=th.complex128, device="cuda")

    def status(fn):
        with pytest.raises(vie.VieError) as e:
            fn()
        return e.value.status

    bad = vie.VIE_ERR_INVALID_ARG
    x0 = buf.data_ptr()
    # off the 16-byte grid (the c64 kernels read complex pairs as one 16-byte load)
    assert status(lambda: tiny_op.apply(x0 + 8, y.data_ptr(), 1, vie.C64, 0)) == bad
    assert status(lambda: tiny_op.apply(x0, y.data_ptr() + 8, 1, vie.BF16X3, vie.FUSE_PRECOND)) == bad
    assert status(lambda: tiny_op.precond(x0 + 8, y.data_ptr(), 1, vie.C64)) == bad
    # overlapping input and output
    assert status(lambda: tiny_op.apply(x0, x0 + 16, 1, vie.C64, 0)) == bad
    assert status(lambda: tiny_op.apply(x0, x0, 1, vie.C64, vie.FUSE_PRECOND)) == bad
    # float64 factors wanted, an unknown precision, a dense apply of two columns
    assert status(lambda: tiny_op.apply(x128.data_ptr(), y128.data_ptr(), 1, vie.C128, 0)) == bad
    assert status(lambda: tiny_op.apply(x0, y.data_ptr(), 1, 99, 0)) == bad
    assert status(lambda: tiny_op.apply(x0, y.data_ptr(), 2, vie.C64, vie.DENSE)) == bad
    assert status(lambda: tiny_op.apply(x0, y.data_ptr(), 0, vie.C64, 0)) == bad
    # the context is still usable and the rejected calls wrote nothing
    th.cuda.synchronize()
    assert th.count_nonzero(y).item() == 0
    buf[:n] = 1 + 1j
    tiny_op.apply(x0, y.data_ptr(), 1, vie.C64, 0)
    th.cuda.synchronize()
    assert th.isfinite(th.view_as_real(y[:n])).all().item() and th.count_nonzero(y[:n]).item() == n
