"""GPU parity on three-level quadtrees: the solve paths (complex float32 single
RHS, BF16x3 lockstep multi-RHS, the batched union and a served request) on an
8 x 8 array of 3^3-voxel cubes and an 8 x 8 graded array (three cube sides),
against the oracle's dense direct solution of the same discrete system
(Sec. 6.2: the reference solution is the LU solve), and the tensor-core apply
the far-field amplitude and the near field against the oracle element by element.

The dense solutions (6,912 unknowns each) are written by
tests/golden/make_multilevel_golden.py, which calls only the oracle.
"""
import os
import time

import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, compress as OC
from oracle import fields as OF

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_10586_gb300 import vie  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def golden(name):
    d = np.load(os.path.join(GOLDEN, name + ".npz"))
    return d["khat"], d["pol"], d["I"]


GEOM = {"mid_8x8_nv3": lambda: workloads.square_array(8, 3),
        "graded_8x8_nv3": lambda: workloads.graded_array(8, 3, 0)}


@pytest.fixture(scope="module")
def ctx():
    c = vie.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ops(ctx):
    out = {}
    for name, mk in GEOM.items():
        op = vie.Operator(ctx, mk())
        info = op.compress(1e-4, vie.C64)
        out[name] = (op, info)
    yield out
    for op, _ in out.values():
        op.close()


@pytest.mark.parametrize("name", list(GEOM))
def test_three_level_tree(ops, name):
    op, info = ops[name]
    levels = sorted({b["level"] for b in op.far_blocks(with_factors=False)})
    assert levels == [2, 3] and info["levels"] == 3


@pytest.mark.parametrize("name", list(GEOM))
def test_single_rhs_c64_solve_matches_dense(ops, name):
    op, _ = ops[name]
    kh, pol, ref = golden(name)
    I, st, status = op.solve(kh[:1], pol[:1], tol=1e-6)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    assert rel(I[:, 0], ref[:, 0]) <= 5e-4


@pytest.mark.parametrize("name", list(GEOM))
def test_bf16x3_lockstep_solve_matches_dense(ops, name):
    op, _ = ops[name]
    kh, pol, ref = golden(name)
    I, st, status = op.solve(kh, pol, tol=1e-6, precision=vie.BF16X3)
    assert status == vie.VIE_OK and st["residual"] <= 1e-6
    for c in range(len(kh)):
        assert rel(I[:, c], ref[:, c]) <= 5e-4, c


@pytest.mark.parametrize("precision", [vie.C64, vie.BF16X3])
def test_batch_matches_dense(ops, precision):
    names = list(GEOM)
    gold = [golden(n) for n in names]
    Is, stats, status = vie.solve_batch([ops[n][0] for n in names], [(kh, pol) for kh, pol, _ in gold],
                                        tol=1e-6, precision=precision)
    assert status == vie.VIE_OK
    for (kh, pol, ref), I, st in zip(gold, Is, stats):
        assert st["residual"] <= 1e-6
        for c in range(len(kh)):
            assert rel(I[:, c], ref[:, c]) <= 5e-4


def test_served_requests_match_dense(ctx):
    srv = vie.Server(ctx, max_inflight=2, tol=1e-4)
    tickets = []
    for name, mk in GEOM.items():
        kh, pol, _ = golden(name)
        tickets.append((name, srv.submit(mk(), kh, pol)))
    for name, t in tickets:
        r = None
        deadline = time.time() + 300
        while r is None and time.time() < deadline:
            r = srv.poll(t, timeout_ms=1000)
        assert r is not None and r["status"] == vie.VIE_OK
        _, _, ref = golden(name)
        for c in range(ref.shape[1]):
            assert rel(r["I"][:, c], ref[:, c]) <= 5e-4
    srv.stop()


@pytest.mark.parametrize("nrhs", [3, 16])
def test_bf16x3_apply_matches_oracle_on_exported_factors(ctx, nrhs):
    # 8 x 8 array of 4^3-voxel cubes (240 unknowns per atom, three levels): the
    # tensor-core apply, rows of three atoms, against the oracle applying the
    # exported factors of every block that touches them in float64
    g = workloads.square_array(8, 4)
    P = problem_from_geometry(g)
    op = vie.Operator(ctx, g)
    op.compress(1e-4, vie.C64)
    npp = op.np
    xs = workloads.random_complex(op.n, 11, cols=nrhs)
    X = torch.from_numpy(np.ascontiguousarray(xs.T).astype(np.complex64)).cuda()
    Y = torch.empty_like(X)
    op.apply(X.data_ptr(), Y.data_ptr(), nrhs, vie.BF16X3, 0)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    x = xs.astype(np.complex64).astype(np.complex128)
    meta = op.far_blocks(with_factors=False)
    Zs = A.self_block(P, 0)
    for atom in (0, 27, 63):
        rows = slice(atom * npp, (atom + 1) * npp)
        idx = [i for i, b in enumerate(meta) if atom in set(b["tatoms"].tolist())]
        ref = Zs @ x[rows]
        for b in op.far_blocks(indices=idx):
            slot = list(b["tatoms"]).index(atom)
            ref = ref + b["Q"][slot * npp:(slot + 1) * npp] @ (b["R"] @ x[OC.atom_rows(P, b["satoms"])])
        assert rel(y[:, rows].T, ref) < 5e-5, atom
    op.close()


def test_far_field_amplitude_matches_oracle(ctx, tiny_dense):
    # vie_fields mode 0 element by element against the oracle's far field of the
    # same current, in directions spread over the sphere
    P, Z, b, kh, pol = tiny_dense
    op = vie.Operator(ctx, workloads.config("tiny")[0])
    op.compress(1e-4, vie.C64)
    I, _, status = op.solve(kh[None], pol[None], tol=1e-8)
    assert status == vie.VIE_OK
    dirs, _ = OF.sphere_rule(6, 8)
    E = op.far_field(I, dirs)[0]                       # npts x 3
    ref = OF.far_field(P, I[:, 0], dirs)
    assert np.max(np.abs(E - ref)) <= 1e-10 * np.max(np.abs(ref))
    op.close()


def test_near_field_matches_oracle(ctx, tiny_dense):
    # vie_fields mode 1 element by element against the oracle's near field of
    # the same current, at points above, beside and between the atoms
    P, Z, b, kh, pol = tiny_dense
    op = vie.Operator(ctx, workloads.config("tiny")[0])
    op.compress(1e-4, vie.C64)
    I, _, status = op.solve(kh[None], pol[None], tol=1e-8)
    assert status == vie.VIE_OK
    pts = np.array([[0.0, 0.0, 0.5], [0.3, -0.2, 0.25], [1.5, 0.0, 0.0], [0.0, 0.0, 0.0], [-3.0, 2.0, 1.0]])
    E = op.near_field(I, pts)[0]
    ref = OF.near_field(P, I[:, 0], pts)
    assert np.max(np.abs(E - ref)) <= 1e-10 * np.max(np.abs(ref))
    # a refused point set leaves the context usable
    with pytest.raises(vie.VieError):
        op.near_field(I, np.array([[np.nan, 0.0, 0.0]]))
    assert np.allclose(op.near_field(I, pts[:1])[0], E[:1], rtol=1e-14, atol=0)
    op.close()


def test_compression_second_pass_for_high_ranks(ctx, ops, monkeypatch):
    # a batch whose blocks need more basis room than its first pass reserved
    # (forced here: room for 32 ranks) is compressed again with the full room;
    # the operator then solves like the one compressed in one pass
    name = "mid_8x8_nv3"
    kh, pol, ref = golden(name)
    monkeypatch.setenv("VIE_TEST_RANK_TRY", "32")
    op = vie.Operator(ctx, GEOM[name]())
    info = op.compress(1e-4, vie.C64)
    monkeypatch.delenv("VIE_TEST_RANK_TRY")
    base = ops[name][1]
    assert max(b["rank"] for b in op.far_blocks(with_factors=False)) > 32
    assert abs(info["factor_entries"] - base["factor_entries"]) <= 0.1 * base["factor_entries"]
    I, st, status = op.solve(kh[:1], pol[:1], tol=1e-6)
    assert status == vie.VIE_OK
    assert rel(I[:, 0], ref[:, 0]) <= 5e-4
    op.close()
