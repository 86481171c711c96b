"""Serving (continuous batching): requests of different sizes submitted while
others run are admitted as slots and memory free up, run concurrently on their
own streams, and give the same result as when solved alone."""
import time

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


def _requests():
    rng = np.random.default_rng(8)
    out = []
    for i, ns in enumerate((3, 6, 4, 7, 5, 3, 8, 4)):
        lam = float(rng.uniform(0.9, 1.1))
        eps = float(rng.uniform(8, 14))
        g = workloads.square_array(ns, 3 if i % 2 == 0 else 2, 0.2, 0.4, eps, lam)
        kh, pol = workloads.random_directions(1 + i % 3, seed=100 + i)
        out.append((g, kh, pol))
    return out


def test_mix_equals_alone_and_requests_overlap():
    ctx = vie.Context(0)
    reqs = _requests()
    srv = vie.Server(ctx, max_inflight=3, tol=1e-4)
    tickets = []
    for g, kh, pol in reqs:
        tickets.append(srv.submit(g, kh, pol))
        time.sleep(0.005)                      # arrivals while others run
    results = []
    for t in tickets:
        r = None
        deadline = time.time() + 300
        while r is None and time.time() < deadline:
            r = srv.poll(t, timeout_ms=1000)
        assert r is not None, "request did not finish"
        results.append(r)
    srv.stop()
    # concurrency: some request started before another one finished
    spans = sorted((r["t_start"], r["t_done"]) for r in results)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for (g, kh, pol), r in zip(reqs, results):
        assert r["status"] == vie.VIE_OK and r["stats"]["residual"] <= 1e-6
        op = vie.Operator(ctx, g)
        op.compress(1e-4, vie.C64)
        I, st, status = op.solve(kh, pol, tol=1e-6)
        op.close()
        assert status == vie.VIE_OK
        assert rel(r["I"], I) <= 1e-10              # the same alone and in the mix
    # accuracy of two of them against the oracle's dense solve
    for idx in (0, 5):
        g, kh, pol = reqs[idx]
        P = problem_from_geometry(g)
        Z = A.dense_matrix(P)
        for c in range(len(kh)):
            ref = np.linalg.solve(Z, A.rhs(P, kh[c], pol[c]))
            assert rel(results[idx]["I"][:, c], ref) <= 5e-4
    ctx.close()


def test_admission_rejects_oversized_request():
    ctx = vie.Context(0)
    srv = vie.Server(ctx, max_inflight=2, hbm_budget=256 << 20)   # 256 MiB
    g = workloads.square_array(48, 3)
    kh, pol = workloads.normal_incidence()
    with pytest.raises(vie.VieError) as e:
        srv.submit(g, kh, pol)
    assert e.value.status == vie.VIE_ERR_ADMISSION
    small = workloads.square_array(2, 2)
    t = srv.submit(small, kh, pol)
    r = srv.poll(t, timeout_ms=120000)
    assert r is not None and r["status"] == vie.VIE_OK
    srv.stop()
    ctx.close()


def test_underestimated_footprint_backs_off_instead_of_failing(monkeypatch):
    # the footprint model scaled down 50x: each slot's context caps its
    # allocations at the admitted footprint, so the requests run into the cap
    # (a host-side refusal before cudaMalloc), go back to the head of the queue
    # with twice the footprint and finish once enough is free; the results are
    # those of plain solves
    monkeypatch.setenv("VIE_TEST_FOOTPRINT_SCALE", "0.02")
    ctx = vie.Context(0)
    srv = vie.Server(ctx, max_inflight=3, hbm_budget=6 << 30, tol=1e-4)
    reqs = _requests()[:5]
    tickets = [srv.submit(g, kh, pol) for g, kh, pol in reqs]
    results = []
    for t in tickets:
        r = None
        deadline = time.time() + 300
        while r is None and time.time() < deadline:
            r = srv.poll(t, timeout_ms=1000)
        assert r is not None
        results.append(r)
    srv.stop()
    assert all(r["status"] == vie.VIE_OK for r in results)
    assert any(r["retries"] > 0 for r in results)
    for r in results:
        assert r["peak"] <= r["footprint"]        # what ran stayed inside its cap
    for (g, kh, pol), r in zip(reqs, results):
        op = vie.Operator(ctx, g)
        op.compress(1e-4, vie.C64)
        I, _, status = op.solve(kh, pol, tol=1e-6)
        op.close()
        assert status == vie.VIE_OK and rel(r["I"], I) <= 1e-10
    ctx.close()


def test_request_that_cannot_fit_is_rejected_after_back_off(monkeypatch):
    # admitted by an underestimate but larger than the whole budget: after the
    # back-off reaches the budget the request is rejected; the server goes on
    monkeypatch.setenv("VIE_TEST_FOOTPRINT_SCALE", "0.001")
    ctx = vie.Context(0)
    srv = vie.Server(ctx, max_inflight=1, hbm_budget=64 << 20, tol=1e-4)
    kh, pol = workloads.normal_incidence()
    t = srv.submit(workloads.square_array(24, 3), kh, pol)
    r = None
    deadline = time.time() + 300
    while r is None and time.time() < deadline:
        r = srv.poll(t, timeout_ms=1000)
    assert r is not None and r["status"] == vie.VIE_ERR_ADMISSION and r["retries"] > 0
    monkeypatch.delenv("VIE_TEST_FOOTPRINT_SCALE")
    t2 = srv.submit(workloads.square_array(2, 2), kh, pol)
    r2 = srv.poll(t2, timeout_ms=120000)
    assert r2 is not None and r2["status"] == vie.VIE_OK
    srv.stop()
    ctx.close()
