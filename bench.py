#!/usr/bin/env python
"""Benchmark: solves/s of the QR-compressed VIE solver on one GB300.

A step is one solve from geometry of a named workload: vie_assemble (grid
hierarchy, float64 self blocks and their inverses), vie_compress (every far
block formed on the device and compressed, complex float32 factors) and
vie_solve (mixed-precision GMRES of every right-hand side to a relative
residual of 1e-6).  `value` = right-hand sides solved per second with the
solution kept on the device; `e2e` goes through the same C-ABI with host
buffers (geometry in, current out).

Workloads (`--workload`, default multirhs):
  multirhs  32 x 32 array of 4^3-voxel cubes, 245,760 unknowns, 64 right-hand
            sides (32 polar angles x 2 polarisations), tolerance 1e-4, far
            apply of the inner GMRES on the tensor cores (BF16x3)
  graded    64 x 64 graded array (three cube sides along a lens phase), 4^3
            voxels, 983,040 unknowns, 16 right-hand sides, tolerance 1e-3; its
            resonant atoms keep GMRES above 1e-6 within the 3,000-iteration
            budget, reported as "converged": false
  scale     16 x 16 array of 6^3-voxel cubes, 193,536 unknowns, 1 right-hand
            side, complex float32 applies
`roofline` is the compressed apply of the inner iteration (the solve's
dominant kernel pair) timed with CUDA events on the final operator; the factor
planes are far larger than L2, so no flush is needed between applies.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload W] [--impl cuda|reference]
Multi-GPU: one process per GPU (torchrun); the solves are independent
replicas (no collective), value = all ranks' solves / max rank time.
"""
import os

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

TOL_SOLVE = 1e-6
DEFAULT_WORKLOAD = "multirhs"
# Measured DRAM bytes (read + write) of one fused apply, keyed by (workload,
# right-hand sides, BF16x3): u1w_kernel<2> 27.24 + 1.17 GB, u2w_kernel<2> 30.32
# + 0.12 GB, type_gemm<float2> 0.25 + 0.10 GB in one ncu pass
# (dram__bytes_read.sum + dram__bytes_write.sum) over the 64-RHS apply of the
# 32 x 32 array, `bench.py --profile`.  Only valid for the kernels and the
# operator it was taken on; remove an entry when either changes.  (The entry
# for the 64-RHS apply of the 32 x 32 array, 59.2e9, was taken on factors
# compressed from float32-table blocks, whose ranks are many times larger.)
APPLY_TRAFFIC = {}

# Per workload: geometry, incident waves, compression tolerance, inner-apply
# precision ("C64" or "BF16X3"), restart length and, for the CPU oracle's
# time model, the operator's counts as this library measured them on a GB300
# (the oracle cannot build the coarse blocks within a bounded sample):
# sum over far blocks of m n r (the unpivoted QR's work), of (m + n) r (the
# apply's), and the slowest right-hand side's GMRES iterations.
WORKLOADS = {
    "multirhs": dict(
        geometry=lambda: workloads.square_array(32, 4),
        incident=lambda: workloads.angle_sweep(32, 60.0),
        tol=1e-4, precision="BF16X3", restart=60,
        desc="32x32 array of eps=12 cubes (side 0.2, pitch 0.4, lambda 1), 4^3 voxels, 245760 unknowns, "
             "64 RHS (32 polar angles 0-60 deg at azimuth 0 x TE/TM)",
        # factors from float64 tables: factor entries and iterations measured; sum m n r from the
        # planned far blocks with the measured mean rank per level (66 / 59.5 / 54.5 / 51.5 at
        # levels 2-5), scaled to the measured factor entries
        model=dict(mnr=3.9e12, factor_entries=2.30e9, iterations=231)),
    "graded": dict(
        geometry=lambda: workloads.graded_array(64, 4, 0),
        incident=lambda: workloads.random_directions(16, 0),
        tol=1e-3, precision="BF16X3", restart=300, max_iters=3000, may_not_converge=True,
        desc="64x64 graded array (cube sides 0.15/0.2/0.25 along a lens phase, F from seed 0), 4^3 voxels, "
             "983040 unknowns, 16 RHS (seed 0, within 20 deg of normal incidence); compression tolerance 1e-3 "
             "(at 1e-4 the factors would need ~970 GB)",
        # counts of the factors from float32 tables (not re-measured from float64 tables)
        model=dict(mnr=2.4e13, factor_entries=7.12e9, iterations=3000)),
    "vogel": dict(
        geometry=lambda: workloads.vogel_gold(2000, nv=3),
        incident=workloads.normal_incidence,
        tol=1e-4, precision="C64", restart=300, max_iters=3000,
        desc="Vogel spiral of 2000 gold meta-atoms (eps = -9.428 - 1.513j, radius lambda/6, equal-volume cubes of "
             "3^3 voxels), 216000 unknowns, 1 RHS at normal incidence; aperiodic, so no two far blocks share factors",
        # counts of the factors from float32 tables (not re-measured from float64 tables)
        model=dict(mnr=9.38e12, factor_entries=3.56e9, iterations=183)),
    "scale": dict(
        geometry=lambda: workloads.square_array(16, 6),
        incident=workloads.normal_incidence,
        tol=1e-4, precision="C64", restart=60,
        desc="16x16 array of eps=12 cubes (side 0.2, pitch 0.4, lambda 1), 6^3 voxels, 193536 unknowns, 1 RHS",
        # counts of the factors from float32 tables (not re-measured from float64 tables)
        model=dict(mnr=2.1e12, factor_entries=3.58e9, iterations=52)),
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return (d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0),
                "measured")
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def reduce_max(v, dist=None, device="cpu"):
    """Max over ranks of a per-rank time (identity without a process group)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, max_ms, nrhs=1):
    """Right-hand sides solved per second by the whole job: every rank solves
    `steps` problems of `nrhs` right-hand sides (replicas)."""
    return world * steps * nrhs / (max_ms * 1e-3)


# ----------------------------------------------------------------------------
# CPU oracle baseline (the oracle as it stands, on the host cores)
# ----------------------------------------------------------------------------
_ORACLE_RATES = r'''
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import workloads
from oracle import problem_from_geometry, assembly as A, compress as OC, krylov as K, tree as OT
spec = json.loads(sys.argv[2])
g = workloads.__dict__[spec["gen"]](*spec["args"])
P = problem_from_geometry(g)
npp = P.mesh(0).n_faces
rng = np.random.default_rng(5)
out = {}
# atom-pair block assembly (the oracle forms every far entry; no pair is reused)
pairs = [(0, 1), (0, P.n_atoms - 1), (P.n_atoms // 2, P.n_atoms // 2 + 3)]
t0 = time.perf_counter()
blks = [A.cross_block(P, a, b) for a, b in pairs]
out["t_pair"] = (time.perf_counter() - t0) / len(pairs)
# unpivoted Householder QR at the tolerance: seconds per unit of m n r
t0 = time.perf_counter()
units = 0.0
for B in blks:
    Q, R, _ = OC.householder_qr_truncated(B, spec["tol"])
    units += B.shape[0] * B.shape[1] * max(1, R.shape[0])
out["t_qr_unit"] = (time.perf_counter() - t0) / units
# compressed apply of those factors: seconds per factor entry (m + n) r
facs = [OC.householder_qr_truncated(B, spec["tol"])[:2] for B in blks]
x = rng.standard_normal(npp) + 1j * rng.standard_normal(npp)
ent = sum((Q.shape[0] + R.shape[1]) * R.shape[0] for Q, R in facs)
reps, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < 0.5 or reps < 3:
    for Q, R in facs:
        Q @ (R @ x)
    reps += 1
out["t_entry"] = (time.perf_counter() - t0) / reps / ent
# self-block assembly (once per distinct type), when asked for
if spec.get("with_self"):
    t0 = time.perf_counter()
    A.self_block(P, 0)
    out["t_self_block"] = time.perf_counter() - t0
# self part of the apply and the block-Jacobi preconditioner, per atom: the
# oracle's routines on a well-conditioned complex matrix of the block's size
Zs = rng.standard_normal((npp, npp)) + 1j * rng.standard_normal((npp, npp)) + 4.0 * npp ** 0.5 * np.eye(npp)
reps, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < 0.3 or reps < 3:
    Zs @ x
    reps += 1
out["t_self_atom"] = (time.perf_counter() - t0) / reps
M = K.BlockJacobi(P, {0: Zs})
sub = min(P.n_atoms, 16)
y = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
t0 = time.perf_counter()
for a in range(sub):
    LU, piv = M.fact[0]
    s = slice(P.offsets[a], P.offsets[a + 1])
    K.lu_solve(LU, piv, y[s])
out["t_prec_atom"] = (time.perf_counter() - t0) / sub
# modified Gram-Schmidt: one vdot + one axpy on vectors of n
v = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
w = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
reps, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < 0.3 or reps < 3:
    h = np.vdot(v, w)
    w = w - h * v
    reps += 1
out["t_mgs_pair"] = (time.perf_counter() - t0) / reps
L, blocks = OT.build_tree(P.centres)
out["n_pairs"] = P.n_atoms * (P.n_atoms - 1)
out["n"] = P.n
out["N"] = P.n_atoms
out["T"] = len(set(P.types.tolist()))
print(json.dumps(out))
'''

_ORACLE_APPLY = r'''
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import workloads
from oracle import problem_from_geometry, compress as OC
spec = json.loads(sys.argv[2])
g = workloads.__dict__[spec["gen"]](*spec["args"])
P = problem_from_geometry(g)
d = np.load(sys.argv[3], allow_pickle=True)
sb = {int(t): d["self_%d" % t] for t in spec["types"]}
blocks = [(d["ta_%d" % i], d["sa_%d" % i], d["Q_%d" % i], d["R_%d" % i]) for i in range(spec["nblocks"])]
far = OC.operator_from_factors(P, sb, blocks)
near = OC.operator_from_factors(P, sb, [])
x = np.random.default_rng(3).standard_normal(P.n) + 1j * np.random.default_rng(4).standard_normal(P.n)
def timed(op):
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 1.0 or reps < 2:
        op.apply(x)
        reps += 1
    return (time.perf_counter() - t0) / reps
tn = timed(near)
tf = timed(far)
print(json.dumps({"t_near": tn, "t_far_sample": max(tf - tn, 0.0)}))
'''


def _geom_spec(name):
    """How the oracle subprocess regenerates the workload's geometry."""
    return {"multirhs": ("square_array", [32, 4]), "graded": ("graded_array", [64, 4, 0]),
            "scale": ("square_array", [16, 6]), "vogel": ("vogel_gold", [2000, 3])}[name]


def _run_oracle(code, args, threads, timeout=600):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, "-c", code, ROOT] + args, capture_output=True, text=True, env=env,
                       timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


_SELF_BLOCK_S = {}


def oracle_model(name, nrhs, counts=None):
    """Seconds of one solve of the workload by the CPU oracle as it stands,
    single-threaded, extrapolated from a bounded sample: per-unit rates of the
    oracle's own steps timed on this host (atom-pair assembly, unpivoted
    Householder QR, compressed apply, block-Jacobi solve, modified
    Gram-Schmidt), times the workload's unit counts (`counts`, else the
    recorded ones).  Returns (seconds, rates, description)."""
    wl = WORKLOADS[name]
    gen, gargs = _geom_spec(name)
    first = name not in _SELF_BLOCK_S
    spec = {"gen": gen, "args": gargs, "tol": wl["tol"], "with_self": first}
    t0 = time.perf_counter()
    r = _run_oracle(_ORACLE_RATES, [json.dumps(spec)], 1)
    wall = time.perf_counter() - t0
    if first:
        _SELF_BLOCK_S[name] = r["t_self_block"]
    r["t_self_block"] = _SELF_BLOCK_S[name]
    c = dict(wl["model"])
    if counts:
        c.update({k: v for k, v in counts.items() if v})
    restart = wl["restart"]
    mean_j = min(restart, c["iterations"]) / 2.0 + 1.0
    t_assemble = r["t_pair"] * r["n_pairs"] + r["t_self_block"] * r["T"]
    t_qr = r["t_qr_unit"] * c["mnr"]
    t_apply = r["t_entry"] * c["factor_entries"] + r["t_self_atom"] * r["N"]
    t_prec = r["t_prec_atom"] * r["N"]
    t_mgs = r["t_mgs_pair"] * mean_j
    t_iter = t_apply + t_prec + t_mgs
    total = t_assemble + t_qr + nrhs * c["iterations"] * t_iter
    desc = (f"oracle (numpy float64, 1 thread) per-unit rates timed on this host in {wall:.1f} s: self-block "
            f"assembly {r['t_self_block']:.1f} s x {r['T']} types (timed once per run); atom-pair "
            f"assembly {r['t_pair']:.3f} s x {r['n_pairs']} pairs; unpivoted Householder QR "
            f"{r['t_qr_unit']:.2e} s per m n r unit x {c['mnr']:.3g}; compressed apply {r['t_entry']:.2e} s per "
            f"factor entry x {c['factor_entries']:.3g} + self blocks; block-Jacobi LU solve "
            f"{r['t_prec_atom']:.2e} s per atom; modified Gram-Schmidt {r['t_mgs_pair']:.2e} s per vector pair x "
            f"{mean_j:.0f}; {c['iterations']} GMRES iterations x {nrhs} right-hand sides (one at a time)")
    return total, r, desc


def oracle_apply_sample(op, name, vie, max_entries=3e7):
    """The oracle's float64 compressed apply of the GPU's exported factors on
    a sample of far blocks (every level), timed single-threaded and on all
    host cores, scaled to one full apply.  Returns a dict."""
    wl = WORKLOADS[name]
    gen, gargs = _geom_spec(name)
    meta = op.far_blocks(with_factors=False)
    npp = op.np
    by_level = {}
    for i, b in enumerate(meta):
        by_level.setdefault(b["level"], []).append(i)
    total_ent = sum((len(b["tatoms"]) + len(b["satoms"])) * npp * b["rank"] for b in meta)
    pick = []
    budget = max_entries / max(1, len(by_level))
    for lev, ids in sorted(by_level.items()):
        step = max(1, len(ids) // 16)
        used = 0.0
        for i in ids[::step]:
            b = meta[i]
            e = (len(b["tatoms"]) + len(b["satoms"])) * npp * b["rank"]
            if used + e > budget and used > 0:
                break
            pick.append(i)
            used += e
    blocks = op.far_blocks(indices=pick)
    types = sorted(set(wl["geometry"]().types.tolist()))
    arrs = {"self_%d" % t: op.export_block(0, t) for t in types}
    samp_ent = 0
    for k, b in enumerate(blocks):
        arrs["ta_%d" % k] = b["tatoms"]
        arrs["sa_%d" % k] = b["satoms"]
        arrs["Q_%d" % k] = b["Q"]
        arrs["R_%d" % k] = b["R"]
        samp_ent += (b["Q"].shape[0] + b["R"].shape[1]) * b["rank"]
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "sample.npz")
        np.savez(f, **arrs)
        spec = json.dumps({"gen": gen, "args": gargs, "types": types, "nblocks": len(blocks)})
        one = _run_oracle(_ORACLE_APPLY, [spec, f], 1)
        allc = _run_oracle(_ORACLE_APPLY, [spec, f], cores())
    scale = total_ent / max(1, samp_ent)
    return {"sample_blocks": len(blocks), "sample_entries": int(samp_ent), "total_entries": int(total_ent),
            "s_per_apply_1core": one["t_near"] + one["t_far_sample"] * scale,
            "s_per_apply_allcore": allc["t_near"] + allc["t_far_sample"] * scale, "cores_all": cores()}


def oracle_tiny_pipeline():
    """The whole oracle pipeline on the 4x4 array of 3^3 cubes (1,728 unknowns),
    single-threaded: dense assembly, textbook LU solve, QR-recursive compression
    at 1e-4 and preconditioned GMRES to 1e-6 (seconds, measured)."""
    code = r'''
import json, sys, time
sys.path.insert(0, sys.argv[1])
import workloads
from oracle import problem_from_geometry, assembly as A, compress as OC, krylov as K, direct as D
g, kh, pol = workloads.config("tiny")
t0 = time.perf_counter()
P = problem_from_geometry(g)
Z = A.dense_matrix(P); b = A.rhs(P, kh[0], pol[0])
LU, piv = D.lu_factor(Z); x = D.lu_solve(LU, piv, b)
op = OC.compress_dense(P, Z, 1e-4)
xg, info = K.gmres(op.apply, b, K.BlockJacobi(P, op.self_blocks).apply, tol=1e-6, restart=60)
print(json.dumps({"s": time.perf_counter() - t0, "iterations": info["iterations"]}))
'''
    return _run_oracle(code, [], 1)


def run_reference(args):
    """--impl reference: the oracle as it stands (CPU, one thread), on rank 0 only.
    Every step times the oracle's per-unit rates on a bounded sample of the
    workload and scales them to one solve of all its right-hand sides."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    nrhs = len(wl["incident"]()[0])
    times, desc = [], ""
    for i in range(args.warmup + args.steps):
        total, _, desc = oracle_model(args.workload, nrhs)
        if i >= args.warmup:
            times.append(total)
    v = nrhs / statistics.mean(times)
    line = {"metric": "solves/s", "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "nrhs": nrhs},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": desc,
                             "extrapolated": True},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# other modes
# ----------------------------------------------------------------------------
def run_serving(args):
    """--serving: the Poisson request stream (20 req/s; arrays of 8x8..48x48 cubes of
    3^3 voxels; lambda ~ U[0.9, 1.1], eps ~ U[8, 14]; 1-8 RHS) through vie_serve with
    continuous batching; reports solves/s (right-hand sides per second) and the
    p50/p99 latency from submit to result."""
    import threading
    import torch
    from paper_2603_10586_gb300 import vie
    torch.cuda.set_device(0)
    ctx = vie.Context(0)
    warm = workloads.serving_stream(args.warmup, seed=99)
    reqs = workloads.serving_stream(args.requests, seed=0)
    srv = vie.Server(ctx, max_inflight=args.slots, tol=1e-4)
    for r in warm:                                   # warm-up, not timed
        srv.poll(srv.submit(r.geometry, r.khat, r.pol), timeout_ms=600000)
    tickets = [None] * len(reqs)
    t_start = time.perf_counter()

    def feeder():
        for i, r in enumerate(reqs):
            delay = r.arrival_s - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            tickets[i] = srv.submit(r.geometry, r.khat, r.pol)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    res = []
    for t in tickets:
        out = None
        while out is None:
            out = srv.poll(t, timeout_ms=1000)
        res.append(out)
    srv.stop()
    lat = sorted(r["t_done"] - r["t_submit"] for r in res)
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    busy = max(r["t_done"] for r in res) - min(r["t_start"] for r in res)
    rhs = sum(r["nrhs"] for r in res)
    ok = sum(1 for r in res if r["status"] == 0)
    line = {"metric": "serving solves/s", "value": rhs / span, "unit": "solves/s", "n_gpus": 1,
            "requests": len(res), "completed_ok": ok, "requests_per_s": len(res) / span,
            "sustainable_requests_per_s": len(res) / busy, "offered_requests_per_s": 20.0,
            "retries": sum(r["retries"] for r in res),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "service_s": {"p50": float(np.percentile([r["t_done"] - r["t_start"] for r in res], 50)),
                          "p99": float(np.percentile([r["t_done"] - r["t_start"] for r in res], 99))},
            "footprints": [{"ns": q.ns, "nrhs": r["nrhs"], "model": r["footprint"], "peak": r["peak"]}
                           for q, r in zip(reqs, res)],
            "higher_is_better": True, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "serving", "slots": args.slots, "rate_hz": 20.0,
                       "arrays": "8x8..48x48 cubes of 3^3 voxels", "tol_compress": 1e-4,
                       "tol_solve": TOL_SOLVE}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_batch(args):
    """--batch: the serving mix (arrays of 8x8..SxS cubes of 3^3 voxels, S =
    --batch-max-side (48), lambda ~ U[0.9, 1.1], eps ~ U[8, 14], 1-8 RHS;
    --batch-requests problems (8), seed 7) solved one vie_solve after another and as one
    vie_solve_batch (block-diagonal union, one persistent apply launch per phase
    over all problems), operators built beforehand.  Reports right-hand sides
    per second both ways, each the median of three runs, and the largest
    difference between the two solutions."""
    import torch
    from paper_2603_10586_gb300 import vie
    torch.cuda.set_device(0)
    ctx = vie.Context(0)
    reqs = workloads.serving_stream(args.batch_requests, seed=7, ns_range=(8, args.batch_max_side))
    ops = []
    for r in reqs:
        op = vie.Operator(ctx, r.geometry)
        op.compress(1e-4, vie.C64)
        ops.append(op)
    nrhs = sum(len(r.khat) for r in reqs)
    out = {"metric": "batched solves/s", "unit": "solves/s", "problems": len(reqs), "nrhs": nrhs,
           "sides": [8, args.batch_max_side],
           "sizes": [r.ns for r in reqs], "n": [op.n for op in ops], "precision": {}}
    for prec, name in ((vie.C64, "c64"), (vie.BF16X3, "bf16x3")):
        seq_t, bat_t = [], []
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            seq = [op.solve(r.khat, r.pol, tol=TOL_SOLVE, precision=prec)[0] for op, r in zip(ops, reqs)]
            torch.cuda.synchronize()
            seq_t.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            bat, st, status = vie.solve_batch(ops, [(r.khat, r.pol) for r in reqs], tol=TOL_SOLVE, precision=prec)
            torch.cuda.synchronize()
            bat_t.append(time.perf_counter() - t0)
            assert status == vie.VIE_OK
        diff = max(float(np.linalg.norm(a - b) / np.linalg.norm(a)) for a, b in zip(seq, bat))
        ts, tb = float(np.median(seq_t)), float(np.median(bat_t))
        out["precision"][name] = {"sequential_s": ts, "batched_s": tb, "sequential": nrhs / ts,
                                  "batched": nrhs / tb, "speedup": ts / tb, "max_rel_diff": diff}
    print(json.dumps(out), flush=True)
    for op in ops:
        op.close()
    ctx.close()
    return 0


def run_methods(args):
    """--methods: the Krylov methods on one operator of the workload, all
    right-hand sides, inner applies as the workload's: lockstep GMRES (each
    right-hand side in its own Krylov space), block GMRES (one space for all)
    and BiCGStab.  Reports time, iterations, applies, residual and the largest
    relative difference from the lockstep solution; the operator is built
    once, outside the timed solves."""
    import torch
    from paper_2603_10586_gb300 import vie
    torch.cuda.set_device(0)
    ctx = vie.Context(0)
    wl = WORKLOADS[args.workload]
    kh, pol = wl["incident"]()
    prec = getattr(vie, wl["precision"])
    op = vie.Operator(ctx, wl["geometry"]())
    op.compress(wl["tol"], vie.C64)
    maxit = args.max_iters or wl.get("max_iters", 20000)
    out = {"metric": "Krylov methods", "workload": args.workload, "nrhs": len(kh), "max_applies": maxit,
           "methods": {}}
    ref = None
    for name, method, restart in (("gmres_lockstep", vie.GMRES, wl["restart"]), ("block_gmres", vie.BLOCK_GMRES, 60),
                                  ("bicgstab", vie.BICGSTAB, 0)):
        # the same budget of operator applications: BiCGStab applies twice per iteration
        mi = maxit if method != vie.BICGSTAB else max(1, maxit // 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        I, st, status = op.solve(kh, pol, tol=TOL_SOLVE, precision=prec, restart=restart, max_iters=mi, method=method)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if ref is None:
            ref = I
        diff = max(float(np.linalg.norm(I[:, c] - ref[:, c]) / np.linalg.norm(ref[:, c])) for c in range(len(kh)))
        out["methods"][name] = {"s": t, "status": status, "iterations": st["iterations"], "applies": st["applies"],
                                "refinements": st["refinements"], "residual": st["residual"],
                                "true_residual": st["true_residual"], "max_rel_diff_vs_lockstep": diff,
                                "solves_per_s": len(kh) / t}
    print(json.dumps(out), flush=True)
    op.close()
    ctx.close()
    return 0


def run_builders(args):
    """--builders: the two far-block builders on one operator of the workload,
    each compressing from geometry: the adaptive randomised range finder
    (vie_compress) and the cross approximation with full pivoting of Sec. 6.5
    (vie_compress_cross).  One untimed range-finder compression first (library
    and cuBLAS set-up), then each builder --builder-reps times (median).  Reports
    compression time, ranks, factor entries and, for the cross approximation,
    the bandwidth of its residual passes (bytes read and written / device time
    of its step loops) against the measured HBM peak; then one solve per builder
    (the workload's right-hand sides and inner precision) with its residuals and
    the largest relative difference between the two solutions."""
    import torch
    from paper_2603_10586_gb300 import vie
    torch.cuda.set_device(0)
    ctx = vie.Context(0)
    wl = WORKLOADS[args.workload]
    kh, pol = wl["incident"]()
    prec = getattr(vie, wl["precision"])
    if args.builders_side:
        g = workloads.square_array(args.builders_side, 4)
        geom = "%dx%d array of eps=12 cubes (side 0.2, pitch 0.4, lambda 1), 4^3 voxels, %d unknowns" % (
            args.builders_side, args.builders_side, g.unknowns())
    else:
        g = wl["geometry"]()
        geom = wl["desc"]
    hbm, _, _, peak_kind = peaks()
    warm = vie.Operator(ctx, g)
    warm.compress(wl["tol"], vie.C64)
    warm.close()
    out = {"metric": "compression builders", "workload": args.workload, "geometry": geom, "tol_compress": wl["tol"],
           "reps": args.builder_reps, "builders": {}}
    sols = {}
    for name, method in (("range_finder", vie.COMPRESS_RANGE_FINDER), ("cross_full_pivoting", vie.COMPRESS_CROSS)):
        ts = []
        for rep in range(args.builder_reps):
            op = vie.Operator(ctx, g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = op.compress(wl["tol"], vie.C64, method=method)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            if rep + 1 < args.builder_reps:
                op.close()
        I, st, status = op.solve(kh, pol, tol=TOL_SOLVE, precision=prec, restart=wl["restart"],
                                 max_iters=wl.get("max_iters", 20000))
        sols[name] = I
        rec = {"compress_s": float(np.median(ts)), "compress_s_all": ts, "rank_mean": info["rank_mean"],
               "rank_max": info["rank_max"], "factor_entries": info["factor_entries"],
               "stored_entries": info["stored_entries"], "solve_status": status,
               "iterations": st["iterations"], "residual": st["residual"], "true_residual": st["true_residual"]}
        if method == vie.COMPRESS_CROSS:
            gbs = info["cross_bytes"] / max(info["t_cross_s"], 1e-12) / 1e9
            rec["residual_passes"] = {"bytes": info["cross_bytes"], "device_s": info["t_cross_s"], "GB/s": gbs,
                                      "peak_GB/s": hbm, "frac": gbs / hbm, "peak_kind": peak_kind,
                                      "note": "each step reads and writes every active block's residual once "
                                              "(m n complex float32 entries); the device time includes the "
                                              "select kernels and the host's reads of the active count"}
        out["builders"][name] = rec
        op.close()
    a, b = sols["range_finder"], sols["cross_full_pivoting"]
    out["max_rel_diff_between_solutions"] = max(
        float(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(a[:, c])) for c in range(a.shape[1]))
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def run_profile(args):
    """--profile: one untimed solve from geometry of the workload followed by 10
    inner-iteration applies, for ncu captures (no warm-up, no timing, no
    baseline).  --profile-case small uses a smaller array of the same kind
    (factors still above L2) and skips the solve."""
    import torch
    from paper_2603_10586_gb300 import vie
    torch.cuda.set_device(0)
    ctx = vie.Context(0)
    wl = WORKLOADS[args.workload]
    kh, pol = wl["incident"]()
    if args.profile_case == "small":
        g = {"multirhs": lambda: workloads.square_array(16, 4), "graded": lambda: workloads.graded_array(24, 4, 0),
             "scale": lambda: workloads.square_array(8, 6),
             "vogel": lambda: workloads.vogel_gold(500, nv=3)}[args.workload]()
    else:
        g = wl["geometry"]()
    prec = getattr(vie, wl["precision"])
    op = vie.Operator(ctx, g)
    info = op.compress(wl["tol"], vie.C64)
    k = len(kh)
    if args.profile_case != "small":
        out = torch.empty((k, op.n), dtype=torch.complex128, device="cuda")
        # host-launched Arnoldi steps (launch = 1: the same kernels as the graph) so that a
        # profiler's launch list sees every kernel of the solve
        op.solve(kh, pol, tol=TOL_SOLVE, precision=prec, restart=wl["restart"], out_ptr=out.data_ptr(), launch=1,
                 max_iters=wl.get("max_iters", 20000))
    x = torch.randn((k, op.n), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(10 if args.profile_case != "small" else 3):
        op.apply(x.data_ptr(), y.data_ptr(), k, prec, vie.FUSE_PRECOND)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "workload": args.workload, "n": op.n, "nrhs": k,
                      "factor_entries": info["factor_entries"]}), flush=True)
    op.close()
    ctx.close()
    return 0


# ----------------------------------------------------------------------------
# the timed solve
# ----------------------------------------------------------------------------
def time_apply(op, vie, torch, k, prec, reps):
    x = torch.randn((k, op.n), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        op.apply(x.data_ptr(), y.data_ptr(), k, prec, vie.FUSE_PRECOND)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record()
    for _ in range(reps):
        op.apply(x.data_ptr(), y.data_ptr(), k, prec, vie.FUSE_PRECOND)
    a1.record()
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-float64 single-RHS comparison")
    ap.add_argument("--applies", type=int, default=10)
    ap.add_argument("--serving", action="store_true", help="the request-stream workload instead")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--batch", action="store_true", help="sequential against batched solves of the serving mix")
    ap.add_argument("--batch-max-side", type=int, default=48, help="largest array side of the --batch mix")
    ap.add_argument("--batch-requests", type=int, default=8, help="problems of the --batch mix")
    ap.add_argument("--methods", action="store_true", help="lockstep GMRES, block GMRES and BiCGStab compared")
    ap.add_argument("--max-iters", type=int, default=0, help="iteration budget of --methods (0: the workload's)")
    ap.add_argument("--builders", action="store_true",
                    help="range finder against cross approximation (full pivoting) as the far-block builder")
    ap.add_argument("--builder-reps", type=int, default=1, help="compressions per builder of --builders")
    ap.add_argument("--builders-side", type=int, default=0,
                    help="--builders on an NxN array of 4^3-voxel cubes instead of the workload's geometry")
    ap.add_argument("--profile", action="store_true", help="one untimed step for ncu captures")
    ap.add_argument("--profile-case", default="full", choices=["full", "small"])
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.batch:
        return run_batch(args)
    if args.methods:
        return run_methods(args)
    if args.builders:
        return run_builders(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2603_10586_gb300 import vie

    wl = WORKLOADS[args.workload]
    g = wl["geometry"]()
    kh, pol = wl["incident"]()
    nrhs = len(kh)
    prec = getattr(vie, wl["precision"])
    ctx = vie.Context(local)
    n = g.unknowns()
    out = torch.empty((nrhs, n), dtype=torch.complex128, device="cuda")
    h2d = (g.centres.nbytes + g.types.nbytes + g.sides.nbytes + g.nvs.nbytes + 16 * len(g.eps)
           + kh.nbytes + 2 * pol.real.nbytes)
    state = {}

    def step(host):
        op = vie.Operator(ctx, g)
        op.compress(wl["tol"], vie.C64)
        I, stats, status = op.solve(kh, pol, tol=TOL_SOLVE, restart=wl["restart"], precision=prec,
                                    max_iters=wl.get("max_iters", 20000), out_ptr=None if host else out.data_ptr())
        state["converged"] = status == vie.VIE_OK
        if status != vie.VIE_OK and not wl.get("may_not_converge"):
            raise RuntimeError(f"solve did not converge: {stats['residual']}")
        state["stats"], state["info"] = stats, op.info()
        if "keep" in state:
            state["keep"].close()
        state["keep"] = op
        return I

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    clocks = Clocks(local)
    barrier()
    l0 = vie.kernel_launches()
    clocks.start()
    lat = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(False)
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    ev1.record()
    barrier()
    clk = clocks.stop()
    launches = vie.kernel_launches() - l0
    total_ms = ev0.elapsed_time(ev1)
    stats, info = state["stats"], state["info"]

    # end to end through the C-ABI with host buffers (geometry in, current out)
    e2e_steps = max(1, min(args.steps, 2))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(e2e_steps):
        I_host = step(True)
    e1.record()
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    # roofline of the inner-iteration apply (fused P^-1 Zs x) on the last operator
    op = state["keep"]
    apply_ms = time_apply(op, vie, torch, nrhs, prec, args.applies)
    info = op.info()
    hbm, tf_burst, tf_sust, peak_kind = peaks()
    alg_bytes = 8.0 * (info["factor_entries"] + info["n_types"] * info["np"] ** 2) + 16.0 * info["n"] * nrhs
    achieved = alg_bytes / (apply_ms * 1e-3) / 1e9
    # the library's default far-apply kernel for this many right-hand sides
    far = ("u1w/u2w<1> (tcgen05 BF16x3, warp-specialised, bulk-TMA A planes)" if nrhs <= 16 else
           "u1w/u2w<2> (tcgen05 BF16x3, warp-specialised, two row tiles per B tile, bulk-TMA A planes)")
    # DRAM bytes of one fused apply (far kernels + type_gemm) from a one-pass ncu capture of
    # `bench.py --profile` on the same workload and kernels
    traffic = APPLY_TRAFFIC.get((args.workload, nrhs, prec == vie.BF16X3))
    roof = {"kernel": (f"far apply {far} + type_gemm, fused P^-1 Zs x, {nrhs} RHS") if prec == vie.BF16X3
            else "far apply + type_gemm, fused P^-1 Zs x (c64, 1 RHS)",
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_kind": peak_kind, "algorithmic_bytes": alg_bytes, "apply_ms": apply_ms,
            "traffic": traffic,
            "note": "algorithmic bytes: every far block's factors once (8 (m+n) r), the distinct self/inverse "
                    "blocks once, x read and y written once per right-hand side"}
    if prec == vie.BF16X3:
        moved = info["packed_bytes"] + 16.0 * info["n"] * nrhs
        roof["moved_bytes"] = moved
        roof["moved_frac"] = moved / (apply_ms * 1e-3) / 1e9 / hbm
        flops = 24.0 * nrhs * info["factor_entries"]
        roof["tensor_tflops"] = flops / (apply_ms * 1e-3) / 1e12
        roof["tensor_frac_of_sustained"] = roof["tensor_tflops"] / tf_sust
        roof["note"] += ("; moved_bytes: the bf16 planes the packed kernels stream (tiles padded to 128 rows, "
                         "K to 32); tensor work 24 s (m+n) r bf16 flops")
    else:
        roof["stored_factor_bytes"] = 8 * info["stored_entries"]
        roof["stored_frac"] = 8 * info["stored_entries"] / (apply_ms * 1e-3) / 1e9 / hbm
        if info["stored_entries"] < info["factor_entries"]:
            # translated copies share factors and the single-RHS kernels read a shared
            # factor once per group of up to four copies: the per-block bytes are not
            # what the kernel moves, so the headline fraction is taken on the stored
            # factor bytes (a lower bound of what it moves) and the per-block one kept aside
            stored = 8.0 * (info["stored_entries"] + info["n_types"] * info["np"] ** 2) + 16.0 * info["n"] * nrhs
            roof["per_block_achieved"], roof["per_block_frac"] = achieved, achieved / hbm
            roof["achieved"] = stored / (apply_ms * 1e-3) / 1e9
            roof["frac"] = roof["achieved"] / hbm
            roof["algorithmic_bytes"] = stored
            roof["note"] = ("bytes of the stored factors once (translated copies share storage), the distinct "
                            "self/inverse blocks once, x read and y written once; per_block_*: every block's "
                            "factors once, which the shared-factor kernels do not read")

    # accuracy of the result: the all-float64 single-RHS GPU solve (c128 factors)
    accuracy = {"residual_preconditioned": stats["residual"], "true_residual": stats["true_residual"],
                "tol_solve": TOL_SOLVE}
    fp64 = None
    if rank == 0 and not args.no_fp64 and args.workload != "graded":
        opd = vie.Operator(ctx, g)
        t0 = time.perf_counter()
        opd.compress(wl["tol"], vie.C128)
        tcomp = time.perf_counter() - t0
        c = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Id, std, sd = opd.solve(kh[c:c + 1], pol[c:c + 1], tol=TOL_SOLVE, precision=vie.C128, restart=wl["restart"],
                                max_iters=20000)
        torch.cuda.synchronize()
        tsol = time.perf_counter() - t0
        opd.close()
        diff = float(np.linalg.norm(I_host[:, c] - Id[:, 0]) / np.linalg.norm(Id[:, 0]))
        per_step = total_ms / args.steps * 1e-3
        fp64 = {"rhs_sampled": [c], "compress_c128_s": tcomp, "solve_s_per_rhs": tsol,
                "solves_per_s": 1.0 / (tcomp / nrhs + tsol),
                "speedup_of_this_solve": (tcomp + nrhs * tsol) / per_step,
                "rel_diff_vs_fp64": diff, "status": sd}
        accuracy["rel_diff_vs_fp64_solve"] = diff

    total_ms = reduce_max(total_ms, dist, "cuda")
    e2e_ms = reduce_max(e2e_ms, dist, "cuda")
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            meta = op.far_blocks(with_factors=False)
            mnr = float(sum(len(b["tatoms"]) * len(b["satoms"]) * b["rank"] for b in meta)) * info["np"] ** 2
            counts = {"factor_entries": info["factor_entries"], "iterations": stats["iterations"], "mnr": mnr}
            t_model, _, desc = oracle_model(args.workload, nrhs, counts)
            cpu = {"value": nrhs / t_model, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": desc,
                   "extrapolated": True, "counts": counts}
            try:
                cpu["apply_sample"] = oracle_apply_sample(op, args.workload, vie)
            except Exception as e:  # the baseline is reported, never required
                cpu["apply_sample"] = {"error": str(e)[:300]}
            try:
                cpu["tiny_pipeline_s"] = oracle_tiny_pipeline()
            except Exception as e:
                cpu["tiny_pipeline_s"] = {"error": str(e)[:300]}
        lat_sorted = sorted(lat)
        line = {
            "metric": "solves/s", "value": whole_job_value(world, args.steps, total_ms, nrhs), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "nrhs": nrhs,
                       "solves": "right-hand sides solved to the residual, per second",
                       "tol_compress": wl["tol"], "tol_solve": TOL_SOLVE, "restart": wl["restart"],
                       "inner_precision": wl["precision"], "parallelism": f"replicas{world}",
                       "l2_flush": "none: factors (GBs) exceed L2"},
            "latency_ms": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
            "breakdown_s": {"assemble": info["t_assemble_s"], "compress": info["t_compress_s"],
                            "solve": stats["t_solve_s"]},
            "solver": {"converged": state["converged"], "iterations": stats["iterations"], "applies": stats["applies"],
                       "refinements": stats["refinements"], "residual": stats["residual"],
                       "true_residual": stats["true_residual"]},
            "accuracy": accuracy,
            "fp64_single_rhs": fp64,
            "operator": {"n": info["n"], "levels": info["levels"], "far_blocks": info["n_far_blocks"],
                         "factor_entries": info["factor_entries"], "stored_entries": info["stored_entries"],
                         "gain": info["gain"], "rank_min": info["rank_min"], "rank_max": info["rank_max"],
                         "rank_mean": info["rank_mean"]},
            "roofline": roof,
            "e2e": {"value": whole_job_value(world, e2e_steps, e2e_ms, nrhs), "unit": "solves/s",
                    "steps": e2e_steps, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(16 * n * nrhs)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if "keep" in state:
        state["keep"].close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
