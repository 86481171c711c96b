"""Thin ctypes binding of libvie (include/vie.h): argument marshalling only.

Every computation happens in the CUDA library.  Device vectors are passed as
raw pointers (e.g. ``torch.Tensor.data_ptr()`` of a contiguous complex64 /
complex128 CUDA tensor); host arrays are numpy arrays.  The binding raises
``VieError`` on any non-zero status and refuses to run without the library.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libvie.so")

VIE_OK = 0
VIE_ERR_INVALID_ARG = -1
VIE_ERR_OOM = -2
VIE_ERR_CUDA = -3
VIE_ERR_NOT_CONVERGED = -4
VIE_ERR_BREAKDOWN = -5
VIE_ERR_NAN = -6
VIE_ERR_TIMEOUT = -7
VIE_ERR_ADMISSION = -8
VIE_ERR_STATE = -9
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "BREAKDOWN",
          -6: "NAN", -7: "TIMEOUT", -8: "ADMISSION", -9: "STATE"}
C64, C128, BF16X3, C64_ACC64 = 1, 2, 3, 4
VAR_SIMT_R1, VAR_SIMT_R2, VAR_SIMT_R4, VAR_SIMT_R8, VAR_MMA_BF16X3, VAR_TCGEN05_BF16X3 = 1, 2, 3, 4, 5, 6
VAR_TCGEN05_PACKED_BF16X3 = 7
VAR_SIMT_SHARED = 8
VAR_TCGEN05_WS_BF16X3 = 9
VAR_TCGEN05_WS2_BF16X3 = 10
COMPRESS_RANGE_FINDER, COMPRESS_CROSS = 0, 1
NOALLOC_SCRATCH_ELEMS = 1 << 22   # VIE_NOALLOC_SCRATCH_ELEMS
FUSE_PRECOND = 1
DENSE = 2
ADJOINT = 4
GMRES, BICGSTAB, BLOCK_GMRES = 0, 1, 2


class VieError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libvie {STATUS.get(status, status)}: {msg}")
        self.status = status


class CtxOpts(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget", C.c_size_t), ("verbose", C.c_int), ("no_sharing", C.c_int)]


class GeometryC(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("centres", C.POINTER(C.c_double)), ("types", C.POINTER(C.c_int)),
                ("n_types", C.c_int), ("sides", C.POINTER(C.c_double)), ("nv", C.POINTER(C.c_int)),
                ("eps", C.POINTER(C.c_double))]


class OpInfo(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("np", C.c_int), ("n_types", C.c_int), ("levels", C.c_int),
                ("n", C.c_int64), ("n_far_blocks", C.c_int64), ("far_entries", C.c_int64),
                ("factor_entries", C.c_int64), ("self_entries", C.c_int64), ("gain", C.c_double),
                ("rank_min", C.c_int), ("rank_max", C.c_int), ("rank_mean", C.c_double),
                ("factor_precision", C.c_int), ("tol", C.c_double), ("apply_bytes", C.c_int64),
                ("t_assemble_s", C.c_double), ("t_compress_s", C.c_double), ("stored_entries", C.c_int64),
                ("packed_bytes", C.c_int64), ("compress_method", C.c_int), ("cross_bytes", C.c_double),
                ("t_cross_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IncidentC(C.Structure):
    _fields_ = [("khat", C.POINTER(C.c_double)), ("pol", C.POINTER(C.c_double))]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_iters", C.c_int), ("precision", C.c_int),
                ("out_on_device", C.c_int), ("precond", C.c_int), ("launch", C.c_int), ("autotune", C.c_int),
                ("method", C.c_int)]


class TuneResult(C.Structure):
    _fields_ = [("variant", C.c_int), ("n_candidates", C.c_int), ("candidates", C.c_int * 16),
                ("ms", C.c_double * 16)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("applies", C.c_int), ("refinements", C.c_int),
                ("residual", C.c_double), ("true_residual", C.c_double), ("t_solve_s", C.c_double),
                ("history", C.c_double * 512), ("n_history", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "history"}
        d["history"] = list(self.history[: self.n_history])
        return d


class ServeOpts(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("hbm_budget", C.c_size_t), ("tol", C.c_double),
                ("solve", SolveOpts)]


class RequestC(C.Structure):
    _fields_ = [("geometry", GeometryC), ("wavelength", C.c_double), ("nrhs", C.c_int), ("inc", IncidentC)]


class ResultC(C.Structure):
    _fields_ = [("status", C.c_int), ("n", C.c_int64), ("nrhs", C.c_int), ("I", C.POINTER(C.c_double)),
                ("stats", SolveStats), ("t_submit_s", C.c_double), ("t_start_s", C.c_double),
                ("t_done_s", C.c_double), ("footprint_bytes", C.c_int64), ("retries", C.c_int),
                ("peak_bytes", C.c_int64)]


EXPORTS = ["vie_create", "vie_destroy", "vie_last_error", "vie_assemble", "vie_compress", "vie_compress_cross",
           "vie_op_destroy",
           "vie_op_get_info", "vie_apply", "vie_precond", "vie_rhs", "vie_solve", "vie_fields",
           "vie_export_block", "vie_far_block_info", "vie_export_far_block", "vie_serve", "vie_submit",
           "vie_poll", "vie_result_free", "vie_server_stop", "vie_footprint_bytes", "vie_kernel_launches",
           "vie_apply_noalloc", "vie_plan_far_blocks", "vie_lpt_assign", "vie_tune", "vie_solve_batch"]

_lib = None


def load():
    """Load libvie (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvie is not built ({LIB_PATH} missing); run "
                          "python -m paper_2603_10586_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
    sig = {
        "vie_create": (C.c_int, [C.POINTER(vp), C.POINTER(CtxOpts)]),
        "vie_destroy": (None, [vp]),
        "vie_last_error": (C.c_char_p, [vp]),
        "vie_assemble": (C.c_int, [vp, C.POINTER(GeometryC), dbl, C.POINTER(vp)]),
        "vie_compress": (C.c_int, [vp, dbl, C.c_int]),
        "vie_compress_cross": (C.c_int, [vp, dbl, C.c_int]),
        "vie_op_destroy": (None, [vp]),
        "vie_op_get_info": (C.c_int, [vp, C.POINTER(OpInfo)]),
        "vie_apply": (C.c_int, [vp, vp, vp, C.c_int, i64, C.c_int, C.c_int, vp]),
        "vie_precond": (C.c_int, [vp, vp, vp, C.c_int, i64, C.c_int, vp]),
        "vie_rhs": (C.c_int, [vp, C.POINTER(IncidentC), C.c_int, vp, i64, vp]),
        "vie_solve": (C.c_int, [vp, C.POINTER(IncidentC), C.c_int, C.POINTER(SolveOpts), vp,
                                C.POINTER(SolveStats)]),
        "vie_fields": (C.c_int, [vp, C.POINTER(IncidentC), vp, C.c_int, C.POINTER(dbl), C.c_int, C.c_int, vp,
                                 C.POINTER(dbl)]),
        "vie_export_block": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]),
        "vie_far_block_info": (C.c_int, [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int)]),
        "vie_export_far_block": (C.c_int, [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp]),
        "vie_serve": (C.c_int, [C.POINTER(vp), vp, C.POINTER(ServeOpts)]),
        "vie_submit": (C.c_int, [vp, C.POINTER(RequestC), C.POINTER(C.c_uint64)]),
        "vie_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(ResultC), C.c_int]),
        "vie_result_free": (None, [C.POINTER(ResultC)]),
        "vie_server_stop": (C.c_int, [vp]),
        "vie_footprint_bytes": (i64, [i64, C.c_int, C.c_int, C.c_int, i64]),
        "vie_kernel_launches": (i64, []),
        "vie_tune": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.POINTER(TuneResult)]),
        "vie_solve_batch": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(IncidentC), C.POINTER(C.c_int),
                                      C.POINTER(SolveOpts), C.POINTER(vp), C.POINTER(SolveStats)]),
        "vie_apply_noalloc": (C.c_int, [vp, vp, vp, C.c_int, i64, vp]),
        "vie_plan_far_blocks": (C.c_int, [C.POINTER(dbl), C.c_int, C.POINTER(C.c_int), C.POINTER(i64),
                                          C.POINTER(C.c_int), i64, C.POINTER(i64)]),
        "vie_lpt_assign": (C.c_int, [C.POINTER(dbl), i64, C.c_int, C.POINTER(C.c_int), C.POINTER(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _stream(stream):
    """Explicit stream handle, else torch's current stream when torch has CUDA
    initialised (its legacy default stream is passed as cudaStreamLegacy = 1),
    else NULL = the library context's own stream."""
    if stream is not None:
        return C.c_void_p(int(stream))
    import sys
    th = sys.modules.get("torch")
    if th is not None and th.cuda.is_available() and th.cuda.is_initialized():
        h = th.cuda.current_stream().cuda_stream
        return C.c_void_p(h if h != 0 else 1)
    return C.c_void_p(0)


def kernel_launches():
    return int(load().vie_kernel_launches())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Context:
    def __init__(self, device=0, hbm_budget=0, verbose=0, no_sharing=0):
        self.L = load()
        self.h = C.c_void_p()
        opts = CtxOpts(device, hbm_budget, verbose, no_sharing)
        st = self.L.vie_create(C.byref(self.h), C.byref(opts))
        if st != VIE_OK:
            raise VieError(st, "vie_create failed")

    def error(self):
        return self.L.vie_last_error(self.h).decode()

    def check(self, st, ok=(VIE_OK,)):
        if st not in ok:
            raise VieError(st, self.error())
        return st

    def close(self):
        if self.h:
            self.L.vie_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _geometry_struct(g):
    arrs = dict(centres=np.ascontiguousarray(g.centres, np.float64).ravel(),
                types=np.ascontiguousarray(g.types, np.int32),
                sides=np.ascontiguousarray(g.sides, np.float64),
                nv=np.ascontiguousarray(g.nvs, np.int32),
                eps=np.ascontiguousarray(np.stack([np.real(g.eps), np.imag(g.eps)], 1), np.float64).ravel())
    s = GeometryC(len(arrs["types"]), _dp(arrs["centres"]), _ip(arrs["types"]), len(arrs["sides"]),
                  _dp(arrs["sides"]), _ip(arrs["nv"]), _dp(arrs["eps"]))
    return s, arrs


def _incident_struct(khat, pol):
    kh = np.ascontiguousarray(np.asarray(khat, np.float64).reshape(-1, 3)).ravel()
    p = np.asarray(pol, np.complex128).reshape(-1, 3)
    pl = np.ascontiguousarray(np.stack([p.real, p.imag], -1), np.float64).ravel()
    return IncidentC(_dp(kh), _dp(pl)), (kh, pl), p.shape[0]


class Operator:
    """A metasurface operator: vie_assemble / vie_compress / vie_apply / ..."""

    def __init__(self, ctx, geometry, wavelength=None):
        self.ctx = ctx
        self.L = ctx.L
        self.h = C.c_void_p()
        gs, keep = _geometry_struct(geometry)
        wl = geometry.wavelength if wavelength is None else wavelength
        ctx.check(self.L.vie_assemble(ctx.h, C.byref(gs), float(wl), C.byref(self.h)))
        self.info()

    def compress(self, tol=1e-4, precision=C64, method=COMPRESS_RANGE_FINDER):
        """vie_compress (method COMPRESS_RANGE_FINDER) or vie_compress_cross (COMPRESS_CROSS)."""
        fn = self.L.vie_compress_cross if method == COMPRESS_CROSS else self.L.vie_compress
        self.ctx.check(fn(self.h, float(tol), int(precision)))
        return self.info()

    def info(self):
        inf = OpInfo()
        self.ctx.check(self.L.vie_op_get_info(self.h, C.byref(inf)))
        self.n = int(inf.n)
        self.np = int(inf.np)
        return inf.as_dict()

    def apply(self, x_ptr, y_ptr, nrhs=1, precision=C64, flags=0, stream=None):
        self.ctx.check(self.L.vie_apply(self.h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(nrhs), self.n,
                                        int(precision), int(flags), _stream(stream)))

    def tune(self, precision=C64, nrhs=1, force=0):
        """vie_tune: time the far-apply variants (or set `force`); returns the choice and timings."""
        r = TuneResult()
        self.ctx.check(self.L.vie_tune(self.h, int(precision), int(nrhs), int(force), C.byref(r)))
        return {"variant": r.variant,
                "ms": {int(r.candidates[i]): float(r.ms[i]) for i in range(r.n_candidates)}}

    def apply_noalloc(self, x_ptr, y_ptr, nrhs=1, stream=None):
        """vie_apply_noalloc: y = Zs x (c64) with the library's static scratch."""
        self.ctx.check(self.L.vie_apply_noalloc(self.h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(nrhs), self.n,
                                                _stream(stream)))

    def precond(self, x_ptr, y_ptr, nrhs=1, precision=C64, stream=None):
        self.ctx.check(self.L.vie_precond(self.h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(nrhs), self.n,
                                          int(precision), _stream(stream)))

    def rhs(self, khat, pol, b_ptr, stream=None):
        inc, keep, nrhs = _incident_struct(khat, pol)
        self.ctx.check(self.L.vie_rhs(self.h, C.byref(inc), nrhs, C.c_void_p(b_ptr), self.n,
                                      _stream(stream)))

    def solve(self, khat, pol, tol=1e-6, restart=60, max_iters=2000, precision=C64, precond=1, out_ptr=None,
              launch=0, autotune=0, method=GMRES):
        """Returns (I (numpy complex128 n x nrhs, or None with out_ptr), stats dict, status)."""
        inc, keep, nrhs = _incident_struct(khat, pol)
        o = SolveOpts(tol, restart, max_iters, precision, 1 if out_ptr else 0, precond, launch, autotune, method)
        st = SolveStats()
        out = None
        if out_ptr is None:
            out = np.zeros((nrhs, self.n), np.complex128)
            ptr = out.ctypes.data_as(C.c_void_p)
        else:
            ptr = C.c_void_p(out_ptr)
        status = self.ctx.check(self.L.vie_solve(self.h, C.byref(inc), nrhs, C.byref(o), ptr, C.byref(st)),
                                ok=(VIE_OK, VIE_ERR_NOT_CONVERGED))
        return (out.T if out is not None else None), st.as_dict(), status

    def sigma(self, I, khat, pol):
        """(extinction, scattering) cross sections per right-hand side."""
        inc, keep, nrhs = _incident_struct(khat, pol)
        I = np.ascontiguousarray(np.asarray(I, np.complex128).T)
        sig = np.zeros(2 * nrhs)
        self.ctx.check(self.L.vie_fields(self.h, C.byref(inc), I.ctypes.data_as(C.c_void_p), nrhs, None, 0, 0,
                                         None, _dp(sig)))
        return sig.reshape(nrhs, 2)

    def far_field(self, I, dirs):
        I = np.ascontiguousarray(np.asarray(I, np.complex128).reshape(self.n, -1).T)
        nrhs = I.shape[0]
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        out = np.zeros((nrhs, d.shape[0], 3), np.complex128)
        self.ctx.check(self.L.vie_fields(self.h, None, I.ctypes.data_as(C.c_void_p), nrhs, _dp(d.ravel()),
                                         d.shape[0], 0, out.ctypes.data_as(C.c_void_p), None))
        return out

    def near_field(self, I, points):
        """vie_fields mode 1: scattered field at points outside the atoms, (nrhs, npts, 3)."""
        I = np.ascontiguousarray(np.asarray(I, np.complex128).reshape(self.n, -1).T)
        nrhs = I.shape[0]
        d = np.ascontiguousarray(np.asarray(points, np.float64).reshape(-1, 3))
        out = np.zeros((nrhs, d.shape[0], 3), np.complex128)
        self.ctx.check(self.L.vie_fields(self.h, None, I.ctypes.data_as(C.c_void_p), nrhs, _dp(d.ravel()),
                                         d.shape[0], 1, out.ctypes.data_as(C.c_void_p), None))
        return out

    def export_block(self, kind, a, b=0, precision=C128):
        """kind 0: self block of type a; 1: interaction block of atoms a != b; 2: inverse of type a."""
        dt = np.complex64 if (kind == 1 and precision == C64) else np.complex128
        out = np.zeros((self.np, self.np), dt, order="F")
        self.ctx.check(self.L.vie_export_block(self.h, int(kind), int(a), int(b), int(precision),
                                               out.ctypes.data_as(C.c_void_p)))
        return out

    def far_blocks(self, with_factors=True, indices=None):
        inf = self.info()
        idx = range(inf["n_far_blocks"]) if indices is None else indices
        out = []
        for i in idx:
            lev, nt, ns, r = C.c_int(), C.c_int(), C.c_int(), C.c_int()
            self.ctx.check(self.L.vie_far_block_info(self.h, i, C.byref(lev), C.byref(nt), C.byref(ns), C.byref(r)))
            ta = np.zeros(nt.value, np.int32)
            sa = np.zeros(ns.value, np.int32)
            Q = R = None
            qp = rp = None
            if with_factors:
                Q = np.zeros((r.value, nt.value * self.np), np.complex128)   # column-major m x r
                R = np.zeros((ns.value * self.np, r.value), np.complex128)   # column-major r x n
                qp, rp = Q.ctypes.data_as(C.c_void_p), R.ctypes.data_as(C.c_void_p)
            self.ctx.check(self.L.vie_export_far_block(self.h, i, _ip(ta), _ip(sa), qp, rp))
            out.append(dict(level=lev.value, tatoms=ta, satoms=sa, rank=r.value,
                            Q=None if Q is None else Q.T, R=None if R is None else R.T))
        return out

    def close(self):
        if self.h:
            self.L.vie_op_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(ops, incidents, tol=1e-6, restart=60, max_iters=2000, precision=C64, launch=0):
    """vie_solve_batch: solve several problems (operators on one context) in one
    lockstep over their block-diagonal union.  incidents[p] = (khat, pol).
    Returns ([I_p numpy complex128 n_p x nrhs_p], [stats dict], status)."""
    B = len(ops)
    ctx = ops[0].ctx
    incs = (IncidentC * B)()
    keep, nr, outs = [], (C.c_int * B)(), []
    for p, (kh, pol) in enumerate(incidents):
        inc, k, n_r = _incident_struct(kh, pol)
        incs[p] = inc
        keep.append(k)
        nr[p] = n_r
        outs.append(np.zeros((n_r, ops[p].n), np.complex128))
    handles = (C.c_void_p * B)(*[op.h.value for op in ops])
    optrs = (C.c_void_p * B)(*[o.ctypes.data for o in outs])
    so = SolveOpts(tol, restart, max_iters, precision, 0, 1, launch, 0, 0)
    stats = (SolveStats * B)()
    status = ctx.check(ctx.L.vie_solve_batch(handles, B, incs, nr, C.byref(so), optrs, stats),
                       ok=(VIE_OK, VIE_ERR_NOT_CONVERGED))
    return [o.T for o in outs], [stats[p].as_dict() for p in range(B)], status


def plan_far_blocks(centres):
    """Host-only: (levels, [(level, target atoms, source atoms)]) as vie_assemble builds them."""
    L = load()
    xy = np.ascontiguousarray(np.asarray(centres, np.float64)[:, :2]).ravel()
    n = len(xy) // 2
    lev, nb, need = C.c_int(), C.c_int64(), C.c_int64()
    st = L.vie_plan_far_blocks(_dp(xy), n, C.byref(lev), C.byref(nb), None, 0, C.byref(need))
    if st != VIE_OK:
        raise VieError(st, "vie_plan_far_blocks")
    buf = np.zeros(max(1, need.value), np.int32)
    st = L.vie_plan_far_blocks(_dp(xy), n, C.byref(lev), C.byref(nb), _ip(buf), need.value, C.byref(need))
    if st != VIE_OK:
        raise VieError(st, "vie_plan_far_blocks")
    out, k = [], 0
    for _ in range(nb.value):
        l, nt, ns = buf[k:k + 3]
        k += 3
        out.append((int(l), buf[k:k + nt].tolist(), buf[k + nt:k + nt + ns].tolist()))
        k += nt + ns
    return lev.value, out


def lpt_assign(weights, n_proc):
    """Host-only greedy least-loaded map: (owner, loads)."""
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    owner = np.zeros(len(w), np.int32)
    loads = np.zeros(n_proc, np.float64)
    st = load().vie_lpt_assign(_dp(w), len(w), int(n_proc), _ip(owner), _dp(loads))
    if st != VIE_OK:
        raise VieError(st, "vie_lpt_assign")
    return owner, loads


def footprint_bytes(n, np_, nrhs, restart, factor_entries):
    return int(load().vie_footprint_bytes(int(n), int(np_), int(nrhs), int(restart), int(factor_entries)))


class Server:
    """vie_serve / vie_submit / vie_poll / vie_server_stop."""

    def __init__(self, ctx, max_inflight=4, hbm_budget=0, tol=1e-4, solve=None):
        self.ctx = ctx
        self.L = ctx.L
        self.h = C.c_void_p()
        so = solve or SolveOpts(1e-6, 60, 2000, C64, 0, 1, 0, 0, 0)
        o = ServeOpts(max_inflight, hbm_budget, tol, so)
        ctx.check(self.L.vie_serve(C.byref(self.h), ctx.h, C.byref(o)))
        self._keep = {}

    def submit(self, geometry, khat, pol):
        gs, keep_g = _geometry_struct(geometry)
        inc, keep_i, nrhs = _incident_struct(khat, pol)
        req = RequestC(gs, float(geometry.wavelength), nrhs, inc)
        t = C.c_uint64()
        st = self.L.vie_submit(self.h, C.byref(req), C.byref(t))
        if st != VIE_OK:
            raise VieError(st, "vie_submit")
        return t.value

    def poll(self, ticket, timeout_ms=60000):
        r = ResultC()
        st = self.L.vie_poll(self.h, C.c_uint64(ticket), C.byref(r), int(timeout_ms))
        if st == VIE_ERR_TIMEOUT:
            return None
        if st != VIE_OK:
            raise VieError(st, "vie_poll")
        I = None
        if r.I:
            I = np.ctypeslib.as_array(r.I, shape=(r.nrhs * r.n * 2,)).copy().view(np.complex128)
            I = I.reshape(r.nrhs, r.n).T
        out = dict(status=r.status, n=r.n, nrhs=r.nrhs, I=I, stats=r.stats.as_dict(), t_submit=r.t_submit_s,
                   t_start=r.t_start_s, t_done=r.t_done_s, footprint=r.footprint_bytes, retries=r.retries,
                   peak=r.peak_bytes)
        self.L.vie_result_free(C.byref(r))
        return out

    def stop(self):
        if self.h:
            self.ctx.check(self.L.vie_server_stop(self.h))
            self.h = C.c_void_p()
