// Left-preconditioned BiCGStab (van der Vorst, 1992): the Krylov method the
// paper weighs against GMRES in Sec. 6, solving P^-1 Zs x = P^-1 b with the
// block-diagonal preconditioner of Sec. 4.  Every right-hand side keeps its
// own recurrence (complex scalars rho, alpha, omega, beta on the device); the
// two operator applications of an iteration serve all of them at once (one
// n x k block, as in the lockstep GMRES).
//
// Precision follows the GMRES: the vectors and the inner products are
// float64, the operator applications inside the recurrence are complex
// float32 (or BF16x3 on the tensor cores); when every recursive residual is
// below the tolerance the preconditioned residual P^-1 (b - Zs x) is
// recomputed float64-accurately, and a column whose true residual is still
// above the tolerance restarts its recurrence from its current iterate with
// that residual (residual replacement: the refinement step).
#include <algorithm>
#include <cmath>

#include "common.h"
#include "cplx.cuh"
#include "krylov.h"

namespace vie {

namespace {

constexpr int kT = 256;

struct Bcg {
    int64_t n;
    int k;
    double2 *x, *r, *rh, *p, *v, *s, *t;  // n x k, column-major
    double2* sc;    // [k][4]: rho, alpha, omega, beta
    double2* dots;  // [k][2]
    double2* part;  // [k][2][nblk]
    double* beta0;  // [k] ||P^-1 b||
    double* res;    // [k] latest recursive residual / beta0
    int* active;    // [k] still iterating
    double tol;
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return d > 0.0 ? (1.0 / d) * cmulc(b, a) : make_double2(0.0, 0.0);  // a conj(b) / |b|^2
}

// partial sums of conj(U_d) W_d over a row slice, d < nd, per active column
__global__ void __launch_bounds__(kT) k_dots(Bcg a, const double2* U0, const double2* W0, const double2* U1,
                                             const double2* W1, int nd, int check_active) {
    const int c = blockIdx.y;
    if (check_active && !a.active[c]) return;
    const int64_t off = (int64_t)c * a.n, stride = (int64_t)gridDim.x * kT;
    double2 acc0 = make_double2(0.0, 0.0), acc1 = make_double2(0.0, 0.0);
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += stride) {
        cfmac(acc0, U0[off + r], W0[off + r]);
        if (nd > 1) cfmac(acc1, U1[off + r], W1[off + r]);
    }
    __shared__ double sh[4][kT / 32];
    double v[4] = {acc0.x, acc0.y, acc1.x, acc1.y};
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if (lane == 0) sh[q][wid] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 2 * nd) {
        const int d = threadIdx.x >> 1, comp = threadIdx.x & 1;
        double s = 0.0;
        for (int w = 0; w < kT / 32; ++w) s += sh[2 * d + comp][w];
        double* dst = reinterpret_cast<double*>(a.part + ((int64_t)c * 2 + d) * gridDim.x + blockIdx.x);
        dst[comp] = s;
    }
}

__global__ void k_dots_reduce(Bcg a, int nd, int nblk, int check_active) {
    const int c = blockIdx.x;
    if (check_active && !a.active[c]) return;
    const int d = threadIdx.x;
    if (d >= nd) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) s += a.part[((int64_t)c * 2 + d) * nblk + b];
    a.dots[c * 2 + d] = s;
}

// scalar recurrences, one thread per column
//  0: rho' = <rh, r>, beta = (rho' / rho) (alpha / omega), rho = rho'
//  1: alpha = rho / <rh, v>
//  2: omega = <t, s> / <t, t>
//  3: res = ||r|| / beta0; a column below the tolerance stops
//  4: (re)start: rho = alpha = omega = 1, beta0 = ||r||, res = 1 (columns with beta0 = 0 stop)
__global__ void k_scalars(Bcg a, int stage, const int* restart) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.k) return;
    double2* sc = a.sc + c * 4;
    const double2 d0 = a.dots[c * 2], d1 = a.dots[c * 2 + 1];
    if (stage == 4) {
        if (!restart[c]) return;
        sc[0] = sc[1] = sc[2] = make_double2(1.0, 0.0);
        sc[3] = make_double2(0.0, 0.0);
        a.res[c] = 1.0;
        a.active[c] = 1;
        return;
    }
    if (!a.active[c]) return;
    if (stage == 0) {
        sc[3] = cmul(cdiv(d0, sc[0]), cdiv(sc[1], sc[2]));
        sc[0] = d0;
    } else if (stage == 1) {
        sc[1] = cdiv(sc[0], d0);
    } else if (stage == 2) {
        sc[2] = cdiv(d0, d1);
    } else {
        const double rn = sqrt(fmax(d0.x, 0.0));
        const double r = a.beta0[c] > 0.0 ? rn / a.beta0[c] : 0.0;
        a.res[c] = r;
        if (!(r > a.tol)) a.active[c] = 0;  // converged (or not finite: stops, reported by the host)
    }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kT) k_upd_p(Bcg a) {
    const int c = blockIdx.y;
    if (!a.active[c]) return;
    const double2 beta = a.sc[c * 4 + 3], omega = a.sc[c * 4 + 2];
    const int64_t off = (int64_t)c * a.n;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT) {
        const double2 q = a.p[off + r] - cmul(omega, a.v[off + r]);
        a.p[off + r] = a.r[off + r] + cmul(beta, q);
    }
}

// s = r - alpha v
__global__ void __launch_bounds__(kT) k_upd_s(Bcg a) {
    const int c = blockIdx.y;
    if (!a.active[c]) return;
    const double2 alpha = a.sc[c * 4 + 1];
    const int64_t off = (int64_t)c * a.n;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT)
        a.s[off + r] = a.r[off + r] - cmul(alpha, a.v[off + r]);
}

// x += alpha p + omega s, r = s - omega t
__global__ void __launch_bounds__(kT) k_upd_xr(Bcg a) {
    const int c = blockIdx.y;
    if (!a.active[c]) return;
    const double2 alpha = a.sc[c * 4 + 1], omega = a.sc[c * 4 + 2];
    const int64_t off = (int64_t)c * a.n;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT) {
        const double2 sv = a.s[off + r];
        a.x[off + r] += cmul(alpha, a.p[off + r]) + cmul(omega, sv);
        a.r[off + r] = sv - cmul(omega, a.t[off + r]);
    }
}

// float32 copy of the active columns of src (zero for the others)
__global__ void __launch_bounds__(kT) k_to32(Bcg a, const double2* __restrict__ src, float2* __restrict__ dst) {
    const int c = blockIdx.y;
    const int64_t off = (int64_t)c * a.n;
    const bool on = a.active[c] != 0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT) {
        const double2 v = on ? src[off + r] : make_double2(0.0, 0.0);
        dst[off + r] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void __launch_bounds__(kT) k_to64(Bcg a, const float2* __restrict__ src, double2* __restrict__ dst) {
    const int c = blockIdx.y;
    if (!a.active[c]) return;
    const int64_t off = (int64_t)c * a.n;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT) {
        const float2 v = src[off + r];
        dst[off + r] = make_double2(v.x, v.y);
    }
}

// restart of the flagged columns from the residual W: r = rh = W, p = v = 0
__global__ void __launch_bounds__(kT) k_restart(Bcg a, const double2* __restrict__ W, const int* restart) {
    const int c = blockIdx.y;
    if (!restart[c]) return;
    const int64_t off = (int64_t)c * a.n;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * kT) {
        const double2 w = W[off + r];
        a.r[off + r] = w;
        a.rh[off + r] = w;
        a.p[off + r] = make_double2(0.0, 0.0);
        a.v[off + r] = make_double2(0.0, 0.0);
    }
}

// R = b - T
__global__ void __launch_bounds__(kT) k_sub(const double2* __restrict__ b, const double2* __restrict__ T,
                                           double2* __restrict__ R, int64_t len) {
    for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < len; i += (int64_t)gridDim.x * kT) R[i] = b[i] - T[i];
}

struct Runner {
    Op& op;
    const vie_solve_opts& o;
    cudaStream_t s;
    int64_t n;
    int k, nblk;
    bool c64;
    DevBuf x, r, rh, p, v, sv, t, sc, dots, part, beta0, res, active, flag, X32, Y32, T, R, W, bn, rn, norms;
    Bcg a{};

    Runner(Op& op_, const vie_solve_opts& o_, int nrhs)
        : op(op_), o(o_), s(op_.ctx->stream), n(op_.n()), k(nrhs) {
        c64 = o.precision != VIE_C128 && o.precond;
        nblk = kr_nblk(n, k, op.ctx->n_sm);
        const size_t vec = (size_t)n * k * sizeof(double2);
        for (DevBuf* d : {&r, &rh, &p, &v, &sv, &t, &T, &R, &W}) d->alloc(vec);
        sc.alloc((size_t)k * 4 * sizeof(double2));
        dots.alloc((size_t)k * 2 * sizeof(double2));
        part.alloc((size_t)k * 2 * nblk * sizeof(double2));
        beta0.alloc(k * sizeof(double));
        res.alloc(k * sizeof(double));
        active.alloc(k * sizeof(int));
        flag.alloc(k * sizeof(int));
        bn.alloc(k * sizeof(double));
        rn.alloc(k * sizeof(double));
        if (c64) {
            X32.alloc((size_t)n * k * sizeof(float2));
            Y32.alloc((size_t)n * k * sizeof(float2));
        }
        op_reserve(op, k, o.precision, s);
        a.n = n;
        a.k = k;
        a.r = r.as<double2>();
        a.rh = rh.as<double2>();
        a.p = p.as<double2>();
        a.v = v.as<double2>();
        a.s = sv.as<double2>();
        a.t = t.as<double2>();
        a.sc = sc.as<double2>();
        a.dots = dots.as<double2>();
        a.part = part.as<double2>();
        a.beta0 = beta0.as<double>();
        a.res = res.as<double>();
        a.active = active.as<int>();
        a.tol = o.tol > 0 ? o.tol : 1e-6;
    }

    void dots_of(const double2* U0, const double2* W0, const double2* U1, const double2* W1, int nd, int chk) {
        k_dots<<<dim3(nblk, k), kT, 0, s>>>(a, U0, W0, U1, W1, nd, chk);
        VIE_CHECK_LAUNCH();
        k_dots_reduce<<<k, 32, 0, s>>>(a, nd, nblk, chk);
        VIE_CHECK_LAUNCH();
    }
    void scalars(int stage, const int* restart = nullptr) {
        k_scalars<<<(k + 127) / 128, 128, 0, s>>>(a, stage, restart);
        VIE_CHECK_LAUNCH();
    }
    // dst = P^-1 Zs src (the inner, recurrence applies)
    void apply(const double2* src, double2* dst) {
        if (c64) {
            k_to32<<<dim3(nblk, k), kT, 0, s>>>(a, src, X32.as<float2>());
            VIE_CHECK_LAUNCH();
            if (o.precision == VIE_BF16X3) op_apply_fused_bf16x3(op, X32.as<float2>(), Y32.as<float2>(), k, s);
            else op_apply_fused32(op, X32.as<float2>(), Y32.as<float2>(), k, s);
            k_to64<<<dim3(nblk, k), kT, 0, s>>>(a, Y32.as<float2>(), dst);
            VIE_CHECK_LAUNCH();
        } else if (o.precond) {
            op_apply_fused64(op, src, dst, k, s);
        } else {
            op_apply64(op, src, dst, k, s);
        }
    }
    // W = P^-1 (b - Zs x) float64-accurate, R = b - Zs x; norms of R into rn
    void true_residual(const double2* b) {
        op_apply64(op, a.x, T.as<double2>(), k, s);
        k_sub<<<(unsigned)std::min<int64_t>(4096, (n * k + kT - 1) / kT), kT, 0, s>>>(b, T.as<double2>(),
                                                                                       R.as<double2>(), n * k);
        VIE_CHECK_LAUNCH();
        if (o.precond) op_precond64(op, R.as<double2>(), W.as<double2>(), k, s);
        else VIE_CUDA(cudaMemcpyAsync(W.p, R.p, (size_t)n * k * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }
    std::vector<double> colnorms(const double2* A) {
        dots_of(A, A, nullptr, nullptr, 1, 0);
        std::vector<double2> h(2 * k);
        VIE_CUDA(cudaMemcpyAsync(h.data(), dots.p, 2 * k * sizeof(double2), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
        std::vector<double> out(k);
        for (int c = 0; c < k; ++c) out[c] = std::sqrt(std::max(h[2 * c].x, 0.0));
        return out;
    }

    GmresOutcome run(const double2* b, double2* Xout) {
        GmresOutcome out;
        a.x = Xout;
        VIE_CUDA(cudaMemsetAsync(Xout, 0, (size_t)n * k * sizeof(double2), s));
        // x = 0: R = b, W = P^-1 b
        VIE_CUDA(cudaMemcpyAsync(R.p, b, (size_t)n * k * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        if (o.precond) op_precond64(op, b, W.as<double2>(), k, s);
        else VIE_CUDA(cudaMemcpyAsync(W.p, b, (size_t)n * k * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        const std::vector<double> bnorm = colnorms(b);
        const std::vector<double> wn0 = colnorms(W.as<double2>());
        VIE_CUDA(cudaMemcpyAsync(beta0.p, wn0.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
        std::vector<int> restart(k), h_active(k), iters(k, 0);
        std::vector<double> h_res(k);
        for (int c = 0; c < k; ++c) restart[c] = wn0[c] > 0.0 ? 1 : 0;
        const int maxit = o.max_iters > 0 ? o.max_iters : 2000;
        int it = 0, applies = 0, refinements = 0;
        out.res.assign(k, 0.0);
        std::vector<double> final_res(k, 0.0);
        while (true) {
            // (re)start the flagged columns from W
            VIE_CUDA(cudaMemcpyAsync(flag.p, restart.data(), k * sizeof(int), cudaMemcpyHostToDevice, s));
            k_restart<<<dim3(nblk, k), kT, 0, s>>>(a, W.as<double2>(), flag.as<int>());
            VIE_CHECK_LAUNCH();
            scalars(4, flag.as<int>());
            VIE_CUDA(cudaMemcpyAsync(h_active.data(), active.p, k * sizeof(int), cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            bool any = std::any_of(h_active.begin(), h_active.end(), [](int x) { return x != 0; });
            while (any && it < maxit) {
                dots_of(a.rh, a.r, nullptr, nullptr, 1, 1);
                scalars(0);
                k_upd_p<<<dim3(nblk, k), kT, 0, s>>>(a);
                VIE_CHECK_LAUNCH();
                apply(a.p, a.v);
                dots_of(a.rh, a.v, nullptr, nullptr, 1, 1);
                scalars(1);
                k_upd_s<<<dim3(nblk, k), kT, 0, s>>>(a);
                VIE_CHECK_LAUNCH();
                apply(a.s, a.t);
                dots_of(a.t, a.s, a.t, a.t, 2, 1);
                scalars(2);
                k_upd_xr<<<dim3(nblk, k), kT, 0, s>>>(a);
                VIE_CHECK_LAUNCH();
                dots_of(a.r, a.r, nullptr, nullptr, 1, 1);
                for (int c = 0; c < k; ++c)
                    if (h_active[c]) ++iters[c];
                scalars(3);
                ++it;
                applies += 2;
                VIE_CUDA(cudaMemcpyAsync(h_active.data(), active.p, k * sizeof(int), cudaMemcpyDeviceToHost, s));
                VIE_CUDA(cudaMemcpyAsync(h_res.data(), res.p, k * sizeof(double), cudaMemcpyDeviceToHost, s));
                VIE_CUDA(cudaStreamSynchronize(s));
                double mx = 0.0;
                for (int c = 0; c < k; ++c) {
                    if (!std::isfinite(h_res[c])) fail(VIE_ERR_NAN, "non-finite residual in BiCGStab");
                    mx = std::max(mx, h_res[c]);
                }
                if ((int)out.hist.size() < 512) out.hist.push_back(mx);
                any = std::any_of(h_active.begin(), h_active.end(), [](int x) { return x != 0; });
            }
            // refinement: the true preconditioned residual of every column
            true_residual(b);
            ++refinements;
            const std::vector<double> wn = colnorms(W.as<double2>());
            bool again = false;
            for (int c = 0; c < k; ++c) {
                final_res[c] = wn0[c] > 0 ? wn[c] / wn0[c] : 0.0;
                restart[c] = (final_res[c] > a.tol && iters[c] < maxit) ? 1 : 0;
                again |= restart[c] != 0;
            }
            if (!again || it >= maxit) break;
        }
        const std::vector<double> rnorm = colnorms(R.as<double2>());
        out.res = final_res;
        out.rnorm = rnorm;
        out.bnorm = bnorm;
        out.iters = iters;
        out.applies = applies;
        out.refinements = refinements;
        return out;
    }
};

}  // namespace

GmresOutcome run_bicgstab(Op& op, const double2* b, double2* X, const vie_solve_opts& o, int nrhs) {
    Runner R(op, o, nrhs);
    return R.run(b, X);
}

}  // namespace vie
