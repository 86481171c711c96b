// Device-resident kernels of the lockstep GMRES (paper Sec. 6: restarted
// GMRES with the Arnoldi process, left-preconditioned by the block diagonal of
// Sec. 4).  Every kernel works on all right-hand sides of a restart cycle at
// once (grid dimension y or z = slot) and reads the Arnoldi step j and the
// per-slot "still iterating" flags from device memory, so a whole cycle runs
// without the host: the Hessenberg matrix, the Givens rotations and the
// residual estimates live on the device too.
//
// Reductions are two-stage with a fixed partition of the rows, so every
// result is the same from run to run.
//
// The basis is stored in one of two float64-accurate forms: float64 (the
// all-float64 solve) or double-float (float4 per complex value, hi + lo: the
// mixed-precision solve, whose inner applies are float32 anyway).  The
// double-float projections and updates run on the float32 pipes, which on
// this GPU are far faster than its float64 units; they carry ~48 significant
// bits per operation, and their sums are reduced in float64.
#include "common.h"
#include "cplx.cuh"
#include "dfloat.cuh"
#include "krylov.h"

namespace vie {

namespace {

constexpr int kT = 256;  // threads of the row kernels
constexpr int kCG = 8;   // basis columns per CTA in the projections

__device__ __forceinline__ double2 ld64(const float2* p, int64_t i) {
    const float2 v = p[i];
    return make_double2(v.x, v.y);
}
__device__ __forceinline__ double2 ld64(const double2* p, int64_t i) { return p[i]; }
__device__ __forceinline__ void st(float2* p, int64_t i, double2 v) { p[i] = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st(double2* p, int64_t i, double2 v) { p[i] = v; }

// sum of v over the CTA (kT threads), valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) s += sh[w];
    return s;
}

// rows of a right-hand-side column and its basis
struct Rows {
    int64_t lo, len;
    double2* V;  // basis vector l at V + l * len
};
__device__ __forceinline__ Rows rows_of(const KrylovArgs& a, int c) {
    return {a.col_lo[c], a.col_len[c], a.V + a.col_voff[c]};
}

__global__ void k_cycle_start(KrylovArgs a, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) a.ctr[KR_J] = 0;
    if (i >= k) return;
    const int c = a.cols[i];
    double2* g = a.g + (int64_t)i * (a.m + 1);
    g[0] = make_double2(a.beta[c], 0.0);
    for (int l = 1; l <= a.m; ++l) g[l] = make_double2(0.0, 0.0);
    a.inv[i] = a.beta[c] > 0.0 ? 1.0 / a.beta[c] : 0.0;
    a.cycling[i] = a.beta[c] > 0.0 && a.iters[c] < a.maxit;
    a.jdone[i] = 0;
}

template <class TX>
__global__ void __launch_bounds__(kT) k_gather(KrylovArgs a, const double2* __restrict__ W, TX* __restrict__ Xg) {
    const int i = blockIdx.y;
    const int c = a.cols[i];
    const Rows R = rows_of(a, c);
    const int64_t n = R.len, stride = (int64_t)gridDim.x * kT;
    TX* x = Xg + (int64_t)i * a.n + R.lo;
    if (!a.cycling[i]) {
        for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += stride) st(x, r, make_double2(0.0, 0.0));
        return;
    }
    const int j = a.ctr[KR_J];
    double2* v = R.V + (int64_t)j * n;
    const double2* src = j == 0 ? W + (int64_t)c * a.n + R.lo : v;
    const double sc = a.inv[i];
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += stride) {
        const double2 e = sc * src[r];
        v[r] = e;
        st(x, r, e);
    }
}

// ---- double-float basis ----------------------------------------------------
// k_gather for a double-float basis: column j (j > 0, stored unnormalised by
// the previous step) is scaled in place; column 0 comes from W (float64)
__global__ void __launch_bounds__(kT) k_gather_df(KrylovArgs a, const double2* __restrict__ W, float2* __restrict__ Xg) {
    const int i = blockIdx.y;
    const int c = a.cols[i];
    const Rows R = rows_of(a, c);
    const int64_t n = R.len, stride = (int64_t)gridDim.x * kT;
    float2* x = Xg + (int64_t)i * a.n + R.lo;
    if (!a.cycling[i]) {
        for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += stride) x[r] = make_float2(0.f, 0.f);
        return;
    }
    const int j = a.ctr[KR_J];
    float4* v = reinterpret_cast<float4*>(R.V) + (int64_t)j * n;
    const double sc = a.inv[i];
    if (j == 0) {
        const double2* src = W + (int64_t)c * a.n + R.lo;
        for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += stride) {
            const float4 e = df_from(sc * src[r]);
            v[r] = e;
            x[r] = make_float2(e.x, e.y);
        }
    } else {
        const float sh = (float)sc, sl = (float)(sc - (double)sh);
        for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += stride) {
            const float4 e = df_scale(v[r], sh, sl);
            v[r] = e;
            x[r] = make_float2(e.x, e.y);
        }
    }
}

// partial h[col] = sum_r conj(V[r, col]) w[r], double-float products and
// per-thread sums, float64 across threads; pass 1 takes w from the float32
// operator output (exact in double-float) and stores it as basis column j+1
template <bool kFirst>
__global__ void __launch_bounds__(kT) k_mdot_df(KrylovArgs a, const float2* __restrict__ Y) {
    const int i = blockIdx.z, cg = blockIdx.y;
    if (!a.cycling[i]) return;
    if (!kFirst && a.reorth && !a.reorth[i]) return;
    const int j = a.ctr[KR_J];
    const int ncols = j + 1;
    if (cg * kCG >= ncols) return;
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const float4* V = reinterpret_cast<const float4*>(R.V);
    float4* w = reinterpret_cast<float4*>(R.V) + (int64_t)(j + 1) * n;
    const float2* y = kFirst ? Y + (int64_t)i * a.n + R.lo : nullptr;
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    float4 acc[kCG];
#pragma unroll
    for (int c = 0; c < kCG; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    double wn = 0.0;  // pass 1: ||w||^2 partials (blocks of column group 0)
    for (int64_t r = r0 + threadIdx.x; r < r1; r += 2 * kT) {
        const bool second = r + kT < r1;
        float4 wv, wv2 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kFirst) {
            const float2 y1 = y[r];
            wv = make_float4(y1.x, y1.y, 0.f, 0.f);
            if (second) {
                const float2 y2 = y[r + kT];
                wv2 = make_float4(y2.x, y2.y, 0.f, 0.f);
            }
            if (cg == 0) {
                w[r] = wv;
                if (second) w[r + kT] = wv2;
                wn += (double)wv.x * wv.x + (double)wv.y * wv.y + (double)wv2.x * wv2.x + (double)wv2.y * wv2.y;
            }
        } else {
            wv = w[r];
            if (second) wv2 = w[r + kT];
        }
        float4 v1[kCG], v2[kCG];
#pragma unroll
        for (int c = 0; c < kCG; ++c) {
            const int col = cg * kCG + c;
            v1[c] = col < ncols ? V[(int64_t)col * n + r] : make_float4(0.f, 0.f, 0.f, 0.f);
            v2[c] = (col < ncols && second) ? V[(int64_t)col * n + r + kT] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < kCG; ++c) {
            df_cmac_conj(acc[c], v1[c], wv);
            df_cmac_conj(acc[c], v2[c], wv2);
        }
    }
    __shared__ double2 sh[kT / 32][kCG];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < kCG; ++c) {
        double re = (double)acc[c].x + (double)acc[c].z, im = (double)acc[c].y + (double)acc[c].w;
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) sh[wid][c] = make_double2(re, im);
    }
    // pass 1: the squared norm of w goes to partial slot j + 1 (<= m < hs), beside the dots
    __shared__ double shn[kT / 32];
    if (kFirst && cg == 0) {
        for (int o = 16; o > 0; o >>= 1) wn += __shfl_down_sync(0xffffffffu, wn, o);
        if (lane == 0) shn[wid] = wn;
    }
    __syncthreads();
    if (threadIdx.x < kCG) {
        const int col = cg * kCG + threadIdx.x;
        if (col < ncols) {
            double2 s = make_double2(0.0, 0.0);
            for (int w2 = 0; w2 < kT / 32; ++w2) s += sh[w2][threadIdx.x];
            a.part[((int64_t)i * a.hs + col) * gridDim.x + blockIdx.x] = s;
        }
    }
    if (kFirst && cg == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < kT / 32; ++w2) t += shn[w2];
        a.part[((int64_t)i * a.hs + ncols) * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
    }
}

// w -= V h (columns 0..j) in double-float; pass 2 also forms the squared-norm
// partials of w (float64)
template <bool kSecond>
__global__ void __launch_bounds__(kT) k_maxpy_df(KrylovArgs a) {
    const int i = blockIdx.y;
    if (!a.cycling[i]) return;
    if (kSecond && a.reorth && !a.reorth[i]) return;  // pass 1's norm partials stand
    const int j = a.ctr[KR_J];
    __shared__ float4 hs[kMaxRestart + 1];
    __shared__ double sh[kT / 32];
    for (int c = threadIdx.x; c <= j; c += kT) hs[c] = df_from(a.h[(int64_t)i * a.hs + c]);
    __syncthreads();
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const float4* V = reinterpret_cast<const float4*>(R.V);
    float4* w = reinterpret_cast<float4*>(R.V) + (int64_t)(j + 1) * n;
    double nacc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        float4 acc = w[r];
        for (int c = 0; c <= j; ++c) df_cmsub(acc, V[(int64_t)c * n + r], hs[c]);
        acc = df_normed(acc);
        w[r] = acc;
        const double2 d = df_to(acc);
        nacc += d.x * d.x + d.y * d.y;
    }
    // the norm of w after this pass: the step's last pass writes the partials k_nsq sums
    const double s = block_sum(nacc, sh);
    if (threadIdx.x == 0) a.npart[(int64_t)i * a.nblk_max + blockIdx.x] = s;
}

// X[:, cols[i]] += V y; with D, the correction V y of slot i is also written
// there in float32 (the input of a residual update), zero for a slot that did
// no step
__global__ void __launch_bounds__(kT) k_xupdate_df(KrylovArgs a, double2* __restrict__ X, float2* __restrict__ D) {
    const int i = blockIdx.y;
    const int jd = a.jdone[i];
    if (jd == 0) {
        if (D) {
            const Rows R = rows_of(a, a.cols[i]);
            float2* d = D + (int64_t)i * a.n + R.lo;
            for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < R.len; r += (int64_t)gridDim.x * kT)
                d[r] = make_float2(0.f, 0.f);
        }
        return;
    }
    __shared__ double2 ys[kMaxRestart];
    for (int l = threadIdx.x; l < jd; l += kT) ys[l] = a.y[(int64_t)i * a.hs + l];
    __syncthreads();
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const float4* V = reinterpret_cast<const float4*>(R.V);
    double2* x = X + (int64_t)a.cols[i] * a.n + R.lo;
    float2* d = D ? D + (int64_t)i * a.n + R.lo : nullptr;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < jd; ++l) cfma(acc, df_to(V[(int64_t)l * n + r]), ys[l]);
        x[r] += acc;
        if (d) d[r] = make_float2((float)acc.x, (float)acc.y);
    }
}

// Wf[:, cols[i]] -= E[:, i] and its squared-norm partials (residual update)
__global__ void __launch_bounds__(kT) k_sub_scatter_norm(KrylovArgs a, const double2* __restrict__ E, double2* Wf) {
    const int i = blockIdx.y;
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* src = E + (int64_t)i * a.n + R.lo;
    double2* dst = Wf + (int64_t)a.cols[i] * a.n + R.lo;
    __shared__ double sh[kT / 32];
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        const double2 v = dst[r] - src[r];
        dst[r] = v;
        acc += v.x * v.x + v.y * v.y;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) a.npart[(int64_t)i * a.nblk_max + blockIdx.x] = s;
}

// partial h[col] = sum_r conj(V[r, col]) w[r] over one row chunk, 8 columns per CTA.
// Pass 1 takes w from the operator output and stores it as basis column j+1.
template <class TW, bool kFirst>
__global__ void __launch_bounds__(kT) k_mdot(KrylovArgs a, const TW* __restrict__ Y) {
    const int i = blockIdx.z, cg = blockIdx.y;
    if (!a.cycling[i]) return;
    const int j = a.ctr[KR_J];
    const int ncols = j + 1;
    if (cg * kCG >= ncols) return;
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* V = R.V;
    double2* w = R.V + (int64_t)(j + 1) * n;
    const TW* y = kFirst ? Y + (int64_t)i * a.n + R.lo : nullptr;
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    double2 acc[kCG];
#pragma unroll
    for (int c = 0; c < kCG; ++c) acc[c] = make_double2(0.0, 0.0);
    // two rows per iteration keep more loads in flight
    for (int64_t r = r0 + threadIdx.x; r < r1; r += 2 * kT) {
        const bool second = r + kT < r1;
        double2 wv, wv2 = make_double2(0.0, 0.0);
        if (kFirst) {
            wv = ld64(y, r);
            if (second) wv2 = ld64(y, r + kT);
            if (cg == 0) {
                w[r] = wv;
                if (second) w[r + kT] = wv2;
            }
        } else {
            wv = w[r];
            if (second) wv2 = w[r + kT];
        }
        double2 v1[kCG], v2[kCG];
#pragma unroll
        for (int c = 0; c < kCG; ++c) {
            const int col = cg * kCG + c;
            v1[c] = col < ncols ? V[(int64_t)col * n + r] : make_double2(0.0, 0.0);
            v2[c] = (col < ncols && second) ? V[(int64_t)col * n + r + kT] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int c = 0; c < kCG; ++c) {
            cfmac(acc[c], v1[c], wv);
            cfmac(acc[c], v2[c], wv2);
        }
    }
    __shared__ double2 sh[kT / 32][kCG];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < kCG; ++c) {
        double re = acc[c].x, im = acc[c].y;
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) sh[wid][c] = make_double2(re, im);
    }
    __syncthreads();
    if (threadIdx.x < kCG) {
        const int col = cg * kCG + threadIdx.x;
        if (col < ncols) {
            double2 s = make_double2(0.0, 0.0);
            for (int w2 = 0; w2 < kT / 32; ++w2) s += sh[w2][threadIdx.x];
            a.part[((int64_t)i * a.hs + col) * gridDim.x + blockIdx.x] = s;
        }
    }
}

// h = sum of the chunk partials (one warp per basis column); the Hessenberg
// column accumulates both passes.
// Double-float basis: pass 2 runs only where pass 1 cancelled much of w
// (selective reorthogonalisation, the criterion of Daniel, Gragg, Kaufman and
// Stewart, 1976): ||w - V h||^2 = ||w||^2 - ||h||^2 against ||w||^2 / 2.
template <bool kFirst>
__global__ void __launch_bounds__(kT) k_reduce(KrylovArgs a, int nchunk) {
    const int i = blockIdx.x;
    if (!a.cycling[i]) return;
    const bool sel = a.df && a.reorth;
    if (!kFirst && sel && !a.reorth[i]) return;
    const int j = a.ctr[KR_J];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double hn[kT / 32];
    double hsq = 0.0;
    for (int col = wid; col <= j; col += kT / 32) {
        const double2* p = a.part + ((int64_t)i * a.hs + col) * nchunk;
        double re = 0.0, im = 0.0;
        for (int x = lane; x < nchunk; x += 32) {
            re += p[x].x;
            im += p[x].y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            const double2 s = make_double2(re, im);
            a.h[(int64_t)i * a.hs + col] = s;
            double2* Hc = a.H + ((int64_t)i * a.m + j) * (a.m + 1);
            if (kFirst) Hc[col] = (a.shift && col == j) ? make_double2(s.x + 1.0, s.y) : s;
            else Hc[col] += s;
            hsq += re * re + im * im;
        }
    }
    if (kFirst && sel) {
        if (lane == 0) hn[wid] = hsq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double h2 = 0.0, w2 = 0.0;
            for (int x = 0; x < kT / 32; ++x) h2 += hn[x];
            const double2* p = a.part + ((int64_t)i * a.hs + j + 1) * nchunk;
            for (int x = 0; x < nchunk; ++x) w2 += p[x].x;
            a.reorth[i] = (w2 - h2 < 0.5 * w2) || !(w2 > 0.0) || !isfinite(w2 - h2) ? 1 : 0;
        }
    }
}

// nsq[slot] = sum of the slot's squared-norm partials (one CTA per slot)
__global__ void __launch_bounds__(kT) k_nsq(KrylovArgs a, int nblk, int check_cycling) {
    const int i = blockIdx.x;
    if (check_cycling && !a.cycling[i]) return;
    __shared__ double sh[kT / 32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kT) acc += a.npart[(int64_t)i * a.nblk_max + b];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) a.nsq[i] = s;
}

// w -= V h (columns 0..j); pass 2 also forms the squared-norm partials of w
template <bool kSecond>
__global__ void __launch_bounds__(kT) k_maxpy(KrylovArgs a) {
    const int i = blockIdx.y;
    if (!a.cycling[i]) return;
    const int j = a.ctr[KR_J];
    __shared__ double2 hs[kMaxRestart + 1];
    __shared__ double sh[kT / 32];
    for (int c = threadIdx.x; c <= j; c += kT) hs[c] = a.h[(int64_t)i * a.hs + c];
    __syncthreads();
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* V = R.V;
    double2* w = R.V + (int64_t)(j + 1) * n;
    double nacc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        double2 acc = w[r];
        for (int c = 0; c <= j; ++c) {
            const double2 v = V[(int64_t)c * n + r], hc = hs[c];
            acc.x -= v.x * hc.x - v.y * hc.y;
            acc.y -= v.x * hc.y + v.y * hc.x;
        }
        w[r] = acc;
        if (kSecond) nacc += acc.x * acc.x + acc.y * acc.y;
    }
    if (kSecond) {
        const double s = block_sum(nacc, sh);
        if (threadIdx.x == 0) a.npart[(int64_t)i * a.nblk_max + blockIdx.x] = s;
    }
}

// one thread per slot: new Hessenberg column, Givens rotations
// G = [[conj c, conj s], [-s, c]], residual estimate |g_{j+1}| / ||M^-1 b||
__global__ void k_givens(KrylovArgs a, int k, int nblk, cudaGraphConditionalHandle hnd, int use_handle) {
    const int i = threadIdx.x;
    const int j = a.ctr[KR_J];
    const int m = a.m;
    bool cyc = i < k && a.cycling[i] != 0;
    double est = 0.0;
    if (cyc) {
        const int c = a.cols[i];
        const double hn = sqrt(a.nsq[i]);
        double2* Hc = a.H + ((int64_t)i * m + j) * (m + 1);
        double2* cs = a.cs + (int64_t)i * m;
        double2* sn = a.sn + (int64_t)i * m;
        double2* g = a.g + (int64_t)i * (m + 1);
        Hc[j + 1] = make_double2(hn, 0.0);
        for (int l = 0; l < j; ++l) {
            const double2 x = Hc[l], y = Hc[l + 1];
            Hc[l] = cmulc(cs[l], x) + cmulc(sn[l], y);
            Hc[l + 1] = cmul(cs[l], y) - cmul(sn[l], x);
        }
        const double2 x = Hc[j], y = Hc[j + 1];
        const double den = sqrt(x.x * x.x + x.y * x.y + y.x * y.x + y.y * y.y);
        const double2 cj = den > 0.0 ? (1.0 / den) * x : make_double2(1.0, 0.0);
        const double2 sj = den > 0.0 ? (1.0 / den) * y : make_double2(0.0, 0.0);
        cs[j] = cj;
        sn[j] = sj;
        Hc[j] = make_double2(den, 0.0);
        Hc[j + 1] = make_double2(0.0, 0.0);
        const double2 gj = g[j];
        g[j + 1] = -1.0 * cmul(sj, gj);
        g[j] = cmulc(cj, gj);
        const int it = a.iters[c] + 1;
        a.iters[c] = it;
        a.jdone[i] = j + 1;
        est = hypot(g[j + 1].x, g[j + 1].y) / a.beta0[c];
        if (!isfinite(est)) {
            a.ctr[KR_NAN] = 1;
            cyc = false;
            est = 0.0;
        } else if (est <= a.tol || hn == 0.0 || it >= a.maxit) {
            cyc = false;
        }
        a.inv[i] = hn > 0.0 ? 1.0 / hn : 0.0;
        a.cycling[i] = cyc ? 1 : 0;
    }
    __shared__ double se[1024];
    se[i] = est;
    const int any = __syncthreads_or(cyc ? 1 : 0);
    if (a.colr && i < k) {
        // the first slot of each problem retires the problem once none of its slots iterates
        const int p = a.col_prob[a.cols[i]];
        const int2 r = a.colr_cycle[p];
        if (i == r.x) {
            int live = 0;
            for (int t = r.x; t < r.y; ++t) live |= a.cycling[t];
            if (!live) a.colr[p] = make_int2(0, 0);
        }
    }
    if (i == 0) {
        double mx = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) mx = fmax(mx, se[t]);
        const int it = a.ctr[KR_IT];
        if (it < 512) a.hist[it] = mx;
        a.ctr[KR_IT] = it + 1;
        a.ctr[KR_APPLIES] += 1;
        const int cont = (any && j + 1 < m) ? 1 : 0;
        if (cont) a.ctr[KR_J] = j + 1;
        a.ctr[KR_CONT] = cont;
        if (use_handle) cudaGraphSetConditional(hnd, (unsigned)cont);
    }
}

// back substitution y = H^-1 g on the rotated (upper triangular) Hessenberg matrix
__global__ void k_backsub(KrylovArgs a, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int jd = a.jdone[i], m = a.m;
    const double2* H = a.H + (int64_t)i * m * (m + 1);
    const double2* g = a.g + (int64_t)i * (m + 1);
    double2* y = a.y + (int64_t)i * a.hs;
    for (int r = jd - 1; r >= 0; --r) {
        double2 acc = g[r];
        for (int l = r + 1; l < jd; ++l) acc -= cmul(H[r + (int64_t)l * (m + 1)], y[l]);
        const double2 d = H[r + (int64_t)r * (m + 1)];
        const double dd = d.x * d.x + d.y * d.y;
        y[r] = dd > 0.0 ? (1.0 / dd) * cmulc(d, acc) : make_double2(0.0, 0.0);
    }
}

__global__ void __launch_bounds__(kT) k_xupdate(KrylovArgs a, double2* __restrict__ X) {
    const int i = blockIdx.y;
    const int jd = a.jdone[i];
    if (jd == 0) return;
    __shared__ double2 ys[kMaxRestart];
    for (int l = threadIdx.x; l < jd; l += kT) ys[l] = a.y[(int64_t)i * a.hs + l];
    __syncthreads();
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* V = R.V;
    double2* x = X + (int64_t)a.cols[i] * a.n + R.lo;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        double2 acc = x[r];
        for (int l = 0; l < jd; ++l) cfma(acc, V[(int64_t)l * n + r], ys[l]);
        x[r] = acc;
    }
}

__global__ void __launch_bounds__(kT) k_gather_cols(KrylovArgs a, const double2* __restrict__ src,
                                                   double2* __restrict__ dst) {
    const int i = blockIdx.y;
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* s = src + (int64_t)a.cols[i] * a.n + R.lo;
    double2* d = dst + (int64_t)i * a.n + R.lo;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) d[r] = s[r];
}

__global__ void __launch_bounds__(kT) k_sub_cols(KrylovArgs a, const double2* __restrict__ b,
                                                const double2* __restrict__ T, double2* __restrict__ R) {
    const int i = blockIdx.y;
    const Rows rw = rows_of(a, a.cols[i]);
    const int64_t n = rw.len;
    const double2* bc = b + (int64_t)a.cols[i] * a.n + rw.lo;
    const double2* t = T + (int64_t)i * a.n + rw.lo;
    double2* rr = R + (int64_t)i * a.n + rw.lo;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) rr[r] = bc[r] - t[r];
}

__global__ void __launch_bounds__(kT) k_scatter_norm(KrylovArgs a, const double2* Wl, double2* W) {
    const int i = blockIdx.y;
    const Rows R = rows_of(a, a.cols[i]);
    const int64_t n = R.len;
    const double2* src = Wl + (int64_t)i * a.n + R.lo;
    double2* dst = W + (int64_t)a.cols[i] * a.n + R.lo;
    __shared__ double sh[kT / 32];
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        const double2 v = src[r];
        if (dst != src) dst[r] = v;
        acc += v.x * v.x + v.y * v.y;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) a.npart[(int64_t)i * a.nblk_max + blockIdx.x] = s;
}

// init = 1: the first residual (sets beta0); 2: a residual from the inner
// precision, which never ends a column's solve (only a float64-accurate one
// may); 0: a float64-accurate refinement residual; 3: a float64-accurate
// residual updated by the inner-precision image of the cycle's correction
// (the host keeps its accumulated error bound below half the tolerance, and it
// ends a column only when it plus that bound is within the tolerance)
__global__ void k_cycle_end(KrylovArgs a, int k, int nblk, int init) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && init == 0) a.ctr[KR_REFIN] += 1;
    if (i >= k) return;
    const int c = a.cols[i];
    const double bn = sqrt(a.nsq[i]);
    if (!isfinite(bn)) a.ctr[KR_NAN] = 1;
    a.beta[c] = bn;
    if (init == 1) {
        a.beta0[c] = bn;
        a.res[c] = bn > 0.0 ? 1.0 : 0.0;
        a.done[c] = bn > 0.0 ? 0 : 1;
        a.iters[c] = 0;
    } else {
        const double r = a.beta0[c] > 0.0 ? bn / a.beta0[c] : 0.0;
        a.res[c] = r;
        // init = 3: an updated residual; it converges when it plus its error bound
        // (the earlier cycles' and this cycle's eps_low |P^-1 Zs d|) is within the tolerance
        const double ub = init == 3 ? a.ubound[c] + (a.beta0[c] > 0.0 ? a.eps_low * a.enorm[c] / a.beta0[c] : 0.0)
                                    : 0.0;
        const bool conv = (init == 0 && r <= a.tol) || (init == 3 && r + ub <= a.tol);
        a.done[c] = (conv || a.iters[c] >= a.maxit || bn == 0.0) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kT) k_colnorm_partial(KrylovArgs a, const double2* __restrict__ A,
                                                       const int* __restrict__ cols, double* part) {
    const int i = blockIdx.y;
    const Rows R = rows_of(a, cols ? cols[i] : i);
    const int64_t n = R.len;
    const double2* x = A + (int64_t)i * a.n + R.lo;
    __shared__ double sh[kT / 32];
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x; r < n; r += (int64_t)gridDim.x * kT) {
        const double2 v = x[r];
        acc += v.x * v.x + v.y * v.y;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = s;
}

__global__ void k_colnorm_final(const double* part, int nblk, int k, const int* cols, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)i * nblk + b];
    out[cols ? cols[i] : i] = sqrt(s);
}

int slot_threads(int k) { return std::max(32, (k + 31) / 32 * 32); }

}  // namespace

int kr_nblk(int64_t n, int k, int n_sm) {
    const int64_t want = ((int64_t)n_sm * 8 + k - 1) / k;       // ~8 CTAs per SM in total
    const int64_t cap = (n + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

int kr_nchunk(int64_t n, int k, int m, int n_sm) {
    const int groups = std::max(1, std::min(4, (m + kCG - 1) / kCG));  // column groups live on average
    const int64_t want = ((int64_t)n_sm * 8 + (int64_t)k * groups - 1) / ((int64_t)k * groups);
    const int64_t cap = (n + 4 * kT - 1) / (4 * kT);
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

void kr_cycle_start(const KrylovArgs& a, int k, cudaStream_t s) {
    k_cycle_start<<<(k + 255) / 256, 256, 0, s>>>(a, k);
    VIE_CHECK_LAUNCH();
}

void kr_gather(const KrylovArgs& a, const double2* W, void* Xg, bool c64, int k, int nblk, cudaStream_t s) {
    dim3 grid(nblk, k);
    if (a.df) {
        if (!c64) fail(VIE_ERR_STATE, "a double-float basis feeds float32 applies");
        k_gather_df<<<grid, kT, 0, s>>>(a, W, static_cast<float2*>(Xg));
    } else if (c64) {
        k_gather<float2><<<grid, kT, 0, s>>>(a, W, static_cast<float2*>(Xg));
    } else {
        k_gather<double2><<<grid, kT, 0, s>>>(a, W, static_cast<double2*>(Xg));
    }
    VIE_CHECK_LAUNCH();
}

void kr_project(const KrylovArgs& a, const void* Y, bool c64, int pass, int k, int nchunk, int nblk, cudaStream_t s) {
    const int ncg = (a.m + kCG - 1) / kCG;
    dim3 gd(nchunk, ncg, k);
    if (pass == 1) {
        if (a.df) k_mdot_df<true><<<gd, kT, 0, s>>>(a, static_cast<const float2*>(Y));
        else if (c64) k_mdot<float2, true><<<gd, kT, 0, s>>>(a, static_cast<const float2*>(Y));
        else k_mdot<double2, true><<<gd, kT, 0, s>>>(a, static_cast<const double2*>(Y));
        VIE_CHECK_LAUNCH();
        k_reduce<true><<<k, kT, 0, s>>>(a, nchunk);
        VIE_CHECK_LAUNCH();
        if (a.df) k_maxpy_df<false><<<dim3(nblk, k), kT, 0, s>>>(a);
        else k_maxpy<false><<<dim3(nblk, k), kT, 0, s>>>(a);
        VIE_CHECK_LAUNCH();
    } else {
        if (a.df) k_mdot_df<false><<<gd, kT, 0, s>>>(a, nullptr);  // returns at once where pass 2 is not needed
        else k_mdot<double2, false><<<gd, kT, 0, s>>>(a, nullptr);
        VIE_CHECK_LAUNCH();
        k_reduce<false><<<k, kT, 0, s>>>(a, nchunk);
        VIE_CHECK_LAUNCH();
        if (a.df) k_maxpy_df<true><<<dim3(nblk, k), kT, 0, s>>>(a);
        else k_maxpy<true><<<dim3(nblk, k), kT, 0, s>>>(a);
        VIE_CHECK_LAUNCH();
        k_nsq<<<k, kT, 0, s>>>(a, nblk, 1);
        VIE_CHECK_LAUNCH();
    }
}

void kr_givens(const KrylovArgs& a, int k, int nblk, cudaGraphConditionalHandle hnd, int use_handle, cudaStream_t s) {
    if (k > 1024) fail(VIE_ERR_INVALID_ARG, "more than 1024 right-hand sides in one solve");
    k_givens<<<1, slot_threads(k), 0, s>>>(a, k, nblk, hnd, use_handle);
    VIE_CHECK_LAUNCH();
}

void kr_update(const KrylovArgs& a, double2* X, int k, int nblk, cudaStream_t s, float2* D) {
    k_backsub<<<(k + 63) / 64, 64, 0, s>>>(a, k);
    VIE_CHECK_LAUNCH();
    if (a.df) k_xupdate_df<<<dim3(nblk, k), kT, 0, s>>>(a, X, D);
    else if (D) fail(VIE_ERR_STATE, "the correction output needs the double-float basis");
    else k_xupdate<<<dim3(nblk, k), kT, 0, s>>>(a, X);
    VIE_CHECK_LAUNCH();
}

__global__ void k_rnorm_from_nsq(KrylovArgs a, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) a.rnorm[a.cols[i]] = sqrt(a.nsq[i]);
}

void kr_rnorm_from_partials(const KrylovArgs& a, int k, int nblk, cudaStream_t s) {
    k_nsq<<<k, kT, 0, s>>>(a, nblk, 0);
    VIE_CHECK_LAUNCH();
    k_rnorm_from_nsq<<<(k + 255) / 256, 256, 0, s>>>(a, k);
    VIE_CHECK_LAUNCH();
}

void kr_sub_scatter_norm(const KrylovArgs& a, const double2* E, double2* Wf, int k, int nblk, cudaStream_t s) {
    if (nblk > a.nblk_max) fail(VIE_ERR_STATE, "norm partials exceed their buffer");
    k_sub_scatter_norm<<<dim3(nblk, k), kT, 0, s>>>(a, E, Wf);
    VIE_CHECK_LAUNCH();
}

void kr_gather_cols(const KrylovArgs& a, const double2* src, double2* dst, int k, int nblk, cudaStream_t s) {
    k_gather_cols<<<dim3(nblk, k), kT, 0, s>>>(a, src, dst);
    VIE_CHECK_LAUNCH();
}

void kr_sub_cols(const KrylovArgs& a, const double2* b, const double2* T, double2* R, int k, int nblk,
                 cudaStream_t s) {
    k_sub_cols<<<dim3(nblk, k), kT, 0, s>>>(a, b, T, R);
    VIE_CHECK_LAUNCH();
}

void kr_scatter_norm(const KrylovArgs& a, const double2* Wl, double2* W, int k, int nblk, cudaStream_t s) {
    if (nblk > a.nblk_max) fail(VIE_ERR_STATE, "norm partials exceed their buffer");
    k_scatter_norm<<<dim3(nblk, k), kT, 0, s>>>(a, Wl, W);
    VIE_CHECK_LAUNCH();
}

void kr_cycle_end(const KrylovArgs& a, int k, int nblk, int init, cudaStream_t s) {
    k_nsq<<<k, kT, 0, s>>>(a, nblk, 0);
    VIE_CHECK_LAUNCH();
    k_cycle_end<<<(k + 255) / 256, 256, 0, s>>>(a, k, nblk, init);
    VIE_CHECK_LAUNCH();
}

void kr_colnorms(const KrylovArgs& a, const double2* A, int k, int nblk, const int* cols, double* d_part,
                 double* d_out, cudaStream_t s) {
    k_colnorm_partial<<<dim3(nblk, k), kT, 0, s>>>(a, A, cols, d_part);
    VIE_CHECK_LAUNCH();
    k_colnorm_final<<<(k + 255) / 256, 256, 0, s>>>(d_part, nblk, k, cols, d_out);
    VIE_CHECK_LAUNCH();
}

}  // namespace vie
