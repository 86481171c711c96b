// QR-recursive compression of the far blocks (paper Sec. 5.2, eq. eq_02;
// Sec. 5.3): each far block A (m x n) is replaced by Q (m x r, orthonormal
// columns) and R = Q^H A (r x n) such that ||A - Q R||_F <= tol ||A||_F.
//
// The paper does not say how its QR factors are computed for large blocks
// (it builds them with a cross approximation, Sec. 6.5; that builder is in
// cross.cu and runs from the same batches).  Here a batch of equally sized
// blocks is formed on the device (complex float32 blocks from float64
// quadrature tables) and compressed together with a blocked adaptive
// randomised range finder:
//   Y = A Omega (Gaussian test matrix), project Y against the current basis
//   (classical Gram-Schmidt), estimate the residual energy
//   ||(I - Q Q^H) A||_F^2 ~ ||Y||_F^2 / s from the projected block, stop when
//   the estimate is below (tol / 3)^2 ||A||_F^2, else orthonormalise the block
//   (Cholesky QR twice, the first Gram matrix accumulated to ~48 bits, a
//   second Gram-Schmidt pass between the two) and append it.
// The factor-of-3 margin makes a violation of the bound improbable for the
// 32-column estimator used here (a chi-square tail below 1/9 of its mean).
// Plain GEMMs go to cuBLAS; the Gram, Cholesky, triangular product, norms,
// random numbers and the column compaction are this file's kernels.
//
// Reciprocity: between two different atoms the quadrature rule is symmetric,
// so the block (J, I) is the transpose of the block (I, J).  Only one block of
// each mirror pair is formed and compressed; its mirror stores the transposed
// factors, Q' = R^T (n x r) and R' = Q^T (r x m), whose product carries exactly
// the same error.  (Q' is then not orthonormal; the apply does not need it.)
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <array>
#include <map>

#include <cuda_bf16.h>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

constexpr int kChunk = 32;    // columns orthonormalised at a time
constexpr int kRankCap = 8192; // largest rank a block may take (larger: error)
// A batch first reserves basis room for a quarter of its blocks' smaller
// dimension, at least kRankTry (the basis buffers and the batch size scale with
// the room); a block that needs more sends its batch back for a second pass
// with room for kRankCap.
constexpr int kRankTry = 2048;
// the first pass's room for blocks of rfull = min(m, n), or VIE_TEST_RANK_TRY
// (a test sets it low to run the second pass)
static int rank_try(int rfull) {
    if (const char* e = std::getenv("VIE_TEST_RANK_TRY")) {
        const int v = std::atoi(e);
        if (v > 0) return std::min(v, kRankCap);
    }
    return std::min(kRankCap, std::max(kRankTry, rfull / 4));
}

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// complex Gaussian with E|w|^2 = 1 (Box-Muller on two 53-bit uniforms)
template <class T2>
__global__ void k_gauss(T2* W, int64_t count, uint64_t seed) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    uint64_t a = splitmix64(seed ^ (uint64_t)(2 * t));
    uint64_t b = splitmix64(seed ^ (uint64_t)(2 * t + 1));
    double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    double r = sqrt(-log(u1));                                    // sqrt(-2 ln u) / sqrt(2)
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    W[t] = mk(decltype(W[0].x)(r * c), decltype(W[0].x)(r * s));
}

// per-batch-entry sum of |x|^2 over `len` contiguous elements (stride between entries)
template <class T2>
__global__ void k_sumsq_partial(const T2* X, int64_t len, int64_t stride, int nchunk, double* part) {
    int b = blockIdx.y, c = blockIdx.x;
    int64_t per = (len + nchunk - 1) / nchunk;
    int64_t lo = c * per, hi = min(len, lo + per);
    const T2* x = X + b * stride;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double re = x[i].x, im = x[i].y;
        acc += re * re + im * im;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)b * nchunk + c] = red[0];
}
__global__ void k_reduce_rows(const double* part, int nchunk, int nb, double* out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(size_t)b * nchunk + c];
    out[b] = s;
}

// partial Gram matrices G = Y^H Y (kChunk x kChunk) over row chunks,
// accumulated in ACC (double2 for a general block; float2 is enough once the
// block is close to orthonormal), stored as double2
template <class T2, class ACC>
__global__ void k_gram_partial(const T2* Y, int m, int64_t stride, int nchunk, double2* part, const int* active) {
    const int b = blockIdx.y, c = blockIdx.x;
    if (!active[b]) return;
    const int per = (m + nchunk - 1) / nchunk;
    const int lo = c * per, hi = min(m, lo + per);
    const T2* y = Y + b * stride;
    using R = decltype(ACC().x);
    __shared__ ACC rows[64][kChunk + 1];
    const int i = threadIdx.x % kChunk, j = threadIdx.x / kChunk;  // 1024 threads
    ACC acc = mk(R(0), R(0));
    const bool upper = i <= j;  // Hermitian: the reduce mirrors the lower triangle
    for (int r0 = lo; r0 < hi; r0 += 64) {
        for (int e = threadIdx.x; e < 64 * kChunk; e += blockDim.x) {
            int rr = e % 64, cc = e / 64;
            int r = r0 + rr;
            rows[rr][cc] = r < hi ? cvt<ACC>(y[r + (int64_t)cc * m]) : mk(R(0), R(0));
        }
        __syncthreads();
        int nr = min(64, hi - r0);
        if (upper)
            for (int rr = 0; rr < nr; ++rr) cfmac(acc, rows[rr][i], rows[rr][j]);
        __syncthreads();
    }
    part[((size_t)b * nchunk + c) * kChunk * kChunk + i + j * kChunk] = cvt<double2>(acc);
}
// Atom-pair blocks are formed once per distinct (types, displacement) and
// placed into every far block that holds that pair: job j copies the np x np
// block `src[j]` (ld np) to rows row_off, columns col_off of its block.
struct PlaceJob {
    int dst, row_off, col_off, src;
};
// With `planes` (float32 blocks only) the destination is written directly in
// the split bf16 layout described below (ld = block height).
template <class T2>
__global__ void k_place_pairs(const PlaceJob* __restrict__ jobs, const T2* __restrict__ ublk, int np,
                              T2* const* __restrict__ dst, int64_t ld, int planes) {
    const PlaceJob jb = jobs[blockIdx.y];
    const T2* src = ublk + (int64_t)jb.src * np * np;
    const int64_t total = (int64_t)np * np;
    if (planes) {
        __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(dst[jb.dst]);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int c = (int)(e / np), r = (int)(e - (int64_t)c * np);
            const T2 v = src[e];
            __nv_bfloat16* col = base + (int64_t)(jb.col_off + c) * 4 * ld + jb.row_off + r;
            const float x = (float)v.x, y = (float)v.y;
            const __nv_bfloat16 xh = __float2bfloat16_rn(x), yh = __float2bfloat16_rn(y);
            col[0] = xh;
            col[ld] = yh;
            col[2 * ld] = __float2bfloat16_rn(x - __bfloat162float(xh));
            col[3 * ld] = __float2bfloat16_rn(y - __bfloat162float(yh));
        }
        return;
    }
    T2* out = dst[jb.dst] + jb.row_off + (int64_t)jb.col_off * ld;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / np), r = (int)(e - (int64_t)c * np);
        out[r + (int64_t)c * ld] = src[e];
    }
}
__global__ void k_gather_norms(const PlaceJob* __restrict__ jobs, int n, const double* __restrict__ unorm,
                               double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = unorm[jobs[j].src];
}

// The first Gram of the float32 compressor in double-float arithmetic on the
// float32 pipes (this GPU's float64 rate is a small fraction of its float32
// rate): the float32 inputs are exact, each product is formed exactly with an
// FMA (two-product) and each addition keeps its error (two-sum), ~48 bits as
// the float64 version above gives to within its own rounding.
__device__ __forceinline__ void df_prod_add(float& h, float& l, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float sum = __fadd_rn(h, p);
    const float bv = __fsub_rn(sum, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bv)), __fsub_rn(p, bv));
    h = sum;
    l = __fadd_rn(l, __fadd_rn(err, e));
}
__global__ void k_gram_partial_df(const float2* Y, int m, int64_t stride, int nchunk, double2* part,
                                  const int* active) {
    const int b = blockIdx.y, c = blockIdx.x;
    if (!active[b]) return;
    const int per = (m + nchunk - 1) / nchunk;
    const int lo = c * per, hi = min(m, lo + per);
    const float2* y = Y + b * stride;
    __shared__ float2 rows[64][kChunk + 1];
    const int i = threadIdx.x % kChunk, j = threadIdx.x / kChunk;  // 1024 threads
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const bool upper = i <= j;  // Hermitian: the reduce mirrors the lower triangle
    for (int r0 = lo; r0 < hi; r0 += 64) {
        for (int e = threadIdx.x; e < 64 * kChunk; e += blockDim.x) {
            int rr = e % 64, cc = e / 64;
            int r = r0 + rr;
            rows[rr][cc] = r < hi ? y[r + (int64_t)cc * m] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        int nr = min(64, hi - r0);
        if (upper)
            for (int rr = 0; rr < nr; ++rr) {
                const float2 a = rows[rr][i], v = rows[rr][j];  // conj(a) v
                df_prod_add(rh, rl, a.x, v.x);
                df_prod_add(rh, rl, a.y, v.y);
                df_prod_add(ih, il, a.x, v.y);
                df_prod_add(ih, il, -a.y, v.x);
            }
        __syncthreads();
    }
    part[((size_t)b * nchunk + c) * kChunk * kChunk + i + j * kChunk] =
        make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

__global__ void k_gram_reduce(const double2* part, int nchunk, double2* G, const int* active) {
    const int b = blockIdx.x;
    if (!active[b]) return;
    const int e = threadIdx.x;  // kChunk^2 threads
    const int i = e % kChunk, j = e / kChunk;
    if (i > j) return;
    double2 s = make_double2(0, 0);
    for (int c = 0; c < nchunk; ++c) s += part[((size_t)b * nchunk + c) * kChunk * kChunk + e];
    G[(size_t)b * kChunk * kChunk + e] = s;
    G[(size_t)b * kChunk * kChunk + j + i * kChunk] = make_double2(s.x, -s.y);
}

// Cholesky G = L L^H (float64, one block per batch entry) and Minv = L^-H
// (upper triangular) so that Y Minv has orthonormal columns.  A pivot below
// 1e-8 of the largest diagonal (a column norm below 1e-4 of the largest after
// the earlier ones are removed) marks the column dead (zero in Minv); what it
// held stays in the residual and is picked up by a later sketch.
template <class T2>
__global__ void __launch_bounds__(kChunk * kChunk) k_chol(const double2* G, T2* Minv, const int* active,
                                                          unsigned char* alive, int rcap, const int* rbase) {
    const int b = blockIdx.x;
    if (!active[b]) return;
    __shared__ double2 L[kChunk][kChunk + 1];
    __shared__ double2 X[kChunk][kChunk + 1];
    __shared__ int dead[kChunk];
    __shared__ double gmax;
    const int tx = threadIdx.x, ty = threadIdx.y;  // column, row
    L[ty][tx] = G[(size_t)b * kChunk * kChunk + ty + tx * kChunk];
    X[ty][tx] = make_double2(ty == tx ? 1.0 : 0.0, 0.0);
    if (ty == 0) dead[tx] = 0;
    __syncthreads();
    if (ty == 0) {
        double v = L[tx][tx].x;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (tx == 0) gmax = v;
    }
    __syncthreads();
    // right-looking Cholesky: one column per step, the trailing update in
    // parallel.  One thread takes the pivot's square root and reciprocal (this
    // GPU's float64 divide and square root are slow); the column is scaled by
    // the reciprocal.
    __shared__ double pinv[kChunk];
    for (int k = 0; k < kChunk; ++k) {
        if (tx == k && ty == k) {
            const double d = L[k][k].x;
            const bool dk = !(d > 1e-8 * gmax) || gmax <= 0.0;
            const double sq = dk ? 1.0 : sqrt(d);
            pinv[k] = dk ? 0.0 : 1.0 / sq;
            L[k][k] = make_double2(sq, 0.0);
            dead[k] = dk;
        }
        __syncthreads();
        if (tx == k && ty > k) {
            const double2 v = L[ty][k];
            L[ty][k] = dead[k] ? make_double2(0, 0) : make_double2(v.x * pinv[k], v.y * pinv[k]);
        }
        __syncthreads();
        if (ty > k && tx > k && tx <= ty) {
            // L[i][j] -= L[i][k] conj(L[j][k])
            double2 a = L[ty][k], c = L[tx][k];
            L[ty][tx].x -= a.x * c.x + a.y * c.y;
            L[ty][tx].y -= a.y * c.x - a.x * c.y;
        }
        __syncthreads();
    }
    // X = L^-1 by forward substitution, all columns at once; X is lower
    // triangular, so column tx only changes from step tx on.  A dead pivot has
    // L[j][j] = 1 and a zero column below it.
    for (int j = 0; j < kChunk; ++j) {
        if (ty == j && tx <= j && !dead[j]) {
            const double r = pinv[j];
            X[j][tx] = make_double2(X[j][tx].x * r, X[j][tx].y * r);
        }
        __syncthreads();
        if (ty > j && tx <= j) {
            double2 a = L[ty][j], x = X[j][tx];
            X[ty][tx].x -= a.x * x.x - a.y * x.y;
            X[ty][tx].y -= a.x * x.y + a.y * x.x;
        }
        __syncthreads();
    }
    // Minv = (L^-1)^H: Minv[i][j] = conj(X[j][i]); dead columns and rows zeroed
    using R = decltype(Minv[0].x);
    const double2 v = X[tx][ty];
    const bool z = dead[ty] || dead[tx];
    Minv[(size_t)b * kChunk * kChunk + ty + tx * kChunk] = z ? mk(R(0), R(0)) : mk(R(v.x), R(-v.y));
    if (tx == 0 && alive && dead[ty]) alive[(size_t)b * rcap + rbase[b] + ty] = 0;
}

// OUT[:, j] = sum_i Y[:, i] Minv[i][j] for active entries (row per thread)
template <class T2>
__global__ void k_trmul(const T2* Y, int m, int64_t ystride, const T2* Minv, const int* active, T2* OUT,
                        int64_t ostride, int64_t ld_out, const int* col0) {
    const int b = blockIdx.y;
    if (!active[b]) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ T2 M[kChunk][kChunk];
    for (int e = threadIdx.x; e < kChunk * kChunk; e += blockDim.x) M[e % kChunk][e / kChunk] = Minv[(size_t)b * kChunk * kChunk + e];
    __syncthreads();
    if (r >= m) return;
    using R = decltype(Y[0].x);
    T2 y[kChunk];
    for (int i = 0; i < kChunk; ++i) y[i] = Y[b * ystride + r + (int64_t)i * m];
    T2* o = OUT + b * ostride + (col0 ? (int64_t)col0[b] * ld_out : 0) + r;
    for (int j = 0; j < kChunk; ++j) {
        T2 acc = mk(R(0), R(0));
        for (int i = 0; i <= j; ++i) cfma(acc, y[i], M[i][j]);
        o[(int64_t)j * ld_out] = acc;
    }
}

// dst = conj(src)
template <class T2>
__global__ void k_conj_copy(const T2* src, T2* dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T2 v = src[i];
        v.y = -v.y;
        dst[i] = v;
    }
}

// copy live columns into the factor store: dst[k] <- src[:, col[k]]
template <class T2>
__global__ void k_gather_cols(const T2* src, int64_t rows, const long long* src_off, const long long* dst_off,
                              T2* dst_base, const T2* src_base) {
    const int k = blockIdx.y;
    const T2* s = src_base + src_off[k];
    T2* d = dst_base + dst_off[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

// ------------------------------------------- split bf16 operands (float32 path)
// The sketch Y = A Omega and the projection R^H = A^H Q run as real bf16
// GEMMs with float32 accumulation on split operands: every float32 value x is
// carried as hi = bf16(x) and lo = bf16(x - hi) (16 significant bits: each
// rounding to bf16 is within 2^-8 relative, so |x - hi - lo| <= 2^-16 |x|).
// Omega is drawn in bf16 (a Gaussian rounded to bf16 is as good a test
// matrix), so the sketch needs hi and lo of A only (two products); R^H takes
// hi.hi + hi.lo + lo.hi.  Both errors stay below ~1e-5 relative, inside the
// tol / 3 margin of the range finder at the float32 tolerances (1e-4 ..
// 1e-3); the Gram-Schmidt projections keep float32 accuracy.
//
// Layout of a formed block after the split: column j of A (8 m bytes as
// complex float32) holds, in the same bytes, [Re hi | Im hi | Re lo | Im lo],
// m bf16 each.  Read with ld = m it is an m x 4n matrix (plane p of column j
// is column 4 j + p); read with ld = 4 m it is a 4 m x n matrix.
using bf16 = __nv_bfloat16;

__device__ __forceinline__ void split_bf16(float x, bf16& hi, bf16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// column per CTA (m even): the whole column is read into shared memory
// before its bytes are rewritten as the four planes, two rows at a time
__global__ void k_split_cols(float2* A, int m) {
    extern __shared__ float4 col4[];
    float2* c = A + (int64_t)blockIdx.x * m;
    const int h = m / 2;
    const float4* c4 = reinterpret_cast<const float4*>(c);
#pragma unroll 4
    for (int i = threadIdx.x; i < h; i += blockDim.x) col4[i] = c4[i];
    __syncthreads();
    __nv_bfloat162* p = reinterpret_cast<__nv_bfloat162*>(c);
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const float4 v = col4[i];  // rows 2i (x, y) and 2i + 1 (z, w)
        bf16 rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
        split_bf16(v.x, rh0, rl0);
        split_bf16(v.y, ih0, il0);
        split_bf16(v.z, rh1, rl1);
        split_bf16(v.w, ih1, il1);
        p[i] = __halves2bfloat162(rh0, rh1);
        p[h + i] = __halves2bfloat162(ih0, ih1);
        p[2 * h + i] = __halves2bfloat162(rl0, rl1);
        p[3 * h + i] = __halves2bfloat162(il0, il1);
    }
}

// The real 4n x 2s right-hand side B of the sketch (ld 4n) from a complex
// Gaussian W (n x s) rounded to bf16: rows 4j and 4j+2 hold [Re W_j, Im W_j],
// rows 4j+1 and 4j+3 hold [-Im W_j, Re W_j], so that with A read as m x 4n
// the product is [Re(A W) | Im(A W)] (m x 2s).
__global__ void k_gauss_bf16(bf16* B, int n, int s, uint64_t seed) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * s) return;
    const int j = (int)(t % n), c = (int)(t / n);
    uint64_t a = splitmix64(seed ^ (uint64_t)(2 * t));
    uint64_t b = splitmix64(seed ^ (uint64_t)(2 * t + 1));
    double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    double r = sqrt(-log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    const bf16 wr = __float2bfloat16_rn((float)(r * cs)), wi = __float2bfloat16_rn((float)(r * sn));
    const bf16 nwi = __hneg(wi);
    const int64_t ld = 4 * (int64_t)n, c0 = (int64_t)c * ld, c1 = (int64_t)(s + c) * ld;
    for (int h = 0; h < 2; ++h) {
        const int64_t row = 4 * (int64_t)j + 2 * h;
        B[row + c0] = wr;
        B[row + c1] = wi;
        B[row + 1 + c0] = nwi;
        B[row + 1 + c1] = wr;
    }
}

// Right-hand sides of R^H = A^H Q from Q (m x r complex, ld m):
// Bh (4m x 2r, ld 4m): column c = [Re Q; Im Q; Re Q; Im Q]_c (hi parts),
// column r + c = [Im Q; -Re Q; Im Q; -Re Q]_c; Bl (2m x 2r, ld 2m): the lo
// parts of the first halves.  With A read as 4m x n, A^T Bh + A_hi^T Bl =
// [Re R^H | Im R^H] (n x 2r).
__global__ void k_split_q(const float2* Q, int m, int r, int64_t qstride, bf16* Bh, int64_t hstride, bf16* Bl,
                          int64_t lstride) {
    const int b = blockIdx.y;
    const float2* q = Q + b * qstride;
    bf16* bh = Bh + b * hstride;
    bf16* bl = Bl + b * lstride;
    const int64_t total = (int64_t)m * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / m), i = (int)(e - (int64_t)c * m);
        const float2 v = q[i + (int64_t)c * m];
        bf16 rh, rl, ih, il;
        split_bf16(v.x, rh, rl);
        split_bf16(v.y, ih, il);
        const bf16 nrh = __hneg(rh), nrl = __hneg(rl);
        bf16* h0 = bh + (int64_t)c * 4 * m;
        bf16* h1 = bh + (int64_t)(r + c) * 4 * m;
        h0[i] = rh; h0[m + i] = ih; h0[2 * m + i] = rh; h0[3 * m + i] = ih;
        h1[i] = ih; h1[m + i] = nrh; h1[2 * m + i] = ih; h1[3 * m + i] = nrh;
        bf16* l0 = bl + (int64_t)c * 2 * m;
        bf16* l1 = bl + (int64_t)(r + c) * 2 * m;
        l0[i] = rl; l0[m + i] = il;
        l1[i] = il; l1[m + i] = nrl;
    }
}

// out[list[y]] (rows x cols complex, ld rows) from F[list[y]] (rows x 2 cols
// real, ld rows: real parts then imaginary parts)
__global__ void k_join_planes(const float* F, int rows, int cols, int64_t fstride, float2* out, int64_t ostride,
                              const int* list) {
    const int b = list ? list[blockIdx.y] : (int)blockIdx.y;
    const float* f = F + b * fstride;
    float2* o = out + b * ostride;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        o[e] = make_float2(f[e], f[e + total]);
}

void gemm_bf16(cublasHandle_t h, cublasOperation_t ta, int m, int n, int k, const bf16* A, int lda, long long sa,
               const bf16* B, int ldb, long long sb, float beta, float* C, int ldc, long long sc, int batch) {
    const float one = 1.f;
    if (batch == 1)
        VIE_BLAS(cublasGemmEx(h, ta, CUBLAS_OP_N, m, n, k, &one, A, CUDA_R_16BF, lda, B, CUDA_R_16BF, ldb, &beta, C,
                              CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT));
    else
        VIE_BLAS(cublasGemmStridedBatchedEx(h, ta, CUBLAS_OP_N, m, n, k, &one, A, CUDA_R_16BF, lda, sa, B, CUDA_R_16BF,
                                            ldb, sb, &beta, C, CUDA_R_32F, ldc, sc, batch, CUBLAS_COMPUTE_32F,
                                            CUBLAS_GEMM_DEFAULT));
}

// largest block height whose column fits the split kernel's shared memory
constexpr int kSplitMaxRows = 200 * 1024 / 8;

// ------------------------------------------------------------------ cuBLAS
template <class T> struct Blas;
template <> struct Blas<float> {
    using T2 = float2;
    static void gemm_ptr(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                         const T2* const* A, int lda, const T2* const* B, int ldb, T2 beta, T2* const* C, int ldc,
                         int batch) {
        VIE_BLAS(cublasCgemmBatched(h, ta, tb, m, n, k, (const cuComplex*)&alpha, (const cuComplex* const*)A, lda,
                                    (const cuComplex* const*)B, ldb, (const cuComplex*)&beta, (cuComplex* const*)C,
                                    ldc, batch));
    }
    static void gemm1(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                      const T2* A, int lda, const T2* B, int ldb, T2 beta, T2* C, int ldc) {
        VIE_BLAS(cublasCgemm(h, ta, tb, m, n, k, (const cuComplex*)&alpha, (const cuComplex*)A, lda,
                             (const cuComplex*)B, ldb, (const cuComplex*)&beta, (cuComplex*)C, ldc));
    }
    static void gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                     const T2* A, int lda, long long sa, const T2* B, int ldb, long long sb, T2 beta, T2* C, int ldc,
                     long long sc, int batch) {
        VIE_BLAS(cublasCgemmStridedBatched(h, ta, tb, m, n, k, (const cuComplex*)&alpha, (const cuComplex*)A, lda, sa,
                                           (const cuComplex*)B, ldb, sb, (const cuComplex*)&beta, (cuComplex*)C, ldc,
                                           sc, batch));
    }
};
template <> struct Blas<double> {
    using T2 = double2;
    static void gemm_ptr(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                         const T2* const* A, int lda, const T2* const* B, int ldb, T2 beta, T2* const* C, int ldc,
                         int batch) {
        VIE_BLAS(cublasZgemmBatched(h, ta, tb, m, n, k, (const cuDoubleComplex*)&alpha,
                                    (const cuDoubleComplex* const*)A, lda, (const cuDoubleComplex* const*)B, ldb,
                                    (const cuDoubleComplex*)&beta, (cuDoubleComplex* const*)C, ldc, batch));
    }
    static void gemm1(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                      const T2* A, int lda, const T2* B, int ldb, T2 beta, T2* C, int ldc) {
        VIE_BLAS(cublasZgemm(h, ta, tb, m, n, k, (const cuDoubleComplex*)&alpha, (const cuDoubleComplex*)A, lda,
                             (const cuDoubleComplex*)B, ldb, (const cuDoubleComplex*)&beta, (cuDoubleComplex*)C, ldc));
    }
    static void gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, T2 alpha,
                     const T2* A, int lda, long long sa, const T2* B, int ldb, long long sb, T2 beta, T2* C, int ldc,
                     long long sc, int batch) {
        VIE_BLAS(cublasZgemmStridedBatched(h, ta, tb, m, n, k, (const cuDoubleComplex*)&alpha,
                                           (const cuDoubleComplex*)A, lda, sa, (const cuDoubleComplex*)B, ldb, sb,
                                           (const cuDoubleComplex*)&beta, (cuDoubleComplex*)C, ldc, sc, batch));
    }
};

// ------------------------------------------------------------------ driver
struct BlockFactors {
    int rank = 0;
    int64_t q_off = 0, rh_off = 0;  // into the staging store of its batch
};

template <class T>
struct Compressor {
    using T2 = typename C2<T>::t;
    Op& op;
    double tol;
    cudaStream_t s;
    cublasHandle_t h;
    std::vector<DevBuf> stores;          // staging factor stores (one per batch)
    std::vector<std::pair<int, int64_t>> where;  // per block: (store, offset of Q); R^H follows Q
    std::map<std::tuple<int, int, int>, int> class_rank;  // (level, offsets) -> largest rank seen
    uint64_t seed = 0x5eed0001ull;
    bool cross = false;  // cross approximation with full pivoting instead of the range finder

    Compressor(Op& o, double t) : op(o), tol(t), s(o.ctx->stream), h(o.ctx->blas) {}

    void sumsq(const T2* X, int64_t len, int64_t stride, int nb, double* out, DevBuf& part) {
        int nchunk = (int)std::min<int64_t>(256, std::max<int64_t>(1, len / 65536));
        size_t need = (size_t)nb * nchunk * sizeof(double);
        if (part.bytes < need) part.alloc(need);
        k_sumsq_partial<T2><<<dim3(nchunk, nb), 256, 0, s>>>(X, len, stride, nchunk, part.as<double>());
        VIE_CHECK_LAUNCH();
        k_reduce_rows<<<(nb + 127) / 128, 128, 0, s>>>(part.as<double>(), nchunk, nb, out);
        VIE_CHECK_LAUNCH();
    }

    // Per-block pointers of one chunk's projections, for the listed blocks:
    // [Q_q ...][Y_q ...][C_q ...] (the table is read by the GEMMs in stream order)
    void proj_ptrs(DevBuf& buf, const std::vector<int>& list, T2* Qb, int64_t qs, T2* Yb, int64_t ys, T2* Cbb,
                   int64_t cs) {
        const size_t L = list.size();
        if (L == 0) return;
        std::vector<T2*> hp(3 * L);
        for (size_t i = 0; i < L; ++i) {
            hp[i] = Qb + list[i] * qs;
            hp[L + i] = Yb + list[i] * ys;
            hp[2 * L + i] = Cbb + list[i] * cs;
        }
        VIE_CUDA(cudaMemcpyAsync(buf.p, hp.data(), hp.size() * sizeof(T2*), cudaMemcpyHostToDevice, s));
    }
    // one classical Gram-Schmidt pass of the chunks against their blocks' first K
    // basis columns: C = Q^H Y, Y -= Q C
    void project(const DevBuf& buf, int L, int K, int m, int ldc, int ncol) {
        if (L == 0 || K == 0) return;
        T2* const* p = buf.as<T2* const>();
        const T2 one = mk(T(1), T(0)), zero = mk(T(0), T(0)), mone = mk(T(-1), T(0));
        Blas<T>::gemm_ptr(h, CUBLAS_OP_C, CUBLAS_OP_N, K, ncol, m, one, (const T2* const*)p, m,
                          (const T2* const*)(p + L), m, zero, p + 2 * L, ldc, L);
        Blas<T>::gemm_ptr(h, CUBLAS_OP_N, CUBLAS_OP_N, m, ncol, K, mone, (const T2* const*)p, m,
                          (const T2* const*)(p + 2 * L), ldc, one, p + L, m, L);
    }

    double tim[5] = {0, 0, 0, 0, 0};  // form, sketch loop, R, compaction, total
    double mark() {
        if (!op.ctx->verbose) return 0.0;
        VIE_CUDA(cudaStreamSynchronize(s));
        return now_s();
    }

    // atom-pair blocks into dst: complex float32 entries come from float64
    // tables (float32 tables leave noise near the tolerance in far blocks)
    void form(const PairJob* jobs, int n_jobs, void* const* dst, const int64_t* ld, double* norm) {
        if (std::is_same<T, float>::value)
            assemble_pairs_f32_from_f64(op, jobs, n_jobs, dst, ld, s, norm);
        else
            assemble_pairs<T>(op, jobs, n_jobs, dst, ld, s, norm);
    }

    // The Galerkin block of two distinct atoms depends only on their types and
    // displacement.  Unless sharing is off, each distinct (types, displacement)
    // among the jobs is formed once into a scratch block and copied to every
    // position that holds it; otherwise every job is formed in place.
    // norm (device, per job): squared Frobenius norm of the job's block.
    // With `planes` the copies are written in the split bf16 layout; returns
    // whether they were (the blocks formed in place are complex float32).
    bool form_pairs(const std::vector<PairJob>& jobs, const std::vector<void*>& dst, const std::vector<int64_t>& ld,
                    double* norm, bool planes) {
        const int np = op.np;
        if (!op.ctx->no_sharing) {
            double span = 0.0;
            for (double c : op.centres) span = std::max(span, std::abs(c));
            const double qu = 1e-9 * std::max(span, 1e-30);
            std::map<std::array<long long, 5>, int> uid;
            std::vector<PairJob> ujobs;
            std::vector<PlaceJob> place(jobs.size());
            for (size_t j = 0; j < jobs.size(); ++j) {
                const int a = jobs[j].a, b = jobs[j].b;
                std::array<long long, 5> key{op.types[a], op.types[b],
                                             std::llround((op.centres[3 * b] - op.centres[3 * a]) / qu),
                                             std::llround((op.centres[3 * b + 1] - op.centres[3 * a + 1]) / qu),
                                             std::llround((op.centres[3 * b + 2] - op.centres[3 * a + 2]) / qu)};
                auto it = uid.find(key);
                int u;
                if (it == uid.end()) {
                    u = (int)ujobs.size();
                    uid.emplace(key, u);
                    ujobs.push_back(PairJob{a, b, u, 0, 0});
                } else {
                    u = it->second;
                }
                place[j] = PlaceJob{jobs[j].dst, jobs[j].row_off, jobs[j].col_off, u};
            }
            const size_t ubytes = ujobs.size() * (size_t)np * np * sizeof(T2);
            // worth it when pairs repeat, and when the distinct blocks fit a modest scratch
            if (ujobs.size() * 2 <= jobs.size() && ubytes <= ((size_t)16 << 30)) {
                DevBuf ublk(ubytes), unorm(ujobs.size() * sizeof(double));
                std::vector<void*> udst(ujobs.size());
                std::vector<int64_t> uld(ujobs.size(), np);
                for (size_t u = 0; u < ujobs.size(); ++u) udst[u] = ublk.as<T2>() + u * (size_t)np * np;
                DevBuf dj, dd, dl, dp, dq;
                upload(dj, ujobs);
                upload(dd, udst);
                upload(dl, uld);
                form(dj.as<PairJob>(), (int)ujobs.size(), dd.as<void* const>(), dl.as<int64_t>(),
                                  unorm.as<double>());
                upload(dp, place);
                upload(dq, dst);
                // every destination block of one batch has the same leading dimension
                for (size_t j0 = 0; j0 < place.size(); j0 += 65535) {
                    const int cnt = (int)std::min<size_t>(65535, place.size() - j0);
                    k_place_pairs<T2><<<dim3(std::min(64, (np * np + 255) / 256), cnt), 256, 0, s>>>(
                        dp.as<PlaceJob>() + j0, ublk.as<T2>(), np, dq.as<T2* const>(), ld[0], planes ? 1 : 0);
                    VIE_CHECK_LAUNCH();
                }
                k_gather_norms<<<((int)place.size() + 255) / 256, 256, 0, s>>>(dp.as<PlaceJob>(), (int)place.size(),
                                                                           unorm.as<double>(), norm);
                VIE_CHECK_LAUNCH();
                VIE_CUDA(cudaStreamSynchronize(s));  // scratch goes out of scope
                return planes;
            }
        }
        DevBuf dj, dd, dl;
        upload(dj, jobs);
        upload(dd, dst);
        upload(dl, ld);
        form(dj.as<PairJob>(), (int)jobs.size(), dd.as<void* const>(), dl.as<int64_t>(), norm);
        return false;
    }

    // Copy the factors of one batch into a new staging store: for block q of
    // ids, the live columns j < r[q] of Q (Q + q qs + j m, m rows) and of R^H
    // (RH + q rs + j n, n rows), where alive (per block alive_stride flags,
    // null: every column) marks the live ones.  Sets the blocks' ranks and
    // staging places and returns the ranks.
    std::vector<int> stash(const std::vector<int>& ids, int m, int n, const DevBuf& Q, int64_t qs, const DevBuf& RH,
                           int64_t rs, const std::vector<int>& r, const unsigned char* alive, int64_t alive_stride) {
        const int nb = (int)ids.size();
        auto live = [&](int q, int j) { return alive == nullptr || alive[(size_t)q * alive_stride + j] != 0; };
        std::vector<int> rank(nb, 0);
        int64_t total = 0;
        for (int q = 0; q < nb; ++q) {
            for (int j = 0; j < r[q]; ++j) rank[q] += live(q, j) ? 1 : 0;
            total += (int64_t)rank[q] * (m + n);
            total = (total + 31) / 32 * 32;
        }
        DevBuf store((size_t)std::max<int64_t>(total, 32) * sizeof(T2));
        std::vector<long long> so, dof;  // Q columns then R^H columns
        std::vector<long long> so2, dof2;
        int64_t off = 0;
        int sidx = (int)stores.size();
        for (int q = 0; q < nb; ++q) {
            FarBlock& b = op.blocks[ids[q]];
            b.rank = rank[q];
            where[ids[q]] = {sidx, off};
            int kk = 0;
            for (int j = 0; j < r[q]; ++j) {
                if (!live(q, j)) continue;
                so.push_back((long long)q * qs + (long long)j * m);
                dof.push_back(off + (int64_t)kk * m);
                so2.push_back((long long)q * rs + (long long)j * n);
                dof2.push_back(off + (int64_t)rank[q] * m + (int64_t)kk * n);
                ++kk;
            }
            off += (int64_t)rank[q] * (m + n);
            off = (off + 31) / 32 * 32;
            int& cr = class_rank[{b.level, b.dist, b.dmin}];
            cr = std::max(cr, rank[q]);
        }
        if (!so.empty()) {
            DevBuf a1, a2, a3, a4;
            upload(a1, so);
            upload(a2, dof);
            upload(a3, so2);
            upload(a4, dof2);
            for (size_t c0 = 0; c0 < so.size(); c0 += 65535) {
                int cnt = (int)std::min<size_t>(65535, so.size() - c0);
                k_gather_cols<T2><<<dim3(std::min(64, (m + 255) / 256), cnt), 256, 0, s>>>(
                    nullptr, m, a1.as<long long>() + c0, a2.as<long long>() + c0, store.as<T2>(), Q.as<T2>());
                k_gather_cols<T2><<<dim3(std::min(64, (n + 255) / 256), cnt), 256, 0, s>>>(
                    nullptr, n, a3.as<long long>() + c0, a4.as<long long>() + c0, store.as<T2>(), RH.as<T2>());
                VIE_CHECK_LAUNCH();
            }
            VIE_CUDA(cudaStreamSynchronize(s));
        }
        stores.push_back(std::move(store));
        return rank;
    }

    // compress one batch of equally sized blocks with basis room for `cap`
    // ranks; returns false, having stored nothing, when a block needs more and
    // cap < kRankCap (the caller then runs the batch again with kRankCap)
    bool batch(const std::vector<int>& ids, int s0_hint, int cap = kRankCap) {
        double t0 = mark();
        const int nb = (int)ids.size();
        const FarBlock& b0 = op.blocks[ids[0]];
        const int m = b0.m, n = b0.n, np = op.np;
        const int rfull = std::min(m, n);
        const int rcap = std::min(rfull, std::min(cap, kRankCap));
        const int rcap_pad = ((rcap + kChunk - 1) / kChunk) * kChunk;
        const int64_t mn = (int64_t)m * n;

        // float32 path: the formed blocks become split bf16 planes
        const char* sp = std::getenv("VIE_COMPRESS_SPLIT");
        const bool split = !cross && std::is_same<T, float>::value && m <= kSplitMaxRows && m % 2 == 0 &&
                           !(sp && sp[0] == '0');
        bool in_planes = false;
        // 1. form the blocks (col-major m x n, ld = m) and their squared norms
        DevBuf A((size_t)nb * mn * sizeof(T2)), jobnorm;
        {
            std::vector<PairJob> jobs;
            std::vector<void*> dst(nb);
            std::vector<int64_t> ld(nb, m);
            for (int q = 0; q < nb; ++q) {
                const FarBlock& b = op.blocks[ids[q]];
                dst[q] = A.as<T2>() + (size_t)q * mn;
                for (int i = 0; i < b.nt; ++i)
                    for (int j = 0; j < b.ns; ++j)
                        jobs.push_back(PairJob{op.block_atoms[b.t_off + i], op.block_atoms[b.s_off + j], q, i * np,
                                               j * np});
            }
            jobnorm.alloc(jobs.size() * sizeof(double));
            in_planes = form_pairs(jobs, dst, ld, jobnorm.as<double>(), split);
        }
        double t1 = mark();
        tim[0] += t1 - t0;
        DevBuf part, normA((size_t)nb * sizeof(double)), est((size_t)nb * sizeof(double));
        // ||A||_F^2 of each block: the sum over its (contiguous) atom-pair jobs
        k_reduce_rows<<<(nb + 127) / 128, 128, 0, s>>>(jobnorm.as<double>(), b0.nt * b0.ns, nb, normA.as<double>());
        VIE_CHECK_LAUNCH();
        std::vector<double> hnorm(nb);
        VIE_CUDA(cudaMemcpyAsync(hnorm.data(), normA.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (cross) {
            // 2'. cross approximation with full pivoting: Q = U, R^H = conj(V)
            DevBuf U((size_t)nb * m * rcap_pad * sizeof(T2)), VH((size_t)nb * n * rcap_pad * sizeof(T2));
            std::vector<int> rk;
            const CrossStats cs = cross_full_batch<T2>(A.as<T2>(), nb, m, n, normA.as<double>(), tol, rcap, rfull,
                                                       U.as<T2>(), (int64_t)m * rcap_pad, VH.as<T2>(),
                                                       (int64_t)n * rcap_pad, rk, op.ctx->n_sm, s);
            if (cs.flags & 2) fail(VIE_ERR_NAN, "cross approximation: a far block has non-finite entries");
            if (op.ctx->verbose && (cs.flags & 1)) {
                VIE_CUDA(cudaStreamSynchronize(s));
                for (int q = 0; q < nb; ++q)
                    if (rk[q] >= rcap)
                        fprintf(stderr, "[vie]   level %d block %d (%d x %d): %d crosses leave ||E||/||A|| = %.3e\n",
                                b0.level, ids[q], m, n, rk[q], std::sqrt(cs.resid2[q] / std::max(hnorm[q], 1e-300)));
            }
            if (cs.flags & 1) {
                if (cap < kRankCap) return false;  // again, with room for kRankCap
                fail(VIE_ERR_BREAKDOWN, "far block needs a rank above " + std::to_string(kRankCap) +
                                            " at this tolerance");
            }
            op.cross_bytes += cs.bytes;
            op.t_cross += cs.seconds;
            A.release();
            double t2 = mark();
            tim[1] += t2 - t1;
            stash(ids, m, n, U, (int64_t)m * rcap_pad, VH, (int64_t)n * rcap_pad, rk, nullptr, 0);
            double t4 = mark();
            tim[3] += t4 - t2;
            if (op.ctx->verbose) {
                int rsum = 0, rmx = 0;
                for (int q = 0; q < nb; ++q) { rsum += rk[q]; rmx = std::max(rmx, rk[q]); }
                double rel = 0.0;
                for (int q = 0; q < nb; ++q) rel = std::max(rel, std::sqrt(cs.resid2[q] / std::max(hnorm[q], 1e-300)));
                fprintf(stderr, "[vie]   level %d batch %d x (%d x %d): cross steps %lld mean rank %.1f max %d "
                        "max ||E||/||A|| %.2e | form %.3f cross %.3f (%.0f GB/s) pack %.3f s\n", b0.level, nb, m, n,
                        (long long)cs.passes, (double)rsum / nb, rmx, rel, t1 - t0, t2 - t1,
                        cs.bytes / std::max(cs.seconds, 1e-12) * 1e-9, t4 - t2);
            }
            return true;
        }
        const bf16* Ap = reinterpret_cast<const bf16*>(A.p);
        if (split && !in_planes) {  // formed in place as complex float32: split now
            const size_t smem = (size_t)m * sizeof(float2);
            VIE_CUDA(cudaFuncSetAttribute(k_split_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_split_cols<<<(unsigned)((int64_t)nb * n), 512, smem, s>>>(reinterpret_cast<float2*>(A.p), m);
            VIE_CHECK_LAUNCH();
        }

        // 2. adaptive range finder
        DevBuf Q((size_t)nb * m * rcap_pad * sizeof(T2));
        VIE_CUDA(cudaMemsetAsync(Q.p, 0, Q.bytes, s));
        DevBuf alive((size_t)nb * rcap_pad);
        VIE_CUDA(cudaMemsetAsync(alive.p, 1, alive.bytes, s));
        DevBuf Cb((size_t)nb * rcap_pad * kChunk * sizeof(T2));
        DevBuf gpart, G((size_t)nb * kChunk * kChunk * sizeof(double2)), Minv((size_t)nb * kChunk * kChunk * sizeof(T2));
        DevBuf d_active(nb * sizeof(int)), d_rbase(nb * sizeof(int));
        DevBuf pbuf1((size_t)3 * nb * sizeof(void*)), pbuf2((size_t)3 * nb * sizeof(void*)), Cpan;
        std::vector<int> r(nb, 0), conv(nb, 0);
        // first sketch: the rank prior of this block class (one pass over A), then
        // 32-column passes for the blocks that still need more
        int s0 = std::min(std::max(kChunk, s0_hint), rcap_pad);
        int step = 0;
        const double thr = (tol / 3.0) * (tol / 3.0);
        VIE_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < nb; ++q)
            if (!(hnorm[q] > 0)) conv[q] = 1;  // an all-zero block has rank 0
        while (true) {
            int rmax = *std::max_element(r.begin(), r.end());
            bool all = std::all_of(conv.begin(), conv.end(), [](int c) { return c; });
            if (all) break;
            // later sketches grow with the rank still being found (half of it, 32 to
            // 256 columns): fewer passes over the formed blocks; columns are still
            // orthogonalised and tested 32 at a time, so the ranks do not change
            int rlive = 0;
            for (int q = 0; q < nb; ++q)
                if (!conv[q]) rlive = std::max(rlive, r[q]);
            int scols = step == 0 ? s0 : std::min(256, std::max(kChunk, ((rlive / 2 + kChunk - 1) / kChunk) * kChunk));
            scols = std::min(scols, rcap_pad - rmax);
            if (scols <= 0) {
                // the unconverged blocks fill the reserved room: with room for every
                // column of the block the basis is exact; otherwise run again with
                // more room (or, at kRankCap, give up)
                if (rcap < rfull) {
                    if (cap < kRankCap) return false;
                    fail(VIE_ERR_BREAKDOWN,
                         "far block needs a rank above " + std::to_string(kRankCap) + " at this tolerance");
                }
                for (int q = 0; q < nb; ++q) conv[q] = 1;
                break;
            }
            DevBuf Y((size_t)nb * m * scols * sizeof(T2));
            const uint64_t sseed = seed + 7919ull * step;
            ++step;
            const T2 one = mk(T(1), T(0)), zero = mk(T(0), T(0)), mone = mk(T(-1), T(0));
            if (split) {
                // [Re Y | Im Y] = A (m x 4n planes) B (4n x 2 scols), then joined
                DevBuf Wb((size_t)8 * n * scols * sizeof(bf16)), Yf((size_t)nb * m * 2 * scols * sizeof(float));
                k_gauss_bf16<<<(unsigned)(((int64_t)n * scols + 255) / 256), 256, 0, s>>>(Wb.as<bf16>(), n, scols,
                                                                                          sseed);
                VIE_CHECK_LAUNCH();
                std::vector<int> list;
                for (int q = 0; q < nb; ++q)
                    if (!conv[q]) list.push_back(q);
                const long long fs = 2LL * m * scols;
                if ((int)list.size() == nb) {
                    gemm_bf16(h, CUBLAS_OP_N, m, 2 * scols, 4 * n, Ap, m, 4 * mn, Wb.as<bf16>(), 4 * n, 0, 0.f,
                              Yf.as<float>(), m, fs, nb);
                } else {
                    std::vector<const void*> pa, pb;
                    std::vector<void*> pc;
                    for (int q : list) {
                        pa.push_back(Ap + (size_t)q * 4 * mn);
                        pb.push_back(Wb.p);
                        pc.push_back(Yf.as<float>() + (size_t)q * fs);
                    }
                    DevBuf da, db, dc;
                    upload(da, pa);
                    upload(db, pb);
                    upload(dc, pc);
                    const float f1 = 1.f, f0 = 0.f;
                    VIE_BLAS(cublasGemmBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, 2 * scols, 4 * n, &f1,
                                                 da.as<const void* const>(), CUDA_R_16BF, m, db.as<const void* const>(),
                                                 CUDA_R_16BF, 4 * n, &f0, dc.as<void* const>(), CUDA_R_32F, m,
                                                 (int)list.size(), CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT));
                    VIE_CUDA(cudaStreamSynchronize(s));
                }
                DevBuf dl;
                upload(dl, list);
                k_join_planes<<<dim3((unsigned)std::min<int64_t>(1024, ((int64_t)m * scols + 255) / 256),
                                     (unsigned)list.size()),
                                256, 0, s>>>(Yf.as<float>(), m, scols, fs, reinterpret_cast<float2*>(Y.p),
                                             (int64_t)m * scols, dl.as<int>());
                VIE_CHECK_LAUNCH();
                VIE_CUDA(cudaStreamSynchronize(s));  // Wb, Yf go out of scope
            } else {
              DevBuf W((size_t)n * scols * sizeof(T2));
              k_gauss<T2><<<(unsigned)(((int64_t)n * scols + 255) / 256), 256, 0, s>>>(W.as<T2>(),
                                                                                       (int64_t)n * scols, sseed);
              VIE_CHECK_LAUNCH();
              if (step == 1) {
                Blas<T>::gemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, scols, n, one, A.as<T2>(), m, mn, W.as<T2>(), n, 0, zero,
                              Y.as<T2>(), m, (long long)m * scols, nb);
              } else {
                std::vector<const T2*> pa, pb;
                std::vector<T2*> pc;
                for (int q = 0; q < nb; ++q)
                    if (!conv[q]) {
                        pa.push_back(A.as<T2>() + (size_t)q * mn);
                        pb.push_back(W.as<T2>());
                        pc.push_back(Y.as<T2>() + (size_t)q * m * scols);
                    }
                DevBuf da, db, dc;
                upload(da, pa);
                upload(db, pb);
                upload(dc, pc);
                Blas<T>::gemm_ptr(h, CUBLAS_OP_N, CUBLAS_OP_N, m, scols, n, one, da.as<const T2* const>(), m,
                                  db.as<const T2* const>(), n, zero, dc.as<T2* const>(), m, (int)pa.size());
              }
              VIE_CUDA(cudaStreamSynchronize(s));  // W goes out of scope
            }
            // Classical Gram-Schmidt of the new columns: the panel once against the
            // basis it starts from (one GEMM pair for all of its columns), each
            // 32-column chunk once against the columns this panel has added, and
            // after its normalisation once more against the whole basis (Cholesky
            // QR, pass 2 below).  The blocks still growing all hold rmax
            // columns; converged ones are left out.
            const int rp = rmax;
            if (rp > 0) {
                std::vector<int> live;
                for (int q = 0; q < nb; ++q)
                    if (!conv[q]) live.push_back(q);
                const size_t need = (size_t)nb * rp * scols * sizeof(T2);
                if (Cpan.bytes < need) Cpan.alloc(need);
                proj_ptrs(pbuf1, live, Q.as<T2>(), (int64_t)m * rcap_pad, Y.as<T2>(), (int64_t)m * scols,
                          Cpan.as<T2>(), (int64_t)rp * scols);
                project(pbuf1, (int)live.size(), rp, m, rp, scols);
            }
            for (int c0 = 0; c0 < scols; c0 += kChunk) {
                T2* Yc = Y.as<T2>() + (int64_t)c0 * m;
                const long long ys = (long long)m * scols;
                rmax = *std::max_element(r.begin(), r.end());
                std::vector<int> live;
                for (int q = 0; q < nb; ++q)
                    if (!conv[q]) live.push_back(q);
                if (rmax > rp) {
                    proj_ptrs(pbuf1, live, Q.as<T2>() + (int64_t)rp * m, (int64_t)m * rcap_pad, Yc, ys, Cb.as<T2>(),
                              (int64_t)rcap_pad * kChunk);
                    project(pbuf1, (int)live.size(), rmax - rp, m, rcap_pad, kChunk);
                }
                sumsq(Yc, (int64_t)m * kChunk, ys, nb, est.as<double>(), part);
                std::vector<double> he(nb);
                VIE_CUDA(cudaMemcpyAsync(he.data(), est.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
                VIE_CUDA(cudaStreamSynchronize(s));
                std::vector<int> active(nb, 0), rbase(nb, 0);
                bool any = false;
                for (int q = 0; q < nb; ++q) {
                    if (!conv[q] && he[q] / kChunk <= thr * hnorm[q]) conv[q] = 1;
                    if (!conv[q] && r[q] + kChunk > rcap_pad) {
                        if (rcap < rfull && cap < kRankCap) return false;  // again, with room for kRankCap
                        if (rcap < rfull)
                            fail(VIE_ERR_BREAKDOWN, "far block needs a rank above " + std::to_string(kRankCap) +
                                                        " at this tolerance");
                        conv[q] = 1;  // full basis of the block's range: exact
                    }
                    active[q] = !conv[q];
                    rbase[q] = r[q];
                    any |= active[q];
                }
                if (!any) break;
                VIE_CUDA(cudaMemcpyAsync(d_active.p, active.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
                VIE_CUDA(cudaMemcpyAsync(d_rbase.p, rbase.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
                // Cholesky QR, twice
                int nchunk = std::max(1, std::min(64, m / 256));
                size_t gneed = (size_t)nb * nchunk * kChunk * kChunk * sizeof(double2);
                if (gpart.bytes < gneed) gpart.alloc(gneed);
                std::vector<int> act;
                for (int q = 0; q < nb; ++q)
                    if (active[q]) act.push_back(q);
                if (rmax > 0)
                    proj_ptrs(pbuf2, act, Q.as<T2>(), (int64_t)m * rcap_pad, Yc, ys, Cb.as<T2>(),
                              (int64_t)rcap_pad * kChunk);
                for (int pass = 0; pass < 2; ++pass) {
                    if (pass == 1 && rmax > 0) {
                        // the normalisation above scales up whatever overlap with the
                        // basis the float32 projection left behind: project once more
                        project(pbuf2, (int)act.size(), rmax, m, rcap_pad, kChunk);
                    }
                    if (pass == 0) {
                        if constexpr (std::is_same<T2, float2>::value)
                            k_gram_partial_df<<<dim3(nchunk, nb), 1024, 0, s>>>(Yc, m, ys, nchunk,
                                                                                gpart.as<double2>(),
                                                                                d_active.as<int>());
                        else
                            k_gram_partial<T2, double2><<<dim3(nchunk, nb), 1024, 0, s>>>(
                                Yc, m, ys, nchunk, gpart.as<double2>(), d_active.as<int>());
                    }
                    else
                        k_gram_partial<T2, T2><<<dim3(nchunk, nb), 1024, 0, s>>>(Yc, m, ys, nchunk,
                                                                               gpart.as<double2>(),
                                                                               d_active.as<int>());
                    VIE_CHECK_LAUNCH();
                    k_gram_reduce<<<nb, kChunk * kChunk, 0, s>>>(gpart.as<double2>(), nchunk, G.as<double2>(),
                                                                 d_active.as<int>());
                    VIE_CHECK_LAUNCH();
                    k_chol<T2><<<nb, dim3(kChunk, kChunk), 0, s>>>(G.as<double2>(), Minv.as<T2>(),
                                                                    d_active.as<int>(), alive.as<unsigned char>(),
                                                                    rcap_pad, d_rbase.as<int>());
                    VIE_CHECK_LAUNCH();
                    if (pass == 0) {
                        // in place: Yc <- Yc Minv (rows are independent)
                        k_trmul<T2><<<dim3((m + 127) / 128, nb), 128, 0, s>>>(Yc, m, ys, Minv.as<T2>(),
                                                                             d_active.as<int>(), Yc, ys, m, nullptr);
                    } else {
                        k_trmul<T2><<<dim3((m + 127) / 128, nb), 128, 0, s>>>(
                            Yc, m, ys, Minv.as<T2>(), d_active.as<int>(), Q.as<T2>(), (int64_t)m * rcap_pad, m,
                            d_rbase.as<int>());
                    }
                    VIE_CHECK_LAUNCH();
                }
                for (int q = 0; q < nb; ++q)
                    if (active[q]) r[q] += kChunk;
            }
        }

        double t2 = mark();
        tim[1] += t2 - t1;
        // 3. R^H = A^H Q (n x rmax per block)
        int rmax = *std::max_element(r.begin(), r.end());
        std::vector<unsigned char> halive((size_t)nb * rcap_pad);
        VIE_CUDA(cudaMemcpyAsync(halive.data(), alive.p, halive.size(), cudaMemcpyDeviceToHost, s));
        DevBuf RH((size_t)nb * n * std::max(rmax, 1) * sizeof(T2));
        if (rmax > 0 && split) {
            // [Re R^H | Im R^H] = A^T Bh + A_hi^T Bl (A read as 4m x n), joined per block
            const float2* Qf = reinterpret_cast<const float2*>(Q.p);
            float2* RHf = reinterpret_cast<float2*>(RH.p);
            if (mn >= ((int64_t)1 << 22)) {
                DevBuf Bh((size_t)8 * m * rmax * sizeof(bf16)), Bl((size_t)4 * m * rmax * sizeof(bf16)),
                    F((size_t)2 * n * rmax * sizeof(float));
                for (int q = 0; q < nb; ++q) {
                    if (r[q] <= 0) continue;
                    const int rq = r[q];
                    k_split_q<<<dim3((unsigned)std::min<int64_t>(4096, ((int64_t)m * rq + 255) / 256), 1), 256, 0,
                                s>>>(Qf + (size_t)q * m * rcap_pad, m, rq, 0, Bh.as<bf16>(), 0, Bl.as<bf16>(), 0);
                    VIE_CHECK_LAUNCH();
                    gemm_bf16(h, CUBLAS_OP_T, n, 2 * rq, 4 * m, Ap + (size_t)q * 4 * mn, 4 * m, 0, Bh.as<bf16>(),
                              4 * m, 0, 0.f, F.as<float>(), n, 0, 1);
                    gemm_bf16(h, CUBLAS_OP_T, n, 2 * rq, 2 * m, Ap + (size_t)q * 4 * mn, 4 * m, 0, Bl.as<bf16>(),
                              2 * m, 0, 1.f, F.as<float>(), n, 0, 1);
                    k_join_planes<<<dim3((unsigned)std::min<int64_t>(4096, ((int64_t)n * rq + 255) / 256), 1), 256,
                                    0, s>>>(F.as<float>(), n, rq, 0, RHf + (size_t)q * n * rmax, 0, nullptr);
                    VIE_CHECK_LAUNCH();
                }
                VIE_CUDA(cudaStreamSynchronize(s));
            } else {
                const long long hs = 8LL * m * rmax, ls = 4LL * m * rmax, fs = 2LL * n * rmax;
                DevBuf Bh((size_t)nb * hs * sizeof(bf16)), Bl((size_t)nb * ls * sizeof(bf16)),
                    F((size_t)nb * fs * sizeof(float));
                k_split_q<<<dim3((unsigned)std::min<int64_t>(1024, ((int64_t)m * rmax + 255) / 256), nb), 256, 0,
                            s>>>(Qf, m, rmax, (int64_t)m * rcap_pad, Bh.as<bf16>(), hs, Bl.as<bf16>(), ls);
                VIE_CHECK_LAUNCH();
                gemm_bf16(h, CUBLAS_OP_T, n, 2 * rmax, 4 * m, Ap, 4 * m, 4 * mn, Bh.as<bf16>(), 4 * m, hs, 0.f,
                          F.as<float>(), n, fs, nb);
                gemm_bf16(h, CUBLAS_OP_T, n, 2 * rmax, 2 * m, Ap, 4 * m, 4 * mn, Bl.as<bf16>(), 2 * m, ls, 1.f,
                          F.as<float>(), n, fs, nb);
                k_join_planes<<<dim3((unsigned)std::min<int64_t>(1024, ((int64_t)n * rmax + 255) / 256), nb), 256, 0,
                                s>>>(F.as<float>(), n, rmax, fs, RHf, (int64_t)n * rmax, nullptr);
                VIE_CHECK_LAUNCH();
                VIE_CUDA(cudaStreamSynchronize(s));
            }
        } else if (rmax > 0) {
            const T2 one = mk(T(1), T(0)), zero = mk(T(0), T(0));
            if (mn >= ((int64_t)1 << 22)) {
                // large blocks: one GEMM per block with its own rank
                for (int q = 0; q < nb; ++q)
                    if (r[q] > 0)
                        Blas<T>::gemm1(h, CUBLAS_OP_C, CUBLAS_OP_N, n, r[q], m, one, A.as<T2>() + (size_t)q * mn, m,
                                       Q.as<T2>() + (size_t)q * m * rcap_pad, m, zero,
                                       RH.as<T2>() + (size_t)q * n * rmax, n);
            } else {
                Blas<T>::gemm(h, CUBLAS_OP_C, CUBLAS_OP_N, n, rmax, m, one, A.as<T2>(), m, mn, Q.as<T2>(), m,
                              (long long)m * rcap_pad, zero, RH.as<T2>(), n, (long long)n * rmax, nb);
            }
        }
        VIE_CUDA(cudaStreamSynchronize(s));
        double t3 = mark();
        tim[2] += t3 - t2;
        A.release();

        // 4. compact the live columns into a staging store
        const std::vector<int> rank = stash(ids, m, n, Q, (int64_t)m * rcap_pad, RH, (int64_t)n * rmax, r,
                                            halive.data(), rcap_pad);
        double t4 = mark();
        tim[3] += t4 - t3;
        if (op.ctx->verbose) {
            int rsum = 0, rmx = 0;
            for (int q = 0; q < nb; ++q) { rsum += rank[q]; rmx = std::max(rmx, rank[q]); }
            fprintf(stderr, "[vie]   level %d batch %d x (%d x %d): s0 %d steps %d mean rank %.1f max %d | form %.3f "
                    "sketch %.3f R %.3f pack %.3f s\n", b0.level, nb, m, n, s0, step, (double)rsum / nb, rmx,
                    t1 - t0, t2 - t1, t3 - t2, t4 - t3);
        }
        return true;
    }

    // Translated copies: two far blocks with the same level, the same atom
    // types and the same atom positions relative to their first target atom
    // are the same matrix (the entries depend on the atoms' types and relative
    // positions only; the copies differ by the rounding of the centres).  The
    // first block of each such class is its representative; the others share
    // its factors.  Classes are keyed on the displacements quantised far below
    // any geometric scale, so only exact translates are joined.
    std::vector<int> canon;
    void find_classes() {
        const size_t nb = op.blocks.size();
        canon.resize(nb);
        for (size_t i = 0; i < nb; ++i) canon[i] = (int)i;
        if (op.ctx->no_sharing) return;
        double span = 0.0;
        for (double c : op.centres) span = std::max(span, std::abs(c));
        const double q = 1e-9 * std::max(span, 1e-30);
        std::map<std::vector<long long>, int> first;
        std::vector<long long> key;
        for (size_t i = 0; i < nb; ++i) {
            const FarBlock& b = op.blocks[i];
            key.clear();
            key.push_back(b.level);
            key.push_back(b.nt);
            key.push_back(b.ns);
            const int a0 = op.block_atoms[b.t_off];
            auto add = [&](int a) {
                key.push_back(op.types[a]);
                for (int d = 0; d < 3; ++d)
                    key.push_back(std::llround((op.centres[3 * a + d] - op.centres[3 * a0 + d]) / q));
            };
            for (int x = 0; x < b.nt; ++x) add(op.block_atoms[b.t_off + x]);
            for (int x = 0; x < b.ns; ++x) add(op.block_atoms[b.s_off + x]);
            auto it = first.find(key);
            if (it == first.end()) first.emplace(key, (int)i);
            else canon[i] = it->second;
        }
    }

    void run() {
        where.assign(op.blocks.size(), {-1, 0});
        find_classes();
        // Of each pair of mirror classes the one whose representative comes first
        // is compressed; the other representative takes the transposed factors
        // (reciprocity, below).  Representatives are grouped by (level, m, n, box
        // distance), coarse levels first; blocks of one group have similar
        // ranks: one pilot block learns the rank, the rest start from a sketch
        // of that size plus a margin.
        std::map<std::tuple<int, int, int, int, int>, std::vector<int>> groups;
        for (size_t i = 0; i < op.blocks.size(); ++i) {
            auto& b = op.blocks[i];
            b.derived = false;
            if (canon[i] != (int)i) continue;  // shares its representative's factors
            b.derived = b.mirror >= 0 && canon[b.mirror] < (int)i;
            if (b.derived) continue;
            // with shared copies a distance group holds one to three
            // representatives: compress all representatives of a level and
            // shape in one batch (their bases grow together) instead of one
            // pilot after another
            if (op.ctx->no_sharing) groups[{b.level, b.m, b.n, b.dist, b.dmin}].push_back((int)i);
            else groups[{b.level, b.m, b.n, 0, 0}].push_back((int)i);
        }
        const size_t budget = std::max<size_t>((size_t)2 << 30, std::min<size_t>(op.ctx->budget / 3, (size_t)48 << 30));
        for (auto& g : groups) {
            std::vector<int> ids = g.second;
            int lev = std::get<0>(g.first), m = std::get<1>(g.first), n = std::get<2>(g.first);
            std::tuple<int, int, int> cls{lev, std::get<3>(g.first), std::get<4>(g.first)};
            // blocks per batch for basis room of `cap` ranks (blocks run along grid y)
            auto batch_size = [&](int cap) {
                const size_t rc = std::min<size_t>(std::min(m, n), (size_t)cap + kChunk);
                const size_t per = ((size_t)m * n + (size_t)m * rc + (size_t)n * rc + (size_t)m * 2 * kChunk) * sizeof(T2);
                int b = (int)std::max<size_t>(1, std::min<size_t>(4096, budget / per));
                if (const char* e = std::getenv("VIE_COMPRESS_MAX_BATCH")) b = std::max(1, std::min(b, std::atoi(e)));
                return b;
            };
            auto hint_of = [&]() {
                auto it = class_rank.find(cls);
                return it == class_rank.end() ? kChunk : ((it->second + kChunk + kChunk - 1) / kChunk) * kChunk;
            };
            const int try_cap = rank_try(std::min(m, n));
            // run a sub-batch with room for kRankTry ranks; if one of its blocks needs
            // more, again in batches sized for kRankCap
            auto run = [&](const std::vector<int>& sub) {
                if (batch(sub, hint_of(), try_cap)) return;
                const int bw = batch_size(kRankCap);
                for (size_t j0 = 0; j0 < sub.size(); j0 += bw)
                    batch(std::vector<int>(sub.begin() + j0, sub.begin() + std::min(sub.size(), j0 + bw)), hint_of(),
                          kRankCap);
            };
            const int bs = batch_size(try_cap);
            size_t i0 = 0;
            if (op.ctx->no_sharing && !class_rank.count(cls) && ids.size() > 1 && (size_t)m * n >= ((size_t)1 << 20)) {
                run({ids[0]});  // pilot
                i0 = 1;
            }
            for (; i0 < ids.size(); i0 += bs)
                run(std::vector<int>(ids.begin() + i0, ids.begin() + std::min(ids.size(), i0 + bs)));
        }
        // consolidate into one factor store: derived representatives take their
        // mirror class's rank, shared blocks their representative's rank and storage
        op.factor_entries = 0;
        op.stored_entries = 0;
        for (size_t i = 0; i < op.blocks.size(); ++i) {
            auto& b = op.blocks[i];
            if (b.derived) b.rank = op.blocks[canon[b.mirror]].rank;
        }
        int64_t total = 0;
        std::vector<int64_t> qoff(op.blocks.size());
        for (size_t i = 0; i < op.blocks.size(); ++i) {
            auto& b = op.blocks[i];
            if (canon[i] != (int)i) continue;
            qoff[i] = total;
            total += (int64_t)b.rank * (b.m + b.n);
            total = (total + 31) / 32 * 32;
        }
        op.d_factors.alloc((size_t)std::max<int64_t>(total, 32) * sizeof(T2));
        for (size_t i = 0; i < op.blocks.size(); ++i) {
            auto& b = op.blocks[i];
            if (canon[i] != (int)i) {
                const FarBlock& c = op.blocks[canon[i]];
                b.rank = c.rank;
                b.q_off = c.q_off;
                b.rh_off = c.rh_off;
                op.factor_entries += (int64_t)b.rank * (b.m + b.n);
                continue;
            }
            b.q_off = qoff[i];
            b.rh_off = qoff[i] + (int64_t)b.rank * b.m;
            op.factor_entries += (int64_t)b.rank * (b.m + b.n);
            op.stored_entries += (int64_t)b.rank * (b.m + b.n);
            if (b.rank == 0) continue;
            if (!b.derived) {
                const T2* src = stores[where[i].first].template as<T2>() + where[i].second;
                VIE_CUDA(cudaMemcpyAsync(op.d_factors.as<T2>() + b.q_off, src,
                                         (size_t)b.rank * (b.m + b.n) * sizeof(T2), cudaMemcpyDeviceToDevice, s));
            } else {
                // mirror of block p (A' = A_p^T): Q' = conj(R_p^H), R'^H = conj(Q_p)
                const int pi = canon[b.mirror];
                const FarBlock& p = op.blocks[pi];
                const T2* src = stores[where[pi].first].template as<T2>() + where[pi].second;
                const int64_t nq = (int64_t)p.rank * p.m, nr = (int64_t)p.rank * p.n;
                k_conj_copy<T2><<<(unsigned)std::min<int64_t>(4096, (nr + 255) / 256), 256, 0, s>>>(
                    src + nq, op.d_factors.as<T2>() + b.q_off, nr);
                k_conj_copy<T2><<<(unsigned)std::min<int64_t>(4096, (nq + 255) / 256), 256, 0, s>>>(
                    src, op.d_factors.as<T2>() + b.rh_off, nq);
                VIE_CHECK_LAUNCH();
            }
        }
        VIE_CUDA(cudaStreamSynchronize(s));
        stores.clear();
    }
};

}  // namespace

void compress_operator(Op& op, double tol, int prec, int method) {
    VIE_BLAS(cublasSetStream(op.ctx->blas, op.ctx->stream));
    // float32-accurate GEMMs on the bf16 tensor cores (BF16x9), float64-accurate
    // fixed-point emulation for the c128 path, where cuBLAS finds them faster
    // (VIE_GEMM_EMULATION=0 keeps plain float32/float64 arithmetic)
    const char* em = std::getenv("VIE_GEMM_EMULATION");
    if (!(em && em[0] == '0')) {
        VIE_BLAS(cublasSetMathMode(op.ctx->blas, (cublasMath_t)(CUBLAS_FP32_EMULATED_BF16X9_MATH |
                                                                CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH)));
        // the formed blocks and sketches are finite: skip the emulation's
        // inf/NaN scans of every operand
        VIE_BLAS(cublasSetEmulationSpecialValuesSupport(op.ctx->blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE));
        const char* es = std::getenv("VIE_GEMM_EMULATION_STRATEGY");
        VIE_BLAS(cublasSetEmulationStrategy(op.ctx->blas, (es && es[0] == 'p') ? CUBLAS_EMULATION_STRATEGY_PERFORMANT
                                                                                 : CUBLAS_EMULATION_STRATEGY_EAGER));
    } else {
        VIE_BLAS(cublasSetMathMode(op.ctx->blas, CUBLAS_DEFAULT_MATH));
    }
    op.d_factors.release();
    for (auto& b : op.blocks) b.rank = 0;
    op.cmethod = method;
    op.cross_bytes = 0;
    op.t_cross = 0;
    if (prec == VIE_C128) {
        Compressor<double> c(op, tol);
        c.cross = method == 1;
        c.run();
    } else {
        Compressor<float> c(op, tol);
        c.cross = method == 1;
        c.run();
    }
    op.fprec = prec == VIE_C128 ? VIE_C128 : VIE_C64;
    op.tol = tol;
    build_apply_lists(op);
}

}  // namespace vie
