// Compressed far-field apply (paper Sec. 5.2, eq. eq_02): for every far block
// b = (target box I, source box J),  F_I += Q_b (R_b x_J),  evaluated as
//   phase 1:  t_b = R_b x_J        (r_b values per right-hand side)
//   phase 2:  F_a = sum_b Q_b[rows of atom a] t_b   for every atom a
// Both phases are persistent kernels over static work lists that the greedy
// least-loaded rule of App. C (weights = factor bytes) maps onto the CTAs.
// Every output element is written once by one thread (no atomics), so the
// result does not depend on the schedule or on other work on the GPU.
//
// Storage: Q_b is m_b x r_b column-major; R_b is kept as R_b^H (n_b x r_b
// column-major, i.e. conj(R_b) row-major), so both phases stream their
// factor with unit stride; complex values are interleaved and pairs of
// complex float32 move as one 16-byte load.
#include <mutex>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

template <class T2> struct Pair { T2 a, b; };

__device__ __forceinline__ Pair<float2> ldpair(const float2* p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double2> ldpair(const double2* p) {
    return {__ldg(p), __ldg(p + 1)};
}
// streaming (read-once) variant for the factors
__device__ __forceinline__ Pair<float2> ldpair_stream(const float2* p) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double2> ldpair_stream(const double2* p) {
    return {__ldcs(p), __ldcs(p + 1)};
}

template <class T2> __device__ __forceinline__ T2 shfl_down2(T2 v, int o) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, o);
    v.y = __shfl_down_sync(0xffffffffu, v.y, o);
    return v;
}

// ---------------------------------------------------------------------------
// Accumulation.  Float32 and float64 vectors accumulate in their own
// precision.  For the float64 refinement residual the vectors come split into
// float32 head + tail (float4: re_h, im_h, re_l, im_l) and the products with
// the exact float32 factors are summed in double-float arithmetic: each
// product is formed exactly with an FMA (Dekker's two-product), each addition
// keeps its rounding error (Knuth's two-sum), so a sum carries about 48
// significant bits while every operation runs on the float32 pipes (the
// float64 pipe of this GPU is a small fraction of the float32 one).
// ---------------------------------------------------------------------------
struct Dfc { float rh, rl, ih, il; };  // (rh + rl) + j (ih + il)

template <class TX> struct AccOf { using t = TX; };
template <> struct AccOf<float4> { using t = Dfc; };

template <class TA> __device__ __forceinline__ TA acc_zero();
template <> __device__ __forceinline__ float2 acc_zero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 acc_zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ Dfc acc_zero<Dfc>() { return {0.f, 0.f, 0.f, 0.f}; }

// acc += conj(a) x  and  acc += a x
__device__ __forceinline__ void mac_conj(float2& acc, float2 a, float2 x) { cfmac(acc, a, x); }
__device__ __forceinline__ void mac_conj(double2& acc, float2 a, double2 x) { cfmac(acc, cvt<double2>(a), x); }
__device__ __forceinline__ void mac_conj(double2& acc, double2 a, double2 x) { cfmac(acc, a, x); }
__device__ __forceinline__ void mac(float2& acc, float2 a, float2 x) { cfma(acc, a, x); }
__device__ __forceinline__ void mac(double2& acc, float2 a, double2 x) { cfma(acc, cvt<double2>(a), x); }
__device__ __forceinline__ void mac(double2& acc, double2 a, double2 x) { cfma(acc, a, x); }

// (h, l) += a (bh + bl): the product a bh exactly as p + e, the tail a bl
// folded into e, then h + p by two-sum with its error and e added to l.
// The _rn intrinsics keep the compiler from fusing these steps.
__device__ __forceinline__ void df_acc(float& h, float& l, float a, float bh, float bl) {
    const float p = __fmul_rn(a, bh);
    float e = fmaf(a, bh, -p);
    e = fmaf(a, bl, e);
    const float sum = __fadd_rn(h, p);
    const float bv = __fsub_rn(sum, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bv)), __fsub_rn(p, bv));
    h = sum;
    l = __fadd_rn(l, __fadd_rn(err, e));
}
__device__ __forceinline__ void mac_conj(Dfc& acc, float2 a, float4 x) {
    df_acc(acc.rh, acc.rl, a.x, x.x, x.z);
    df_acc(acc.rh, acc.rl, a.y, x.y, x.w);
    df_acc(acc.ih, acc.il, a.x, x.y, x.w);
    df_acc(acc.ih, acc.il, -a.y, x.x, x.z);
}
__device__ __forceinline__ void mac(Dfc& acc, float2 a, float4 x) {
    df_acc(acc.rh, acc.rl, a.x, x.x, x.z);
    df_acc(acc.rh, acc.rl, -a.y, x.y, x.w);
    df_acc(acc.ih, acc.il, a.x, x.y, x.w);
    df_acc(acc.ih, acc.il, a.y, x.x, x.z);
}

__device__ __forceinline__ void acc_add(float2& a, float2 b) { a += b; }
__device__ __forceinline__ void acc_add(double2& a, double2 b) { a += b; }
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    const float sum = __fadd_rn(h, bh);
    const float bv = __fsub_rn(sum, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bv)), __fsub_rn(bh, bv));
    h = sum;
    l = __fadd_rn(__fadd_rn(l, bl), err);
}
__device__ __forceinline__ void acc_add(Dfc& a, const Dfc& b) {
    df_add(a.rh, a.rl, b.rh, b.rl);
    df_add(a.ih, a.il, b.ih, b.il);
}

__device__ __forceinline__ float2 acc_shfl_down(float2 v, int o) { return shfl_down2(v, o); }
__device__ __forceinline__ double2 acc_shfl_down(double2 v, int o) { return shfl_down2(v, o); }
__device__ __forceinline__ Dfc acc_shfl_down(Dfc v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.rh, o), __shfl_down_sync(0xffffffffu, v.rl, o),
            __shfl_down_sync(0xffffffffu, v.ih, o), __shfl_down_sync(0xffffffffu, v.il, o)};
}

__device__ __forceinline__ void store(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void store(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void store(double2* p, const Dfc& v) {
    *p = make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}
// renormalised head + tail (fast two-sum, the head dominates)
__device__ __forceinline__ void store(float4* p, const Dfc& v) {
    const float sr = __fadd_rn(v.rh, v.rl), si = __fadd_rn(v.ih, v.il);
    *p = make_float4(sr, si, __fsub_rn(v.rl, __fsub_rn(sr, v.rh)), __fsub_rn(v.il, __fsub_rn(si, v.ih)));
}

__device__ __forceinline__ Pair<float4> ldpair(const float4* p) { return {__ldg(p), __ldg(p + 1)}; }

// ---------------------------------------------------------------------------
// phase 1: one warp per group of ROWS rows of R_b, lanes stride over columns
// ---------------------------------------------------------------------------
template <class TF, class TX, int ROWS>
__global__ void __launch_bounds__(256, 3) p1_kernel(const FarBlockDev* __restrict__ blocks,
                                                 const int* __restrict__ batoms, const int4* __restrict__ items,
                                                 const int* __restrict__ cta_ptr, const TF* __restrict__ factors,
                                                 const TX* __restrict__ x, int64_t ldx, int np,
                                                 TX* __restrict__ t, int64_t ldt, int nrhs,
                                                 const int2* __restrict__ colr) {
    using TA = typename AccOf<TX>::t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const FarBlockDev B = blocks[item.x];
        const TF* RH = factors + B.rh_off;
        const int* S = batoms + B.s_off;
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);  // right-hand sides of this problem
        for (int k = item.y + warp * ROWS; k < item.z; k += nwarps * ROWS) {
            const int nrow = min(ROWS, item.z - k);
            const TF* rows[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) rows[r] = RH + (int64_t)(k + min(r, nrow - 1)) * B.n;
            for (int c0 = cr.x; c0 < cr.y; ++c0) {
                TA acc[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) acc[r] = acc_zero<TA>();
                const TX* xc = x + (int64_t)c0 * ldx;
                // column c = 2 lane + 64 i; two positions (c, c + 64) per iteration;
                // (slot, off) of each tracked incrementally
                int c = 2 * lane;
                int slot = c / np, off = c - slot * np;
                for (; c + 64 < B.n; c += 128) {
                    int off2 = off + 64, slot2 = slot;
                    while (off2 >= np) { off2 -= np; ++slot2; }
                    Pair<TX> xa = ldpair(xc + (int64_t)S[slot] * np + off);
                    Pair<TX> xb = ldpair(xc + (int64_t)S[slot2] * np + off2);
                    Pair<TF> ra[ROWS], rb[ROWS];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        ra[r] = ldpair_stream(rows[r] + c);
                        rb[r] = ldpair_stream(rows[r] + c + 64);
                    }
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        mac_conj(acc[r], ra[r].a, xa.a);
                        mac_conj(acc[r], ra[r].b, xa.b);
                        mac_conj(acc[r], rb[r].a, xb.a);
                        mac_conj(acc[r], rb[r].b, xb.b);
                    }
                    off = off2 + 64;
                    slot = slot2;
                    while (off >= np) { off -= np; ++slot; }
                }
                if (c < B.n) {
                    Pair<TX> xa = ldpair(xc + (int64_t)S[slot] * np + off);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        Pair<TF> ra = ldpair_stream(rows[r] + c);
                        mac_conj(acc[r], ra.a, xa.a);
                        mac_conj(acc[r], ra.b, xa.b);
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    TA v = acc[r];
                    for (int o = 16; o > 0; o >>= 1) acc_add(v, acc_shfl_down(v, o));
                    if (lane == 0 && r < nrow) store(&t[B.tvec_off + k + r + (int64_t)c0 * ldt], v);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// phase 2: item = (atom a, rows p0..p1 of a).  256 threads = 64 row pairs x
// 4 rank groups; each thread streams Q column segments of 2 rows and the
// partial sums of the 4 rank groups are added in a fixed order at the end.
// ---------------------------------------------------------------------------
template <class TF, class TX, class TO>
__global__ void __launch_bounds__(256) p2_kernel(const FarBlockDev* __restrict__ blocks,
                                                 const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                 const int* __restrict__ csr, const int2* __restrict__ ent,
                                                 const TF* __restrict__ factors, const TX* __restrict__ t,
                                                 int64_t ldt, int np, TO* __restrict__ F, int64_t ldf, int nrhs,
                                                 const int2* __restrict__ colr) {
    using TA = typename AccOf<TX>::t;
    __shared__ TA red[3][64][2];
    const int rp = threadIdx.x & 63, kg = threadIdx.x >> 6;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int a = item.x;
        const int row = item.y + 2 * rp;
        const bool active = row < item.z;
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y; ++c0) {
            TA acc0 = acc_zero<TA>(), acc1 = acc_zero<TA>();
            if (active) {
                for (int e = csr[a]; e < csr[a + 1]; ++e) {
                    const int2 en = ent[e];
                    const FarBlockDev B = blocks[en.x];
                    const TF* Q = factors + B.q_off + (int64_t)en.y * np + row;
                    const TX* tb = t + B.tvec_off + (int64_t)c0 * ldt;
                    int k = kg;
                    for (; k + 28 < B.rank; k += 32) {
                        Pair<TF> q[8];
                        TX tv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) q[u] = ldpair_stream(Q + (int64_t)(k + 4 * u) * B.m);
#pragma unroll
                        for (int u = 0; u < 8; ++u) tv[u] = tb[k + 4 * u];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            mac(acc0, q[u].a, tv[u]);
                            mac(acc1, q[u].b, tv[u]);
                        }
                    }
                    for (; k < B.rank; k += 4) {
                        Pair<TF> q0 = ldpair_stream(Q + (int64_t)k * B.m);
                        const TX t0 = tb[k];
                        mac(acc0, q0.a, t0);
                        mac(acc1, q0.b, t0);
                    }
                }
            }
            if (kg > 0) {
                red[kg - 1][rp][0] = acc0;
                red[kg - 1][rp][1] = acc1;
            }
            __syncthreads();
            if (kg == 0 && active) {
                for (int g = 0; g < 3; ++g) {
                    acc_add(acc0, red[g][rp][0]);
                    acc_add(acc1, red[g][rp][1]);
                }
                TO* out = F + (int64_t)a * np + row + (int64_t)c0 * ldf;
                store(out, acc0);
                store(out + 1, acc1);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// several right-hand sides: every factor element is read once per group of NR
// right-hand sides (the single-RHS kernels above re-read it per column)
// ---------------------------------------------------------------------------
template <class TF, class TX, int NR>
__global__ void __launch_bounds__(256, 2) p1m_kernel(const FarBlockDev* __restrict__ blocks,
                                                  const int* __restrict__ batoms, const int4* __restrict__ items,
                                                  const int* __restrict__ cta_ptr, const TF* __restrict__ factors,
                                                  const TX* __restrict__ x, int64_t ldx, int np,
                                                  TX* __restrict__ t, int64_t ldt, int nrhs,
                                                  const int2* __restrict__ colr) {
    using TA = typename AccOf<TX>::t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const FarBlockDev B = blocks[item.x];
        const TF* RH = factors + B.rh_off;
        const int* S = batoms + B.s_off;
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int k = item.y + warp * 2; k < item.z; k += nwarps * 2) {
            const bool two = k + 1 < item.z;
            const TF* row0 = RH + (int64_t)k * B.n;
            const TF* row1 = RH + (int64_t)(two ? k + 1 : k) * B.n;
            for (int c0 = cr.x; c0 < cr.y; c0 += NR) {
                const int nr = min(NR, cr.y - c0);
                TA a0[NR], a1[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) a0[r] = a1[r] = acc_zero<TA>();
                int c = 2 * lane;
                int slot = c / np, off = c - slot * np;
                for (; c < B.n; c += 64) {
                    Pair<TF> ra = ldpair_stream(row0 + c);
                    Pair<TF> rb = ldpair_stream(row1 + c);
                    const TX* xb = x + (int64_t)S[slot] * np + off + (int64_t)c0 * ldx;
                    // all right-hand sides' x pairs of this step in flight before the products
                    Pair<TX> xv[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) xv[r] = ldpair(xb + (int64_t)(r < nr ? r : 0) * ldx);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (r < nr) {
                            mac_conj(a0[r], ra.a, xv[r].a);
                            mac_conj(a0[r], ra.b, xv[r].b);
                            mac_conj(a1[r], rb.a, xv[r].a);
                            mac_conj(a1[r], rb.b, xv[r].b);
                        }
                    }
                    off += 64;
                    while (off >= np) { off -= np; ++slot; }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    TA v0 = a0[r], v1 = a1[r];
                    for (int o = 16; o > 0; o >>= 1) {
                        acc_add(v0, acc_shfl_down(v0, o));
                        acc_add(v1, acc_shfl_down(v1, o));
                    }
                    if (lane == 0 && r < nr) {
                        store(&t[B.tvec_off + k + (int64_t)(c0 + r) * ldt], v0);
                        if (two) store(&t[B.tvec_off + k + 1 + (int64_t)(c0 + r) * ldt], v1);
                    }
                }
            }
        }
    }
}

template <class TF, class TX, class TO, int NR>
__global__ void __launch_bounds__(256, 2) p2m_kernel(const FarBlockDev* __restrict__ blocks,
                                                  const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                  const int* __restrict__ csr, const int2* __restrict__ ent,
                                                  const TF* __restrict__ factors, const TX* __restrict__ t,
                                                  int64_t ldt, int np, TO* __restrict__ F, int64_t ldf, int nrhs,
                                                  const int2* __restrict__ colr) {
    using TA = typename AccOf<TX>::t;
    __shared__ TA red[3][64][2][NR];
    const int rp = threadIdx.x & 63, kg = threadIdx.x >> 6;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int a = item.x;
        const int row = item.y + 2 * rp;
        const bool active = row < item.z;
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y; c0 += NR) {
            const int nr = min(NR, cr.y - c0);
            TA a0[NR], a1[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) a0[r] = a1[r] = acc_zero<TA>();
            if (active) {
                for (int e = csr[a]; e < csr[a + 1]; ++e) {
                    const int2 en = ent[e];
                    const FarBlockDev B = blocks[en.x];
                    const TF* Q = factors + B.q_off + (int64_t)en.y * np + row;
                    const TX* tb = t + B.tvec_off + (int64_t)c0 * ldt;
                    // two rank steps (k, k + 4) per iteration: both steps' loads are in
                    // flight before the products; each accumulator still adds k, k + 4,
                    // k + 8, ... in order
                    for (int k = kg; k < B.rank; k += 8) {
                        const bool two = k + 4 < B.rank;
                        const Pair<TF> q0 = ldpair_stream(Q + (int64_t)k * B.m);
                        const Pair<TF> q1 = ldpair_stream(Q + (int64_t)(two ? k + 4 : k) * B.m);
                        TX tv0[NR], tv1[NR];
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            tv0[r] = tb[k + (int64_t)(r < nr ? r : 0) * ldt];
                            tv1[r] = tb[(two ? k + 4 : k) + (int64_t)(r < nr ? r : 0) * ldt];
                        }
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (r < nr) {
                                mac(a0[r], q0.a, tv0[r]);
                                mac(a1[r], q0.b, tv0[r]);
                                if (two) {
                                    mac(a0[r], q1.a, tv1[r]);
                                    mac(a1[r], q1.b, tv1[r]);
                                }
                            }
                        }
                    }
                }
            }
            if (kg > 0)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    red[kg - 1][rp][0][r] = a0[r];
                    red[kg - 1][rp][1][r] = a1[r];
                }
            __syncthreads();
            if (kg == 0 && active) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r >= nr) continue;
                    TA v0 = a0[r], v1 = a1[r];
                    for (int g = 0; g < 3; ++g) {
                        acc_add(v0, red[g][rp][0][r]);
                        acc_add(v1, red[g][rp][1][r]);
                    }
                    TO* out = F + (int64_t)a * np + row + (int64_t)(c0 + r) * ldf;
                    store(out, v0);
                    store(out + 1, v1);
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Shared factors, one right-hand side (column `col` of x; t and P hold that
// column only).  An item covers up to NR blocks of one class (the same R and
// Q): cmem[item.x .. item.x + item.w) lists them.
// Phase 1: t_j = R x[S_j] for each member j, every R element read once per
// item; the row layout and summation order follow p1m_kernel.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256, 3) p1c_kernel(const FarBlockDev* __restrict__ blocks,
                                                  const int* __restrict__ batoms, const int4* __restrict__ items,
                                                  const int* __restrict__ cta_ptr, const int* __restrict__ cmem,
                                                  const float2* __restrict__ factors, const float2* __restrict__ x,
                                                  int np, float2* __restrict__ t, const int2* __restrict__ colr,
                                                  int col) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int* mem = cmem + item.x;
        const int nm = item.w;
        const FarBlockDev B = blocks[mem[0]];
        if (colr) {
            const int2 cr = colr[B.prob];
            if (col < cr.x || col >= cr.y) continue;
        }
        const float2* RH = factors + B.rh_off;
        const int* S[NR];
        long long to[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const FarBlockDev Bj = blocks[mem[min(r, nm - 1)]];
            S[r] = batoms + Bj.s_off;
            to[r] = Bj.tvec_off;
        }
        for (int k = item.y + warp * 2; k < item.z; k += nwarps * 2) {
            const bool two = k + 1 < item.z;
            const float2* row0 = RH + (int64_t)k * B.n;
            const float2* row1 = RH + (int64_t)(two ? k + 1 : k) * B.n;
            float2 a0[NR], a1[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) a0[r] = a1[r] = make_float2(0.f, 0.f);
            int c = 2 * lane;
            int slot = c / np, off = c - slot * np;
            for (; c < B.n; c += 64) {
                const Pair<float2> ra = ldpair_stream(row0 + c);
                const Pair<float2> rb = ldpair_stream(row1 + c);
                // every member's x pair in flight before the products (S[r] of a
                // missing member repeats the last one, so the loads stay in bounds)
                Pair<float2> xv[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) xv[r] = ldpair(x + (int64_t)S[r][slot] * np + off);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r < nm) {
                        mac_conj(a0[r], ra.a, xv[r].a);
                        mac_conj(a0[r], ra.b, xv[r].b);
                        mac_conj(a1[r], rb.a, xv[r].a);
                        mac_conj(a1[r], rb.b, xv[r].b);
                    }
                }
                off += 64;
                while (off >= np) { off -= np; ++slot; }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float2 v0 = a0[r], v1 = a1[r];
                for (int o = 16; o > 0; o >>= 1) {
                    v0 += shfl_down2(v0, o);
                    v1 += shfl_down2(v1, o);
                }
                if (lane == 0 && r < nm) {
                    t[to[r] + k] = v0;
                    if (two) t[to[r] + k + 1] = v1;
                }
            }
        }
    }
}

// Phase 2 partials: item = (members, target slot sl, rows p0..p1 of the slot
// packed as p0 | p1 << 16).  P[poff_j + sl np + row] = Q[sl rows] t_j, every
// Q element read once per item; 64 row pairs x 4 rank groups as in p2m_kernel.
template <int NR>
__global__ void __launch_bounds__(256, 3) p2c_kernel(const FarBlockDev* __restrict__ blocks,
                                                  const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                  const int* __restrict__ cmem, const long long* __restrict__ poff,
                                                  const float2* __restrict__ factors, const float2* __restrict__ t,
                                                  int np, float2* __restrict__ P, const int2* __restrict__ colr,
                                                  int col) {
    __shared__ float2 red[3][64][2][NR];
    const int rp = threadIdx.x & 63, kg = threadIdx.x >> 6;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int* mem = cmem + item.x;
        const int nm = item.w, sl = item.y, p0 = item.z & 0xffff, p1 = item.z >> 16;
        const FarBlockDev B = blocks[mem[0]];
        if (colr) {
            const int2 cr = colr[B.prob];
            if (col < cr.x || col >= cr.y) continue;  // uniform over the CTA
        }
        const int row = p0 + 2 * rp;
        const bool active = row < p1;
        long long to[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) to[r] = blocks[mem[min(r, nm - 1)]].tvec_off;
        float2 a0[NR], a1[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) a0[r] = a1[r] = make_float2(0.f, 0.f);
        if (active) {
            const float2* Q = factors + B.q_off + (int64_t)sl * np + row;
            int k = kg;
            for (; k + 12 < B.rank; k += 16) {
                Pair<float2> q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) q[u] = ldpair_stream(Q + (int64_t)(k + 4 * u) * B.m);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // the members' t values loaded unconditionally, so that they can be
                    // issued ahead (to[r] of a missing member repeats the last one)
                    float2 tv[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) tv[r] = t[to[r] + k + 4 * u];
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (r < nm) {
                            mac(a0[r], q[u].a, tv[r]);
                            mac(a1[r], q[u].b, tv[r]);
                        }
                }
            }
            for (; k < B.rank; k += 4) {
                const Pair<float2> q = ldpair_stream(Q + (int64_t)k * B.m);
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (r < nm) {
                        const float2 tv = t[to[r] + k];
                        mac(a0[r], q.a, tv);
                        mac(a1[r], q.b, tv);
                    }
            }
        }
        if (kg > 0)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                red[kg - 1][rp][0][r] = a0[r];
                red[kg - 1][rp][1][r] = a1[r];
            }
        __syncthreads();
        if (kg == 0 && active) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (r >= nm) continue;
                float2 v0 = a0[r], v1 = a1[r];
                for (int g = 0; g < 3; ++g) {
                    v0 += red[g][rp][0][r];
                    v1 += red[g][rp][1][r];
                }
                float2* out = P + poff[mem[r]] + (int64_t)sl * np + row;
                out[0] = v0;
                out[1] = v1;
            }
        }
        __syncthreads();
    }
}

// F[a rows] = sum of the partial products of the (block, slot) entries of atom
// a, in the order of its entry list (deterministic); one row per thread
__global__ void __launch_bounds__(128) p2r_kernel(const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                 const int* __restrict__ csr, const int2* __restrict__ ent,
                                                 const long long* __restrict__ poff, const float2* __restrict__ P,
                                                 int np, float2* __restrict__ F, const int2* __restrict__ colr,
                                                 int col) {
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int a = item.x, row = item.y + (int)threadIdx.x;
        if (row >= item.z) continue;
        if (colr) {
            const int2 cr = colr[item.w];
            if (col < cr.x || col >= cr.y) continue;
        }
        float2 acc = make_float2(0.f, 0.f);
        for (int e = csr[a]; e < csr[a + 1]; ++e) {
            const int2 en = ent[e];
            acc += P[poff[en.x] + (int64_t)en.y * np + row];
        }
        F[(int64_t)a * np + row] = acc;
    }
}

}  // namespace

void shared_reserve(Op& op) {
    const size_t need = (size_t)std::max<int64_t>(op.part_total, 1) * sizeof(float2);
    if (op.d_part.bytes < need) op.d_part.alloc(need);
    const size_t nt = (size_t)std::max<int64_t>(op.t_total, 1) * sizeof(float2);
    if (op.d_t.bytes < nt) op.d_t.alloc(nt);
}

void apply_far_shared(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    shared_reserve(op);
    const float2* fac = op.fac<float2>();
    float2* t = op.d_t.as<float2>();
    float2* P = op.d_part.as<float2>();
    const FarBlockDev* bl = op.d_blocks.as<FarBlockDev>();
    for (int c = 0; c < nrhs; ++c) {
        if (op.n_c1_items > 0) {
            p1c_kernel<Op::kShareGroup><<<op.n_cta_c, 256, 0, s>>>(bl, op.d_block_atoms.as<int>(), op.d_c1_items.as<int4>(),
                                                     op.d_c1_cta.as<int>(), op.d_cmem.as<int>(), fac, x + c * ldx,
                                                     op.np, t, op.colr, c);
            VIE_CHECK_LAUNCH();
        }
        if (op.n_c2_items > 0) {
            p2c_kernel<Op::kShareGroup><<<op.n_cta_c, 256, 0, s>>>(bl, op.d_c2_items.as<int4>(), op.d_c2_cta.as<int>(),
                                                     op.d_cmem.as<int>(), op.d_poff.as<long long>(), fac, t, op.np,
                                                     P, op.colr, c);
            VIE_CHECK_LAUNCH();
        }
        p2r_kernel<<<op.n_cta, 128, 0, s>>>(op.d_p2_items.as<int4>(), op.d_p2_cta.as<int>(), op.d_p2_csr.as<int>(),
                                            op.d_p2_ent.as<int2>(), op.d_poff.as<long long>(), P, op.np,
                                            F + c * ldf, op.colr, c);
        VIE_CHECK_LAUNCH();
    }
}

template <class TF, class TX>
void apply_far(Op& op, const TX* x, int64_t ldx, TX* F, int64_t ldf, int nrhs, cudaStream_t s) {
    size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(TX);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const TF* fac = op.fac<TF>();
    const int nc = op.n_cta;
    if (nrhs > 1) {
        const int ncm = op.n_cta_m;
        if (op.n_p1_items > 0) {
            p1m_kernel<TF, TX, 4><<<ncm, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
                                                      op.d_p1m_items.as<int4>(), op.d_p1m_cta.as<int>(), fac, x, ldx,
                                                      op.np, op.d_t.as<TX>(), op.t_total, nrhs, op.colr);
            VIE_CHECK_LAUNCH();
        }
        p2m_kernel<TF, TX, TX, 4><<<ncm, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_p2m_items.as<int4>(),
                                                  op.d_p2m_cta.as<int>(), op.d_p2_csr.as<int>(), op.d_p2_ent.as<int2>(),
                                                  fac, op.d_t.as<TX>(), op.t_total, op.np, F, ldf, nrhs, op.colr);
        VIE_CHECK_LAUNCH();
        return;
    }
    if (op.n_p1_items > 0) {
        p1_kernel<TF, TX, 4><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
                                                op.d_p1_items.as<int4>(), op.d_p1_cta.as<int>(), fac, x, ldx,
                                                op.np, op.d_t.as<TX>(), op.t_total, nrhs, op.colr);
        VIE_CHECK_LAUNCH();
    }
    p2_kernel<TF, TX, TX><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_p2_items.as<int4>(),
                                         op.d_p2_cta.as<int>(), op.d_p2_csr.as<int>(), op.d_p2_ent.as<int2>(),
                                         fac, op.d_t.as<TX>(), op.t_total, op.np, F, ldf, nrhs, op.colr);
    VIE_CHECK_LAUNCH();
}

template void apply_far<float2, float2>(Op&, const float2*, int64_t, float2*, int64_t, int, cudaStream_t);
template void apply_far<double2, double2>(Op&, const double2*, int64_t, double2*, int64_t, int, cudaStream_t);

// complex float32 far apply with nr right-hand sides per factor read (1, 2, 4, 8):
// the tile shapes the autotuner chooses between
void apply_far_simt32(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, int nr,
                      cudaStream_t s) {
    const size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const float2* fac = op.fac<float2>();
    float2* t = op.d_t.as<float2>();
    const int nc = op.n_cta;
    const FarBlockDev* bl = op.d_blocks.as<FarBlockDev>();
#define VIE_P1M(NR)                                                                                                   \
    p1m_kernel<float2, float2, NR><<<op.n_cta_m, 256, 0, s>>>(bl, op.d_block_atoms.as<int>(), op.d_p1m_items.as<int4>(), \
                                                              op.d_p1m_cta.as<int>(), fac, x, ldx, op.np, t, op.t_total, \
                                                              nrhs, op.colr)
#define VIE_P2M(NR)                                                                                                  \
    p2m_kernel<float2, float2, float2, NR><<<op.n_cta_m, 256, 0, s>>>(bl, op.d_p2m_items.as<int4>(),                \
                                                                      op.d_p2m_cta.as<int>(), op.d_p2_csr.as<int>(), \
                                                                      op.d_p2_ent.as<int2>(), fac, t, op.t_total,   \
                                                                      op.np, F, ldf, nrhs, op.colr)
    if (op.n_p1_items > 0) {
        switch (nr) {
            case 1: p1_kernel<float2, float2, 4><<<nc, 256, 0, s>>>(bl, op.d_block_atoms.as<int>(),
                                                                    op.d_p1_items.as<int4>(), op.d_p1_cta.as<int>(),
                                                                    fac, x, ldx, op.np, t, op.t_total, nrhs, op.colr); break;
            case 2: VIE_P1M(2); break;
            case 4: VIE_P1M(4); break;
            case 8: VIE_P1M(8); break;
            default: fail(VIE_ERR_INVALID_ARG, "unknown SIMT tile");
        }
        VIE_CHECK_LAUNCH();
    }
    switch (nr) {
        case 1: p2_kernel<float2, float2, float2><<<nc, 256, 0, s>>>(bl, op.d_p2_items.as<int4>(),
                                                                     op.d_p2_cta.as<int>(), op.d_p2_csr.as<int>(),
                                                                     op.d_p2_ent.as<int2>(), fac, t, op.t_total,
                                                                     op.np, F, ldf, nrhs, op.colr); break;
        case 2: VIE_P2M(2); break;
        case 4: VIE_P2M(4); break;
        case 8: VIE_P2M(8); break;
        default: fail(VIE_ERR_INVALID_ARG, "unknown SIMT tile");
    }
    VIE_CHECK_LAUNCH();
#undef VIE_P1M
#undef VIE_P2M
}

namespace {
// x (complex float64, n x nrhs, leading dimension ldx) -> float32 head + tail
__global__ void k_split_hl(const double2* __restrict__ x, int64_t ldx, int64_t n, int nrhs, float4* __restrict__ xs) {
    const int64_t total = n * nrhs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / n, r = i - c * n;
        const double2 v = x[r + c * ldx];
        const float hr = (float)v.x, hi = (float)v.y;
        xs[i] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
    }
}
}  // namespace

// F = far part of Zs x for complex float32 factors and complex float64 vectors,
// summed in double-float arithmetic (the float64 refinement residual)
void apply_far_df(Op& op, const double2* x, int64_t ldx, double2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "the double-float apply needs VIE_C64 factors");
    const int64_t n = op.n();
    const size_t need_t = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float4);
    const size_t need_x = (size_t)n * nrhs * sizeof(float4);
    if (op.d_t.bytes < need_t) op.d_t.alloc(need_t);
    if (op.d_xs.bytes < need_x) op.d_xs.alloc(need_x);
    float4* xs = op.d_xs.as<float4>();
    float4* t = op.d_t.as<float4>();
    const float2* fac = op.fac<float2>();
    const int nc = op.n_cta;
    k_split_hl<<<op.ctx->n_sm * 8, 256, 0, s>>>(x, ldx, n, nrhs, xs);
    VIE_CHECK_LAUNCH();
    if (nrhs > 1) {
        const int ncm = op.n_cta_m;
        if (op.n_p1_items > 0) {
            p1m_kernel<float2, float4, 4><<<ncm, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(),
                                                              op.d_block_atoms.as<int>(), op.d_p1m_items.as<int4>(),
                                                              op.d_p1m_cta.as<int>(), fac, xs, n, op.np, t,
                                                              op.t_total, nrhs, op.colr);
            VIE_CHECK_LAUNCH();
        }
        p2m_kernel<float2, float4, double2, 4><<<ncm, 256, 0, s>>>(
            op.d_blocks.as<FarBlockDev>(), op.d_p2m_items.as<int4>(), op.d_p2m_cta.as<int>(), op.d_p2_csr.as<int>(),
            op.d_p2_ent.as<int2>(), fac, t, op.t_total, op.np, F, ldf, nrhs, op.colr);
        VIE_CHECK_LAUNCH();
        return;
    }
    if (op.n_p1_items > 0) {
        p1_kernel<float2, float4, 4><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
                                                        op.d_p1_items.as<int4>(), op.d_p1_cta.as<int>(), fac, xs, n,
                                                        op.np, t, op.t_total, nrhs, op.colr);
        VIE_CHECK_LAUNCH();
    }
    p2_kernel<float2, float4, double2><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_p2_items.as<int4>(),
                                                          op.d_p2_cta.as<int>(), op.d_p2_csr.as<int>(),
                                                          op.d_p2_ent.as<int2>(), fac, t, op.t_total, op.np, F, ldf,
                                                          nrhs, op.colr);
    VIE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Allocation-free apply: the phase-1 vector t lives in a fixed device array
// of this module instead of memory obtained with cudaMalloc, and the far part
// is accumulated straight into y.  Host code cannot use the array's name as
// a device address, so its address is looked up once per device.
// ---------------------------------------------------------------------------
constexpr int64_t kStaticScratchElems = VIE_NOALLOC_SCRATCH_ELEMS;  // complex float32: 32 MiB per device
static __device__ __align__(256) float2 g_static_scratch[kStaticScratchElems];

namespace {
std::mutex g_static_mu;
float2* g_static_addr[256] = {};

float2* static_scratch_address(int device) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (device < 0 || device >= 256) fail(VIE_ERR_INVALID_ARG, "device ordinal out of range");
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            fail(VIE_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                   cudaGetErrorString(e));
        g_static_addr[device] = static_cast<float2*>(p);
    }
    return g_static_addr[device];
}
}  // namespace

// y = Zs x with complex float32 factors and vectors; the caller has made the
// operator's device current
void apply_static(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "the allocation-free apply needs VIE_C64 factors");
    const int64_t need = std::max<int64_t>(op.t_total, 1) * nrhs;
    if (need > kStaticScratchElems)
        fail(VIE_ERR_INVALID_ARG, "allocation-free apply: " + std::to_string(need) +
                                      " complex scratch elements needed (sum of ranks x nrhs), the static array holds " +
                                      std::to_string(kStaticScratchElems));
    float2* t = static_scratch_address(op.ctx->device);
    const float2* fac = op.fac<float2>();
    const int nc = op.n_cta;
    const int64_t n = op.n();
    // every element of t[0, t_total * nrhs) is written by phase 1 before phase 2
    // reads it, and every element of y by phase 2: nothing needs clearing
    if (op.n_p1_items > 0) {
        p1_kernel<float2, float2, 4><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
                                                        op.d_p1_items.as<int4>(), op.d_p1_cta.as<int>(), fac, x, n,
                                                        op.np, t, op.t_total, nrhs, nullptr);
        VIE_CHECK_LAUNCH();
    }
    p2_kernel<float2, float2, float2><<<nc, 256, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_p2_items.as<int4>(),
                                                 op.d_p2_cta.as<int>(), op.d_p2_csr.as<int>(), op.d_p2_ent.as<int2>(),
                                                 fac, t, op.t_total, op.np, y, n, nrhs, nullptr);
    VIE_CHECK_LAUNCH();
    // y = Z_ii x + y, each element read and written by the same thread
    self_gemm<float2, float2>(op, op.d_zself32.as<float2>(), x, n, y, n, y, n, nrhs, 0, s);
}

}  // namespace vie
