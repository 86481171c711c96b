// Multi-right-hand-side far apply on the tensor cores, split precision BF16x3.
//
// With s right-hand sides the far apply is a pair of dense contractions per
// block, T_b = R_b X_J (r x n . n x s) and F_I += Q_b T_b (m x r . r x s).  Each
// complex float32 operand a is split into bfloat16 hi = bf16(a) and
// lo = bf16(a - hi) for its real and imaginary parts; a real product is
// hi.hi + hi.lo + lo.hi (the lo.lo term, ~2^-16 relative, is dropped) and the
// four real products of a complex product are accumulated in float32:
//   Cr += Ar Br - Ai Bi,   Ci += Ar Bi + Ai Br   (12 bf16 MMAs per 16x8x16 tile).
// A CTA holds a 64-row tile of the output for up to 64 right-hand sides, so each
// factor element is read from HBM once for all of them.  Operands are staged
// through shared memory as bf16 hi/lo planes (row stride KC + 8 elements, which
// makes the fragment loads bank-conflict free) and fed to warp-level
// mma.sync.m16n8k16 (four warps, 16 rows each, eight 8-column tiles).
#include <cuda_bf16.h>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

constexpr int kTM = 64;        // output rows per CTA (4 warps x 16)
constexpr int kTN = 64;        // right-hand sides per pass (8 tiles of 8)
constexpr int kKC = 32;        // K per shared-memory stage
constexpr int kLD = kKC + 8;   // padded row stride (bf16 elements)
constexpr int kThreads = 128;

struct Planes {                // one operand tile as four bf16 planes
    __nv_bfloat16 rh[kTM][kLD], rl[kTM][kLD], ih[kTM][kLD], il[kTM][kLD];
};

__device__ __forceinline__ void split(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ void store_c(Planes& P, int row, int col, float2 v) {
    __nv_bfloat16 h, l;
    split(v.x, h, l);
    P.rh[row][col] = h;
    P.rl[row][col] = l;
    split(v.y, h, l);
    P.ih[row][col] = h;
    P.il[row][col] = l;
}

__device__ __forceinline__ void zero_c(Planes& P, int row, int col) {
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    P.rh[row][col] = z;
    P.rl[row][col] = z;
    P.ih[row][col] = z;
    P.il[row][col] = z;
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment (16 x 16, row-major) of a plane: rows r0 + {g, g+8}, cols kk + {2t, 2t+1, 2t+8, 2t+9}
__device__ __forceinline__ void frag_a(const __nv_bfloat16 (*P)[kLD], int r0, int kk, int g, int t, uint32_t (&a)[4]) {
    a[0] = ld32(&P[r0 + g][kk + 2 * t]);
    a[1] = ld32(&P[r0 + g + 8][kk + 2 * t]);
    a[2] = ld32(&P[r0 + g][kk + 2 * t + 8]);
    a[3] = ld32(&P[r0 + g + 8][kk + 2 * t + 8]);
}

// one K stage: C (warp's 16 rows x 64 columns) += A (16 x kKC) B (kKC x 64)
// A planes are [row][k]; B planes are stored transposed, [n][k]
__device__ __forceinline__ void mma_stage(const Planes& A, const Planes& Bt, int r0, int g, int t, int ntiles,
                                          float (&cr)[8][4], float (&ci)[8][4]) {
#pragma unroll
    for (int kk = 0; kk < kKC; kk += 16) {
        uint32_t arh[4], arl[4], aih[4], ail[4], naih[4], nail[4];
        frag_a(A.rh, r0, kk, g, t, arh);
        frag_a(A.rl, r0, kk, g, t, arl);
        frag_a(A.ih, r0, kk, g, t, aih);
        frag_a(A.il, r0, kk, g, t, ail);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            naih[q] = aih[q] ^ 0x80008000u;  // negate both bf16 halves
            nail[q] = ail[q] ^ 0x80008000u;
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntiles) break;
            const int n = nt * 8 + g;
            const uint32_t brh0 = ld32(&Bt.rh[n][kk + 2 * t]), brh1 = ld32(&Bt.rh[n][kk + 2 * t + 8]);
            const uint32_t brl0 = ld32(&Bt.rl[n][kk + 2 * t]), brl1 = ld32(&Bt.rl[n][kk + 2 * t + 8]);
            const uint32_t bih0 = ld32(&Bt.ih[n][kk + 2 * t]), bih1 = ld32(&Bt.ih[n][kk + 2 * t + 8]);
            const uint32_t bil0 = ld32(&Bt.il[n][kk + 2 * t]), bil1 = ld32(&Bt.il[n][kk + 2 * t + 8]);
            // real part: Ar Br - Ai Bi
            mma(cr[nt], arh, brh0, brh1);
            mma(cr[nt], arh, brl0, brl1);
            mma(cr[nt], arl, brh0, brh1);
            mma(cr[nt], naih, bih0, bih1);
            mma(cr[nt], naih, bil0, bil1);
            mma(cr[nt], nail, bih0, bih1);
            // imaginary part: Ar Bi + Ai Br
            mma(ci[nt], arh, bih0, bih1);
            mma(ci[nt], arh, bil0, bil1);
            mma(ci[nt], arl, bih0, bih1);
            mma(ci[nt], aih, brh0, brh1);
            mma(ci[nt], aih, brl0, brl1);
            mma(ci[nt], ail, brh0, brh1);
        }
    }
}

// C fragment element (e = 0..3) of tile nt: row g + 8 (e >> 1), column nt * 8 + 2 t + (e & 1)
__device__ __forceinline__ int frag_row(int g, int e) { return g + 8 * (e >> 1); }
__device__ __forceinline__ int frag_col(int nt, int t, int e) { return nt * 8 + 2 * t + (e & 1); }

// ---------------------------------------------------------------------------
// phase 1: t_b[k, c] = sum_j conj(RH_b[j, k]) x[J_b(j), c] for 64 rows k of R_b
// item = (block, k0, k1) with k1 - k0 <= 64
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) p1_tc_kernel(const FarBlockDev* __restrict__ blocks,
                                                         const int* __restrict__ batoms,
                                                         const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                         const float2* __restrict__ factors,
                                                         const float2* __restrict__ x, int64_t ldx, int np,
                                                         float2* __restrict__ t, int64_t ldt, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    Planes& A = *reinterpret_cast<Planes*>(smem);
    Planes& Bt = *reinterpret_cast<Planes*>(smem + sizeof(Planes));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const FarBlockDev B = blocks[item.x];
        const float2* RH = factors + B.rh_off;
        const int* S = batoms + B.s_off;
        const int rows = item.z - item.y;
        for (int c0 = 0; c0 < nrhs; c0 += kTN) {
            const int ncol = min(kTN, nrhs - c0);
            const int ntiles = (ncol + 7) / 8;
            float cr[8][4], ci[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int e = 0; e < 4; ++e) cr[a][e] = ci[a][e] = 0.f;
            for (int j0 = 0; j0 < B.n; j0 += kKC) {
                __syncthreads();  // previous stage consumed
                // A: R rows k0 .. k0+63, columns j0 .. j0+31: conj(RH[j + k n])
                for (int e = tid; e < kTM * kKC; e += kThreads) {
                    const int r = e / kKC, j = e % kKC;
                    if (r < rows && j0 + j < B.n) {
                        float2 v = RH[(j0 + j) + (int64_t)(item.y + r) * B.n];
                        store_c(A, r, j, make_float2(v.x, -v.y));
                    } else {
                        zero_c(A, r, j);
                    }
                }
                // B^T: x columns c0 .. c0+63 (as rows), source unknowns j0 .. j0+31
                for (int e = tid; e < kTN * kKC; e += kThreads) {
                    const int c = e / kKC, j = e % kKC;
                    const int jj = j0 + j;
                    if (c < ncol && jj < B.n) {
                        const int slot = jj / np, off = jj - slot * np;
                        store_c(Bt, c, j, x[(int64_t)S[slot] * np + off + (int64_t)(c0 + c) * ldx]);
                    } else {
                        zero_c(Bt, c, j);
                    }
                }
                __syncthreads();
                mma_stage(A, Bt, warp * 16, g, tq, ntiles, cr, ci);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= ntiles) break;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = warp * 16 + frag_row(g, e), c = frag_col(nt, tq, e);
                    if (r < rows && c < ncol)
                        t[B.tvec_off + item.y + r + (int64_t)(c0 + c) * ldt] = make_float2(cr[nt][e], ci[nt][e]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// phase 2: F[a rows p0..p0+63, c] = sum_b Q_b[slot rows, :] t_b[:, c]
// item = (atom a, p0, p1) with p1 - p0 <= 64
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) p2_tc_kernel(const FarBlockDev* __restrict__ blocks,
                                                         const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                         const int* __restrict__ csr, const int2* __restrict__ ent,
                                                         const float2* __restrict__ factors,
                                                         const float2* __restrict__ t, int64_t ldt, int np,
                                                         float2* __restrict__ F, int64_t ldf, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    Planes& A = *reinterpret_cast<Planes*>(smem);
    Planes& Bt = *reinterpret_cast<Planes*>(smem + sizeof(Planes));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1]; ++it) {
        const int4 item = items[it];
        const int a = item.x, p0 = item.y, rows = item.z - item.y;
        for (int c0 = 0; c0 < nrhs; c0 += kTN) {
            const int ncol = min(kTN, nrhs - c0);
            const int ntiles = (ncol + 7) / 8;
            float cr[8][4], ci[8][4];
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) cr[q][e] = ci[q][e] = 0.f;
            for (int en = csr[a]; en < csr[a + 1]; ++en) {
                const int2 eb = ent[en];
                const FarBlockDev B = blocks[eb.x];
                const float2* Q = factors + B.q_off + (int64_t)eb.y * np + p0;
                const float2* tb = t + B.tvec_off;
                for (int k0 = 0; k0 < B.rank; k0 += kKC) {
                    __syncthreads();
                    // A: Q rows p0 .. p0+63 of this atom's slot, rank columns k0 .. k0+31
                    for (int e = tid; e < kTM * kKC; e += kThreads) {
                        const int r = e % kTM, k = e / kTM;  // consecutive threads: consecutive rows
                        if (r < rows && k0 + k < B.rank) store_c(A, r, k, Q[r + (int64_t)(k0 + k) * B.m]);
                        else zero_c(A, r, k);
                    }
                    // B^T: t_b rows k0 .. k0+31 for columns c0 .. c0+63
                    for (int e = tid; e < kTN * kKC; e += kThreads) {
                        const int c = e / kKC, k = e % kKC;
                        if (c < ncol && k0 + k < B.rank) store_c(Bt, c, k, tb[k0 + k + (int64_t)(c0 + c) * ldt]);
                        else zero_c(Bt, c, k);
                    }
                    __syncthreads();
                    mma_stage(A, Bt, warp * 16, g, tq, ntiles, cr, ci);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= ntiles) break;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = warp * 16 + frag_row(g, e), c = frag_col(nt, tq, e);
                    if (r < rows && c < ncol)
                        F[(int64_t)a * np + p0 + r + (int64_t)(c0 + c) * ldf] = make_float2(cr[nt][e], ci[nt][e]);
                }
            }
        }
    }
}

}  // namespace

void apply_far_bf16x3(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "VIE_BF16X3 applies need VIE_C64 factors");
    size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const size_t sm = 2 * sizeof(Planes);  // 40 KiB
    const float2* fac = op.fac<float2>();
    if (op.n_t1_items > 0) {
        p1_tc_kernel<<<op.n_cta_tc, kThreads, sm, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
                                                       op.d_t1_items.as<int4>(), op.d_t1_cta.as<int>(), fac, x, ldx,
                                                       op.np, op.d_t.as<float2>(), op.t_total, nrhs);
        VIE_CHECK_LAUNCH();
    }
    p2_tc_kernel<<<op.n_cta_tc, kThreads, sm, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_t2_items.as<int4>(),
                                                   op.d_t2_cta.as<int>(), op.d_p2_csr.as<int>(), op.d_p2_ent.as<int2>(),
                                                   fac, op.d_t.as<float2>(), op.t_total, op.np, F, ldf, nrhs);
    VIE_CHECK_LAUNCH();
}

}  // namespace vie
