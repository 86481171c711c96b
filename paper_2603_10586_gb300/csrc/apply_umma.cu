// Multi-right-hand-side far apply on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), split precision BF16x3.
//
// With s right-hand sides the far apply is two sets of dense contractions,
//   phase 1:  t_b = R_b X_J           (paper Sec. 5.2, the inner product R x)
//   phase 2:  F_a = sum_b Q_b[a] t_b  (the outer product Q t, per atom a)
// Each complex float32 operand value v is split into bfloat16 hi = bf16(v)
// and lo = bf16(v - hi) for its real and imaginary parts; a real product is
// hi.hi + hi.lo + lo.hi (the lo.lo term, ~2^-16 relative, is dropped), so a
// complex product is twelve bf16 MMAs accumulated in float32:
//   D_r += Ar Br - Ai Bi,   D_i += Ar Bi + Ai Br,
// the minus sign taken by the MMA's negate-A bit.
//
// Tile: 128 output rows (tensor-memory lanes) x up to 64 right-hand sides;
// D_r occupies tensor-memory columns [0, 64) and D_i columns [64, 128).
// The K dimension is staged 32 complex values at a time: the four warps load
// the operands from global memory, split them into bf16 planes and store the
// planes in shared memory in the canonical no-swizzle K-major layout (8x8
// core matrices of 128 contiguous bytes); one thread then issues the 24 MMAs
// of the stage and commits them to an mbarrier, and while the tensor core
// works on one stage the warps fill the other.
//
// Phase 1 stacks the R rows of all blocks that share one source atom list,
// so one gathered x_J feeds up to 128 rows; phase 2 walks one virtual K axis
// made of every (block, rank index) that touches the atom, so short ranks do
// not pad the K stages.
//
// Every wait on an mbarrier gives up after about a second of clock cycles,
// records the failure in an error word and leaves the kernel after freeing
// its tensor memory.
#include <cuda_bf16.h>

#include <cstdlib>
#include <mutex>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

constexpr int kM = 128;                 // output rows per tile
constexpr int kN = 64;                  // right-hand sides per pass
constexpr int kKS = 32;                 // complex K values per stage
constexpr int kThr = 256;               // eight warps (two per tensor-memory lane quarter)
constexpr int kTmemCols = 128;          // D_r: [0, 64), D_i: [64, 128)
constexpr int kChunksA = kM * kKS / 8;  // 16-byte chunks per A plane (512)
constexpr int kChunksB = kN * kKS / 8;  // 16-byte chunks per B plane (256)
constexpr uint32_t kLboA = kM * 16;     // bytes between K-adjacent core matrices of A
constexpr uint32_t kLboB = kN * 16;
constexpr uint32_t kSbo = 128;          // bytes between 8-row groups

// one stage: planes (re hi, re lo, im hi, im lo) of A (128 x 32) and B (64 x 32);
// chunk (row, q) of a plane holds K values 8q .. 8q+7 of that row and sits at
// index q * rows + row, i.e. core matrix (row / 8, q) at q * LBO + (row / 8) * 128
struct Stage {
    uint4 a[4][kChunksA];
    uint4 b[4][kChunksB];
};
constexpr size_t kStageBytes = sizeof(Stage);  // 48 KiB
constexpr size_t kSmemBytes = 2 * kStageBytes;  // two stages: 96 KiB, two CTAs per SM

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, canonical layout without swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture
    return d;                // base offset 0, relative LBO, no swizzle
}

// instruction descriptor of kind::f16: bf16 x bf16 -> f32, both K-major,
// M = 128, N = n
__host__ __device__ constexpr uint32_t idesc(int n, bool neg_a) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// split two floats (K positions 2e, 2e+1) into packed bf16 hi and lo words
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}
// 8 complex values -> the 16-byte chunk of each plane
template <int CHUNKS>
__device__ __forceinline__ void put8(uint4 (*planes)[CHUNKS], int chunk, const float2 (&v)[8]) {
    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split2(v[2 * e].x, v[2 * e + 1].x, rh[e], rl[e]);
        split2(v[2 * e].y, v[2 * e + 1].y, ih[e], il[e]);
    }
    planes[0][chunk] = make_uint4(rh[0], rh[1], rh[2], rh[3]);
    planes[1][chunk] = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    planes[2][chunk] = make_uint4(ih[0], ih[1], ih[2], ih[3]);
    planes[3][chunk] = make_uint4(il[0], il[1], il[2], il[3]);
}

__device__ __forceinline__ void zero8(float2 (&v)[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = make_float2(0.f, 0.f);
}

// the 24 MMAs of one stage (two K steps of 16)
__device__ __forceinline__ void issue_stage(const Stage& st, uint32_t tm, int nmma, bool first) {
    const uint32_t id = idesc(nmma, false), idn = idesc(nmma, true);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        uint64_t A[4], B[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            A[p] = sdesc(smem_u32(&st.a[p][0]) + ks * 2 * kLboA, kLboA);
            B[p] = sdesc(smem_u32(&st.b[p][0]) + ks * 2 * kLboB, kLboB);
        }
        const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
        // planes: 0 re hi, 1 re lo, 2 im hi, 3 im lo
        umma(tm, A[0], B[0], id, acc0);
        umma(tm, A[0], B[1], id, 1u);
        umma(tm, A[1], B[0], id, 1u);
        umma(tm, A[2], B[2], idn, 1u);
        umma(tm, A[2], B[3], idn, 1u);
        umma(tm, A[3], B[2], idn, 1u);
        umma(tm + kN, A[0], B[2], id, acc0);
        umma(tm + kN, A[0], B[3], id, 1u);
        umma(tm + kN, A[1], B[2], id, 1u);
        umma(tm + kN, A[2], B[0], id, 1u);
        umma(tm + kN, A[2], B[1], id, 1u);
        umma(tm + kN, A[3], B[0], id, 1u);
    }
}

// Operand sources.  load_a(row, q, k0, v) fills the 8 values K = k0+8q.. of
// A row `row`; load_b(col, q, k0, v) those of right-hand side `col`.
struct Phase1 {
    // stacked rows of R (conj of the stored R^H rows) times x gathered over the source atoms
    const float2* fac;
    const long long* rowoff;
    const int* rowt;
    const int* S;
    const float2* x;
    int64_t ldx;
    int np, nK, row_begin, rows, c0, ncol;
    __device__ __forceinline__ void load_a(int row, int q, int k0, float2 (&v)[8]) const {
        const int j = k0 + 8 * q;
        if (row >= rows || j >= nK) {
            zero8(v);
            return;
        }
        const float2* src = fac + rowoff[row_begin + row] + j;
        if (j + 8 <= nK) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 w = __ldcs(reinterpret_cast<const float4*>(src) + e);
                v[2 * e] = make_float2(w.x, -w.y);
                v[2 * e + 1] = make_float2(w.z, -w.w);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float2 w = j + e < nK ? __ldcs(src + e) : make_float2(0.f, 0.f);
                v[e] = make_float2(w.x, -w.y);
            }
        }
    }
    __device__ __forceinline__ void load_b(int col, int q, int k0, float2 (&v)[8]) const {
        const int j = k0 + 8 * q;
        if (col >= ncol || j >= nK) {
            zero8(v);
            return;
        }
        const float2* xc = x + (int64_t)(c0 + col) * ldx;
        const int slot = j / np, off = j - slot * np;
        if (j + 8 <= nK && off + 8 <= np) {
            const float4* p = reinterpret_cast<const float4*>(xc + (int64_t)S[slot] * np + off);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 w = __ldg(p + e);
                v[2 * e] = make_float2(w.x, w.y);
                v[2 * e + 1] = make_float2(w.z, w.w);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int jj = j + e;
                if (jj < nK) {
                    const int sl = jj / np, of = jj - sl * np;
                    v[e] = __ldg(xc + (int64_t)S[sl] * np + of);
                } else {
                    v[e] = make_float2(0.f, 0.f);
                }
            }
        }
    }
};

struct Phase2 {
    // rows p0.. of one atom in every Q_b touching it, times the matching t_b entries
    const float2* fac;
    const long long* qoff;
    const int* tidx;
    const float2* t;
    int64_t ldt;
    int64_t kbase;
    int nK, p0, rows, c0, ncol;
    __device__ __forceinline__ void load_a(int row, int q, int k0, float2 (&v)[8]) const {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int kk = k0 + 8 * q + e;
            v[e] = (row < rows && kk < nK) ? __ldcs(fac + qoff[kbase + kk] + p0 + row) : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void load_b(int col, int q, int k0, float2 (&v)[8]) const {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int kk = k0 + 8 * q + e;
            v[e] = (col < ncol && kk < nK) ? __ldg(t + tidx[kbase + kk] + (int64_t)(c0 + col) * ldt)
                                           : make_float2(0.f, 0.f);
        }
    }
};

// A segments: phase 1 keeps the 4 K chunks of a row on neighbouring threads
// (contiguous R rows), phase 2 keeps rows on neighbouring threads (contiguous
// Q columns)
template <bool kRowFast>
__device__ __forceinline__ void a_seg(int s, int& row, int& q) {  // s in [0, 512)
    if (kRowFast) {
        row = s & (kM - 1);
        q = s >> 7;
    } else {
        row = s >> 2;
        q = s & 3;
    }
}

struct Ctl {
    uint64_t mbar[2];  // MMAs of the stage in buffer b done
    uint64_t tma[2];   // packed variant: A of the stage in buffer b landed
    uint32_t tmem;
    int ok;
};

constexpr int kStageChunksA = 4 * kChunksA;      // 16-byte chunks of one packed A stage (2048)
constexpr uint32_t kStageBytesA = kStageChunksA * 16;  // 32 KiB

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// bulk copy global -> shared memory, completion counted on the mbarrier.  The
// factor planes are read once per apply, so their lines are marked first to
// leave L2, in favour of the gathered x / t rows that many tiles read.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void tma_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    const uint64_t pol = l2_evict_first_policy();
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(mbar), "l"(pol)
        : "memory");
}

// One output tile (rows x ncol) over K = nK: stages g0, g0+1, ... of this CTA.
// Returns false when a wait gave up.  On return every thread may read the
// accumulators (when nK > 0).

template <class Src, bool kRowFast>
__device__ bool run_tile(const Src& src, Stage* stages, Ctl& ctl, uint32_t& g, int nK, int nmma) {
    const int tid = threadIdx.x;
    const int nst = (nK + kKS - 1) / kKS;
    for (int st = 0; st < nst; ++st, ++g) {
        const int k0 = st * kKS;
        Stage& S = stages[g & 1];
        // A: 512 segments of 8 values, B: 256 (two and one per thread)
        float2 va[2][8], vb[8];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int row, q;
            a_seg<kRowFast>(tid + i * kThr, row, q);
            src.load_a(row, q, k0, va[i]);
        }
        src.load_b(tid >> 2, tid & 3, k0, vb);
        // the stage buffer is free once the MMAs issued two stages ago are done
        if (tid == 0) ctl.ok = (g < 2) ? 1 : (mbar_wait(smem_u32(&ctl.mbar[g & 1]), ((g >> 1) - 1) & 1) ? 1 : 0);
        __syncthreads();
        if (!ctl.ok) return false;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int row, q;
            a_seg<kRowFast>(tid + i * kThr, row, q);
            put8<kChunksA>(S.a, q * kM + row, va[i]);
        }
        put8<kChunksB>(S.b, (tid & 3) * kN + (tid >> 2), vb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            fence_after();
            issue_stage(S, ctl.tmem, nmma, st == 0);
            umma_commit(smem_u32(&ctl.mbar[g & 1]));
        }
    }
    if (nst > 0) {
        const uint32_t gl = g - 1;
        if (tid == 0) ctl.ok = mbar_wait(smem_u32(&ctl.mbar[gl & 1]), (gl >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!ctl.ok) return false;
        fence_after();
    }
    return true;
}

// The packed variant: the A operand of every stage is already split into bf16
// planes in the stage layout (packA, 32 KiB per stage), so one thread moves
// it with a bulk copy, one stage ahead, while the warps split only B.
// `alive` (thread 0's) turns false when a wait gave up.
__device__ __forceinline__ void issue_a(Ctl& ctl, Stage* stages, uint32_t g, const uint4* src) {
    const uint32_t mb = smem_u32(&ctl.tma[g & 1]);
    mbar_expect_tx(mb, kStageBytesA);
    tma_bulk(smem_u32(&stages[g & 1].a[0][0]), src, kStageBytesA, mb);
}

template <class Src>
__device__ bool run_tile_tma(const Src& src, const uint4* packA, Stage* stages, Ctl& ctl, uint32_t& g, int nK,
                             int nmma, bool& alive) {
    const int tid = threadIdx.x;
    const int nst = (nK + kKS - 1) / kKS;
    for (int st = 0; st < nst; ++st, ++g) {
        Stage& S = stages[g & 1];
        float2 vb[8];
        src.load_b(tid >> 2, tid & 3, st * kKS, vb);
        if (tid == 0) {
            // a buffer is free once the MMAs issued two stages before it are done
            if (st == 0 && alive) {
                if (g >= 2) alive = mbar_wait(smem_u32(&ctl.mbar[g & 1]), ((g >> 1) - 1) & 1);
                if (alive) issue_a(ctl, stages, g, packA);
            }
            if (st + 1 < nst && alive) {
                const uint32_t g1 = g + 1;
                if (g1 >= 2) alive = mbar_wait(smem_u32(&ctl.mbar[g1 & 1]), ((g1 >> 1) - 1) & 1);
                if (alive) issue_a(ctl, stages, g1, packA + (int64_t)(st + 1) * kStageChunksA);
            }
            ctl.ok = alive ? 1 : 0;
        }
        __syncthreads();
        if (!ctl.ok) return false;
        put8<kChunksB>(S.b, (tid & 3) * kN + (tid >> 2), vb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && alive) {
            alive = mbar_wait(smem_u32(&ctl.tma[g & 1]), (g >> 1) & 1);
            if (alive) {
                fence_after();
                issue_stage(S, ctl.tmem, nmma, st == 0);
                umma_commit(smem_u32(&ctl.mbar[g & 1]));
            }
        }
    }
    if (nst > 0) {
        const uint32_t gl = g - 1;
        if (tid == 0) {
            if (alive) alive = mbar_wait(smem_u32(&ctl.mbar[gl & 1]), (gl >> 1) & 1);
            ctl.ok = alive ? 1 : 0;
        }
        __syncthreads();
        if (!ctl.ok) return false;
        fence_after();
    }
    return true;
}

// out[rowidx(r) + c * ld] = (D_r, D_i)[r, c] for r < rows, c < ncol (zeros when nK == 0).
// A warp reads the tensor-memory lanes of its quarter (warp % 4); warps 0-3
// take columns 0-31, warps 4-7 columns 32-63.
template <class RowIdx>
__device__ void epilogue(const Ctl& ctl, bool have, int rows, int ncol, RowIdx rowidx, float2* out, int64_t ld) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;
    const uint32_t base = ctl.tmem + ((uint32_t)(quarter * 32) << 16);
    const bool mine = r < rows;
    const int64_t ri = mine ? rowidx(r) : 0;
    for (int cb = half * 32; cb < min(ncol, half * 32 + 32); cb += 16) {
        float vr[16], vi[16];
        if (have) {
            tmem_ld16(base + cb, vr);
            tmem_ld16(base + kN + cb, vi);
            tmem_wait_ld();
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) vr[i] = vi[i] = 0.f;
        }
        if (mine) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (cb + i < ncol) out[ri + (int64_t)(cb + i) * ld] = make_float2(vr[i], vi[i]);
        }
    }
    fence_before();
    __syncthreads();  // accumulators read before the next tile overwrites them
}

__device__ void setup(Ctl& ctl) {
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&ctl.mbar[0]));
        mbar_init(smem_u32(&ctl.mbar[1]));
        mbar_init(smem_u32(&ctl.tma[0]));
        mbar_init(smem_u32(&ctl.tma[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
}

// leave: if a wait gave up, give the tensor core one more bounded chance to
// finish what was issued, then free the tensor memory
__device__ void teardown(Ctl& ctl, bool failed, uint32_t g, int* err) {
    if (failed) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            if (g > 0) mbar_wait(smem_u32(&ctl.mbar[(g - 1) & 1]), ((g - 1) >> 1) & 1);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ctl.tmem), "r"(kTmemCols)
                     : "memory");
}

__global__ void __launch_bounds__(kThr) u1_kernel(const FarBlockDev* __restrict__ blocks,
                                                  const int* __restrict__ batoms, const int4* __restrict__ items,
                                                  const int* __restrict__ cta_ptr,
                                                  const long long* __restrict__ rowoff, const int* __restrict__ rowt,
                                                  const float2* __restrict__ fac, const float2* __restrict__ x,
                                                  int64_t ldx, int np, float2* __restrict__ t, int64_t ldt, int nrhs,
                                                  const int2* __restrict__ colr, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Stage* stages = reinterpret_cast<Stage*>(smem);
    __shared__ Ctl ctl;
    setup(ctl);
    uint32_t g = 0;
    bool failed = false;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1] && !failed; ++it) {
        const int4 item = items[it];
        const FarBlockDev B = blocks[item.x];
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);  // right-hand sides of this problem
        for (int c0 = cr.x; c0 < cr.y && !failed; c0 += kN) {
            Phase1 src{fac, rowoff, rowt, batoms + B.s_off, x, ldx, np, B.n, item.y, item.z, c0, min(kN, cr.y - c0)};
            const int nmma = max(16, (src.ncol + 15) / 16 * 16);
            if (!run_tile<Phase1, false>(src, stages, ctl, g, B.n, nmma)) {
                failed = true;
                break;
            }
            const int* rt = rowt + item.y;
            epilogue(ctl, B.n > 0, item.z, src.ncol, [rt](int r) { return (int64_t)rt[r]; }, t + (int64_t)c0 * ldt,
                     ldt);
        }
    }
    teardown(ctl, failed, g, err);
}

__global__ void __launch_bounds__(kThr) u2_kernel(const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                  const long long* __restrict__ qoff, const int* __restrict__ tidx,
                                                  const long long* __restrict__ kptr, const float2* __restrict__ fac,
                                                  const float2* __restrict__ t, int64_t ldt, int np,
                                                  float2* __restrict__ F, int64_t ldf, int nrhs,
                                                  const int2* __restrict__ colr, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Stage* stages = reinterpret_cast<Stage*>(smem);
    __shared__ Ctl ctl;
    setup(ctl);
    uint32_t g = 0;
    bool failed = false;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1] && !failed; ++it) {
        const int4 item = items[it];
        const int a = item.x, p0 = item.y, rows = item.z - item.y;
        const long long kb = kptr[a];
        const int nK = (int)(kptr[a + 1] - kb);
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y && !failed; c0 += kN) {
            Phase2 src{fac, qoff, tidx, t, ldt, kb, nK, p0, rows, c0, min(kN, cr.y - c0)};
            const int nmma = max(16, (src.ncol + 15) / 16 * 16);
            if (!run_tile<Phase2, true>(src, stages, ctl, g, nK, nmma)) {
                failed = true;
                break;
            }
            const int64_t rb = (int64_t)a * np + p0;
            epilogue(ctl, nK > 0, rows, src.ncol, [rb](int r) { return rb + r; }, F + (int64_t)c0 * ldf, ldf);
        }
    }
    teardown(ctl, failed, g, err);
}

// ---- packed variant ---------------------------------------------------------
// pack: one CTA per work item writes the item's A operand, stage after stage,
// in the shared-memory stage layout (zero padding past the last row / K value)
__global__ void __launch_bounds__(kThr) pack1_kernel(const FarBlockDev* __restrict__ blocks,
                                                     const int4* __restrict__ items, const long long* __restrict__ pk,
                                                     const long long* __restrict__ rowoff,
                                                     const float2* __restrict__ fac, int np, uint4* __restrict__ out) {
    const int4 item = items[blockIdx.x];
    const FarBlockDev B = blocks[item.x];
    const Phase1 src{fac, rowoff, nullptr, nullptr, nullptr, 0, np, B.n, item.y, item.z, 0, 0};
    const int nst = (B.n + kKS - 1) / kKS;
    uint4* base = out + pk[blockIdx.x] * kStageChunksA;
    for (int st = 0; st < nst; ++st) {
        uint4(*planes)[kChunksA] = reinterpret_cast<uint4(*)[kChunksA]>(base + (int64_t)st * kStageChunksA);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int row, q;
            a_seg<false>(threadIdx.x + i * kThr, row, q);
            float2 v[8];
            src.load_a(row, q, st * kKS, v);
            put8<kChunksA>(planes, q * kM + row, v);
        }
    }
}

__global__ void __launch_bounds__(kThr) pack2_kernel(const int4* __restrict__ items, const long long* __restrict__ pk,
                                                     const long long* __restrict__ qoff,
                                                     const long long* __restrict__ kptr,
                                                     const float2* __restrict__ fac, uint4* __restrict__ out) {
    const int4 item = items[blockIdx.x];
    const int a = item.x;
    const long long kb = kptr[a];
    const int nK = (int)(kptr[a + 1] - kb);
    const Phase2 src{fac, qoff, nullptr, nullptr, 0, kb, nK, item.y, item.z - item.y, 0, 0};
    const int nst = (nK + kKS - 1) / kKS;
    uint4* base = out + pk[blockIdx.x] * kStageChunksA;
    for (int st = 0; st < nst; ++st) {
        uint4(*planes)[kChunksA] = reinterpret_cast<uint4(*)[kChunksA]>(base + (int64_t)st * kStageChunksA);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int row, q;
            a_seg<true>(threadIdx.x + i * kThr, row, q);
            float2 v[8];
            src.load_a(row, q, st * kKS, v);
            put8<kChunksA>(planes, q * kM + row, v);
        }
    }
}

__global__ void __launch_bounds__(kThr) u1p_kernel(const FarBlockDev* __restrict__ blocks,
                                                   const int* __restrict__ batoms, const int4* __restrict__ items,
                                                   const int* __restrict__ cta_ptr, const long long* __restrict__ pk,
                                                   const uint4* __restrict__ pack, const int* __restrict__ rowt,
                                                   const float2* __restrict__ x, int64_t ldx, int np,
                                                   float2* __restrict__ t, int64_t ldt, int nrhs,
                                                   const int2* __restrict__ colr, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Stage* stages = reinterpret_cast<Stage*>(smem);
    __shared__ Ctl ctl;
    setup(ctl);
    uint32_t g = 0;
    bool failed = false, alive = true;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1] && !failed; ++it) {
        const int4 item = items[it];
        const FarBlockDev B = blocks[item.x];
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y && !failed; c0 += kN) {
            Phase1 src{nullptr, nullptr, rowt, batoms + B.s_off, x, ldx, np, B.n, item.y, item.z, c0,
                       min(kN, cr.y - c0)};
            const int nmma = max(16, (src.ncol + 15) / 16 * 16);
            if (!run_tile_tma(src, pack + pk[it] * kStageChunksA, stages, ctl, g, B.n, nmma, alive)) {
                failed = true;
                break;
            }
            const int* rt = rowt + item.y;
            epilogue(ctl, B.n > 0, item.z, src.ncol, [rt](int r) { return (int64_t)rt[r]; }, t + (int64_t)c0 * ldt,
                     ldt);
        }
    }
    teardown(ctl, failed, g, err);
}

__global__ void __launch_bounds__(kThr) u2p_kernel(const int4* __restrict__ items, const int* __restrict__ cta_ptr,
                                                   const long long* __restrict__ pk, const uint4* __restrict__ pack,
                                                   const int* __restrict__ tidx, const long long* __restrict__ kptr,
                                                   const float2* __restrict__ t, int64_t ldt, int np,
                                                   float2* __restrict__ F, int64_t ldf, int nrhs,
                                                   const int2* __restrict__ colr, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Stage* stages = reinterpret_cast<Stage*>(smem);
    __shared__ Ctl ctl;
    setup(ctl);
    uint32_t g = 0;
    bool failed = false, alive = true;
    for (int it = cta_ptr[blockIdx.x]; it < cta_ptr[blockIdx.x + 1] && !failed; ++it) {
        const int4 item = items[it];
        const int a = item.x, p0 = item.y, rows = item.z - item.y;
        const long long kb = kptr[a];
        const int nK = (int)(kptr[a + 1] - kb);
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y && !failed; c0 += kN) {
            Phase2 src{nullptr, nullptr, tidx, t, ldt, kb, nK, p0, rows, c0, min(kN, cr.y - c0)};
            const int nmma = max(16, (src.ncol + 15) / 16 * 16);
            if (!run_tile_tma(src, pack + pk[it] * kStageChunksA, stages, ctl, g, nK, nmma, alive)) {
                failed = true;
                break;
            }
            const int64_t rb = (int64_t)a * np + p0;
            epilogue(ctl, nK > 0, rows, src.ncol, [rb](int r) { return rb + r; }, F + (int64_t)c0 * ldf, ldf);
        }
    }
    teardown(ctl, failed, g, err);
}

// ---- warp-specialised variant ---------------------------------------------
// One persistent CTA per SM; the roles run concurrently and meet on mbarriers
// instead of CTA-wide barriers:
//   warp 4     one thread starts the bulk copy of the pre-split A planes of
//              every K stage (32 KiB) into the next free slot of a ring of 3
//              to 5 stages (as many as fit beside the B planes of the widest
//              tile), running ahead of everything else;
//   warps 5-12 up to four groups of two warps (no more than the ring has
//              stages) load, split and store the B operand (x gathered over
//              the source atoms, or t) of a stage; group q takes the stages
//              g = q mod G and gathers a stage's values into registers before
//              it waits for the stage's slot, so the loads of G stages are in
//              flight while the MMAs run;
//   warp 13    one thread issues the 8 MMAs of a stage once its A copy has
//              landed and its B planes are stored, and commits them to the
//              slot's "empty" barrier (the producers refill it) and, at the end
//              of a tile, to the tile's accumulator barrier;
//   warps 0-3  epilogue: read the finished tile from tensor memory (warp w
//              owns lanes 32w..32w+31) and store it.  Tensor memory holds two
//              accumulator buffers, so the MMAs of the next tile run while the
//              previous one drains.
// The MMAs are fewer and wider than in u1p/u2p.  With B stored as two stacks
// of planes, S1 = [Br_hi; Bi_hi; Br_lo; Bi_lo] and S2 = [-Bi_hi; Br_hi; -Bi_lo;
// Br_lo] (N = ncol rows each; the negation is exact in bf16), a K step is four
// MMAs into one accumulator of 4 ncol columns [Re_a | Im_a | Re_b | Im_b]:
//   Ar_hi x S1 (N = 4 ncol), Ai_hi x S2 (4 ncol), Ar_lo x S1[0:2 ncol],
//   Ai_lo x S2[0:2 ncol],
// and the epilogue adds Re = Re_a + Re_b, Im = Im_a + Im_b.  The products are
// those of the twelve-MMA form (hi.hi + hi.lo + lo.hi of every real product);
// each A plane is read by one MMA instead of two to four, which nearly halves
// the tensor core's shared-memory operand traffic.  The float32 sums are
// grouped differently, so the results agree with u1p/u2p to rounding.
// Every wait gives up after `lim` clock cycles: the waiting role raises the
// CTA's abort flag, every role leaves its loop at its next check, and before
// the tensor memory is freed and the CTA exits, the bulk copies that were
// started and the MMAs that were issued are waited for (with the normal ~1 s
// limit).  The error word then tells the host.
constexpr int kWsMaxStages = 6;
constexpr int kWsThr = 448;  // 14 warps
constexpr int kWsWarpTma = 4, kWsWarpB0 = 5, kWsWarpMma = 13;
constexpr int kWsGroups = (kWsWarpMma - kWsWarpB0) / 2;  // B-producer groups of two warps
constexpr int kWsTmemCols = 512;                          // accumulators [Re_a | Im_a | Re_b | Im_b] of 4 nmax columns
constexpr int kWsSmemBytes = 224 * 1024;                  // the ring

// Two tile shapes share the code.  MT = 1: one 128-row M tile per B tile and
// 32 K values per stage (two MMA K steps).  MT = 2: two M tiles (256 rows: the
// two row tiles of one target atom, or two consecutive row tiles of one
// source group) share one B tile, 16 K values per stage (one K step), so the
// B operand is gathered and split once for twice the factor rows.  Either way
// a stage carries 32 KiB of A planes.
template <int MT>
struct WsGeom {
    static constexpr int KS = 32 / MT;                                  // K values per stage
    static constexpr int KQ = KS / 8;                                   // 16-byte K chunks per row and stage
    static constexpr int KSTEPS = KS / 16;                              // MMA K steps per stage
    static constexpr uint32_t kPlaneBytes = (uint32_t)kM * KS * 2;      // one bf16 plane of one M tile
    static constexpr uint32_t kTileBytes = 4 * kPlaneBytes;             // its four planes
    static constexpr uint32_t kABytes = MT * kTileBytes;                // 32 KiB
    // stage bytes: the A planes, then two B stacks of 4 KQ nmax chunks
    __host__ __device__ static constexpr uint32_t stride(int nmax) { return kABytes + 2u * 4u * KQ * nmax * 16u; }
    __host__ __device__ static constexpr int stages(int nmax) {
        return (int)(kWsSmemBytes / stride(nmax)) < kWsMaxStages ? (int)(kWsSmemBytes / stride(nmax)) : kWsMaxStages;
    }
    // accumulator buffers: each holds MT accumulators of 4 nmax columns
    __host__ __device__ static constexpr int nbuf(int nmax) { return kWsTmemCols / (MT * 4 * nmax) >= 2 ? 2 : 1; }
};
static_assert(WsGeom<1>::stages(64) == 3 && WsGeom<1>::stages(16) == 5, "ring sizes");
static_assert(WsGeom<2>::stages(64) == 4 && WsGeom<2>::stages(16) == 6, "ring sizes");
static_assert(WsGeom<1>::kABytes == kStageBytesA && WsGeom<2>::kABytes == kStageBytesA, "A bytes per stage");
static_assert(WsGeom<2>::stride(16) % 1024 == 0 && WsGeom<1>::stride(16) % 1024 == 0, "stage alignment");

// The ring: ns stages of `stride` bytes.  A stage holds the A planes (MT = 1:
// the packed layout of one 32-K stage, one bulk copy; MT = 2: per M tile the
// half of a packed stage that holds 16 of its K values, four copies), then the
// two B stacks; chunk (slot, row, q) of a stack sits at q (4 nmma) + slot nmma
// + row.  nmax, the widest tile's column count rounded up to 16, sets the
// stride, and the stage count is what fits: for MT = 1, 5 stages up to 16
// right-hand sides, 4 up to 48, 3 up to 64; for MT = 2, 6, 5 and 4.
struct WsRing {
    unsigned char* base;
    uint32_t stride, bstack;  // bytes per stage; chunks per B stack
    uint32_t ns;              // stages
    uint32_t abytes;          // A bytes per stage
    __device__ __forceinline__ uint4* a(uint32_t slot) const { return reinterpret_cast<uint4*>(base + slot * stride); }
    __device__ __forceinline__ uint4* b(uint32_t slot, int k) const {
        return reinterpret_cast<uint4*>(base + slot * stride + abytes) + k * bstack;
    }
};
template <int MT>
__device__ __forceinline__ WsRing ws_ring(unsigned char* smem, int nmax) {
    return WsRing{smem, WsGeom<MT>::stride(nmax), 4u * WsGeom<MT>::KQ * nmax, (uint32_t)WsGeom<MT>::stages(nmax),
                  WsGeom<MT>::kABytes};
}

__device__ __forceinline__ uint4 neg_bf16x8(uint4 v) {
    return make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
}

// 8 complex values of B (column `row`, K chunk q) into both stacks
__device__ __forceinline__ void put8_ws(uint4* b0, uint4* b1, int nmma, int row, int q, const float2 (&v)[8]) {
    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split2(v[2 * e].x, v[2 * e + 1].x, rh[e], rl[e]);
        split2(v[2 * e].y, v[2 * e + 1].y, ih[e], il[e]);
    }
    const uint4 RH = make_uint4(rh[0], rh[1], rh[2], rh[3]), RL = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    const uint4 IH = make_uint4(ih[0], ih[1], ih[2], ih[3]), IL = make_uint4(il[0], il[1], il[2], il[3]);
    const int base = q * 4 * nmma + row;
    b0[base] = RH;
    b0[base + nmma] = IH;
    b0[base + 2 * nmma] = RL;
    b0[base + 3 * nmma] = IL;
    b1[base] = neg_bf16x8(IH);
    b1[base + nmma] = RH;
    b1[base + 2 * nmma] = neg_bf16x8(IL);
    b1[base + 3 * nmma] = RL;
}

// the four wide MMAs of one K step (16) of M tile planes `a` (plane stride
// `pb` bytes) against the B stacks at byte offset `boff` into the accumulator
// at tm
__device__ __forceinline__ void mma_kstep_ws(uint32_t a, uint32_t pb, uint32_t b0, uint32_t b1, uint32_t tm,
                                             int nmma, uint32_t acc0) {
    const uint32_t id4 = idesc(4 * nmma, false), id2 = idesc(2 * nmma, false);
    const uint32_t lbob = (uint32_t)(4 * nmma * 16);
    uint64_t A[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) A[p] = sdesc(a + p * pb, kLboA);
    const uint64_t B1 = sdesc(b0, lbob), B2 = sdesc(b1, lbob);
    // planes: 0 re hi, 1 re lo, 2 im hi, 3 im lo
    umma(tm, A[0], B1, id4, acc0);
    umma(tm, A[2], B2, id4, 1u);
    umma(tm, A[1], B1, id2, 1u);
    umma(tm, A[3], B2, id2, 1u);
}

struct WsCtl {
    uint64_t full_a[kWsMaxStages];  // A copies of the slot landed (1 arrival + bytes)
    uint64_t full_b[kWsMaxStages];  // B planes of the slot stored (the stage's 2 producer warps)
    uint64_t empty[kWsMaxStages];   // MMAs that read the slot are done (1 commit)
    uint64_t acc_full[2];        // accumulator buffer holds a finished tile (1 commit)
    uint64_t acc_empty[2];       // epilogue has read the buffer (4 epilogue warps)
    uint32_t tmem;
    volatile int abort;
    uint32_t g_tma, g_mma;       // stages whose A copy was started / whose MMAs were issued
};

__device__ __forceinline__ void mbar_init_n(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// bounded wait with a caller-given limit
__device__ __forceinline__ bool mbar_wait_lim(uint32_t mbar, uint32_t parity, long long lim) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > lim) return false;
    }
}

// The tiles of this CTA, in the same order for every role: (item, or pair of
// items with one B operand, 64-column pass).  nst = K stages (0: nothing to
// multiply, the output is zero); rows[m] = 0 marks an absent second M tile;
// pk[m] = the M tile's first stage in the packed planes.
struct WsTile1 {
    Phase1 src;
    int nst, nmma;
    int rows[2];
    const int* rt[2];
    long long pk[2];
};

template <int MT, class Role>
__device__ void ws_tiles1(const FarBlockDev* blocks, const int* batoms, const int4* items, const int4* items_b,
                          const long long* pk, const long long* pk_b, int it0, int it1, const int* rowt,
                          const float2* x, int64_t ldx, int np, int nrhs, const int2* colr, volatile int* abort,
                          Role&& role) {
    for (int it = it0; it < it1 && !*abort; ++it) {
        const int4 item = items[it];
        const int4 ib = MT == 2 ? items_b[it] : make_int4(0, 0, 0, 0);
        const FarBlockDev B = blocks[item.x];
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y && !*abort; c0 += kN) {
            WsTile1 T{Phase1{nullptr, nullptr, rowt, batoms + B.s_off, x, ldx, np, B.n, item.y, item.z, c0,
                             min(kN, cr.y - c0)},
                      (B.n + WsGeom<MT>::KS - 1) / WsGeom<MT>::KS,
                      0,
                      {item.z, ib.z},
                      {rowt + item.y, rowt + ib.y},
                      {pk[it], MT == 2 ? pk_b[it] : 0}};
            T.nmma = max(16, (T.src.ncol + 15) / 16 * 16);
            if (!role(T, it, c0)) return;
        }
    }
}

struct WsTile2 {
    Phase2 src;
    int nst, nmma;
    int rows[2];
    int64_t rb[2];
    long long pk[2];
};

template <int MT, class Role>
__device__ void ws_tiles2(const int4* items, const int4* items_b, const long long* pk, const long long* pk_b,
                          int it0, int it1, const int* tidx, const long long* kptr, const float2* t, int64_t ldt,
                          int np, int nrhs, const int2* colr, volatile int* abort, Role&& role) {
    for (int it = it0; it < it1 && !*abort; ++it) {
        const int4 item = items[it];
        const int4 ib = MT == 2 ? items_b[it] : make_int4(item.x, 0, 0, 0);
        const int a = item.x, p0 = item.y, rows = item.z - item.y;
        const long long kb = kptr[a];
        const int nK = (int)(kptr[a + 1] - kb);
        const int2 cr = colr ? colr[item.w] : make_int2(0, nrhs);
        for (int c0 = cr.x; c0 < cr.y && !*abort; c0 += kN) {
            WsTile2 T{Phase2{nullptr, nullptr, tidx, t, ldt, kb, nK, p0, rows, c0, min(kN, cr.y - c0)},
                      (nK + WsGeom<MT>::KS - 1) / WsGeom<MT>::KS,
                      0,
                      {rows, ib.z - ib.y},
                      {(int64_t)a * np + p0, (int64_t)a * np + ib.y},
                      {pk[it], MT == 2 ? pk_b[it] : 0}};
            T.nmma = max(16, (T.src.ncol + 15) / 16 * 16);
            if (!role(T, it, c0)) return;
        }
    }
}

__device__ void ws_setup(WsCtl& ctl, uint32_t ns) {
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < ns; ++i) {
            mbar_init_n(smem_u32(&ctl.full_a[i]), 1);
            mbar_init_n(smem_u32(&ctl.full_b[i]), 2);
            mbar_init_n(smem_u32(&ctl.empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init_n(smem_u32(&ctl.acc_full[i]), 1);
            mbar_init_n(smem_u32(&ctl.acc_empty[i]), 4);
        }
        ctl.abort = 0;
        ctl.g_tma = 0;
        ctl.g_mma = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == kWsWarpMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl.tmem)),
                     "r"(kWsTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
}

// wait for what is still in flight (started copies, issued MMAs), free the
// tensor memory, report an abort
__device__ void ws_teardown(WsCtl& ctl, uint32_t ns, int* err) {
    __syncthreads();
    if (threadIdx.x == kWsWarpTma * 32) {  // the thread that started the copies
        for (uint32_t g = ctl.g_mma; g < ctl.g_tma; ++g)
            mbar_wait_lim(smem_u32(&ctl.full_a[g % ns]), (g / ns) & 1, kWaitCycles);
    }
    if (threadIdx.x == kWsWarpMma * 32 && ctl.g_mma > 0) {  // the thread that issued the MMAs
        const uint32_t g = ctl.g_mma - 1;
        mbar_wait_lim(smem_u32(&ctl.empty[g % ns]), (g / ns) & 1, kWaitCycles);
    }
    if (threadIdx.x == 0 && ctl.abort) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if ((threadIdx.x >> 5) == kWsWarpMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ctl.tmem), "r"(kWsTmemCols)
                     : "memory");
}

// The roles over one phase's tiles.  enumerate: a callable enumerating the
// CTA's tiles (ws_tiles1 / ws_tiles2 bound to their arguments); out(T, m, r,
// c, v): stores row r of M tile m, column c of the tile, to its destination.
template <int MT, class TileT, class Enum, class Out>
__device__ void ws_run(WsCtl& ctl, const WsRing& ring, int nmax, const uint4* pack, long long lim, Enum&& enumerate,
                       Out&& out) {
    using G = WsGeom<MT>;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &ctl.abort;
    const uint32_t accs = 4u * nmax;  // columns of one accumulator
    const uint32_t nbuf = (uint32_t)G::nbuf(nmax);
    if (warp == kWsWarpTma) {
        // ---- A copies, one thread
        if (lane == 0) {
            uint32_t g = 0;
            enumerate([&](const TileT& T, int, int) -> bool {
                for (int st = 0; st < T.nst; ++st, ++g) {
                    const uint32_t slot = g % ring.ns;
                    if (g >= ring.ns && !mbar_wait_lim(smem_u32(&ctl.empty[slot]), ((g / ring.ns) - 1) & 1, lim))
                        *abort = 1;
                    if (*abort) return false;
                    const uint32_t mb = smem_u32(&ctl.full_a[slot]);
                    if (MT == 1) {
                        mbar_expect_tx(mb, kStageBytesA);
                        tma_bulk(smem_u32(ring.a(slot)), pack + (T.pk[0] + st) * kStageChunksA, kStageBytesA, mb);
                    } else {
                        // M tile m, plane p: chunks 2h kM .. 2h kM + 2 kM of plane p of
                        // packed stage st / 2 (h = st mod 2), 4 KiB
                        const int nt = T.rows[1] > 0 ? 2 : 1;
                        mbar_expect_tx(mb, nt * G::kTileBytes);
                        for (int m = 0; m < nt; ++m)
                            for (int p = 0; p < 4; ++p)
                                tma_bulk(smem_u32(ring.a(slot)) + m * G::kTileBytes + p * G::kPlaneBytes,
                                         pack + (T.pk[m] + st / 2) * kStageChunksA + p * kChunksA +
                                             (st & 1) * 2 * kM,
                                         G::kPlaneBytes, mb);
                    }
                    ctl.g_tma = g + 1;
                }
                return true;
            });
        }
        __syncwarp();
    } else if (warp >= kWsWarpB0 && warp < kWsWarpMma) {
        // ---- B operands: group q (two warps, 64 threads) takes the stages
        // g = q mod G and fills ring slot g mod ns, G = min(4, ns) groups.  It
        // loads a stage's values into registers before it waits for the slot,
        // so the gather from L2 overlaps the MMAs that still read the slot.
        // G <= ns keeps every wait on a slot's "empty" barrier within one
        // phase of it: the group's previous stage g - G waited for the MMAs of
        // stage g - G - ns >= g - 2 ns, so the phase of stage g - ns that this
        // wait asks for is the barrier's current or last completed one, never
        // one that a parity test would confuse with an older phase.
        const int q = (warp - kWsWarpB0) >> 1;
        const int gtid = tid - (kWsWarpB0 + 2 * q) * 32;
        const uint32_t ngroups = ring.ns < (uint32_t)kWsGroups ? ring.ns : (uint32_t)kWsGroups;
        uint32_t g = 0;
        if ((uint32_t)q < ngroups) enumerate([&](const TileT& T, int, int) -> bool {
            for (int st = 0; st < T.nst; ++st, ++g) {
                if (g % ngroups != (uint32_t)q) continue;
                const uint32_t slot = g % ring.ns;
                // all loads of the stage first (up to four segments of 8 values
                // per thread), then the wait, the split and the stores;
                // neighbouring threads take neighbouring columns of one K
                // chunk, so their 16-byte stores fill whole shared-memory
                // wavefronts
                const int nm = T.nmma, nseg = nm * G::KQ;
                float2 vb[4][8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int seg = gtid + 64 * u;
                    if (seg < nseg) T.src.load_b(seg % nm, seg / nm, st * G::KS, vb[u]);
                }
                if (g >= ring.ns) {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait_lim(smem_u32(&ctl.empty[slot]), ((g / ring.ns) - 1) & 1, lim);
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) *abort = 1;
                }
                if (*abort) return false;
                uint4* b0 = ring.b(slot, 0);
                uint4* b1 = ring.b(slot, 1);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int seg = gtid + 64 * u;
                    if (seg < nseg) put8_ws(b0, b1, nm, seg % nm, seg / nm, vb[u]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl.full_b[slot]));
            }
            return true;
        });
    } else if (warp == kWsWarpMma) {
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t g = 0, t = 0;
            enumerate([&](const TileT& T, int, int) -> bool {
                if (T.nst == 0) return true;
                const uint32_t ab = t % nbuf, use = t / nbuf;
                if (use >= 1 && !mbar_wait_lim(smem_u32(&ctl.acc_empty[ab]), (use - 1) & 1, lim)) {
                    *abort = 1;
                    return false;
                }
                const uint32_t tm = ctl.tmem + ab * MT * accs;
                const int nt = T.rows[1] > 0 && MT == 2 ? 2 : 1;
                for (int st = 0; st < T.nst; ++st, ++g) {
                    const uint32_t slot = g % ring.ns, par = (g / ring.ns) & 1;
                    if (*abort || !mbar_wait_lim(smem_u32(&ctl.full_a[slot]), par, lim) ||
                        !mbar_wait_lim(smem_u32(&ctl.full_b[slot]), par, lim)) {
                        *abort = 1;
                        return false;
                    }
                    fence_after();
                    const uint32_t a = smem_u32(ring.a(slot)), b0 = smem_u32(ring.b(slot, 0)),
                                   b1 = smem_u32(ring.b(slot, 1));
                    const uint32_t lbob = (uint32_t)(4 * T.nmma * 16);
#pragma unroll
                    for (int ks = 0; ks < G::KSTEPS; ++ks)
                        for (int m = 0; m < nt; ++m)
                            mma_kstep_ws(a + m * G::kTileBytes + ks * 2 * kLboA, G::kPlaneBytes, b0 + ks * 2 * lbob,
                                         b1 + ks * 2 * lbob, tm + m * accs, T.nmma, (st == 0 && ks == 0) ? 0u : 1u);
                    umma_commit(smem_u32(&ctl.empty[slot]));
                    ctl.g_mma = g + 1;
                }
                umma_commit(smem_u32(&ctl.acc_full[ab]));
                ++t;
                return true;
            });
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 0-3, tensor-memory lane quarter = warp)
        uint32_t t = 0;
        const int r = warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        enumerate([&](const TileT& T, int, int) -> bool {
            const int ncol = T.src.ncol;
            const int nt = T.rows[1] > 0 && MT == 2 ? 2 : 1;
            if (T.nst == 0) {
                for (int m = 0; m < nt; ++m)
                    if (r < T.rows[m])
                        for (int c = 0; c < ncol; ++c) out(T, m, r, c, make_float2(0.f, 0.f));
                return true;
            }
            const uint32_t ab = t % nbuf, use = t / nbuf;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_lim(smem_u32(&ctl.acc_full[ab]), use & 1, lim);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                *abort = 1;
                return false;
            }
            fence_after();
            const int nm = T.nmma;
            for (int m = 0; m < nt; ++m) {
                const uint32_t base = ctl.tmem + (ab * MT + m) * accs + lane_base;
                for (int cb = 0; cb < ncol; cb += 16) {
                    float ra[16], ia[16], rb[16], ib[16];
                    tmem_ld16(base + cb, ra);
                    tmem_ld16(base + nm + cb, ia);
                    tmem_ld16(base + 2 * nm + cb, rb);
                    tmem_ld16(base + 3 * nm + cb, ib);
                    tmem_wait_ld();
                    if (r < T.rows[m]) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (cb + i < ncol) out(T, m, r, cb + i, make_float2(ra[i] + rb[i], ia[i] + ib[i]));
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.acc_empty[ab]));
            ++t;
            return true;
        });
    }
}

template <int MT>
__global__ void __launch_bounds__(kWsThr, 1) u1w_kernel(const FarBlockDev* __restrict__ blocks,
                                                        const int* __restrict__ batoms, const int4* __restrict__ items,
                                                        const int4* __restrict__ items_b,
                                                        const int* __restrict__ cta_ptr,
                                                        const long long* __restrict__ pk,
                                                        const long long* __restrict__ pk_b,
                                                        const uint4* __restrict__ pack, const int* __restrict__ rowt,
                                                        const float2* __restrict__ x, int64_t ldx, int np,
                                                        float2* __restrict__ t, int64_t ldt, int nrhs,
                                                        const int2* __restrict__ colr, int nmax, int* err,
                                                        long long lim) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const WsRing ring = ws_ring<MT>(smem, nmax);
    __shared__ WsCtl ctl;
    ws_setup(ctl, ring.ns);
    const int it0 = cta_ptr[blockIdx.x], it1 = cta_ptr[blockIdx.x + 1];
    ws_run<MT, WsTile1>(
        ctl, ring, nmax, pack, lim,
        [&](auto&& role) {
            ws_tiles1<MT>(blocks, batoms, items, items_b, pk, pk_b, it0, it1, rowt, x, ldx, np, nrhs, colr,
                          &ctl.abort, role);
        },
        [&](const WsTile1& T, int m, int r, int c, float2 v) {
            t[(int64_t)T.rt[m][r] + (int64_t)(T.src.c0 + c) * ldt] = v;
        });
    ws_teardown(ctl, ring.ns, err);
}

template <int MT>
__global__ void __launch_bounds__(kWsThr, 1) u2w_kernel(const int4* __restrict__ items,
                                                        const int4* __restrict__ items_b,
                                                        const int* __restrict__ cta_ptr,
                                                        const long long* __restrict__ pk,
                                                        const long long* __restrict__ pk_b,
                                                        const uint4* __restrict__ pack, const int* __restrict__ tidx,
                                                        const long long* __restrict__ kptr,
                                                        const float2* __restrict__ t, int64_t ldt, int np,
                                                        float2* __restrict__ F, int64_t ldf, int nrhs,
                                                        const int2* __restrict__ colr, int nmax, int* err,
                                                        long long lim) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const WsRing ring = ws_ring<MT>(smem, nmax);
    __shared__ WsCtl ctl;
    ws_setup(ctl, ring.ns);
    const int it0 = cta_ptr[blockIdx.x], it1 = cta_ptr[blockIdx.x + 1];
    ws_run<MT, WsTile2>(
        ctl, ring, nmax, pack, lim,
        [&](auto&& role) {
            ws_tiles2<MT>(items, items_b, pk, pk_b, it0, it1, tidx, kptr, t, ldt, np, nrhs, colr, &ctl.abort, role);
        },
        [&](const WsTile2& T, int m, int r, int c, float2 v) { F[T.rb[m] + r + (int64_t)(T.src.c0 + c) * ldf] = v; });
    ws_teardown(ctl, ring.ns, err);
}

std::once_flag g_umma_attr_once;

}  // namespace

void umma_prepare(Op& op, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "the tcgen05 apply needs VIE_C64 factors");
    build_umma_lists(op);
    std::call_once(g_umma_attr_once, [] {
        cudaFuncSetAttribute(u1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        cudaFuncSetAttribute(u2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        cudaFuncSetAttribute(u1p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        cudaFuncSetAttribute(u2p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        cudaFuncSetAttribute(u1w_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemBytes);
        cudaFuncSetAttribute(u2w_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemBytes);
        cudaFuncSetAttribute(u1w_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemBytes);
        cudaFuncSetAttribute(u2w_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemBytes);
    });
    if (!op.d_err.p) {
        op.d_err.alloc(sizeof(int));
        VIE_CUDA(cudaMemsetAsync(op.d_err.p, 0, sizeof(int), s));
    }
}

void apply_far_umma(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    umma_prepare(op, s);
    if (((uintptr_t)x & 15) || (ldx & 1)) fail(VIE_ERR_INVALID_ARG, "tensor-core apply: x must be 16-byte aligned");
    const size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const float2* fac = op.fac<float2>();
    if (op.n_u1_items > 0) {
        u1_kernel<<<op.n_cta_u, kThr, kSmemBytes, s>>>(
            op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(), op.d_u1_items.as<int4>(), op.d_u1_cta.as<int>(),
            op.d_u1_rowoff.as<long long>(), op.d_u1_rowt.as<int>(), fac, x, ldx, op.np, op.d_t.as<float2>(),
            op.t_total, nrhs, op.colr, op.d_err.as<int>());
        VIE_CHECK_LAUNCH();
    }
    u2_kernel<<<op.n_cta_u, kThr, kSmemBytes, s>>>(
        op.d_u2_items.as<int4>(), op.d_u2_cta.as<int>(), op.d_u2_qoff.as<long long>(), op.d_u2_tidx.as<int>(),
        op.d_u2_kptr.as<long long>(), fac, op.d_t.as<float2>(), op.t_total, op.np, F, ldf, nrhs, op.colr,
        op.d_err.as<int>());
    VIE_CHECK_LAUNCH();
}

size_t umma_pack_bytes(const Op& op) { return (size_t)(op.u1_stages + op.u2_stages) * kStageBytesA; }

bool umma_pack(Op& op, cudaStream_t s) {
    umma_prepare(op, s);
    if (op.umma_packed) return true;
    if (op.umma_pack_failed) return false;
    const size_t b1 = (size_t)op.u1_stages * kStageBytesA, b2 = (size_t)op.u2_stages * kStageBytesA;
    size_t free_b = 0, total_b = 0;
    VIE_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (b1 + b2 + ((size_t)1 << 30) > free_b) {  // keep 1 GiB for the solver
        op.umma_pack_failed = true;
        return false;
    }
    op.d_u1_pack.alloc(std::max<size_t>(b1, 16));
    op.d_u2_pack.alloc(std::max<size_t>(b2, 16));
    if (op.n_u1_items > 0) {
        pack1_kernel<<<op.n_u1_items, kThr, 0, s>>>(op.d_blocks.as<FarBlockDev>(), op.d_u1_items.as<int4>(),
                                                    op.d_u1_pk.as<long long>(), op.d_u1_rowoff.as<long long>(),
                                                    op.fac<float2>(), op.np, op.d_u1_pack.as<uint4>());
        VIE_CHECK_LAUNCH();
    }
    if (op.n_u2_items > 0) {
        pack2_kernel<<<op.n_u2_items, kThr, 0, s>>>(op.d_u2_items.as<int4>(), op.d_u2_pk.as<long long>(),
                                                    op.d_u2_qoff.as<long long>(), op.d_u2_kptr.as<long long>(),
                                                    op.fac<float2>(), op.d_u2_pack.as<uint4>());
        VIE_CHECK_LAUNCH();
    }
    op.umma_packed = true;
    return true;
}

void apply_far_umma_packed(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    if (!umma_pack(op, s)) {  // not enough memory for the packed planes: the kernel that splits A itself
        apply_far_umma(op, x, ldx, F, ldf, nrhs, s);
        return;
    }
    if (((uintptr_t)x & 15) || (ldx & 1)) fail(VIE_ERR_INVALID_ARG, "tensor-core apply: x must be 16-byte aligned");
    const size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    if (op.n_u1_items > 0) {
        u1p_kernel<<<op.n_cta_u, kThr, kSmemBytes, s>>>(
            op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(), op.d_u1_items.as<int4>(), op.d_u1_cta.as<int>(),
            op.d_u1_pk.as<long long>(), op.d_u1_pack.as<uint4>(), op.d_u1_rowt.as<int>(), x, ldx, op.np,
            op.d_t.as<float2>(), op.t_total, nrhs, op.colr, op.d_err.as<int>());
        VIE_CHECK_LAUNCH();
    }
    u2p_kernel<<<op.n_cta_u, kThr, kSmemBytes, s>>>(
        op.d_u2_items.as<int4>(), op.d_u2_cta.as<int>(), op.d_u2_pk.as<long long>(), op.d_u2_pack.as<uint4>(),
        op.d_u2_tidx.as<int>(), op.d_u2_kptr.as<long long>(), op.d_t.as<float2>(), op.t_total, op.np, F, ldf, nrhs,
        op.colr, op.d_err.as<int>());
    VIE_CHECK_LAUNCH();
}

// Wait limit of the warp-specialised kernels in clock cycles: ~1 s, or the
// value of VIE_TEST_WAIT_CYCLES (a test of the timeout path sets it to 0 so
// that the first wait gives up; the kernels then drain and report).
static long long ws_wait_limit() {
    const char* e = std::getenv("VIE_TEST_WAIT_CYCLES");
    if (e && *e) {
        const long long v = std::atoll(e);
        return v < 0 ? 0 : v;
    }
    return kWaitCycles;
}

// MT = 1: variant 9 over the one-CTA-per-SM item lists; MT = 2: variant 10
// over the lists of item pairs that share their B operand.
template <int MT>
static void apply_far_ws(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    if (!umma_pack(op, s)) {  // not enough memory for the packed planes: the kernel that splits A itself
        apply_far_umma(op, x, ldx, F, ldf, nrhs, s);
        return;
    }
    if (((uintptr_t)x & 15) || (ldx & 1)) fail(VIE_ERR_INVALID_ARG, "tensor-core apply: x must be 16-byte aligned");
    const size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(float2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const long long lim = ws_wait_limit();
    const int nc = op.ctx->n_sm;
    // the widest tile: 64 columns, or all of them when fewer (a tile never
    // spans two problems' column ranges, so it is no wider than this either)
    const int nmax = std::max(16, (std::min(nrhs, kN) + 15) / 16 * 16);
    const size_t smem = (size_t)WsGeom<MT>::stages(nmax) * WsGeom<MT>::stride(nmax);
    const bool two = MT == 2;
    if (op.n_u1_items > 0) {
        u1w_kernel<MT><<<nc, kWsThr, smem, s>>>(
            op.d_blocks.as<FarBlockDev>(), op.d_block_atoms.as<int>(),
            (two ? op.d_x1_items : op.d_w1_items).as<int4>(), two ? op.d_x1_items_b.as<int4>() : nullptr,
            (two ? op.d_x1_cta : op.d_w1_cta).as<int>(), (two ? op.d_x1_pk : op.d_w1_pk).as<long long>(),
            two ? op.d_x1_pk_b.as<long long>() : nullptr, op.d_u1_pack.as<uint4>(), op.d_u1_rowt.as<int>(), x, ldx,
            op.np, op.d_t.as<float2>(), op.t_total, nrhs, op.colr, nmax, op.d_err.as<int>(), lim);
        VIE_CHECK_LAUNCH();
    }
    u2w_kernel<MT><<<nc, kWsThr, smem, s>>>(
        (two ? op.d_x2_items : op.d_w2_items).as<int4>(), two ? op.d_x2_items_b.as<int4>() : nullptr,
        (two ? op.d_x2_cta : op.d_w2_cta).as<int>(), (two ? op.d_x2_pk : op.d_w2_pk).as<long long>(),
        two ? op.d_x2_pk_b.as<long long>() : nullptr, op.d_u2_pack.as<uint4>(), op.d_u2_tidx.as<int>(),
        op.d_u2_kptr.as<long long>(), op.d_t.as<float2>(), op.t_total, op.np, F, ldf, nrhs, op.colr, nmax,
        op.d_err.as<int>(), lim);
    VIE_CHECK_LAUNCH();
}

void apply_far_umma_ws(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    apply_far_ws<1>(op, x, ldx, F, ldf, nrhs, s);
}

void apply_far_umma_ws2(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s) {
    apply_far_ws<2>(op, x, ldx, F, ldf, nrhs, s);
}

}  // namespace vie
