// Far-apply variants and the autotuner that chooses between them.
//
// The far part of a complex float32 apply has several implementations: the
// SIMT kernels with 1, 2, 4 or 8 right-hand sides per factor read (register
// tiles), the SIMT kernels that apply translated copies of a block together
// (one factor read per group of copies), and for split-precision requests the
// warp-MMA and the tcgen05 tensor-core kernels.  Which is fastest depends on the right-hand-side count
// and on the operator (rank distribution, atom size), so the choice is made by
// timing on the operator itself and is remembered per power-of-two bucket of
// the right-hand-side count.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace vie {

namespace {

int bucket(int nrhs) {
    int b = 0;
    while ((2 << b) <= nrhs && b < 30) ++b;
    return b;
}

bool admissible(int precision, int v) {
    if ((v >= VIE_VAR_SIMT_R1 && v <= VIE_VAR_SIMT_R8) || v == VIE_VAR_SIMT_SHARED) return true;
    return precision == VIE_BF16X3 &&
           (v == VIE_VAR_MMA_BF16X3 || v == VIE_VAR_TCGEN05_BF16X3 || v == VIE_VAR_TCGEN05_PACKED_BF16X3 ||
            v == VIE_VAR_TCGEN05_WS_BF16X3 || v == VIE_VAR_TCGEN05_WS2_BF16X3);
}

int default_variant(const Op& op, int precision, int nrhs) {
    // one right-hand side: read shared factors once per group of copies when
    // the operator has translated copies
    if (nrhs == 1) return op.share_mean > 1.5 ? VIE_VAR_SIMT_SHARED : VIE_VAR_SIMT_R1;
    // BF16x3: the warp-specialised kernel with one row tile per B tile streams
    // the A planes fastest while the B operand is narrow (8.6 ms per apply of
    // the 32 x 32 array of 4^3 cubes at 16 columns); wider, the gathers of B
    // bound it and two row tiles per B tile win (9.7 / 11.3 / 12.7 ms at 32 /
    // 48 / 64 columns, against 11.2 / 16.4 / 19.8 ms)
    if (precision == VIE_BF16X3 && nrhs >= 8)
        return nrhs <= 16 ? VIE_VAR_TCGEN05_WS_BF16X3 : VIE_VAR_TCGEN05_WS2_BF16X3;
    return VIE_VAR_SIMT_R4;
}

}  // namespace

int far_variant(const Op& op, int precision, int nrhs) {
    auto it = op.variant.find({precision, bucket(nrhs)});
    return it != op.variant.end() ? it->second : default_variant(op, precision, nrhs);
}

void far32(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, int precision, cudaStream_t s) {
    switch (far_variant(op, precision, nrhs)) {
        case VIE_VAR_SIMT_R1: apply_far_simt32(op, x, ldx, F, ldf, nrhs, 1, s); break;
        case VIE_VAR_SIMT_R2: apply_far_simt32(op, x, ldx, F, ldf, nrhs, 2, s); break;
        case VIE_VAR_SIMT_R4: apply_far_simt32(op, x, ldx, F, ldf, nrhs, 4, s); break;
        case VIE_VAR_SIMT_R8: apply_far_simt32(op, x, ldx, F, ldf, nrhs, 8, s); break;
        case VIE_VAR_MMA_BF16X3: apply_far_bf16x3(op, x, ldx, F, ldf, nrhs, s); break;
        case VIE_VAR_TCGEN05_BF16X3: apply_far_umma(op, x, ldx, F, ldf, nrhs, s); break;
        case VIE_VAR_TCGEN05_PACKED_BF16X3: apply_far_umma_packed(op, x, ldx, F, ldf, nrhs, s); break;
        case VIE_VAR_SIMT_SHARED: apply_far_shared(op, x, ldx, F, ldf, nrhs, s); break;
        case VIE_VAR_TCGEN05_WS_BF16X3: apply_far_umma_ws(op, x, ldx, F, ldf, nrhs, s); break;
        case VIE_VAR_TCGEN05_WS2_BF16X3: apply_far_umma_ws2(op, x, ldx, F, ldf, nrhs, s); break;
        default: fail(VIE_ERR_STATE, "unknown far-apply variant");
    }
}

int tune_far(Op& op, int precision, int nrhs, cudaStream_t s, std::vector<int>& cand, std::vector<double>& ms) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "vie_tune: needs VIE_C64 factors");
    if (precision != VIE_C64 && precision != VIE_BF16X3) fail(VIE_ERR_INVALID_ARG, "vie_tune: VIE_C64 or VIE_BF16X3");
    if (nrhs < 1 || nrhs > 1024) fail(VIE_ERR_INVALID_ARG, "vie_tune: 1 to 1024 right-hand sides");
    cand.clear();
    ms.clear();
    for (int v = VIE_VAR_SIMT_R1; v <= VIE_VAR_TCGEN05_WS2_BF16X3; ++v) {
        if (!admissible(precision, v)) continue;
        if (v >= VIE_VAR_SIMT_R2 && v <= VIE_VAR_SIMT_R8 && nrhs == 1) continue;  // same as R1
        if (v == VIE_VAR_SIMT_SHARED && nrhs > 1) continue;  // one column at a time
        cand.push_back(v);
    }
    const int64_t n = op.n();
    DevBuf x((size_t)n * nrhs * sizeof(float2)), F((size_t)n * nrhs * sizeof(float2));
    VIE_CUDA(cudaMemsetAsync(x.p, 0, (size_t)n * nrhs * sizeof(float2), s));
    if (precision == VIE_BF16X3) {
        umma_prepare(op, s);
        umma_pack(op, s);
    }
    cudaEvent_t e0, e1;
    VIE_CUDA(cudaEventCreate(&e0));
    VIE_CUDA(cudaEventCreate(&e1));
    // time all columns of the operator (a batched solve's column table does not apply here)
    struct ColrGuard {
        Op& o;
        const int2* saved;
        ~ColrGuard() { o.colr = saved; }
    } guard{op, op.colr};
    op.colr = nullptr;
    const auto key = std::make_pair(precision, bucket(nrhs));
    const auto saved = op.variant.find(key) != op.variant.end() ? op.variant[key] : 0;
    int best = 0;
    double best_ms = 1e300;
    try {
        for (int v : cand) {
            op.variant[key] = v;
            far32(op, x.as<float2>(), n, F.as<float2>(), n, nrhs, precision, s);  // warm-up
            double t = 1e300;
            for (int r = 0; r < 3; ++r) {
                VIE_CUDA(cudaEventRecord(e0, s));
                far32(op, x.as<float2>(), n, F.as<float2>(), n, nrhs, precision, s);
                VIE_CUDA(cudaEventRecord(e1, s));
                VIE_CUDA(cudaEventSynchronize(e1));
                float m = 0.f;
                VIE_CUDA(cudaEventElapsedTime(&m, e0, e1));
                t = std::min(t, (double)m);
            }
            ms.push_back(t);
            if (t < best_ms) {
                best_ms = t;
                best = v;
            }
        }
    } catch (...) {
        if (saved) op.variant[key] = saved;
        else op.variant.erase(key);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op.variant[key] = best;
    return best;
}

int tune_entry(Op& op, int precision, int nrhs, int force, vie_tune_result* res, cudaStream_t s) {
    std::vector<int> cand;
    std::vector<double> ms;
    int v;
    if (force > 0) {
        if (!admissible(precision, force)) fail(VIE_ERR_INVALID_ARG, "vie_tune: variant not admissible for precision");
        if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "vie_tune: needs VIE_C64 factors");
        if (nrhs < 1 || nrhs > 1024) fail(VIE_ERR_INVALID_ARG, "vie_tune: 1 to 1024 right-hand sides");
        op.variant[{precision, bucket(nrhs)}] = force;
        v = force;
    } else {
        v = tune_far(op, precision, nrhs, s, cand, ms);
    }
    if (res) {
        res->variant = v;
        res->n_candidates = (int)std::min<size_t>(16, cand.size());
        for (int i = 0; i < res->n_candidates; ++i) {
            res->candidates[i] = cand[i];
            res->ms[i] = ms[i];
        }
    }
    return VIE_OK;
}

bool tuned(const Op& op, int precision, int nrhs) { return op.variant.count({precision, bucket(nrhs)}) > 0; }

}  // namespace vie
