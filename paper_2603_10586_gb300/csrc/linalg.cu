#include <algorithm>
// Dense kernels around the self blocks (paper Sec. 4, eq. diagprecond):
// explicit inverse of each distinct Z_ii by Gauss-Jordan elimination with
// partial pivoting (float64), precision conversions, and the per-type block
// product Y = M B (+ A) over all atoms of one type (the self part of the
// operator, the preconditioner and the fused P^-1 Z form).
#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

// The augmented matrix Maug = [A | I] is np x 2np, column-major (ld = np).
// one block: pick the pivot of column k, swap rows, normalise the pivot row,
// save the elimination factors of column k
__global__ void gj_pivot(double2* M, int np, int k, double2* fac, int* status) {
    __shared__ double best[1024];
    __shared__ int bidx[1024];
    double b = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < np; i += blockDim.x) {
        double2 v = M[i + (int64_t)k * np];
        double a = v.x * v.x + v.y * v.y;
        if (a > b) { b = a; bi = i; }
    }
    best[threadIdx.x] = b;
    bidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            double o = best[threadIdx.x + s];
            int oi = bidx[threadIdx.x + s];
            if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
                best[threadIdx.x] = o;
                bidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    int p = bidx[0];
    if (best[0] <= 0.0) {
        if (threadIdx.x == 0) *status = 1;
        return;
    }
    // swap rows k and p
    if (p != k)
        for (int j = threadIdx.x; j < 2 * np; j += blockDim.x) {
            double2 a = M[k + (int64_t)j * np], c = M[p + (int64_t)j * np];
            M[k + (int64_t)j * np] = c;
            M[p + (int64_t)j * np] = a;
        }
    __syncthreads();
    double2 piv = M[k + (int64_t)k * np];
    double den = piv.x * piv.x + piv.y * piv.y;
    double2 inv = make_double2(piv.x / den, -piv.y / den);
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * np; j += blockDim.x) M[k + (int64_t)j * np] = cmul(M[k + (int64_t)j * np], inv);
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) fac[i] = i == k ? make_double2(0, 0) : M[i + (int64_t)k * np];
}

__global__ void gj_eliminate(double2* M, int np, int k, const double2* fac) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t cols = 2 * np - k;
    if (t >= (int64_t)np * cols) return;
    int i = (int)(t % np);
    int j = k + (int)(t / np);
    if (i == k) return;
    double2 f = fac[i];
    double2 r = M[k + (int64_t)j * np];
    double2 v = M[i + (int64_t)j * np];
    v.x -= f.x * r.x - f.y * r.y;
    v.y -= f.x * r.y + f.y * r.x;
    M[i + (int64_t)j * np] = v;
}

// Maug = [A | I] and the extraction of A^-1, through device pointer tables (a
// captured graph replays them for several blocks)
__global__ void gj_init_ptr(const double2* const* A, double2* M, int np) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)np * 2 * np) return;
    int i = (int)(t % np), j = (int)(t / np);
    M[t] = j < np ? (*A)[i + (int64_t)j * np] : make_double2(i == j - np ? 1.0 : 0.0, 0.0);
}

__global__ void gj_extract_ptr(const double2* M, double2* const* inv, int np) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)np * np) return;
    (*inv)[t] = M[t + (int64_t)np * np];
}

__global__ void c128_to_c64(const double2* s, float2* d, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) d[t] = make_float2((float)s[t].x, (float)s[t].y);
}
__global__ void c64_to_c128(const float2* s, double2* d, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) d[t] = make_double2(s[t].x, s[t].y);
}

// ---------------------------------------------------------------------------
// Y[:, col] = M B[:, col] (+ ADD[:, col]) for the columns col = (atom of the
// type, rhs).  M: np x np column-major.  Vector element (row r of atom a, rhs c)
// lives at a * np + r + c * ld.  32 x 32 output tile per CTA (enough CTAs for a
// few hundred atoms), 256 threads, each a 2 x 2 sub-tile; K staged through
// shared memory 32 at a time.
// ADD may be Y itself (y = Z_ii x + y in place): every output element is read
// from ADD and then written to Y by the one thread that owns it, so ADD and Y
// carry no __restrict__ and ADD is read through the ordinary (coherent) path.
// B must not overlap Y.
// ---------------------------------------------------------------------------
template <class TM, class TX>
__global__ void __launch_bounds__(256) type_gemm(const TM* __restrict__ M, int np, const int* __restrict__ atoms,
                                                 int n_atoms, int nrhs, const TX* __restrict__ B, int64_t ldb,
                                                 const TX* ADD, int64_t ldadd, TX* Y, int64_t ldy,
                                                 const int2* __restrict__ colr, int prob) {
    using R = decltype(TM().x);
    using TA = typename C2<R>::t;
    constexpr int BM = 32, BN = 32, BK = 32;
    __shared__ TA sM[BK][BM + 1];
    __shared__ TA sB[BK][BN + 1];
    // right-hand sides of this type's problem (all of them for a single operator)
    const int2 cr = colr ? colr[prob] : make_int2(0, nrhs);
    const int ncols = n_atoms * (cr.y - cr.x);
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
    if (col0 >= ncols) return;
    const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;  // 16 x 16 threads, 2 x 2 each
    TA acc[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc[a][b] = mk(R(0), R(0));
    // column -> (atom, rhs) base offsets for the B loads of this tile
    for (int k0 = 0; k0 < np; k0 += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += 256) {
            int kk = e / BM, r = e % BM;
            int gr = row0 + r, gk = k0 + kk;
            sM[kk][r] = (gr < np && gk < np) ? cvt<TA>(M[gr + (int64_t)gk * np]) : mk(R(0), R(0));
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            int kk = e % BK, c = e / BK;
            int gc = col0 + c, gk = k0 + kk;
            TA v = mk(R(0), R(0));
            if (gc < ncols && gk < np) {
                int a = atoms[gc % n_atoms], rhs = cr.x + gc / n_atoms;
                v = cvt<TA>(B[(int64_t)a * np + gk + (int64_t)rhs * ldb]);
            }
            sB[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            TA mv[2], bv[2];
            for (int a = 0; a < 2; ++a) mv[a] = sM[kk][tr + 16 * a];
            for (int b = 0; b < 2; ++b) bv[b] = sB[kk][tc + 16 * b];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) cfma(acc[a][b], mv[a], bv[b]);
        }
        __syncthreads();
    }
    for (int b = 0; b < 2; ++b) {
        int gc = col0 + tc + 16 * b;
        if (gc >= ncols) continue;
        int a_ = atoms[gc % n_atoms], rhs = cr.x + gc / n_atoms;
        for (int a = 0; a < 2; ++a) {
            int gr = row0 + tr + 16 * a;
            if (gr >= np) continue;
            TA v = acc[a][b];
            if (ADD) v += cvt<TA>(ADD[(int64_t)a_ * np + gr + (int64_t)rhs * ldadd]);
            Y[(int64_t)a_ * np + gr + (int64_t)rhs * ldy] = cvt<TX>(v);
        }
    }
}

}  // namespace

void invert_self_blocks(Op& op) {
    const int np = op.np;
    cudaStream_t s = op.ctx->stream;
    op.d_inv64.alloc((size_t)op.T * np * np * sizeof(double2));
    DevBuf M((size_t)np * 2 * np * sizeof(double2)), fac(np * sizeof(double2)), st(sizeof(int));
    VIE_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
    // the 2 np pivot and elimination launches of a type are captured once into
    // a CUDA graph and replayed for every type (one graph launch per type
    // instead of 2 np kernel launches); the graph reads the type's block
    // through the pointer table `src`
    DevBuf src(sizeof(const double2*)), dst(sizeof(double2*));
    cudaGraphExec_t exec = nullptr;
    {
        VIE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            const int64_t tot = (int64_t)np * 2 * np;
            gj_init_ptr<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src.as<const double2*>(), M.as<double2>(), np);
            for (int k = 0; k < np; ++k) {
                gj_pivot<<<1, 1024, 0, s>>>(M.as<double2>(), np, k, fac.as<double2>(), st.as<int>());
                int64_t work = (int64_t)np * (2 * np - k);
                gj_eliminate<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(M.as<double2>(), np, k,
                                                                            fac.as<double2>());
            }
            gj_extract_ptr<<<(unsigned)(((int64_t)np * np + 255) / 256), 256, 0, s>>>(M.as<double2>(),
                                                                                     dst.as<double2*>(), np);
        } catch (...) {
            cudaStreamEndCapture(s, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw;
        }
        VIE_CUDA(cudaStreamEndCapture(s, &graph));
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) fail(VIE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    struct ExecGuard {
        cudaGraphExec_t e;
        ~ExecGuard() { cudaGraphExecDestroy(e); }
    } guard{exec};
    for (int t = 0; t < op.T; ++t) {
        const double2* A = op.d_zself64.as<double2>() + (size_t)t * np * np;
        double2* Inv = op.d_inv64.as<double2>() + (size_t)t * np * np;
        VIE_CUDA(cudaMemcpyAsync(src.p, &A, sizeof(A), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(dst.p, &Inv, sizeof(Inv), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaGraphLaunch(exec, s));
        VIE_CUDA(cudaStreamSynchronize(s));  // the pointer table is rewritten for the next type
        VIE_COUNT_LAUNCH(2 * np + 2);
    }
    int status = 0;
    VIE_CUDA(cudaMemcpyAsync(&status, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    if (status) fail(VIE_ERR_BREAKDOWN, "a meta-atom self block is singular");
}

void convert_c128_to_c64(const void* src, void* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    c128_to_c64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)src, (float2*)dst, n);
    VIE_CHECK_LAUNCH();
}
void convert_c64_to_c128(const void* src, void* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    c64_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float2*)src, (double2*)dst, n);
    VIE_CHECK_LAUNCH();
}

template <class T2>
__global__ void k_conj(const T2* src, T2* dst, int64_t n) {  // may run in place
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T2 v = src[i];
        dst[i] = mk(v.x, -v.y);
    }
}

template <class T2>
__global__ void k_conj_transpose(const T2* __restrict__ src, T2* __restrict__ dst, int np) {
    const int64_t base = (int64_t)blockIdx.y * np * np;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)np * np;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % np, c = e / np;
        const T2 v = src[base + c + r * np];  // element (c, r) of the source
        dst[base + e] = mk(v.x, -v.y);
    }
}

void conj_copy(const void* src, void* dst, int64_t n, bool c128, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned g = (unsigned)std::min<int64_t>(8192, (n + 255) / 256);
    if (c128) k_conj<double2><<<g, 256, 0, s>>>((const double2*)src, (double2*)dst, n);
    else k_conj<float2><<<g, 256, 0, s>>>((const float2*)src, (float2*)dst, n);
    VIE_CHECK_LAUNCH();
}

void conj_transpose_blocks(const void* src, void* dst, int T, int np, bool c128, cudaStream_t s) {
    const dim3 g((unsigned)std::min<int64_t>(1024, ((int64_t)np * np + 255) / 256), T);
    if (c128) k_conj_transpose<double2><<<g, 256, 0, s>>>((const double2*)src, (double2*)dst, np);
    else k_conj_transpose<float2><<<g, 256, 0, s>>>((const float2*)src, (float2*)dst, np);
    VIE_CHECK_LAUNCH();
}

// mode 0: Y = M X + C   (self part plus far part C)
// mode 1: Y = X + M C   (fused preconditioner: X + Z_D^-1 (far part))
// mode 2: Y = M X       (plain block product, e.g. the preconditioner)
template <class TM, class TX>
void self_gemm(Op& op, const TM* M, const TX* X, int64_t ldx, const TX* C, int64_t ldc, TX* Y, int64_t ldy,
               int nrhs, int mode, cudaStream_t s) {
    const int np = op.np;
    for (int t = 0; t < op.T; ++t) {
        int na = op.type_atom_off[t + 1] - op.type_atom_off[t];
        if (na == 0) continue;
        const int* atoms = op.d_atoms_by_type.as<int>() + op.type_atom_off[t];
        const TM* Mt = M + (size_t)t * np * np;
        dim3 grid((np + 31) / 32, (na * nrhs + 31) / 32);
        const TX* Bop = mode == 1 ? C : X;
        int64_t ldb = mode == 1 ? ldc : ldx;
        const TX* ADD = mode == 0 ? C : (mode == 1 ? X : nullptr);
        int64_t ldadd = mode == 0 ? ldc : ldx;
        const int prob = op.type_prob.empty() ? 0 : op.type_prob[t];
        type_gemm<TM, TX><<<grid, 256, 0, s>>>(Mt, np, atoms, na, nrhs, Bop, ldb, ADD, ldadd, Y, ldy, op.colr, prob);
        VIE_CHECK_LAUNCH();
    }
}

template void self_gemm<float2, float2>(Op&, const float2*, const float2*, int64_t, const float2*, int64_t,
                                        float2*, int64_t, int, int, cudaStream_t);
template void self_gemm<double2, double2>(Op&, const double2*, const double2*, int64_t, const double2*, int64_t,
                                          double2*, int64_t, int, int, cudaStream_t);

}  // namespace vie
