// Cross approximation with full pivoting of a batch of assembled far blocks
// (paper Sec. 6.5: the compressed operator is built by local assembly and then
// a "full-cross" approximation of each block, after Kurz, Rain and Rjasanow).
//
// Every block of the batch is held formed (m x n, column-major) and is turned
// into its residual in place.  Step k of one block takes the entry of largest
// modulus of the residual E_k, (i_k, j_k), with ties to the smallest column and
// then the smallest row, and removes the cross through it:
//   u_k = E_k[:, j_k] / s,  v_k = E_k[i_k, :] s / E_k[i_k, j_k],  s = |E_k[i_k, j_k]|^(1/2),
//   E_{k+1} = E_k - u_k v_k^T   (row i_k and column j_k set to zero).
// The two factors carry the same scale (|u|, |v| <= s).  The whole residual is
// at hand, so its Frobenius norm is exact, and a block stops at the first k with
// ||E_k||_F <= tol ||A||_F.  A ~ U V^T is stored as Q = U and R^H = conj(V),
// the layout the range finder writes (Q is then not orthonormal; the apply
// does not need it).
//
// One step is two launches over the blocks still active:
//   update: E -= u_k v_k^T tile by tile (128 rows x 64 columns per CTA, a
//           persistent grid over the active blocks' tiles), with the tile's
//           largest |e|^2, its position and its sum of |e|^2;
//   select: one CTA per block reduces the tile partials in a fixed order,
//           tests the stopping rule and writes the next cross into U and V.
// The residual pass is HBM-bound: a step reads and writes m n entries per
// active block; the tile partials and the crosses are O(m + n + tiles).
#include <algorithm>
#include <climits>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

constexpr int kXRows = 128;   // rows of a tile (one per thread)
constexpr int kXCols = 64;    // columns of a tile
constexpr int kXAhead = 8;    // columns each thread loads before it updates them
constexpr int kXSel = 256;    // threads of the select CTA

template <class R>
struct XPart {
    R val;      // largest |e|^2 of the tile
    int i, j;   // its position
    double ss;  // sum of |e|^2 over the tile
};

// (a, ja, ia) comes before (b, jb, ib): larger modulus, then smaller column, then smaller row
template <class R>
__device__ __forceinline__ bool before(R a, int ja, int ia, R b, int jb, int ib) {
    return a > b || (a == b && (ja < jb || (ja == jb && ia < ib)));
}

// fixed-order reduction of (val, i, j, ss) over a CTA of NT threads; thread 0 gets the result
template <class R, int NT>
__device__ __forceinline__ void cta_reduce(R& val, int& i, int& j, double& ss) {
    __shared__ R s_val[NT / 32];
    __shared__ int s_i[NT / 32], s_j[NT / 32];
    __shared__ double s_ss[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const R ov = __shfl_down_sync(0xffffffffu, val, off);
        const int oi = __shfl_down_sync(0xffffffffu, i, off);
        const int oj = __shfl_down_sync(0xffffffffu, j, off);
        ss += __shfl_down_sync(0xffffffffu, ss, off);
        if (before(ov, oj, oi, val, j, i)) {
            val = ov;
            i = oi;
            j = oj;
        }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_val[w] = val;
        s_i[w] = i;
        s_j[w] = j;
        s_ss[w] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int x = 1; x < NT / 32; ++x) {
            ss += s_ss[x];
            if (before(s_val[x], s_j[x], s_i[x], val, j, i)) {
                val = s_val[x];
                i = s_i[x];
                j = s_j[x];
            }
        }
    }
    __syncthreads();
}

__global__ void k_cross_init(int nb, int* rank, int* list0, int* cnt, unsigned long long* passes) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nb) {
        rank[q] = 0;
        list0[q] = q;
    }
    if (q == 0) {
        cnt[0] = nb;
        cnt[1] = 0;
        cnt[2] = 0;  // flags: 1 a block needs more room, 2 a residual is not finite
        *passes = 0;
    }
}

// E[q] -= u v^T for the active blocks (subtract = 0: scan A only), with the
// per-tile partials.  Units (active block, tile) run on a persistent grid.
template <class T2, class R>
__global__ void __launch_bounds__(kXRows) k_cross_update(T2* __restrict__ E, int m, int n, int64_t es,
                                                         const T2* __restrict__ U, int64_t us,
                                                         const T2* __restrict__ VH, int64_t vs,
                                                         const int* __restrict__ rank, const int2* __restrict__ piv,
                                                         const int* __restrict__ list, const int* __restrict__ cnt_in,
                                                         int* cnt_clear, int tiles_m, int ntile,
                                                         XPart<R>* __restrict__ part, int subtract) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt_clear = 0;
    const int64_t units = (int64_t)(*cnt_in) * ntile;
    for (int64_t w = blockIdx.x; w < units; w += gridDim.x) {
        const int q = list[w / ntile];
        const int t = (int)(w % ntile);
        const int i = (t % tiles_m) * kXRows + (int)threadIdx.x;
        const int j0 = (t / tiles_m) * kXCols;
        const int j1 = min(n, j0 + kXCols);
        T2* e = E + (int64_t)q * es;
        R best = R(-1);
        int bi = 0, bj = 0;
        R ssr = R(0);
        if (i < m) {
            T2 u = mk(R(0), R(0));
            const T2* vh = VH;
            int pi = -1, pj = -1;
            if (subtract) {
                const int k = rank[q];
                u = U[(int64_t)q * us + (int64_t)k * m + i];
                vh = VH + (int64_t)q * vs + (int64_t)k * n;
                const int2 p = piv[q];
                pi = p.x;
                pj = p.y;
            }
            for (int jb = j0; jb < j1; jb += kXAhead) {
                T2 x[kXAhead];
#pragma unroll
                for (int c = 0; c < kXAhead; ++c)
                    if (jb + c < j1) x[c] = e[i + (int64_t)(jb + c) * m];
#pragma unroll
                for (int c = 0; c < kXAhead; ++c) {
                    const int j = jb + c;
                    if (j < j1) {
                        if (subtract) {
                            const T2 h = vh[j];  // conj(v_j)
                            T2 y = x[c];
                            y.x -= u.x * h.x + u.y * h.y;
                            y.y -= u.y * h.x - u.x * h.y;
                            if (i == pi || j == pj) y = mk(R(0), R(0));
                            x[c] = y;
                            e[i + (int64_t)j * m] = y;
                        }
                        const R a = x[c].x * x[c].x + x[c].y * x[c].y;
                        ssr += a;
                        if (a > best) {
                            best = a;
                            bi = i;
                            bj = j;
                        }
                    }
                }
            }
        }
        double ss = (double)ssr;
        cta_reduce<R, kXRows>(best, bi, bj, ss);
        if (threadIdx.x == 0) part[(int64_t)q * ntile + t] = XPart<R>{best, bi, bj, ss};
    }
}

// One CTA per active block: the residual's norm and largest entry from the
// tile partials, the stopping rule, and the next cross into U and V.
template <class T2, class R>
__global__ void __launch_bounds__(kXSel) k_cross_select(const T2* __restrict__ E, int m, int n, int64_t es,
                                                        T2* __restrict__ U, int64_t us, T2* __restrict__ VH,
                                                        int64_t vs, int* rank, int2* piv,
                                                        const double* __restrict__ anorm2, double tol2, int rcap,
                                                        int rfull, const int* __restrict__ list_in,
                                                        const int* __restrict__ cnt_in, int* list_out, int* cnt_out,
                                                        int* flags, unsigned long long* passes, int ntile,
                                                        const XPart<R>* __restrict__ part, int counted,
                                                        double* resid2) {
    __shared__ int s_go, s_k, s_pi, s_pj;
    const int cnt = *cnt_in;
    for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
        const int q = list_in[w];
        const XPart<R>* pp = part + (int64_t)q * ntile;
        R best = R(-1);
        int bi = 0, bj = 0;
        double ss = 0.0;
        for (int t = threadIdx.x; t < ntile; t += kXSel) {
            const XPart<R> x = pp[t];
            ss += x.ss;
            if (before(x.val, x.j, x.i, best, bj, bi)) {
                best = x.val;
                bi = x.i;
                bj = x.j;
            }
        }
        cta_reduce<R, kXSel>(best, bi, bj, ss);
        if (threadIdx.x == 0) {
            const int k = rank[q] + (counted ? 1 : 0);
            rank[q] = k;
            resid2[q] = ss;
            int go = 1;
            if (!(ss <= 1e300)) {  // NaN or infinite residual
                atomicOr(flags, 2);
                go = 0;
            } else if (ss <= tol2 * anorm2[q] || !(best > R(0))) {
                go = 0;
            } else if (k >= rcap) {
                if (rcap < rfull) atomicOr(flags, 1);
                go = 0;
            }
            s_go = go;
            s_k = k;
            s_pi = bi;
            s_pj = bj;
            if (go) {
                piv[q] = make_int2(bi, bj);
                list_out[atomicAdd(cnt_out, 1)] = q;
                atomicAdd(passes, 1ull);
            }
        }
        __syncthreads();
        if (s_go) {
            const int k = s_k, pi = s_pi, pj = s_pj;
            const T2* e = E + (int64_t)q * es;
            const T2 p = e[pi + (int64_t)pj * m];
            const R ap = sqrt(p.x * p.x + p.y * p.y);
            const R sq = sqrt(ap);
            const R is = R(1) / sq;
            const R g = (sq / ap) / ap;
            const T2 f = mk(p.x * g, -p.y * g);  // s / p
            T2* uk = U + (int64_t)q * us + (int64_t)k * m;
            T2* vk = VH + (int64_t)q * vs + (int64_t)k * n;
            for (int i = threadIdx.x; i < m; i += kXSel) uk[i] = is * e[i + (int64_t)pj * m];
            for (int j = threadIdx.x; j < n; j += kXSel) {
                const T2 v = cmul(e[pi + (int64_t)j * m], f);
                vk[j] = mk(v.x, -v.y);
            }
        }
        __syncthreads();
    }
}

}  // namespace

template <class T2>
CrossStats cross_full_batch(T2* E, int nb, int m, int n, const double* d_anorm2, double tol, int rcap, int rfull,
                            T2* U, int64_t us, T2* VH, int64_t vs, std::vector<int>& rank, int n_sm,
                            cudaStream_t s) {
    using R = decltype(T2().x);
    CrossStats st;
    rank.assign(nb, 0);
    if (nb <= 0) return st;
    const int64_t es = (int64_t)m * n;
    const int tiles_m = (m + kXRows - 1) / kXRows;
    const int64_t ntile64 = (int64_t)tiles_m * ((n + kXCols - 1) / kXCols);
    if (ntile64 > INT_MAX / 2 || rcap > std::min(m, n)) fail(VIE_ERR_INVALID_ARG, "cross approximation: block too large");
    const int ntile = (int)ntile64;
    DevBuf d_rank(nb * sizeof(int)), d_piv(nb * sizeof(int2)), d_list(2 * (size_t)nb * sizeof(int)),
        d_cnt(4 * sizeof(int)), d_passes(sizeof(unsigned long long)), d_resid(nb * sizeof(double)),
        d_part((size_t)nb * ntile * sizeof(XPart<R>));
    int* list[2] = {d_list.as<int>(), d_list.as<int>() + nb};
    int* cnt = d_cnt.as<int>();
    struct Events {  // destroyed on every exit, errors included
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    VIE_CUDA(cudaEventCreate(&ev.a));
    VIE_CUDA(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    VIE_CUDA(cudaEventRecord(e0, s));
    k_cross_init<<<(nb + 255) / 256, 256, 0, s>>>(nb, d_rank.as<int>(), list[0], cnt,
                                                   d_passes.as<unsigned long long>());
    VIE_CHECK_LAUNCH();
    const int grid_u = std::max(1, n_sm) * 8;
    const int grid_s = std::min(nb, std::max(1, n_sm) * 2);
    const double tol2 = tol * tol;
    auto step = [&](int t) {
        const int a = t & 1;
        k_cross_update<T2, R><<<grid_u, kXRows, 0, s>>>(E, m, n, es, U, us, VH, vs, d_rank.as<int>(),
                                                        d_piv.as<int2>(), list[a], cnt + a, cnt + (a ^ 1), tiles_m,
                                                        ntile, d_part.as<XPart<R>>(), t > 0 ? 1 : 0);
        VIE_CHECK_LAUNCH();
        k_cross_select<T2, R><<<grid_s, kXSel, 0, s>>>(E, m, n, es, U, us, VH, vs, d_rank.as<int>(),
                                                       d_piv.as<int2>(), d_anorm2, tol2, rcap, rfull, list[a],
                                                       cnt + a, list[a ^ 1], cnt + (a ^ 1), cnt + 2,
                                                       d_passes.as<unsigned long long>(), ntile,
                                                       d_part.as<XPart<R>>(), t > 0 ? 1 : 0, d_resid.as<double>());
        VIE_CHECK_LAUNCH();
    };
    // every active block gains one cross per step and leaves at rank rcap, so
    // the loop ends by step rcap; the host reads the active count every 16 steps
    int h_cnt = nb;
    for (int t = 0; t <= rcap + 1; ++t) {
        step(t);
        if (t % 16 == 15 || t >= rcap) {
            VIE_CUDA(cudaMemcpyAsync(&h_cnt, cnt + ((t & 1) ^ 1), sizeof(int), cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            if (h_cnt == 0) break;
        }
    }
    VIE_CUDA(cudaEventRecord(e1, s));
    int h_flags = 0;
    unsigned long long h_passes = 0;
    VIE_CUDA(cudaMemcpyAsync(&h_flags, cnt + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(&h_passes, d_passes.p, sizeof(h_passes), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(rank.data(), d_rank.p, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
    st.resid2.resize(nb);
    VIE_CUDA(cudaMemcpyAsync(st.resid2.data(), d_resid.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    VIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (h_cnt != 0) fail(VIE_ERR_BREAKDOWN, "cross approximation did not end within its rank room");
    st.flags = h_flags;
    st.seconds = ms * 1e-3;
    // the scan reads every block once; each cross pass reads and writes one block
    st.bytes = (double)sizeof(T2) * (double)es * ((double)nb + 2.0 * (double)h_passes);
    st.passes = (int64_t)h_passes;
    return st;
}

template CrossStats cross_full_batch<float2>(float2*, int, int, int, const double*, double, int, int, float2*, int64_t,
                                             float2*, int64_t, std::vector<int>&, int, cudaStream_t);
template CrossStats cross_full_batch<double2>(double2*, int, int, int, const double*, double, int, int, double2*,
                                              int64_t, double2*, int64_t, std::vector<int>&, int, cudaStream_t);

}  // namespace vie
