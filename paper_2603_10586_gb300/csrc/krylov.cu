// Float64 vector kernels of the Krylov solver (paper Sec. 6: GMRES with the
// Arnoldi process): norms, the multi-vector dot products and updates of
// classical Gram-Schmidt, scaling and residual formation.  Reductions are
// two-stage with a fixed chunking, so results are reproducible run to run.
#include "common.h"
#include "cplx.cuh"
#include "krylov.h"

namespace vie {

namespace {

constexpr int kRed = 256;   // CTAs in the first reduction stage
constexpr int kMaxCols = 64;

__global__ void k_norm2_partial(const double2* x, int64_t n, double* part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        acc += v.x * v.x + v.y * v.y;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_sum(const double* part, int n, double* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// h[j] = sum_i conj(V[i, j]) w[i], j < ncols; partial sums per CTA
__global__ void k_mdot_partial(const double2* V, int64_t ldv, int ncols, const double2* w, int64_t n,
                               double2* part) {
    double2 acc[kMaxCols];
    for (int j = 0; j < ncols; ++j) acc[j] = make_double2(0, 0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 wv = w[i];
        for (int j = 0; j < ncols; ++j) cfmac(acc[j], V[i + j * ldv], wv);
    }
    __shared__ double2 red[256];
    for (int j = 0; j < ncols; ++j) {
        red[threadIdx.x] = acc[j];
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = red[0];
        __syncthreads();
    }
}
__global__ void k_mdot_reduce(const double2* part, int nchunk, double2* h) {
    int j = blockIdx.x;
    __shared__ double2 red[256];
    double2 acc = make_double2(0, 0);
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x) acc += part[(size_t)j * nchunk + c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[j] = red[0];
}

// w += sign * V h
__global__ void k_maxpy(const double2* V, int64_t ldv, int ncols, const double2* h, double sign, double2* w,
                        int64_t n) {
    __shared__ double2 hs[kMaxCols];
    if ((int)threadIdx.x < ncols) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = w[i];
        for (int j = 0; j < ncols; ++j) {
            double2 p = cmul(V[i + j * ldv], hs[j]);
            acc.x += sign * p.x;
            acc.y += sign * p.y;
        }
        w[i] = acc;
    }
}

__global__ void k_scale(const double2* x, double a, double2* y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}
// y = a - b
__global__ void k_sub(const double2* a, const double2* b, double2* y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a[i] - b[i];
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(kRed * 4, (n + 255) / 256); }

}  // namespace

double knorm2(const double2* x, int64_t n, KrylovScratch& ks, cudaStream_t s) {
    k_norm2_partial<<<kRed, 256, 0, s>>>(x, n, ks.part.as<double>());
    k_sum<<<1, 256, 0, s>>>(ks.part.as<double>(), kRed, ks.scalar.as<double>());
    VIE_CHECK_LAUNCH();
    double v = 0;
    VIE_CUDA(cudaMemcpyAsync(&v, ks.scalar.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    return v;
}

void kmdot(const double2* V, int64_t ldv, int ncols, const double2* w, int64_t n, double2* d_h, KrylovScratch& ks,
           cudaStream_t s) {
    if (ncols > kMaxCols) fail(VIE_ERR_INVALID_ARG, "restart length above 63");
    k_mdot_partial<<<kRed, 256, 0, s>>>(V, ldv, ncols, w, n, ks.part2.as<double2>());
    k_mdot_reduce<<<ncols, 256, 0, s>>>(ks.part2.as<double2>(), kRed, d_h);
    VIE_CHECK_LAUNCH();
}

void kmaxpy(const double2* V, int64_t ldv, int ncols, const double2* d_h, double sign, double2* w, int64_t n,
            cudaStream_t s) {
    k_maxpy<<<grid_for(n), 256, 0, s>>>(V, ldv, ncols, d_h, sign, w, n);
    VIE_CHECK_LAUNCH();
}

void kscale(const double2* x, double a, double2* y, int64_t n, cudaStream_t s) {
    k_scale<<<grid_for(n), 256, 0, s>>>(x, a, y, n);
    VIE_CHECK_LAUNCH();
}

void ksub(const double2* a, const double2* b, double2* y, int64_t n, cudaStream_t s) {
    k_sub<<<grid_for(n), 256, 0, s>>>(a, b, y, n);
    VIE_CHECK_LAUNCH();
}

void KrylovScratch::init() {
    part.alloc(kRed * sizeof(double));
    part2.alloc((size_t)kRed * kMaxCols * sizeof(double2));
    scalar.alloc(sizeof(double));
}

}  // namespace vie
