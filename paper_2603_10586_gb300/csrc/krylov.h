// Float64 Krylov vector kernels (see krylov.cu).
#pragma once
#include "common.h"

namespace vie {

struct KrylovScratch {
    DevBuf part, part2, scalar;
    void init();
};

double knorm2(const double2* x, int64_t n, KrylovScratch& ks, cudaStream_t s);  // sum |x|^2 (synchronises)
void kmdot(const double2* V, int64_t ldv, int ncols, const double2* w, int64_t n, double2* d_h, KrylovScratch& ks,
           cudaStream_t s);
void kmaxpy(const double2* V, int64_t ldv, int ncols, const double2* d_h, double sign, double2* w, int64_t n,
            cudaStream_t s);
void kscale(const double2* x, double a, double2* y, int64_t n, cudaStream_t s);
void ksub(const double2* a, const double2* b, double2* y, int64_t n, cudaStream_t s);

// operator applications used by the solver (solve.cpp / api.cpp)
// y = P^-1 Zs x in complex float32 (fused preconditioner), x, y: n x nrhs, ld = n
void op_apply_fused32(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s);
// y = P^-1 Zs x with the far part on the tensor cores (BF16x3), float32 vectors
void op_apply_fused_bf16x3(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s);
// y = Zs x with float64 vectors; factors in their stored precision (float64 accumulation)
void op_apply64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);
// y = P^-1 Zs x in float64 (needs C128 factors for an all-float64 solve)
void op_apply_fused64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);
// y = Z_D^-1 x in float64
void op_precond64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);

}  // namespace vie
