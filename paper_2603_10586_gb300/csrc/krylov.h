// Device-resident lockstep GMRES state and kernels (see krylov.cu), and the
// operator applications the solver uses (api.cpp).
#pragma once
#include "common.h"

namespace vie {

// Longest restart cycle (basis vectors per right-hand side, minus one).
constexpr int kMaxRestart = 512;

// Counters kept on the device.
enum : int {
    KR_J = 0,        // Arnoldi step within the current restart cycle
    KR_IT = 1,       // lockstep iterations so far (all cycles)
    KR_APPLIES = 2,  // operator applications
    KR_REFIN = 3,    // float64 refinement residuals
    KR_NAN = 4,      // a non-finite residual was seen
    KR_CONT = 5,     // another Arnoldi step follows in this cycle
    KR_NCTR = 8
};

// Pointers into the solver's device state, passed by value to every kernel.
// Slot i (< k) of a restart cycle works on column cols[i] of the n x nrhs
// right-hand side, solution and residual arrays.  Column c only uses rows
// [col_lo[c], col_lo[c] + col_len[c]) of them (all n rows for one operator;
// its own problem's rows for a batched block-diagonal operator), and its
// Krylov basis is col_len[c] x (m+1) at V + col_voff[c].
struct KrylovArgs {
    int64_t n;
    const long long* col_lo;
    const long long* col_len;
    const long long* col_voff;
    int m;            // restart length (<= kMaxRestart)
    int hs;           // per-slot stride of h, y and the projection partials (>= m + 1)
    int df;           // 1: the basis is double-float (float4 per value), 0: float64
    int shift;        // 1: the step applies E = P^-1 Zs - I; the Hessenberg column adds the identity
    int nblk_max;     // row blocks the norm partials are laid out for
    double tol;
    int maxit;
    double eps_low;   // error bound of one inner-precision product (updated residuals)
    double* ubound;   // [nrhs] accumulated error bound of a column's updated residual (host-written)
    double* enorm;    // [nrhs] |P^-1 Zs d| of the cycle's correction (updated residuals)
    double2* V;       // per column: col_len x (m+1) basis (float64, or double-float in the same bytes)
    double2* H;       // [slot][m][m+1] Hessenberg columns (rotated in place)
    double2* g;       // [slot][m+1] rotated right-hand side of the least-squares problem
    double2* cs;      // [slot][m] Givens cosines
    double2* sn;      // [slot][m] Givens sines
    double2* h;       // [slot][hs] coefficients of the current Gram-Schmidt pass
    double2* y;       // [slot][hs] least-squares solution of the cycle
    double2* part;    // [slot][hs][nchunk] projection partial sums
    double* npart;    // [slot][nblk_max] squared-norm partial sums
    double* nsq;      // [slot] their total
    double* inv;      // [slot] scale the next gather applies to its basis column
    int* cycling;     // [slot] still iterating in this cycle
    int* reorth;      // [slot] double-float basis: the step needs Gram-Schmidt pass 2 (null: always)
    int* jdone;       // [slot] Arnoldi steps done in this cycle
    int* cols;        // [slot] right-hand-side column of the slot
    int* iters;       // [nrhs] Arnoldi steps per column (all cycles)
    int* done;        // [nrhs] converged or out of iterations
    double* beta0;    // [nrhs] ||M^-1 b||
    double* beta;     // [nrhs] norm of the latest refinement residual
    double* res;      // [nrhs] beta / beta0
    double* rnorm;    // [nrhs] ||b - Zs x|| at the latest refinement
    double* hist;     // [512] largest estimated residual per lockstep iteration
    int* ctr;         // [KR_NCTR]
    // batched operators only (null otherwise): problem of every column, the
    // cycle's slot range of every problem, and the table the apply kernels read,
    // in which a problem whose right-hand sides have all stopped iterating in
    // this cycle gets an empty range (its work items are skipped)
    const int* col_prob;
    const int2* colr_cycle;
    int2* colr;
};

// launch shapes: row blocks of the (rows, slot) kernels and row chunks of the
// projections, chosen so that one launch covers the GPU a few times over
int kr_nblk(int64_t n, int k, int n_sm);
int kr_nchunk(int64_t n, int k, int m, int n_sm);

void kr_cycle_start(const KrylovArgs& a, int k, cudaStream_t s);
// Xg[:, i] = basis column j of slot i, scaled to unit norm (column 0 comes from W)
void kr_gather(const KrylovArgs& a, const double2* W, void* Xg, bool c64, int k, int nblk, cudaStream_t s);
// classical Gram-Schmidt pass 1 (w from the operator output Y) or pass 2 (w = basis column j+1)
void kr_project(const KrylovArgs& a, const void* Y, bool c64, int pass, int k, int nchunk, int nblk, cudaStream_t s);
// Givens update of the Hessenberg column, residual estimate, end-of-step test;
// with use_handle the continue flag also drives the enclosing graph loop
void kr_givens(const KrylovArgs& a, int k, int nblk, cudaGraphConditionalHandle hnd, int use_handle, cudaStream_t s);
// X[:, cols[i]] += V_i y_i with y_i = H_i^-1 g_i; with D (double-float basis only)
// the correction V_i y_i is also written to D[:, i] in float32
void kr_update(const KrylovArgs& a, double2* X, int k, int nblk, cudaStream_t s, float2* D = nullptr);
// rnorm[cols[i]] = the square root of slot i's squared-norm partials
void kr_rnorm_from_partials(const KrylovArgs& a, int k, int nblk, cudaStream_t s);
// Wf[:, cols[i]] -= E[:, i] and its squared-norm partials
void kr_sub_scatter_norm(const KrylovArgs& a, const double2* E, double2* Wf, int k, int nblk, cudaStream_t s);
// dst[:, i] = src[:, cols[i]] (the rows of that column)
void kr_gather_cols(const KrylovArgs& a, const double2* src, double2* dst, int k, int nblk, cudaStream_t s);
// R[:, i] = b[:, cols[i]] - T[:, i]
void kr_sub_cols(const KrylovArgs& a, const double2* b, const double2* T, double2* R, int k, int nblk, cudaStream_t s);
// W[:, cols[i]] = Wl[:, i] (W may equal Wl with cols the identity) and its squared-norm partials
void kr_scatter_norm(const KrylovArgs& a, const double2* Wl, double2* W, int k, int nblk, cudaStream_t s);
// beta, res and done of the slots' columns from the norm partials; init = 1 also
// sets beta0; init = 2 marks a residual of the inner precision (it ends no
// solve); init = 3 an updated float64 residual (it ends a solve when it plus its
// error bound, ubound + eps_low enorm / beta0, is within the tolerance)
void kr_cycle_end(const KrylovArgs& a, int k, int nblk, int init, cudaStream_t s);
// norms of the k columns of A (n x k, column i holding the rows of column
// cols ? cols[i] : i) into d_out[cols ? cols[i] : i]; d_part holds k * nblk doubles
void kr_colnorms(const KrylovArgs& a, const double2* A, int k, int nblk, const int* cols, double* d_part,
                 double* d_out, cudaStream_t s);

// Rows of every right-hand-side column: all n rows for one operator, the
// column's own problem for a batched (block-diagonal) operator, whose
// columns are grouped by problem.
struct ColumnLayout {
    std::vector<long long> lo, len;
    std::vector<int> prob;  // problem of each column
    int nprob = 1;
    static ColumnLayout single(int64_t n, int nrhs) {
        ColumnLayout L;
        L.lo.assign(nrhs, 0);
        L.len.assign(nrhs, n);
        L.prob.assign(nrhs, 0);
        return L;
    }
};

// outcome of one lockstep solve, per right-hand-side column
struct GmresOutcome {
    std::vector<double> res, rnorm, bnorm, hist;
    std::vector<int> iters;
    int applies = 0, refinements = 0;
};
void check_solve_opts(const Op& op, const vie_solve_opts* o, int nrhs);
// restarted GMRES of every column of b (device, n x nrhs) into X
GmresOutcome run_gmres(Op& op, const ColumnLayout& lay, const double2* b, double2* X, const vie_solve_opts& o,
                       int nrhs);
// block GMRES over one Krylov space shared by the nrhs columns (blockgmres.cpp)
GmresOutcome run_block_gmres(Op& op, const double2* b, double2* X, const vie_solve_opts& o, int nrhs);
// left-preconditioned BiCGStab of every column of b (device, n x nrhs) into X (bicgstab.cu)
GmresOutcome run_bicgstab(Op& op, const double2* b, double2* X, const vie_solve_opts& o, int nrhs);
// stats of columns [c0, c1); returns VIE_OK or VIE_ERR_NOT_CONVERGED
int fill_stats(const GmresOutcome& r, int c0, int c1, double tol, double t0, vie_solve_stats* st);

// operator applications used by the solver (solve.cpp / api.cpp)
// y = Zs x in complex float32 or with the far part in BF16x3 (precision), x, y: n x nrhs, ld = n
void op_apply_plain32(Op& op, const float2* x, float2* y, int nrhs, int precision, cudaStream_t s);
// y = P^-1 Zs x in complex float32 (fused preconditioner), x, y: n x nrhs, ld = n
void op_apply_fused32(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s);
// y = P^-1 Zs x with the far part on the tensor cores (BF16x3), float32 vectors
void op_apply_fused_bf16x3(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s);
// P^-1 Zs x - x (= Z_D^-1 times the far part of Zs x) in the inner precision (VIE_C64 or VIE_BF16X3)
void op_apply_shift32(Op& op, const float2* x, float2* y, int nrhs, int precision, cudaStream_t s);
// y = Zs x with float64 vectors; factors in their stored precision (float64 accumulation)
void op_apply64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);
// y = P^-1 Zs x in float64 (needs C128 factors for an all-float64 solve)
void op_apply_fused64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);
// y = Z_D^-1 x in float64
void op_precond64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s);
// size the operator's apply workspaces for nrhs float64 columns (no allocation
// may happen while a CUDA graph is being captured)
void op_reserve(Op& op, int nrhs, int precision, cudaStream_t s);

}  // namespace vie
