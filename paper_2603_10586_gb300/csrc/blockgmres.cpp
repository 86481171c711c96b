// Block GMRES (one block Krylov space shared by all right-hand sides): the
// multi-RHS form of the GMRES of Sec. 6, left-preconditioned by the
// block diagonal of Sec. 4.  With s right-hand sides every step applies the
// operator to one n x s block and orthogonalises it against the whole block
// basis, so each right-hand side's residual is minimised over a space s times
// larger than its own Krylov space after the same number of applies.
//
//   R0 = P^-1 (B - Zs X) = V0 S0                (CholQR2)
//   step j:  W = P^-1 Zs Vj;  H_ij = Vi^H W, W -= Vi H_ij for i <= j (block
//            classical Gram-Schmidt, twice);  W = V_{j+1} H_{j+1,j} (CholQR2)
//   the block Hessenberg H ((j+2)s x (j+1)s) is reduced by Householder
//   reflections on the host as it grows; the rotated right-hand side gives
//   each column's residual estimate; at the end of a cycle Y solves the
//   triangular system and X += V Y.
// Precision: inner applies in complex float32 (or BF16x3), the basis and the
// block Gram-Schmidt in float64 (cuBLAS complex GEMMs), the residual that
// starts each cycle float64-accurate (refinement).  The Cholesky factors
// (s x s) and the reflections are computed on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.h"
#include "krylov.h"

namespace vie {

namespace {

using cplx = std::complex<double>;

// lower Cholesky factor of the Hermitian positive definite s x s matrix G
// (column-major); returns false if a pivot is not positive
bool cholesky(std::vector<cplx>& G, int s) {
    for (int j = 0; j < s; ++j) {
        double d = G[j + (size_t)j * s].real();
        for (int k = 0; k < j; ++k) d -= std::norm(G[j + (size_t)k * s]);
        if (!(d > 0.0)) return false;
        const double l = std::sqrt(d);
        G[j + (size_t)j * s] = l;
        for (int i = j + 1; i < s; ++i) {
            cplx v = G[i + (size_t)j * s];
            for (int k = 0; k < j; ++k) v -= G[i + (size_t)k * s] * std::conj(G[j + (size_t)k * s]);
            G[i + (size_t)j * s] = v / l;
        }
        for (int i = 0; i < j; ++i) G[i + (size_t)j * s] = 0.0;
    }
    return true;
}

struct Runner {
    Op& op;
    const vie_solve_opts& o;
    cudaStream_t st;
    cublasHandle_t h;
    int64_t n;
    int s, m;
    bool c64;
    DevBuf V, W, X32, Y32, R, T, C, G, S;
    // host: rotated block Hessenberg, its reflectors, the rotated right-hand side
    std::vector<cplx> Hb, refl, g;
    std::vector<double> tau;

    Runner(Op& op_, const vie_solve_opts& o_, int nrhs)
        : op(op_), o(o_), st(op_.ctx->stream), h(op_.ctx->blas), n(op_.n()), s(nrhs) {
        // block steps per cycle: the block basis holds (m+1) s vectors and the
        // host-side reduction of the block Hessenberg costs O((m s)^2 s) per
        // cycle, so m is kept to (m+1) s <= 512
        m = std::max(1, std::min(o.restart > 0 ? o.restart : 60, 512 / std::max(1, s) - 1));
        c64 = o.precision != VIE_C128 && o.precond;
        const size_t blk = (size_t)n * s * sizeof(double2);
        V.alloc(blk * (m + 1));
        W.alloc(blk);
        R.alloc(blk);
        T.alloc(blk);
        if (c64) {
            X32.alloc((size_t)n * s * sizeof(float2));
            Y32.alloc((size_t)n * s * sizeof(float2));
        }
        C.alloc((size_t)(m + 1) * s * s * sizeof(double2));
        G.alloc((size_t)s * s * sizeof(double2));
        S.alloc((size_t)s * s * sizeof(double2));
        op_reserve(op, s, o.precision, st);
        VIE_BLAS(cublasSetStream(h, st));
    }

    double2* Vj(int j) { return V.as<double2>() + (size_t)j * n * s; }

    void zgemm(cublasOperation_t ta, int mm, int nn, int kk, cplx alpha, const double2* A, int lda, const double2* B,
               int ldb, cplx beta, double2* Cm, int ldc) {
        VIE_BLAS(cublasZgemm(h, ta, CUBLAS_OP_N, mm, nn, kk, reinterpret_cast<const cuDoubleComplex*>(&alpha),
                             reinterpret_cast<const cuDoubleComplex*>(A), lda,
                             reinterpret_cast<const cuDoubleComplex*>(B), ldb,
                             reinterpret_cast<const cuDoubleComplex*>(&beta), reinterpret_cast<cuDoubleComplex*>(Cm),
                             ldc));
    }

    // Y = P^-1 Zs X for one n x s block (inner precision)
    void apply(const double2* X, double2* Y) {
        if (c64) {
            convert_c128_to_c64(X, X32.p, n * s, st);
            if (o.precision == VIE_BF16X3) op_apply_fused_bf16x3(op, X32.as<float2>(), Y32.as<float2>(), s, st);
            else op_apply_fused32(op, X32.as<float2>(), Y32.as<float2>(), s, st);
            convert_c64_to_c128(Y32.p, Y, n * s, st);
        } else if (o.precond) {
            op_apply_fused64(op, X, Y, s, st);
        } else {
            op_apply64(op, X, Y, s, st);
        }
    }

    // A (n x s) = Q Rq with orthonormal Q (in place) and upper Rq (host, s x s),
    // by Cholesky QR twice; false on a rank-deficient block
    bool cholqr2(double2* A, std::vector<cplx>& Rq) {
        std::vector<cplx> Rtot(s * (size_t)s, 0.0);
        for (int i = 0; i < s; ++i) Rtot[i + (size_t)i * s] = 1.0;
        for (int pass = 0; pass < 2; ++pass) {
            zgemm(CUBLAS_OP_C, s, s, (int)n, 1.0, A, (int)n, A, (int)n, 0.0, G.as<double2>(), s);
            std::vector<cplx> Gh(s * (size_t)s);
            VIE_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaStreamSynchronize(st));
            if (!cholesky(Gh, s)) return false;
            // U = L^H (upper); A := A U^-1
            std::vector<cplx> U(s * (size_t)s, 0.0);
            for (int i = 0; i < s; ++i)
                for (int j = i; j < s; ++j) U[i + (size_t)j * s] = std::conj(Gh[j + (size_t)i * s]);
            VIE_CUDA(cudaMemcpyAsync(S.p, U.data(), U.size() * sizeof(cplx), cudaMemcpyHostToDevice, st));
            const cplx one = 1.0;
            VIE_BLAS(cublasZtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT,
                                 (int)n, s, reinterpret_cast<const cuDoubleComplex*>(&one),
                                 reinterpret_cast<const cuDoubleComplex*>(S.p), s,
                                 reinterpret_cast<cuDoubleComplex*>(A), (int)n));
            // Rtot := U Rtot
            std::vector<cplx> Rn(s * (size_t)s, 0.0);
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < s; ++j) {
                    cplx v = 0.0;
                    for (int k = i; k <= j; ++k) v += U[i + (size_t)k * s] * Rtot[k + (size_t)j * s];
                    Rn[i + (size_t)j * s] = v;
                }
            Rtot.swap(Rn);
        }
        Rq.swap(Rtot);
        return true;
    }

    // rows of the full system: (m+1) s; column c of Hb at Hb[c * ldh]
    int ldh() const { return (m + 1) * s; }

    // Householder reflection of column `col` over rows col .. rows-1 of the
    // rotated Hessenberg: stored in refl[col], tau[col]
    void reflect(int col, int rows) {
        const int L = ldh();
        cplx* a = &Hb[(size_t)col * L];
        double nx = 0.0;
        for (int r = col; r < rows; ++r) nx += std::norm(a[r]);
        nx = std::sqrt(nx);
        cplx* v = &refl[(size_t)col * L];
        std::fill(v, v + L, cplx(0.0));
        if (nx == 0.0) {
            tau[col] = 0.0;
            return;
        }
        const cplx a0 = a[col];
        const cplx ph = std::abs(a0) > 0 ? a0 / std::abs(a0) : cplx(1.0);
        const cplx alpha = -ph * nx;  // a -> alpha e_col
        v[col] = a0 - alpha;
        for (int r = col + 1; r < rows; ++r) v[r] = a[r];
        double vn = 0.0;
        for (int r = col; r < rows; ++r) vn += std::norm(v[r]);
        tau[col] = vn > 0 ? 2.0 / vn : 0.0;
        a[col] = alpha;
        for (int r = col + 1; r < rows; ++r) a[r] = 0.0;
    }
    // apply reflection `col` (I - tau v v^H) to the column x (rows col .. rows-1)
    void apply_reflect(int col, int rows, cplx* x) const {
        const cplx* v = &refl[(size_t)col * ldh()];
        cplx d = 0.0;
        for (int r = col; r < rows; ++r) d += std::conj(v[r]) * x[r];
        d *= tau[col];
        for (int r = col; r < rows; ++r) x[r] -= d * v[r];
    }

    GmresOutcome run(const double2* B, double2* X) {
        GmresOutcome out;
        const double tol = o.tol > 0 ? o.tol : 1e-6;
        const int maxit = o.max_iters > 0 ? o.max_iters : 2000;
        const int L = ldh();
        VIE_CUDA(cudaMemsetAsync(X, 0, (size_t)n * s * sizeof(double2), st));
        std::vector<double> beta0(s), bnorm(s), res(s, 1.0);
        auto colnorms = [&](const double2* A, std::vector<double>& nrm) {
            // diagonal of A^H A
            zgemm(CUBLAS_OP_C, s, s, (int)n, 1.0, A, (int)n, A, (int)n, 0.0, G.as<double2>(), s);
            std::vector<cplx> Gh(s * (size_t)s);
            VIE_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaStreamSynchronize(st));
            for (int c = 0; c < s; ++c) nrm[c] = std::sqrt(std::max(0.0, Gh[c + (size_t)c * s].real()));
        };
        colnorms(B, bnorm);
        // R = P^-1 B (x = 0)
        if (o.precond) op_precond64(op, B, R.as<double2>(), s, st);
        else VIE_CUDA(cudaMemcpyAsync(R.p, B, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        colnorms(R.as<double2>(), beta0);
        int it = 0, applies = 0, refinements = 0;
        std::vector<double> rn(s, 0.0);
        for (int c = 0; c < s; ++c) rn[c] = bnorm[c];
        while (true) {
            bool all = true;
            for (int c = 0; c < s; ++c) all &= !(res[c] > tol);
            if (all || it >= maxit) break;
            // V0 S0 = R
            VIE_CUDA(cudaMemcpyAsync(Vj(0), R.p, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            std::vector<cplx> S0;
            if (!cholqr2(Vj(0), S0)) fail(VIE_ERR_BREAKDOWN, "block GMRES: the residual block is rank deficient");
            Hb.assign((size_t)L * m * s, 0.0);
            refl.assign((size_t)L * m * s, 0.0);
            tau.assign((size_t)m * s, 0.0);
            g.assign((size_t)L * s, 0.0);
            for (int c = 0; c < s; ++c)
                for (int i = 0; i < s; ++i) g[i + (size_t)c * L] = S0[i + (size_t)c * s];
            int jd = 0;
            for (int j = 0; j < m && it < maxit; ++j) {
                apply(Vj(j), W.as<double2>());
                ++applies;
                ++it;
                // block classical Gram-Schmidt against V_0 .. V_j, twice
                std::vector<cplx> Hc((size_t)(j + 1) * s * s, 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    const int K = (j + 1) * s;
                    zgemm(CUBLAS_OP_C, K, s, (int)n, 1.0, Vj(0), (int)n, W.as<double2>(), (int)n, 0.0,
                          C.as<double2>(), K);
                    zgemm(CUBLAS_OP_N, (int)n, s, K, -1.0, Vj(0), (int)n, C.as<double2>(), K, 1.0,
                          W.as<double2>(), (int)n);
                    std::vector<cplx> Ch((size_t)K * s);
                    VIE_CUDA(cudaMemcpyAsync(Ch.data(), C.p, Ch.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
                    VIE_CUDA(cudaStreamSynchronize(st));
                    for (size_t e = 0; e < Ch.size(); ++e) Hc[e] += Ch[e];
                }
                std::vector<cplx> Hn;
                const bool ok = cholqr2(W.as<double2>(), Hn);
                if (ok)
                    VIE_CUDA(cudaMemcpyAsync(Vj(j + 1), W.p, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice,
                                             st));
                // new block column of the Hessenberg: rows 0 .. (j+2) s
                const int rows = (j + 2) * s;
                for (int c = 0; c < s; ++c) {
                    cplx* col = &Hb[(size_t)(j * s + c) * L];
                    for (int i = 0; i < (j + 1) * s; ++i) col[i] = Hc[i + (size_t)c * (j + 1) * s];
                    for (int i = 0; i < s; ++i) col[(j + 1) * s + i] = ok ? Hn[i + (size_t)c * s] : 0.0;
                    for (int p = 0; p < j * s; ++p) apply_reflect(p, rows, col);
                }
                for (int c = 0; c < s; ++c) {
                    const int colx = j * s + c;
                    // earlier reflections of this block, then this column's own
                    for (int p = j * s; p < colx; ++p) apply_reflect(p, rows, &Hb[(size_t)colx * L]);
                    reflect(colx, rows);
                    for (int q = 0; q < s; ++q) apply_reflect(colx, rows, &g[(size_t)q * L]);
                }
                jd = j + 1;
                double worst = 0.0;
                for (int c = 0; c < s; ++c) {
                    double e = 0.0;
                    for (int i = jd * s; i < rows; ++i) e += std::norm(g[i + (size_t)c * L]);
                    const double r = beta0[c] > 0 ? std::sqrt(e) / beta0[c] : 0.0;
                    worst = std::max(worst, r);
                }
                if ((int)out.hist.size() < 512) out.hist.push_back(worst);
                if (worst <= tol || !ok) break;
            }
            // Y: upper-triangular solve with the rotated Hessenberg, X += V Y
            const int K = jd * s;
            std::vector<cplx> Y((size_t)K * s, 0.0);
            for (int c = 0; c < s; ++c)
                for (int i = K - 1; i >= 0; --i) {
                    cplx v = g[i + (size_t)c * L];
                    for (int l = i + 1; l < K; ++l) v -= Hb[i + (size_t)l * L] * Y[l + (size_t)c * K];
                    const cplx d = Hb[i + (size_t)i * L];
                    Y[i + (size_t)c * K] = std::abs(d) > 0 ? v / d : cplx(0.0);
                }
            VIE_CUDA(cudaMemcpyAsync(C.p, Y.data(), Y.size() * sizeof(cplx), cudaMemcpyHostToDevice, st));
            zgemm(CUBLAS_OP_N, (int)n, s, K, 1.0, Vj(0), (int)n, C.as<double2>(), K, 1.0, X, (int)n);
            // refinement: R = P^-1 (B - Zs X), float64-accurate
            op_apply64(op, X, T.as<double2>(), s, st);
            const cplx mone = -1.0;
            VIE_CUDA(cudaMemcpyAsync(W.p, B, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            VIE_BLAS(cublasZaxpy(h, (int)(n * s), reinterpret_cast<const cuDoubleComplex*>(&mone),
                                 reinterpret_cast<const cuDoubleComplex*>(T.p), 1, reinterpret_cast<cuDoubleComplex*>(W.p),
                                 1));
            colnorms(W.as<double2>(), rn);
            if (o.precond) op_precond64(op, W.as<double2>(), R.as<double2>(), s, st);
            else VIE_CUDA(cudaMemcpyAsync(R.p, W.p, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            std::vector<double> wn(s);
            colnorms(R.as<double2>(), wn);
            ++refinements;
            for (int c = 0; c < s; ++c) {
                res[c] = beta0[c] > 0 ? wn[c] / beta0[c] : 0.0;
                if (!std::isfinite(res[c])) fail(VIE_ERR_NAN, "non-finite residual in block GMRES");
            }
        }
        out.res = res;
        out.rnorm = rn;
        out.bnorm = bnorm;
        out.iters.assign(s, it);
        out.applies = applies;
        out.refinements = refinements;
        return out;
    }
};

}  // namespace

GmresOutcome run_block_gmres(Op& op, const double2* b, double2* X, const vie_solve_opts& o, int nrhs) {
    Runner R(op, o, nrhs);
    return R.run(b, X);
}

}  // namespace vie
