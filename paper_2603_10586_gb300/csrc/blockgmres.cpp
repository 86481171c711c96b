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
    int sb = 0;  // width of the current cycle's block (the unconverged columns)
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

    double2* Vj(int j) { return V.as<double2>() + (size_t)j * n * sb; }

    void zgemm(cublasOperation_t ta, int mm, int nn, int kk, cplx alpha, const double2* A, int lda, const double2* B,
               int ldb, cplx beta, double2* Cm, int ldc) {
        VIE_BLAS(cublasZgemm(h, ta, CUBLAS_OP_N, mm, nn, kk, reinterpret_cast<const cuDoubleComplex*>(&alpha),
                             reinterpret_cast<const cuDoubleComplex*>(A), lda,
                             reinterpret_cast<const cuDoubleComplex*>(B), ldb,
                             reinterpret_cast<const cuDoubleComplex*>(&beta), reinterpret_cast<cuDoubleComplex*>(Cm),
                             ldc));
    }

    // Y = P^-1 Zs X for one n x sb block (inner precision)
    void apply(const double2* X, double2* Y) {
        if (c64) {
            convert_c128_to_c64(X, X32.p, n * sb, st);
            if (o.precision == VIE_BF16X3) op_apply_fused_bf16x3(op, X32.as<float2>(), Y32.as<float2>(), sb, st);
            else op_apply_fused32(op, X32.as<float2>(), Y32.as<float2>(), sb, st);
            convert_c64_to_c128(Y32.p, Y, n * sb, st);
        } else if (o.precond) {
            op_apply_fused64(op, X, Y, sb, st);
        } else {
            op_apply64(op, X, Y, sb, st);
        }
    }

    // A (n x sb) = Q Rq with orthonormal Q (in place) and upper Rq (host, s x s),
    // by Cholesky QR twice; false on a rank-deficient block
    bool cholqr2(double2* A, std::vector<cplx>& Rq) {
        std::vector<cplx> Rtot(sb * (size_t)sb, 0.0);
        for (int i = 0; i < sb; ++i) Rtot[i + (size_t)i * sb] = 1.0;
        for (int pass = 0; pass < 2; ++pass) {
            zgemm(CUBLAS_OP_C, sb, sb, (int)n, 1.0, A, (int)n, A, (int)n, 0.0, G.as<double2>(), sb);
            std::vector<cplx> Gh(sb * (size_t)sb);
            VIE_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaStreamSynchronize(st));
            if (!cholesky(Gh, sb)) return false;
            // U = L^H (upper); A := A U^-1
            std::vector<cplx> U(sb * (size_t)sb, 0.0);
            for (int i = 0; i < sb; ++i)
                for (int j = i; j < sb; ++j) U[i + (size_t)j * sb] = std::conj(Gh[j + (size_t)i * sb]);
            VIE_CUDA(cudaMemcpyAsync(S.p, U.data(), U.size() * sizeof(cplx), cudaMemcpyHostToDevice, st));
            const cplx one = 1.0;
            VIE_BLAS(cublasZtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT,
                                 (int)n, sb, reinterpret_cast<const cuDoubleComplex*>(&one),
                                 reinterpret_cast<const cuDoubleComplex*>(S.p), sb,
                                 reinterpret_cast<cuDoubleComplex*>(A), (int)n));
            // Rtot := U Rtot
            std::vector<cplx> Rn(sb * (size_t)sb, 0.0);
            for (int i = 0; i < sb; ++i)
                for (int j = 0; j < sb; ++j) {
                    cplx v = 0.0;
                    for (int k = i; k <= j; ++k) v += U[i + (size_t)k * sb] * Rtot[k + (size_t)j * sb];
                    Rn[i + (size_t)j * sb] = v;
                }
            Rtot.swap(Rn);
        }
        Rq.swap(Rtot);
        return true;
    }

    // rows of the full system: (m+1) sb; column c of Hb at Hb[c * ldh]
    int ldh() const { return (m + 1) * sb; }

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

    // column norms of an n x w block (device), from the diagonal of A^H A
    std::vector<double> colnorms(const double2* A, int w) {
        zgemm(CUBLAS_OP_C, w, w, (int)n, 1.0, A, (int)n, A, (int)n, 0.0, G.as<double2>(), w);
        std::vector<cplx> Gh(w * (size_t)w);
        VIE_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
        VIE_CUDA(cudaStreamSynchronize(st));
        std::vector<double> nrm(w);
        for (int c = 0; c < w; ++c) nrm[c] = std::sqrt(std::max(0.0, Gh[c + (size_t)c * w].real()));
        return nrm;
    }

    GmresOutcome run(const double2* B, double2* X) {
        GmresOutcome out;
        const double tol = o.tol > 0 ? o.tol : 1e-6;
        const int maxit = o.max_iters > 0 ? o.max_iters : 2000;
        const size_t col = (size_t)n * sizeof(double2);
        VIE_CUDA(cudaMemsetAsync(X, 0, (size_t)n * s * sizeof(double2), st));
        const std::vector<double> bnorm = colnorms(B, s);
        // R = P^-1 B (x = 0)
        if (o.precond) op_precond64(op, B, R.as<double2>(), s, st);
        else VIE_CUDA(cudaMemcpyAsync(R.p, B, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        const std::vector<double> beta0 = colnorms(R.as<double2>(), s);
        std::vector<double> res(s), rn = bnorm;
        std::vector<int> iters(s, 0);
        for (int c = 0; c < s; ++c) res[c] = beta0[c] > 0 ? 1.0 : 0.0;
        int it = 0, applies = 0, refinements = 0;
        while (it < maxit) {
            // the cycle's right-hand sides: the columns still above the tolerance
            std::vector<int> act;
            for (int c = 0; c < s; ++c)
                if (res[c] > tol) act.push_back(c);
            if (act.empty()) break;
            const int na = (int)act.size();
            // their residuals, each scaled to unit norm, into W
            std::vector<double> sc(na);
            for (int i = 0; i < na; ++i) {
                double2* w = W.as<double2>() + (size_t)i * n;
                VIE_CUDA(cudaMemcpyAsync(w, R.as<double2>() + (size_t)act[i] * n, col, cudaMemcpyDeviceToDevice, st));
                sc[i] = res[act[i]] * beta0[act[i]];
                const double inv = sc[i] > 0 ? 1.0 / sc[i] : 1.0;
                VIE_BLAS(cublasZdscal(h, (int)n, &inv, reinterpret_cast<cuDoubleComplex*>(w), 1));
            }
            // a basis of their span: pivoted Cholesky of the Gram picks independent
            // columns (dependent right-hand sides, e.g. the same wave twice, are
            // carried by the coefficients S0 instead of widening the block)
            std::vector<int> pick;
            {
                zgemm(CUBLAS_OP_C, na, na, (int)n, 1.0, W.as<double2>(), (int)n, W.as<double2>(), (int)n, 0.0,
                      G.as<double2>(), na);
                std::vector<cplx> Gh(na * (size_t)na);
                VIE_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
                VIE_CUDA(cudaStreamSynchronize(st));
                std::vector<double> d(na);
                std::vector<cplx> Lf(na * (size_t)na, 0.0);  // rows of the partial factor, per picked column
                for (int i = 0; i < na; ++i) d[i] = Gh[i + (size_t)i * na].real();
                std::vector<char> used(na, 0);
                for (int r = 0; r < na; ++r) {
                    int bi = -1;
                    double bv = 0.0;
                    for (int i = 0; i < na; ++i)
                        if (!used[i] && d[i] > bv) { bv = d[i]; bi = i; }
                    // the rest lies in the span to 1e-6 of its norm: below that the
                    // float64 Gram's rounding (~1e-16 sqrt n) would decide the pick,
                    // and what is left out returns in the next cycle's residual
                    if (bi < 0 || bv <= 1e-12) break;
                    used[bi] = 1;
                    pick.push_back(bi);
                    const double l = std::sqrt(bv);
                    // row r of L: L[r][i] = (G[bi][i] - sum_k L[k][bi]^* L[k][i]) / l
                    for (int i = 0; i < na; ++i) {
                        cplx v = Gh[bi + (size_t)i * na];
                        for (int k = 0; k < r; ++k) v -= std::conj(Lf[k + (size_t)bi * na]) * Lf[k + (size_t)i * na];
                        Lf[r + (size_t)i * na] = v / l;
                    }
                    for (int i = 0; i < na; ++i)
                        if (!used[i]) d[i] -= std::norm(Lf[r + (size_t)i * na]);
                }
            }
            if (pick.empty()) break;
            sb = (int)pick.size();
            const int L = ldh();
            for (int i = 0; i < sb; ++i)
                VIE_CUDA(cudaMemcpyAsync(Vj(0) + (size_t)i * n, W.as<double2>() + (size_t)pick[i] * n, col,
                                         cudaMemcpyDeviceToDevice, st));
            std::vector<cplx> Sdummy;
            if (!cholqr2(Vj(0), Sdummy)) fail(VIE_ERR_BREAKDOWN, "block GMRES: the residual block is rank deficient");
            // S0 = V0^H R (sb x na, in the unscaled residuals)
            zgemm(CUBLAS_OP_C, sb, na, (int)n, 1.0, Vj(0), (int)n, W.as<double2>(), (int)n, 0.0, C.as<double2>(), sb);
            std::vector<cplx> S0((size_t)sb * na);
            VIE_CUDA(cudaMemcpyAsync(S0.data(), C.p, S0.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
            VIE_CUDA(cudaStreamSynchronize(st));
            for (int j = 0; j < na; ++j)
                for (int i = 0; i < sb; ++i) S0[i + (size_t)j * sb] *= sc[j];
            Hb.assign((size_t)L * m * sb, 0.0);
            refl.assign((size_t)L * m * sb, 0.0);
            tau.assign((size_t)m * sb, 0.0);
            g.assign((size_t)L * na, 0.0);
            for (int c = 0; c < na; ++c)
                for (int i = 0; i < sb; ++i) g[i + (size_t)c * L] = S0[i + (size_t)c * sb];
            int jd = 0;
            for (int j = 0; j < m && it < maxit; ++j) {
                apply(Vj(j), W.as<double2>());
                ++applies;
                ++it;
                for (int c : act) ++iters[c];
                // block classical Gram-Schmidt against V_0 .. V_j, twice
                const int K = (j + 1) * sb;
                std::vector<cplx> Hc((size_t)K * sb, 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    zgemm(CUBLAS_OP_C, K, sb, (int)n, 1.0, Vj(0), (int)n, W.as<double2>(), (int)n, 0.0,
                          C.as<double2>(), K);
                    zgemm(CUBLAS_OP_N, (int)n, sb, K, -1.0, Vj(0), (int)n, C.as<double2>(), K, 1.0,
                          W.as<double2>(), (int)n);
                    std::vector<cplx> Ch((size_t)K * sb);
                    VIE_CUDA(cudaMemcpyAsync(Ch.data(), C.p, Ch.size() * sizeof(cplx), cudaMemcpyDeviceToHost, st));
                    VIE_CUDA(cudaStreamSynchronize(st));
                    for (size_t e = 0; e < Ch.size(); ++e) Hc[e] += Ch[e];
                }
                std::vector<cplx> Hn;
                const bool ok = cholqr2(W.as<double2>(), Hn);
                if (ok)
                    VIE_CUDA(cudaMemcpyAsync(Vj(j + 1), W.p, (size_t)n * sb * sizeof(double2),
                                             cudaMemcpyDeviceToDevice, st));
                // new block column of the Hessenberg: rows 0 .. (j+2) sb
                const int rows = (j + 2) * sb;
                for (int c = 0; c < sb; ++c) {
                    cplx* cl = &Hb[(size_t)(j * sb + c) * L];
                    for (int i = 0; i < K; ++i) cl[i] = Hc[i + (size_t)c * K];
                    for (int i = 0; i < sb; ++i) cl[K + i] = ok ? Hn[i + (size_t)c * sb] : 0.0;
                    for (int p = 0; p < j * sb; ++p) apply_reflect(p, rows, cl);
                }
                for (int c = 0; c < sb; ++c) {
                    const int colx = j * sb + c;
                    for (int p = j * sb; p < colx; ++p) apply_reflect(p, rows, &Hb[(size_t)colx * L]);
                    reflect(colx, rows);
                    for (int q = 0; q < na; ++q) apply_reflect(colx, rows, &g[(size_t)q * L]);
                }
                jd = j + 1;
                double worst = 0.0;
                for (int c = 0; c < na; ++c) {
                    double e = 0.0;
                    for (int i = jd * sb; i < rows; ++i) e += std::norm(g[i + (size_t)c * L]);
                    const double b0 = beta0[act[c]];
                    worst = std::max(worst, b0 > 0 ? std::sqrt(e) / b0 : 0.0);
                }
                if ((int)out.hist.size() < 512) out.hist.push_back(worst);
                if (worst <= tol || !ok) break;
            }
            // Y: upper-triangular solve with the rotated Hessenberg, X[:, act] += V Y
            const int K = jd * sb;
            std::vector<cplx> Y((size_t)K * na, 0.0);
            for (int c = 0; c < na; ++c)
                for (int i = K - 1; i >= 0; --i) {
                    cplx v = g[i + (size_t)c * L];
                    for (int l = i + 1; l < K; ++l) v -= Hb[i + (size_t)l * L] * Y[l + (size_t)c * K];
                    const cplx d = Hb[i + (size_t)i * L];
                    Y[i + (size_t)c * K] = std::abs(d) > 0 ? v / d : cplx(0.0);
                }
            VIE_CUDA(cudaMemcpyAsync(C.p, Y.data(), Y.size() * sizeof(cplx), cudaMemcpyHostToDevice, st));
            zgemm(CUBLAS_OP_N, (int)n, na, K, 1.0, Vj(0), (int)n, C.as<double2>(), K, 0.0, W.as<double2>(), (int)n);
            const cplx one = 1.0, mone = -1.0;
            for (int i = 0; i < na; ++i)
                VIE_BLAS(cublasZaxpy(h, (int)n, reinterpret_cast<const cuDoubleComplex*>(&one),
                                     reinterpret_cast<const cuDoubleComplex*>(W.as<double2>() + (size_t)i * n), 1,
                                     reinterpret_cast<cuDoubleComplex*>(X + (size_t)act[i] * n), 1));
            // refinement: R = P^-1 (B - Zs X), float64-accurate, all columns
            op_apply64(op, X, T.as<double2>(), s, st);
            VIE_CUDA(cudaMemcpyAsync(W.p, B, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            VIE_BLAS(cublasZaxpy(h, (int)(n * s), reinterpret_cast<const cuDoubleComplex*>(&mone),
                                 reinterpret_cast<const cuDoubleComplex*>(T.p), 1,
                                 reinterpret_cast<cuDoubleComplex*>(W.p), 1));
            rn = colnorms(W.as<double2>(), s);
            if (o.precond) op_precond64(op, W.as<double2>(), R.as<double2>(), s, st);
            else VIE_CUDA(cudaMemcpyAsync(R.p, W.p, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            const std::vector<double> wn = colnorms(R.as<double2>(), s);
            ++refinements;
            for (int c = 0; c < s; ++c) {
                res[c] = beta0[c] > 0 ? wn[c] / beta0[c] : 0.0;
                if (!std::isfinite(res[c])) fail(VIE_ERR_NAN, "non-finite residual in block GMRES");
            }
        }
        out.res = res;
        out.rnorm = rn;
        out.bnorm = bnorm;
        out.iters = iters;
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
