// Left-preconditioned restarted GMRES (paper Sec. 6: Saad-Schultz GMRES with
// the Arnoldi process; Sec. 4: block-diagonal preconditioner P = Z_D).
//
// Mixed precision: inside a restart cycle the operator P^-1 Zs is applied in
// complex float32 (stored c64 factors, float32 accumulation) while the Krylov
// basis, the two-pass classical Gram-Schmidt, the Hessenberg matrix and the
// Givens rotations are float64.  At the end of every cycle the residual
// P^-1 (b - Zs x) is recomputed in float64 (c64 factors read exactly, float64
// accumulation): this is the iterative refinement step, and the stopping test
// uses that true residual.  With VIE_C128 every apply is float64.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"
#include "krylov.h"

namespace vie {

namespace {

struct Gmres {
    Op& op;
    const vie_solve_opts& o;
    cudaStream_t s;
    int64_t n;
    int m;
    KrylovScratch ks;
    DevBuf V, w, x32, y32, h, tmp, r0;

    Gmres(Op& op_, const vie_solve_opts& o_) : op(op_), o(o_), s(op_.ctx->stream), n(op_.n()) {
        m = std::max(1, std::min(o.restart > 0 ? o.restart : 60, 63));
        ks.init();
        V.alloc((size_t)n * (m + 1) * sizeof(double2));
        w.alloc(n * sizeof(double2));
        tmp.alloc(n * sizeof(double2));
        r0.alloc(n * sizeof(double2));
        h.alloc(64 * sizeof(double2));
        if (o.precision != VIE_C128) {
            x32.alloc(n * sizeof(float2));
            y32.alloc(n * sizeof(float2));
        }
    }

    // w = M^-1 Zs v   (M = Z_D or identity)
    void apply_inner(const double2* v, double2* out) {
        if (o.precision == VIE_C128) {
            if (o.precond) op_apply_fused64(op, v, out, 1, s);
            else op_apply64(op, v, out, 1, s);
            return;
        }
        convert_c128_to_c64(v, x32.p, n, s);
        if (o.precond) {
            op_apply_fused32(op, x32.as<float2>(), y32.as<float2>(), 1, s);
            convert_c64_to_c128(y32.p, out, n, s);
        } else {
            op_apply64(op, v, out, 1, s);  // unpreconditioned runs use the float64 apply
        }
    }

    // out = M^-1 (b - Zs x) in float64
    void residual(const double2* b, const double2* x, double2* out) {
        op_apply64(op, x, tmp.as<double2>(), 1, s);
        ksub(b, tmp.as<double2>(), r0.as<double2>(), n, s);
        if (o.precond) op_precond64(op, r0.as<double2>(), out, 1, s);
        else VIE_CUDA(cudaMemcpyAsync(out, r0.p, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }

    // solve one right-hand side; x (device, c128) is overwritten
    int run(const double2* b, double2* x, vie_solve_stats* st, int& iters, int& applies, int& refin,
            double& res_out) {
        VIE_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        double2* V0 = V.as<double2>();
        // r = M^-1 b
        if (o.precond) op_precond64(op, b, w.as<double2>(), 1, s);
        else VIE_CUDA(cudaMemcpyAsync(w.p, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        const double beta0 = std::sqrt(knorm2(w.as<double2>(), n, ks, s));
        if (beta0 == 0.0) {
            res_out = 0.0;
            return VIE_OK;
        }
        const double tol = o.tol > 0 ? o.tol : 1e-6;
        const int maxit = o.max_iters > 0 ? o.max_iters : 2000;
        double beta = beta0;
        std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), hv(m + 1);
        double res = 1.0;
        while (true) {
            kscale(w.as<double2>(), 1.0 / beta, V0, n, s);
            std::fill(g.begin(), g.end(), cd(0));
            g[0] = beta;
            int jdone = 0;
            bool inner_conv = false;
            for (int j = 0; j < m && iters < maxit; ++j) {
                double2* vj = V0 + (size_t)j * n;
                double2* vj1 = V0 + (size_t)(j + 1) * n;
                apply_inner(vj, vj1);
                ++applies;
                // two-pass classical Gram-Schmidt in float64
                std::vector<cd> hsum(j + 1, cd(0));
                for (int pass = 0; pass < 2; ++pass) {
                    kmdot(V0, n, j + 1, vj1, n, h.as<double2>(), ks, s);
                    kmaxpy(V0, n, j + 1, h.as<double2>(), -1.0, vj1, n, s);
                    VIE_CUDA(cudaMemcpyAsync(hv.data(), h.p, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost, s));
                    VIE_CUDA(cudaStreamSynchronize(s));
                    for (int i = 0; i <= j; ++i) hsum[i] += hv[i];
                }
                double hn = std::sqrt(knorm2(vj1, n, ks, s));
                if (hn > 0) kscale(vj1, 1.0 / hn, vj1, n, s);
                for (int i = 0; i <= j; ++i) H[i + (size_t)j * (m + 1)] = hsum[i];
                H[j + 1 + (size_t)j * (m + 1)] = hn;
                // previous rotations, G = [[conj c, conj s], [-s, c]]
                for (int i = 0; i < j; ++i) {
                    cd a = H[i + (size_t)j * (m + 1)], c = H[i + 1 + (size_t)j * (m + 1)];
                    H[i + (size_t)j * (m + 1)] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
                    H[i + 1 + (size_t)j * (m + 1)] = -sn[i] * a + cs[i] * c;
                }
                cd a = H[j + (size_t)j * (m + 1)], c = H[j + 1 + (size_t)j * (m + 1)];
                double den = std::sqrt(std::norm(a) + std::norm(c));
                cs[j] = den > 0 ? a / den : cd(1);
                sn[j] = den > 0 ? c / den : cd(0);
                H[j + (size_t)j * (m + 1)] = den;
                H[j + 1 + (size_t)j * (m + 1)] = 0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = std::conj(cs[j]) * g[j];
                ++iters;
                jdone = j + 1;
                double est = std::abs(g[j + 1]) / beta0;
                if (st && st->n_history < 512) st->history[st->n_history++] = est;
                if (!std::isfinite(est)) fail(VIE_ERR_NAN, "non-finite residual in GMRES");
                if (est <= tol || hn == 0.0) {
                    inner_conv = true;
                    break;
                }
            }
            // y = H^-1 g (upper triangular), x += V y
            std::vector<cd> y(jdone);
            for (int i = jdone - 1; i >= 0; --i) {
                cd acc = g[i];
                for (int l = i + 1; l < jdone; ++l) acc -= H[i + (size_t)l * (m + 1)] * y[l];
                y[i] = acc / H[i + (size_t)i * (m + 1)];
            }
            VIE_CUDA(cudaMemcpyAsync(h.p, y.data(), jdone * sizeof(double2), cudaMemcpyHostToDevice, s));
            kmaxpy(V0, n, jdone, h.as<double2>(), 1.0, x, n, s);
            // float64 refinement residual
            residual(b, x, w.as<double2>());
            ++refin;
            beta = std::sqrt(knorm2(w.as<double2>(), n, ks, s));
            res = beta / beta0;
            (void)inner_conv;
            if (res <= tol) break;
            if (iters >= maxit) break;
            if (beta == 0.0) break;
        }
        res_out = res;
        return res <= tol ? VIE_OK : VIE_ERR_NOT_CONVERGED;
    }
};

}  // namespace

int solve(Op& op, const vie_incident* inc, int nrhs, const vie_solve_opts* o, void* I_out, vie_solve_stats* st) {
    if (op.fprec == 0) fail(VIE_ERR_STATE, "operator is not compressed");
    if (o->precision == VIE_C128 && op.fprec != VIE_C128)
        fail(VIE_ERR_INVALID_ARG, "an all-float64 solve needs VIE_C128 factors");
    cudaStream_t s = op.ctx->stream;
    const int64_t n = op.n();
    double t0 = now_s();
    DevBuf kh(3 * nrhs * sizeof(double)), pl(6 * nrhs * sizeof(double));
    VIE_CUDA(cudaMemcpyAsync(kh.p, inc->khat, 3 * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(pl.p, inc->pol, 6 * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    DevBuf b((size_t)n * nrhs * sizeof(double2));
    rhs_kernel_launch(op, kh.as<double>(), pl.as<double>(), nrhs, b.p, n, s);
    DevBuf xdev;
    double2* X;
    if (o->out_on_device) X = static_cast<double2*>(I_out);
    else {
        xdev.alloc((size_t)n * nrhs * sizeof(double2));
        X = xdev.as<double2>();
    }
    Gmres G(op, *o);
    int status = VIE_OK;
    int iters = 0, applies = 0, refin = 0;
    double worst = 0.0, worst_true = 0.0;
    if (st) st->n_history = 0;
    KrylovScratch ks;
    ks.init();
    DevBuf zx(n * sizeof(double2)), rr(n * sizeof(double2));
    for (int c = 0; c < nrhs; ++c) {
        const double2* bc = b.as<double2>() + (size_t)c * n;
        double2* xc = X + (size_t)c * n;
        double res = 0;
        int stc = G.run(bc, xc, st, iters, applies, refin, res);
        if (stc != VIE_OK) status = stc;
        worst = std::max(worst, res);
        // unpreconditioned relative residual with the compressed operator
        op_apply64(op, xc, zx.as<double2>(), 1, s);
        ksub(bc, zx.as<double2>(), rr.as<double2>(), n, s);
        double rn = std::sqrt(knorm2(rr.as<double2>(), n, ks, s));
        double bn = std::sqrt(knorm2(bc, n, ks, s));
        worst_true = std::max(worst_true, bn > 0 ? rn / bn : 0.0);
    }
    if (!o->out_on_device)
        VIE_CUDA(cudaMemcpyAsync(I_out, X, (size_t)n * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    if (st) {
        st->iterations = iters;
        st->applies = applies;
        st->refinements = refin;
        st->residual = worst;
        st->true_residual = worst_true;
        st->t_solve_s = now_s() - t0;
    }
    return status;
}

}  // namespace vie
