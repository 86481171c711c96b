// Left-preconditioned restarted GMRES (paper Sec. 6: Saad-Schultz GMRES with
// the Arnoldi process; Sec. 4: block-diagonal preconditioner P = Z_D).
//
// Mixed precision: inside a restart cycle the operator P^-1 Zs is applied in
// complex float32 (stored c64 factors, float32 accumulation) while the Krylov
// basis, the two-pass classical Gram-Schmidt, the Hessenberg matrix and the
// Givens rotations are float64.  At the end of every cycle the residual
// P^-1 (b - Zs x) is recomputed in float64 (c64 factors read exactly, float64
// accumulation): this is the iterative refinement step, and the stopping test
// uses that true residual.  With VIE_C128 every apply is float64; with
// VIE_BF16X3 the far part of the inner applies runs on the tensor cores in
// split-precision bf16 (the refinement residual stays float64).
//
// Several right-hand sides advance in lockstep: each Arnoldi step gathers the
// current basis vector of every right-hand side still iterating into one
// n x s block and applies the operator once to all of them, so the factors
// are streamed once per step instead of once per right-hand side.  Each
// right-hand side keeps its own Krylov space, Hessenberg matrix and rotations
// and leaves the lockstep when it has converged.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"
#include "krylov.h"

namespace vie {

namespace {

struct Rhs {
    DevBuf V;                // n x (m+1) float64 complex basis
    std::vector<cd> H, g, cs, sn;
    double beta0 = 0, beta = 0, res = 1;
    bool done = false;       // converged (true residual) or out of iterations
    bool cycling = false;    // still iterating in the current restart cycle
    int jdone = 0, iters = 0;
};

struct Gmres {
    Op& op;
    const vie_solve_opts& o;
    cudaStream_t s;
    int64_t n;
    int m, nrhs;
    KrylovScratch ks;
    std::vector<Rhs> R;
    DevBuf X32, Y32, Xg, Yg, h, tmp, r0, W;

    Gmres(Op& op_, const vie_solve_opts& o_, int nrhs_)
        : op(op_), o(o_), s(op_.ctx->stream), n(op_.n()), nrhs(nrhs_) {
        m = std::max(1, std::min(o.restart > 0 ? o.restart : 60, 63));
        ks.init();
        R.resize(nrhs);
        for (auto& r : R) {
            r.V.alloc((size_t)n * (m + 1) * sizeof(double2));
            r.H.assign((size_t)(m + 1) * m, cd(0));
            r.g.assign(m + 1, cd(0));
            r.cs.assign(m, cd(0));
            r.sn.assign(m, cd(0));
        }
        h.alloc(64 * sizeof(double2));
        tmp.alloc((size_t)n * nrhs * sizeof(double2));
        r0.alloc((size_t)n * nrhs * sizeof(double2));
        W.alloc((size_t)n * nrhs * sizeof(double2));
        Xg.alloc((size_t)n * nrhs * sizeof(double2));
        Yg.alloc((size_t)n * nrhs * sizeof(double2));
        if (o.precision != VIE_C128) {
            X32.alloc((size_t)n * nrhs * sizeof(float2));
            Y32.alloc((size_t)n * nrhs * sizeof(float2));
        }
    }

    // out[:, i] = M^-1 Zs in[:, i] for the k gathered columns (M = Z_D or identity)
    void apply_inner(const double2* in, double2* out, int k) {
        if (o.precision == VIE_C128 || !o.precond) {
            if (o.precond) op_apply_fused64(op, in, out, k, s);
            else op_apply64(op, in, out, k, s);
            return;
        }
        convert_c128_to_c64(in, X32.p, n * k, s);
        if (o.precision == VIE_BF16X3) op_apply_fused_bf16x3(op, X32.as<float2>(), Y32.as<float2>(), k, s);
        else op_apply_fused32(op, X32.as<float2>(), Y32.as<float2>(), k, s);
        convert_c64_to_c128(Y32.p, out, n * k, s);
    }

    // out = M^-1 (b - Zs x) in float64 for all right-hand sides
    void residual(const double2* b, const double2* x, double2* out) {
        op_apply64(op, x, tmp.as<double2>(), nrhs, s);
        ksub(b, tmp.as<double2>(), r0.as<double2>(), n * nrhs, s);
        if (o.precond) op_precond64(op, r0.as<double2>(), out, nrhs, s);
        else VIE_CUDA(cudaMemcpyAsync(out, r0.p, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }

    int run(const double2* b, double2* X, vie_solve_stats* st, int& applies, int& refin) {
        const double tol = o.tol > 0 ? o.tol : 1e-6;
        const int maxit = o.max_iters > 0 ? o.max_iters : 2000;
        VIE_CUDA(cudaMemsetAsync(X, 0, (size_t)n * nrhs * sizeof(double2), s));
        // r = M^-1 b
        if (o.precond) op_precond64(op, b, W.as<double2>(), nrhs, s);
        else VIE_CUDA(cudaMemcpyAsync(W.p, b, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        for (int c = 0; c < nrhs; ++c) {
            Rhs& r = R[c];
            r.beta0 = r.beta = std::sqrt(knorm2(W.as<double2>() + (size_t)c * n, n, ks, s));
            r.done = r.beta0 == 0.0;
            r.res = r.done ? 0.0 : 1.0;
        }
        std::vector<cd> hv(m + 1);
        while (true) {
            std::vector<int> live;
            for (int c = 0; c < nrhs; ++c)
                if (!R[c].done) live.push_back(c);
            if (live.empty()) break;
            for (int c : live) {
                Rhs& r = R[c];
                kscale(W.as<double2>() + (size_t)c * n, 1.0 / r.beta, r.V.as<double2>(), n, s);
                std::fill(r.g.begin(), r.g.end(), cd(0));
                r.g[0] = r.beta;
                r.jdone = 0;
                r.cycling = true;
            }
            for (int j = 0; j < m; ++j) {
                std::vector<int> act;
                for (int c : live)
                    if (R[c].cycling && R[c].iters < maxit) act.push_back(c);
                if (act.empty()) break;
                const int k = (int)act.size();
                for (int i = 0; i < k; ++i)
                    VIE_CUDA(cudaMemcpyAsync(Xg.as<double2>() + (size_t)i * n, R[act[i]].V.as<double2>() + (size_t)j * n,
                                             n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
                apply_inner(Xg.as<double2>(), Yg.as<double2>(), k);
                ++applies;
                double est_max = 0.0;
                for (int i = 0; i < k; ++i) {
                    Rhs& r = R[act[i]];
                    double2* V0 = r.V.as<double2>();
                    double2* vj1 = V0 + (size_t)(j + 1) * n;
                    VIE_CUDA(cudaMemcpyAsync(vj1, Yg.as<double2>() + (size_t)i * n, n * sizeof(double2),
                                             cudaMemcpyDeviceToDevice, s));
                    // two-pass classical Gram-Schmidt in float64
                    std::vector<cd> hsum(j + 1, cd(0));
                    for (int pass = 0; pass < 2; ++pass) {
                        kmdot(V0, n, j + 1, vj1, n, h.as<double2>(), ks, s);
                        kmaxpy(V0, n, j + 1, h.as<double2>(), -1.0, vj1, n, s);
                        VIE_CUDA(cudaMemcpyAsync(hv.data(), h.p, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost, s));
                        VIE_CUDA(cudaStreamSynchronize(s));
                        for (int l = 0; l <= j; ++l) hsum[l] += hv[l];
                    }
                    double hn = std::sqrt(knorm2(vj1, n, ks, s));
                    if (hn > 0) kscale(vj1, 1.0 / hn, vj1, n, s);
                    auto H = [&](int row, int col) -> cd& { return r.H[row + (size_t)col * (m + 1)]; };
                    for (int l = 0; l <= j; ++l) H(l, j) = hsum[l];
                    H(j + 1, j) = hn;
                    // Givens rotations G = [[conj c, conj s], [-s, c]]
                    for (int l = 0; l < j; ++l) {
                        cd a = H(l, j), c2 = H(l + 1, j);
                        H(l, j) = std::conj(r.cs[l]) * a + std::conj(r.sn[l]) * c2;
                        H(l + 1, j) = -r.sn[l] * a + r.cs[l] * c2;
                    }
                    cd a = H(j, j), c2 = H(j + 1, j);
                    double den = std::sqrt(std::norm(a) + std::norm(c2));
                    r.cs[j] = den > 0 ? a / den : cd(1);
                    r.sn[j] = den > 0 ? c2 / den : cd(0);
                    H(j, j) = den;
                    H(j + 1, j) = 0;
                    r.g[j + 1] = -r.sn[j] * r.g[j];
                    r.g[j] = std::conj(r.cs[j]) * r.g[j];
                    ++r.iters;
                    r.jdone = j + 1;
                    double est = std::abs(r.g[j + 1]) / r.beta0;
                    if (!std::isfinite(est)) fail(VIE_ERR_NAN, "non-finite residual in GMRES");
                    est_max = std::max(est_max, est);
                    if (est <= tol || hn == 0.0) r.cycling = false;
                }
                if (st && st->n_history < 512) st->history[st->n_history++] = est_max;
            }
            // x += V y with y = H^-1 g (upper triangular), per right-hand side
            for (int c : live) {
                Rhs& r = R[c];
                if (r.jdone == 0) continue;
                std::vector<cd> y(r.jdone);
                for (int i = r.jdone - 1; i >= 0; --i) {
                    cd acc = r.g[i];
                    for (int l = i + 1; l < r.jdone; ++l) acc -= r.H[i + (size_t)l * (m + 1)] * y[l];
                    y[i] = acc / r.H[i + (size_t)i * (m + 1)];
                }
                VIE_CUDA(cudaMemcpyAsync(h.p, y.data(), r.jdone * sizeof(double2), cudaMemcpyHostToDevice, s));
                kmaxpy(r.V.as<double2>(), n, r.jdone, h.as<double2>(), 1.0, X + (size_t)c * n, n, s);
            }
            // float64 refinement residual for every right-hand side
            residual(b, X, W.as<double2>());
            ++refin;
            for (int c : live) {
                Rhs& r = R[c];
                r.beta = std::sqrt(knorm2(W.as<double2>() + (size_t)c * n, n, ks, s));
                r.res = r.beta / r.beta0;
                if (r.res <= tol || r.iters >= maxit || r.beta == 0.0) r.done = true;
            }
        }
        int status = VIE_OK;
        for (auto& r : R)
            if (r.res > tol) status = VIE_ERR_NOT_CONVERGED;
        return status;
    }
};

}  // namespace

int solve(Op& op, const vie_incident* inc, int nrhs, const vie_solve_opts* o, void* I_out, vie_solve_stats* st) {
    if (op.fprec == 0) fail(VIE_ERR_STATE, "operator is not compressed");
    if (o->precision == VIE_C128 && op.fprec != VIE_C128)
        fail(VIE_ERR_INVALID_ARG, "an all-float64 solve needs VIE_C128 factors");
    if (o->precision != VIE_C128 && o->precision != VIE_C64 && o->precision != VIE_BF16X3 && o->precision != 0)
        fail(VIE_ERR_INVALID_ARG, "solve precision must be VIE_C64, VIE_BF16X3 or VIE_C128");
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
    if (st) st->n_history = 0;
    int applies = 0, refin = 0;
    Gmres G(op, *o, nrhs);
    int status = G.run(b.as<double2>(), X, st, applies, refin);
    // unpreconditioned relative residual with the compressed operator
    KrylovScratch ks;
    ks.init();
    DevBuf zx((size_t)n * nrhs * sizeof(double2)), rr((size_t)n * nrhs * sizeof(double2));
    op_apply64(op, X, zx.as<double2>(), nrhs, s);
    ksub(b.as<double2>(), zx.as<double2>(), rr.as<double2>(), n * nrhs, s);
    double worst = 0.0, worst_true = 0.0;
    int iters = 0;
    for (int c = 0; c < nrhs; ++c) {
        double rn = std::sqrt(knorm2(rr.as<double2>() + (size_t)c * n, n, ks, s));
        double bn = std::sqrt(knorm2(b.as<double2>() + (size_t)c * n, n, ks, s));
        worst_true = std::max(worst_true, bn > 0 ? rn / bn : 0.0);
        worst = std::max(worst, G.R[c].res);
        iters = std::max(iters, G.R[c].iters);
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
