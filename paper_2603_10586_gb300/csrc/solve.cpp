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
// Several right-hand sides advance in lockstep: each Arnoldi step applies the
// operator once to the current basis vectors of all of them (one n x k
// block), so the factors are streamed once per step instead of once per
// right-hand side.  Each right-hand side keeps its own Krylov space,
// Hessenberg matrix and rotations and leaves the lockstep when it converges.
//
// The whole restart cycle runs on the device: the Arnoldi step, the
// orthogonalisation, the Givens updates and the end-of-step test are kernels
// (krylov.cu), and by default one cycle is one CUDA graph whose Arnoldi steps
// sit in a conditional while-node driven by the Givens kernel.  The host only
// reads the per-column convergence flags between cycles.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>

#include "common.h"
#include "krylov.h"

namespace vie {

namespace {

struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    long long pre = 0, body = 0, post = 0;  // kernels per launch of each part
};

struct Gmres {
    Op& op;
    const vie_solve_opts& o;
    const ColumnLayout& lay;
    cudaStream_t s, s_body = nullptr;
    int64_t n;
    int m, nrhs, n_sm;
    bool c64;  // inner applies on float32 vectors
    DevBuf V, H, g, cs, sn, h, y, part, npart, nsq, rpart, inv, cycling, reorth, jdone, cols, iters, done, beta0, beta, res,
        rnorm,
        bnorm, hist, ctr, col_lo, col_len, col_voff, colr, colr_cycle, col_prob;
    std::vector<int2> h_colr;
    DevBuf Xg, Yg, Xl, T, Rl, Wl, W, Rf, enorm, ubound;
    KrylovArgs a{};
    std::map<int, CycleGraph> graphs;
    int* h_pinned = nullptr;  // [KR_NCTR + nrhs] host-visible copy of counters and done flags
    std::vector<double> h_res; // latest residual per column (relative)
    std::vector<double> h_beta0, bound;  // ||P^-1 b|| and the error bound of the updated residual
    bool have_base = false;              // Rf and W hold float64-accurate residuals (possibly updated)
    double eps_low = 1e-4;

    Gmres(Op& op_, const vie_solve_opts& o_, int nrhs_, const ColumnLayout& lay_)
        : op(op_), o(o_), lay(lay_), s(op_.ctx->stream), n(op_.n()), nrhs(nrhs_), n_sm(op_.ctx->n_sm) {
        m = std::max(1, std::min(o.restart > 0 ? o.restart : 60, kMaxRestart));
        c64 = !(o.precision == VIE_C128 || !o.precond);
        const int S = nrhs;
        const int nblk_max = kr_nblk(n, 1, n_sm);
        const int nchunk_max = kr_nchunk(n, 1, m, n_sm);
        // the basis of column c: col_len[c] x (m+1) at col_voff[c]
        std::vector<long long> voff(nrhs);
        long long vtot = 0;
        for (int c = 0; c < nrhs; ++c) {
            voff[c] = vtot;
            vtot += (long long)(m + 1) * lay.len[c];
        }
        V.alloc((size_t)vtot * sizeof(double2));
        upload(col_lo, lay.lo);
        upload(col_len, lay.len);
        upload(col_voff, voff);
        if (lay.nprob > 1) {
            colr.alloc(lay.nprob * sizeof(int2));
            colr_cycle.alloc(lay.nprob * sizeof(int2));
            upload(col_prob, lay.prob);
            h_colr.assign(lay.nprob, make_int2(0, 0));
        }
        H.alloc((size_t)S * m * (m + 1) * sizeof(double2));
        g.alloc((size_t)S * (m + 1) * sizeof(double2));
        cs.alloc((size_t)S * m * sizeof(double2));
        sn.alloc((size_t)S * m * sizeof(double2));
        const int hstride = m + 1;
        h.alloc((size_t)S * hstride * sizeof(double2));
        y.alloc((size_t)S * hstride * sizeof(double2));
        part.alloc((size_t)S * hstride * nchunk_max * sizeof(double2));
        npart.alloc((size_t)S * nblk_max * sizeof(double));
        rpart.alloc((size_t)S * nblk_max * sizeof(double));
        nsq.alloc(S * sizeof(double));
        inv.alloc(S * sizeof(double));
        cycling.alloc(S * sizeof(int));
        reorth.alloc(S * sizeof(int));
        jdone.alloc(S * sizeof(int));
        cols.alloc(S * sizeof(int));
        iters.alloc(nrhs * sizeof(int));
        done.alloc(nrhs * sizeof(int));
        beta0.alloc(nrhs * sizeof(double));
        beta.alloc(nrhs * sizeof(double));
        res.alloc(nrhs * sizeof(double));
        rnorm.alloc(nrhs * sizeof(double));
        bnorm.alloc(nrhs * sizeof(double));
        hist.alloc(512 * sizeof(double));
        ctr.alloc(KR_NCTR * sizeof(int));
        const size_t vec = (size_t)n * nrhs * sizeof(double2);
        Xg.alloc(vec);
        Yg.alloc(vec);
        Xl.alloc(vec);
        T.alloc(vec);
        Rl.alloc(vec);
        Wl.alloc(vec);
        W.alloc(vec);
        if (c64) {
            Rf.alloc(vec);  // b - Zs x per column, the base of residual updates
            enorm.alloc(nrhs * sizeof(double));
            ubound.alloc(nrhs * sizeof(double));
        }
        op_reserve(op, nrhs, o.precision, s);
        VIE_CUDA(cudaMemsetAsync(ctr.p, 0, KR_NCTR * sizeof(int), s));
        VIE_CUDA(cudaMemsetAsync(hist.p, 0, 512 * sizeof(double), s));
        a.n = n;
        a.col_lo = col_lo.as<long long>();
        a.col_len = col_len.as<long long>();
        a.col_voff = col_voff.as<long long>();
        a.col_prob = lay.nprob > 1 ? col_prob.as<int>() : nullptr;
        a.colr_cycle = lay.nprob > 1 ? colr_cycle.as<int2>() : nullptr;
        a.colr = lay.nprob > 1 ? colr.as<int2>() : nullptr;
        a.m = m;
        a.hs = m + 1;
        // float32 inner applies: the Gram-Schmidt in double-float on the float32 pipes
        a.df = c64 ? 1 : 0;
        a.nblk_max = nblk_max;
        a.tol = o.tol > 0 ? o.tol : 1e-6;
        a.maxit = o.max_iters > 0 ? o.max_iters : 2000;
        // relative error of one inner-precision product, with margin (measured: BF16x3
        // <= 5e-5, float32 <= 1e-6): the weight of an updated residual's error bound
        a.eps_low = o.precision == VIE_BF16X3 ? 1e-4 : 1e-5;
        a.ubound = c64 ? ubound.as<double>() : nullptr;
        // mixed precision: the Arnoldi steps apply E = P^-1 Zs - I (the block-Jacobi
        // preconditioned operator is I plus the preconditioned far part), whose
        // Krylov space is the same; the new vector then carries no copy of the
        // previous one for Gram-Schmidt to cancel, the inner-precision error
        // scales with |E v| instead of |v|, and the Hessenberg of I + E is that
        // of E plus the identity
        a.shift = c64 ? 1 : 0;
        a.enorm = c64 ? enorm.as<double>() : nullptr;
        a.V = V.as<double2>();
        a.H = H.as<double2>();
        a.g = g.as<double2>();
        a.cs = cs.as<double2>();
        a.sn = sn.as<double2>();
        a.h = h.as<double2>();
        a.y = y.as<double2>();
        a.part = part.as<double2>();
        a.npart = npart.as<double>();
        a.nsq = nsq.as<double>();
        a.inv = inv.as<double>();
        a.cycling = cycling.as<int>();
        a.reorth = reorth.as<int>();
        a.jdone = jdone.as<int>();
        a.cols = cols.as<int>();
        a.iters = iters.as<int>();
        a.done = done.as<int>();
        a.beta0 = beta0.as<double>();
        a.beta = beta.as<double>();
        a.res = res.as<double>();
        a.rnorm = rnorm.as<double>();
        a.hist = hist.as<double>();
        a.ctr = ctr.as<int>();
        VIE_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h_pinned), (KR_NCTR + nrhs) * sizeof(int)));
    }

    ~Gmres() {
        for (auto& kv : graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (s_body) cudaStreamDestroy(s_body);
        if (h_pinned) cudaFreeHost(h_pinned);
    }

    // Yg = M^-1 Zs Xg for k columns (M = Z_D or the identity)
    void apply_inner(int k, cudaStream_t st) {
        if (!c64) {
            if (o.precond) op_apply_fused64(op, Xg.as<double2>(), Yg.as<double2>(), k, st);
            else op_apply64(op, Xg.as<double2>(), Yg.as<double2>(), k, st);
        } else {
            // E = P^-1 Zs - I; the Hessenberg adds the identity back (a.shift)
            op_apply_shift32(op, Xg.as<float2>(), Yg.as<float2>(), k,
                             o.precision == VIE_BF16X3 ? VIE_BF16X3 : VIE_C64, st);
        }
    }

    // the apply kernels' column table starts every cycle, and its refinement, complete
    void restore_colr(cudaStream_t st) {
        if (lay.nprob > 1)
            VIE_CUDA(cudaMemcpyAsync(colr.p, colr_cycle.p, lay.nprob * sizeof(int2), cudaMemcpyDeviceToDevice, st));
    }

    void launch_pre(int k, cudaStream_t st) {
        restore_colr(st);
        kr_cycle_start(a, k, st);
    }

    void launch_body(int k, cudaStream_t st, cudaGraphConditionalHandle hnd, int use_handle) {
        const int nblk = kr_nblk(n, k, n_sm), nchunk = kr_nchunk(n, k, m, n_sm);
        kr_gather(a, W.as<double2>(), Xg.p, c64, k, nblk, st);
        apply_inner(k, st);
        kr_project(a, Yg.p, c64, 1, k, nchunk, nblk, st);
        kr_project(a, nullptr, c64, 2, k, nchunk, nblk, st);
        kr_givens(a, k, nblk, hnd, use_handle, st);
    }

    // x += V y, then the residual W = M^-1 (b - Zs x) of the slots' columns that
    // starts the next cycle: float64-accurate (the refinement step), or, while
    // the residual is still far above the tolerance (cheap), with the inner
    // apply's precision, which is accurate enough to restart from and never
    // ends a solve
    // post modes: the residual that ends a cycle
    enum { kPostAccurate = 0, kPostCheap = 1, kPostUpdate = 2 };
    void launch_post(int k, const double2* b, double2* X, cudaStream_t st, int mode) {
        const int nblk = kr_nblk(n, k, n_sm);
        restore_colr(st);
        if (mode != kPostUpdate) {
            kr_update(a, X, k, nblk, st);
            launch_residual(k, b, X, st, mode == kPostCheap);
            return;
        }
        // W -= P^-1 Zs d and R -= Zs d for the cycle's correction d = V y,
        // both products in the inner precision: the error they add is below
        // ~1e-4 of |P^-1 Zs d|, which the host accumulates and bounds
        float2* d32 = reinterpret_cast<float2*>(Xg.p);
        float2* e32 = reinterpret_cast<float2*>(Yg.p);
        float2* t32 = reinterpret_cast<float2*>(Xl.p);
        kr_update(a, X, k, nblk, st, d32);
        const int prec = o.precision == VIE_BF16X3 ? VIE_BF16X3 : VIE_C64;
        if (prec == VIE_BF16X3) op_apply_fused_bf16x3(op, d32, e32, k, st);
        else op_apply_fused32(op, d32, e32, k, st);
        op_apply_plain32(op, d32, t32, k, prec, st);
        convert_c64_to_c128(e32, Wl.p, n * k, st);
        convert_c64_to_c128(t32, T.p, n * k, st);
        kr_colnorms(a, Wl.as<double2>(), k, nblk, a.cols, rpart.as<double>(), enorm.as<double>(), st);
        kr_sub_scatter_norm(a, T.as<double2>(), Rf.as<double2>(), k, nblk, st);
        kr_rnorm_from_partials(a, k, nblk, st);
        kr_sub_scatter_norm(a, Wl.as<double2>(), W.as<double2>(), k, nblk, st);
        kr_cycle_end(a, k, nblk, 3, st);
    }

    void launch_residual(int k, const double2* b, const double2* X, cudaStream_t st, bool cheap) {
        const int nblk = kr_nblk(n, k, n_sm);
        kr_gather_cols(a, X, Xl.as<double2>(), k, nblk, st);
        if (cheap) {
            float2* x32 = reinterpret_cast<float2*>(Xg.p);
            float2* y32 = reinterpret_cast<float2*>(Yg.p);
            convert_c128_to_c64(Xl.p, x32, n * k, st);
            op_apply_plain32(op, x32, y32, k, o.precision == VIE_BF16X3 ? VIE_BF16X3 : VIE_C64, st);
            convert_c64_to_c128(y32, T.p, n * k, st);
        } else {
            op_apply64(op, Xl.as<double2>(), T.as<double2>(), k, st);
        }
        kr_sub_cols(a, b, T.as<double2>(), Rl.as<double2>(), k, nblk, st);
        kr_colnorms(a, Rl.as<double2>(), k, nblk, a.cols, rpart.as<double>(), a.rnorm, st);
        if (!cheap && Rf.p) kr_scatter_norm(a, Rl.as<double2>(), Rf.as<double2>(), k, nblk, st);  // update base
        if (o.precond) op_precond64(op, Rl.as<double2>(), Wl.as<double2>(), k, st);
        else VIE_CUDA(cudaMemcpyAsync(Wl.p, Rl.p, (size_t)n * k * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        kr_scatter_norm(a, Wl.as<double2>(), W.as<double2>(), k, nblk, st);
        kr_cycle_end(a, k, nblk, cheap ? 2 : 0, st);
    }

    // one restart cycle as a CUDA graph: pre -> while (continue) { Arnoldi step } -> post
    CycleGraph& graph_for(int k, const double2* b, double2* X, int mode) {
        const int key = 3 * k + mode;
        auto it = graphs.find(key);
        if (it != graphs.end()) return it->second;
        if (!s_body) VIE_CUDA(cudaStreamCreateWithFlags(&s_body, cudaStreamNonBlocking));
        CycleGraph cg;
        const long long c0 = g_kernel_launches.load();
        VIE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            launch_pre(k, s);
            const long long c1 = g_kernel_launches.load();
            cudaStreamCaptureStatus cst;
            cudaGraph_t cap = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            VIE_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cap, &deps, nullptr, &ndeps));
            std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
            cudaGraphConditionalHandle hnd;
            VIE_CUDA(cudaGraphConditionalHandleCreate(&hnd, cap, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};  // the rest zero
            p.conditional.handle = hnd;
            p.conditional.type = cudaGraphCondTypeWhile;
            p.conditional.size = 1;
            cudaGraphNode_t wnode;
            VIE_CUDA(cudaGraphAddNode(&wnode, cap, dv.data(), nullptr, dv.size(), &p));
            cudaGraph_t body = p.conditional.phGraph_out[0];
            VIE_CUDA(cudaStreamBeginCaptureToGraph(s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            try {
                launch_body(k, s_body, hnd, 1);
            } catch (...) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(s_body, &tmp);
                throw;
            }
            VIE_CUDA(cudaStreamEndCapture(s_body, &body));
            const long long c2 = g_kernel_launches.load();
            VIE_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
            launch_post(k, b, X, s, mode);
            const long long c3 = g_kernel_launches.load();
            VIE_CUDA(cudaStreamEndCapture(s, &graph));
            cg.pre = c1 - c0;
            cg.body = c2 - c1;
            cg.post = c3 - c2;
            VIE_COUNT_LAUNCH(-(c3 - c0));  // counted again per executed launch
        } catch (...) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(s, &tmp);
            if (tmp) cudaGraphDestroy(tmp);
            cudaGetLastError();
            throw;
        }
        cudaError_t e = cudaGraphInstantiate(&cg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) fail(VIE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return graphs.emplace(key, cg).first->second;
    }

    void read_state() {
        VIE_CUDA(cudaMemcpyAsync(h_pinned, ctr.p, KR_NCTR * sizeof(int), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaMemcpyAsync(h_pinned + KR_NCTR, done.p, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
        h_res.resize(nrhs);
        VIE_CUDA(cudaMemcpyAsync(h_res.data(), res.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
        // a tensor-core kernel that gave up waiting leaves its output incomplete
        // (and may thereby cause the non-finite values seen next): report it
        // first, and clear the word so that the operator stays usable
        if (op.d_err.p) {
            int e = 0;
            VIE_CUDA(cudaMemcpy(&e, op.d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) {
                VIE_CUDA(cudaMemset(op.d_err.p, 0, sizeof(int)));
                fail(VIE_ERR_TIMEOUT, "a tensor-core kernel gave up waiting for its operands or MMAs");
            }
        }
        if (h_pinned[KR_NAN]) fail(VIE_ERR_NAN, "non-finite residual in GMRES");
    }

    // a batched operator's kernels take each problem's right-hand sides from
    // the column-range table: slots (or columns) [x, y) belong to problem p
    void set_colr(const std::vector<int>& slot_cols) {
        if (lay.nprob <= 1) return;
        std::fill(h_colr.begin(), h_colr.end(), make_int2(0, 0));
        for (int i = 0; i < (int)slot_cols.size(); ++i) {
            int2& r = h_colr[lay.prob[slot_cols[i]]];
            if (r.y == 0) r.x = i;
            r.y = i + 1;
        }
        VIE_CUDA(cudaMemcpyAsync(colr_cycle.p, h_colr.data(), lay.nprob * sizeof(int2), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(colr.p, h_colr.data(), lay.nprob * sizeof(int2), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaStreamSynchronize(s));  // h_colr is reused for the next cycle
        op.colr = colr.as<int2>();
    }

    void run(const double2* b, double2* X) {
        struct ResetColr {
            Op& o;
            ~ResetColr() { o.colr = nullptr; }
        } reset{op};
        VIE_CUDA(cudaMemsetAsync(X, 0, (size_t)n * nrhs * sizeof(double2), s));
        // W = M^-1 b, beta0 = ||W|| per column
        std::vector<int> ident(nrhs);
        for (int c = 0; c < nrhs; ++c) ident[c] = c;
        set_colr(ident);
        if (o.precond) op_precond64(op, b, W.as<double2>(), nrhs, s);
        else VIE_CUDA(cudaMemcpyAsync(W.p, b, (size_t)n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(cols.p, ident.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
        const int nb1 = kr_nblk(n, nrhs, n_sm);
        // x = 0: the unpreconditioned residual is b
        kr_colnorms(a, b, nrhs, nb1, nullptr, rpart.as<double>(), bnorm.as<double>(), s);
        VIE_CUDA(cudaMemcpyAsync(rnorm.p, bnorm.p, nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
        kr_scatter_norm(a, W.as<double2>(), W.as<double2>(), nrhs, nb1, s);
        kr_cycle_end(a, nrhs, nb1, 1, s);
        read_state();
        h_beta0.resize(nrhs);
        VIE_CUDA(cudaMemcpyAsync(h_beta0.data(), beta0.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
        bound.assign(nrhs, 0.0);
        have_base = false;
        eps_low = a.eps_low;
        std::vector<int> live;
        while (true) {
            live.clear();
            for (int c = 0; c < nrhs; ++c)
                if (!h_pinned[KR_NCTR + c]) live.push_back(c);
            if (live.empty()) break;
            const int k = (int)live.size();
            if (o.autotune && c64 && !tuned(op, o.precision == VIE_BF16X3 ? VIE_BF16X3 : VIE_C64, k)) {
                std::vector<int> cand;
                std::vector<double> ms;
                tune_far(op, o.precision == VIE_BF16X3 ? VIE_BF16X3 : VIE_C64, k, s, cand, ms);
            }
            VIE_CUDA(cudaMemcpyAsync(cols.p, live.data(), k * sizeof(int), cudaMemcpyHostToDevice, s));
            set_colr(live);
            const int it0 = h_pinned[KR_IT];
            // the residual that ends this cycle in the inner precision while every
            // live column is still above 1000 x the tolerance (that residual only
            // starts the next cycle; the solve ends on a float64-accurate one)
            double worst = 0.0, bworst = 0.0;
            for (int c : live) {
                worst = std::max(worst, h_res[c]);
                bworst = std::max(bworst, bound[c]);
            }
            const double near = 100.0 * a.tol;
            const bool cheap = c64 && worst > near && it0 + m < a.maxit;
            // from a float64-accurate residual on, updates of it while their
            // accumulated error bound (eps_low |P^-1 Zs d| per cycle, |P^-1 Zs d| ~
            // the residual the cycle removes) stays below half the tolerance; an
            // updated residual ends a column only when it plus its bound is within
            // the tolerance.  Before that base exists: the inner-precision residual
            // while any column is far from the tolerance, else a float64 one.
            const bool upd = c64 && have_base && bworst + eps_low * worst <= 0.5 * a.tol;
            const int mode = upd ? kPostUpdate : cheap ? kPostCheap : kPostAccurate;
            if (mode == kPostUpdate)
                VIE_CUDA(cudaMemcpyAsync(ubound.p, bound.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
            if (o.launch == 1) {
                launch_pre(k, s);
                do {
                    launch_body(k, s, 0, 0);
                    VIE_CUDA(cudaMemcpyAsync(h_pinned, ctr.p, KR_NCTR * sizeof(int), cudaMemcpyDeviceToHost, s));
                    VIE_CUDA(cudaStreamSynchronize(s));
                } while (h_pinned[KR_CONT] && !h_pinned[KR_NAN]);
                launch_post(k, b, X, s, mode);
                read_state();
            } else {
                CycleGraph& cg = graph_for(k, b, X, mode);
                VIE_CUDA(cudaGraphLaunch(cg.exec, s));
                read_state();
                VIE_COUNT_LAUNCH(cg.pre + cg.post + cg.body * (long long)(h_pinned[KR_IT] - it0));
            }
            if (op.ctx->verbose) {
                int n1 = 0, n2 = 0, n3 = 0;
                for (int c : live) {
                    n1 += h_res[c] <= near;
                    n2 += h_res[c] <= 10.0 * a.tol;
                    n3 += h_res[c] <= 2.0 * a.tol;
                }
                fprintf(stderr,
                        "[vie] cycle: %d columns, steps %d..%d, restart residual %s (worst %.2e, bound %.2e; columns "
                        "<= 100/10/2 tol: %d/%d/%d)\n",
                        k, it0, h_pinned[KR_IT], mode == kPostCheap ? "inner" : mode == kPostUpdate ? "updated" : "float64",
                        worst, bworst, n1, n2, n3);
            }
            if (mode == kPostUpdate) {
                // error bound of the update: eps_low |P^-1 Zs d| relative to ||P^-1 b||
                std::vector<double> en(nrhs);
                VIE_CUDA(cudaMemcpyAsync(en.data(), enorm.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
                VIE_CUDA(cudaStreamSynchronize(s));
                for (int c : live) bound[c] += h_beta0[c] > 0 ? eps_low * en[c] / h_beta0[c] : 0.0;
            } else if (mode == kPostAccurate) {
                have_base = true;
                for (int c : live) bound[c] = 0.0;
            } else {
                have_base = false;
                // when a quarter or more of the live columns came near the tolerance
                // (where the inner-precision residual no longer tells), they get a
                // float64-accurate residual now, from the same iterate, so that the
                // converged ones stop before the next cycle; a few near columns do not
                // repay the float64 product (it costs about a cycle's applies) and go
                // on with the rest
                int nclose = 0;
                for (int c : live) nclose += h_res[c] <= near ? 1 : 0;
                const bool close = 4 * nclose >= (int)live.size();
                if (close) {
                    restore_colr(s);
                    launch_residual(k, b, X, s, false);
                    read_state();
                    if (op.ctx->verbose) fprintf(stderr, "[vie] cycle: float64 residual of the same iterate\n");
                    have_base = true;
                    for (int c : live) bound[c] = 0.0;
                }
            }
        }
    }
};

}  // namespace

void check_solve_opts(const Op& op, const vie_solve_opts* o, int nrhs) {
    if (op.fprec == 0) fail(VIE_ERR_STATE, "operator is not compressed");
    if (o->precision == VIE_C128 && op.fprec != VIE_C128)
        fail(VIE_ERR_INVALID_ARG, "an all-float64 solve needs VIE_C128 factors");
    if (o->precision != VIE_C128 && o->precision != VIE_C64 && o->precision != VIE_BF16X3 && o->precision != 0)
        fail(VIE_ERR_INVALID_ARG, "solve precision must be VIE_C64, VIE_BF16X3 or VIE_C128");
    if (o->launch != 0 && o->launch != 1) fail(VIE_ERR_INVALID_ARG, "solve launch must be 0 (graph) or 1 (host loop)");
    if (nrhs < 1 || nrhs > 1024) fail(VIE_ERR_INVALID_ARG, "a solve takes 1 to 1024 right-hand sides");
    if (o->method < 0 || o->method > 2)
        fail(VIE_ERR_INVALID_ARG, "solve method must be 0 (GMRES), 1 (BiCGStab) or 2 (block GMRES)");
}

GmresOutcome run_gmres(Op& op, const ColumnLayout& lay, const double2* b, double2* X, const vie_solve_opts& o,
                       int nrhs) {
    cudaStream_t s = op.ctx->stream;
    Gmres G(op, o, nrhs, lay);
    G.run(b, X);
    GmresOutcome r;
    r.rnorm.resize(nrhs);
    r.bnorm.resize(nrhs);
    r.res.resize(nrhs);
    r.iters.resize(nrhs);
    std::vector<double> hh(512);
    std::vector<int> hc(KR_NCTR);
    VIE_CUDA(cudaMemcpyAsync(r.rnorm.data(), G.rnorm.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(r.bnorm.data(), G.bnorm.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(r.res.data(), G.res.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(r.iters.data(), G.iters.p, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(hh.data(), G.hist.p, 512 * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(hc.data(), G.ctr.p, KR_NCTR * sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    r.applies = hc[KR_APPLIES];
    r.refinements = hc[KR_REFIN];
    r.hist.assign(hh.begin(), hh.begin() + std::min(512, hc[KR_IT]));
    return r;
}

int fill_stats(const GmresOutcome& r, int c0, int c1, double tol, double t0, vie_solve_stats* st) {
    double worst = 0.0, worst_true = 0.0;
    int iters = 0, status = VIE_OK;
    for (int c = c0; c < c1; ++c) {
        worst_true = std::max(worst_true, r.bnorm[c] > 0 ? r.rnorm[c] / r.bnorm[c] : 0.0);
        worst = std::max(worst, r.res[c]);
        iters = std::max(iters, r.iters[c]);
        if (r.res[c] > tol) status = VIE_ERR_NOT_CONVERGED;
    }
    if (st) {
        st->iterations = iters;
        st->applies = r.applies;
        st->refinements = r.refinements;
        st->residual = worst;
        st->true_residual = worst_true;
        st->t_solve_s = now_s() - t0;
        st->n_history = (int)r.hist.size();
        for (int i = 0; i < st->n_history; ++i) st->history[i] = r.hist[i];
    }
    return status;
}

int solve(Op& op, const vie_incident* inc, int nrhs, const vie_solve_opts* o, void* I_out, vie_solve_stats* st) {
    check_solve_opts(op, o, nrhs);
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
    const ColumnLayout lay = ColumnLayout::single(n, nrhs);
    const GmresOutcome r = o->method == 1   ? run_bicgstab(op, b.as<double2>(), X, *o, nrhs)
                           : o->method == 2 ? run_block_gmres(op, b.as<double2>(), X, *o, nrhs)
                                            : run_gmres(op, lay, b.as<double2>(), X, *o, nrhs);
    if (!o->out_on_device) {
        VIE_CUDA(cudaMemcpyAsync(I_out, X, (size_t)n * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
    }
    return fill_stats(r, 0, nrhs, o->tol > 0 ? o->tol : 1e-6, t0, st);
}

}  // namespace vie
