// Serving loop: continuous batching of metasurface solves on one GPU.
//
// Requests (geometry, wavelength, plane waves) queue in arrival order.  A
// fixed set of slots, each with its own CUDA stream and cuBLAS handle, runs
// requests concurrently: a free slot takes the oldest waiting request whose
// modelled HBM footprint (compressed factors, self blocks and inverses,
// Krylov basis, solver vectors, compression workspace) fits in what the
// in-flight requests leave of the budget.  A request that cannot fit even
// alone is rejected (VIE_ERR_ADMISSION).  Every wait is bounded.
//
// The slot's context refuses allocations beyond the footprint its request
// was admitted with, so an under-estimate cannot take memory that another
// request was promised: the allocation fails with VIE_ERR_OOM on the host,
// and the request goes back to the head of the queue with twice the
// footprint (at most the whole budget), to run again once that much is free.
// A request that fails this way with the whole budget is rejected.
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "common.h"

// slot-context hooks of the library (api.cpp)
void ctx_set_cap(vie_ctx* ctx, int64_t cap);
int64_t ctx_peak(vie_ctx* ctx);

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    uint64_t ticket;
    int retries = 0;
    std::vector<double> centres, sides, eps, khat, pol;
    std::vector<int> types, nv;
    int n_atoms, n_types, nrhs;
    double wavelength;
    int64_t footprint;
    double t_submit;
};

struct Done {
    vie_result r{};
    bool ready = false;
};

int64_t model_footprint(const Pending& p, int restart) {
    const int nv = p.nv[0];
    const int np = 3 * (nv + 1) * nv * nv;
    const int64_t n = (int64_t)p.n_atoms * np;
    int levels = 0;
    while ((1LL << (2 * levels)) < p.n_atoms) ++levels;
    // rank model: ~64 per far block row/column per level (measured ranks at
    // tolerance 1e-4 are of this order for sub-wavelength atoms)
    int64_t factor_entries = 2 * n * 64 * std::max(1, levels - 1);
    int64_t b = vie_footprint_bytes(n, np, p.nrhs, restart, factor_entries);
    // compression workspace: the largest batch of formed blocks
    int64_t big = std::min<int64_t>(n, (int64_t)16 * np);
    b += std::min<int64_t>(big * big * 8 * 4, (int64_t)8 << 30);
    // a test of the back-off path scales the model down (VIE_TEST_FOOTPRINT_SCALE)
    if (const char* e = std::getenv("VIE_TEST_FOOTPRINT_SCALE")) {
        const double f = std::atof(e);
        if (f > 0) b = std::max<int64_t>(1 << 20, (int64_t)(b * f));
    }
    return b;
}

}  // namespace

struct vie_server {
    vie_ctx* parent = nullptr;
    vie_serve_opts opts{};
    int device = 0;
    std::vector<vie_ctx*> slots;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::map<uint64_t, Done> results;
    uint64_t next_ticket = 1;
    int64_t inflight_bytes = 0;
    int64_t budget = 0;
    bool stopping = false;
    Clock::time_point t0 = Clock::now();

    double clock_s() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void run_slot(int si) {
        vie_ctx* ctx = slots[si];
        cudaSetDevice(device);
        while (true) {
            Pending p;
            {
                std::unique_lock<std::mutex> lk(mu);
                while (true) {
                    if (!queue.empty() && inflight_bytes + queue.front().footprint <= budget) break;
                    if (stopping && queue.empty()) return;
                    cv_work.wait_for(lk, std::chrono::milliseconds(50));
                }
                p = std::move(queue.front());
                queue.pop_front();
                inflight_bytes += p.footprint;
            }
            vie_result res{};
            res.t_submit_s = p.t_submit;
            res.t_start_s = clock_s();
            res.nrhs = p.nrhs;
            res.footprint_bytes = p.footprint;
            vie_geometry g{p.n_atoms, p.centres.data(), p.types.data(), p.n_types, p.sides.data(), p.nv.data(),
                           p.eps.data()};
            ctx_set_cap(ctx, p.footprint);
            vie_op* op = nullptr;
            int st = vie_assemble(ctx, &g, p.wavelength, &op);
            if (st == VIE_OK) st = vie_compress(op, opts.tol > 0 ? opts.tol : 1e-4, VIE_C64);
            if (st == VIE_OK) {
                vie_op_info info;
                vie_op_get_info(op, &info);
                res.n = info.n;
                res.I = static_cast<double*>(std::malloc((size_t)info.n * p.nrhs * 2 * sizeof(double)));
                vie_incident inc{p.khat.data(), p.pol.data()};
                vie_solve_opts so = opts.solve;
                so.out_on_device = 0;
                st = vie_solve(op, &inc, p.nrhs, &so, res.I, &res.stats);
            }
            if (op) vie_op_destroy(op);
            res.peak_bytes = ctx_peak(ctx);
            if (st == VIE_ERR_OOM) {
                std::free(res.I);
                res.I = nullptr;
                std::lock_guard<std::mutex> lk(mu);
                inflight_bytes -= p.footprint;
                if (p.footprint < budget) {
                    // back off: wait at the head of the queue for twice the memory
                    p.footprint = std::min<int64_t>(budget, 2 * p.footprint);
                    p.retries += 1;
                    queue.push_front(std::move(p));
                    cv_work.notify_all();
                    continue;
                }
                st = VIE_ERR_ADMISSION;  // did not fit with the whole budget
            }
            res.status = st;
            res.retries = p.retries;
            res.t_done_s = clock_s();
            {
                std::lock_guard<std::mutex> lk(mu);
                if (res.status != VIE_ERR_ADMISSION) inflight_bytes -= p.footprint;
                Done& d = results[p.ticket];
                d.r = res;
                d.ready = true;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

extern "C" {

int vie_serve(vie_server** out, vie_ctx* ctx, const vie_serve_opts* opts) {
    if (!out || !ctx || !opts) return VIE_ERR_INVALID_ARG;
    *out = nullptr;
    auto s = std::make_unique<vie_server>();
    s->parent = ctx;
    s->opts = *opts;
    int slots = opts->max_inflight > 0 ? opts->max_inflight : 4;
    cudaGetDevice(&s->device);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return VIE_ERR_CUDA;
    s->budget = opts->hbm_budget ? (int64_t)opts->hbm_budget : (int64_t)(fr > ((size_t)8 << 30) ? fr - ((size_t)8 << 30) : fr / 2);
    for (int i = 0; i < slots; ++i) {
        vie_ctx_opts co{s->device, (size_t)s->budget / slots, 0};
        vie_ctx* c = nullptr;
        int st = vie_create(&c, &co);
        if (st != VIE_OK) {
            for (auto* q : s->slots) vie_destroy(q);
            return st;
        }
        s->slots.push_back(c);
    }
    vie_server* raw = s.get();
    for (int i = 0; i < slots; ++i) raw->workers.emplace_back([raw, i] { raw->run_slot(i); });
    *out = s.release();
    return VIE_OK;
}

int vie_submit(vie_server* s, const vie_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || req->nrhs < 1 || req->geometry.n_atoms < 1 || req->geometry.n_types < 1)
        return VIE_ERR_INVALID_ARG;
    const vie_geometry& g = req->geometry;
    Pending p;
    p.n_atoms = g.n_atoms;
    p.n_types = g.n_types;
    p.nrhs = req->nrhs;
    p.wavelength = req->wavelength;
    p.centres.assign(g.centres, g.centres + 3 * g.n_atoms);
    p.types.assign(g.types, g.types + g.n_atoms);
    p.sides.assign(g.sides, g.sides + g.n_types);
    p.nv.assign(g.nv, g.nv + g.n_types);
    p.eps.assign(g.eps, g.eps + 2 * g.n_types);
    p.khat.assign(req->inc.khat, req->inc.khat + 3 * req->nrhs);
    p.pol.assign(req->inc.pol, req->inc.pol + 6 * req->nrhs);
    p.footprint = model_footprint(p, s->opts.solve.restart);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return VIE_ERR_STATE;
    if (p.footprint > s->budget) return VIE_ERR_ADMISSION;
    p.ticket = s->next_ticket++;
    p.t_submit = s->clock_s();
    *ticket = p.ticket;
    s->results[p.ticket] = Done{};
    s->queue.push_back(std::move(p));
    s->cv_work.notify_all();
    return VIE_OK;
}

int vie_poll(vie_server* s, uint64_t ticket, vie_result* out, int timeout_ms) {
    if (!s || !out) return VIE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return VIE_ERR_INVALID_ARG;
    auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (!s->results[ticket].ready) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->results[ticket].ready)
            return VIE_ERR_TIMEOUT;
    }
    *out = s->results[ticket].r;
    s->results.erase(ticket);
    return VIE_OK;
}

void vie_result_free(vie_result* r) {
    if (!r) return;
    std::free(r->I);
    r->I = nullptr;
}

int vie_server_stop(vie_server* s) {
    if (!s) return VIE_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto* c : s->slots) vie_destroy(c);
    for (auto& kv : s->results) std::free(kv.second.r.I);
    delete s;
    return VIE_OK;
}

}  // extern "C"
