// Several problems in one solve: the block-diagonal union of their compressed
// operators.
//
// Arrays of different size (and wavelength and permittivity) with the same
// meta-atom discretisation are concatenated: atoms, atom types and their
// self blocks, far blocks and their factors.  No far block couples two
// problems, so the union is block diagonal and GMRES on a right-hand side
// that lives in one problem's rows is GMRES on that problem alone.  What the
// union buys is the launch: each phase of the far apply is one persistent
// kernel over the work items of all problems, balanced across the CTAs by
// the greedy least-loaded rule of App. C, and each Arnoldi step of the
// lockstep solve (one CUDA graph per restart cycle) serves every problem.
// The joined operator reads each problem's factors in place (no copy); only
// the small self blocks are concatenated.
// Each item and each self-block product only touches the right-hand sides
// of its own problem (a per-problem column range), and each Krylov vector
// only the rows of its problem.
#include <algorithm>
#include <memory>

#include "common.h"
#include "krylov.h"

namespace vie {

namespace {

void copy_concat(DevBuf& dst, const std::vector<const DevBuf*>& src, const std::vector<size_t>& bytes,
                 cudaStream_t s) {
    size_t total = 0;
    for (size_t b : bytes) total += b;
    dst.alloc(std::max<size_t>(total, 16));
    size_t off = 0;
    for (size_t i = 0; i < src.size(); ++i) {
        if (bytes[i])
            VIE_CUDA(cudaMemcpyAsync(static_cast<char*>(dst.p) + off, src[i]->p, bytes[i], cudaMemcpyDeviceToDevice, s));
        off += bytes[i];
    }
}

}  // namespace

std::unique_ptr<Op> make_union(const std::vector<Op*>& ops) {
    if (ops.empty()) fail(VIE_ERR_INVALID_ARG, "a batch needs at least one operator");
    Op& o0 = *ops[0];
    for (Op* p : ops) {
        if (p->ctx != o0.ctx) fail(VIE_ERR_INVALID_ARG, "batched operators must share one context");
        if (p->fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "batched operators need VIE_C64 factors");
        if (p->np != o0.np) fail(VIE_ERR_INVALID_ARG, "batched operators need the same voxels per meta-atom");
    }
    cudaStream_t s = o0.ctx->stream;
    auto U = std::make_unique<Op>();
    U->ctx = o0.ctx;
    U->np = o0.np;
    U->fprec = VIE_C64;
    U->nprob = (int)ops.size();
    const int np = o0.np;
    std::vector<const DevBuf*> z64, i64, z32, i32;
    std::vector<size_t> b64, b32;
    // the factors stay where they are: offsets from the lowest buffer address
    // (cudaMalloc returns 256-byte aligned addresses, so the distances are
    // whole complex float32 elements)
    const char* base = static_cast<const char*>(o0.d_factors.p);
    for (Op* p : ops) base = std::min(base, static_cast<const char*>(p->d_factors.p));
    U->factors_view = base;
    int atom_off = 0, type_off = 0, batom_off = 0, block_off = 0;
    for (int p = 0; p < (int)ops.size(); ++p) {
        const Op& P = *ops[p];
        const int64_t fac_off = (int64_t)((static_cast<const char*>(P.d_factors.p) - base) / sizeof(float2));
        U->L = std::max(U->L, P.L);
        U->tol = std::max(U->tol, P.tol);
        for (int a = 0; a < P.N; ++a) {
            U->types.push_back(P.types[a] + type_off);
            U->atom_prob.push_back(p);
        }
        for (int t = 0; t < P.T; ++t) U->type_prob.push_back(p);
        for (int x : P.block_atoms) U->block_atoms.push_back(x + atom_off);
        for (const FarBlock& b : P.blocks) {
            FarBlock c = b;
            c.t_off += batom_off;
            c.s_off += batom_off;
            c.q_off += fac_off;
            c.rh_off += fac_off;
            if (c.mirror >= 0) c.mirror += block_off;
            U->blocks.push_back(c);
            U->block_prob.push_back(p);
        }
        U->factor_entries += P.factor_entries;
        const size_t e = (size_t)P.T * np * np;
        z64.push_back(&P.d_zself64);
        i64.push_back(&P.d_inv64);
        b64.push_back(e * sizeof(double2));
        z32.push_back(&P.d_zself32);
        i32.push_back(&P.d_inv32);
        b32.push_back(e * sizeof(float2));
        atom_off += P.N;
        type_off += P.T;
        batom_off += (int)P.block_atoms.size();
        block_off += (int)P.blocks.size();
    }
    U->N = atom_off;
    U->T = type_off;
    copy_concat(U->d_zself64, z64, b64, s);
    copy_concat(U->d_inv64, i64, b64, s);
    copy_concat(U->d_zself32, z32, b32, s);
    copy_concat(U->d_inv32, i32, b32, s);
    U->atoms_of_type.assign(U->T, {});
    for (int a = 0; a < U->N; ++a) U->atoms_of_type[U->types[a]].push_back(a);
    std::vector<int> flat;
    U->type_atom_off.assign(U->T + 1, 0);
    for (int t = 0; t < U->T; ++t) {
        flat.insert(flat.end(), U->atoms_of_type[t].begin(), U->atoms_of_type[t].end());
        U->type_atom_off[t + 1] = (int)flat.size();
    }
    upload(U->d_atoms_by_type, flat.empty() ? std::vector<int>{0} : flat);
    build_apply_lists(*U);
    VIE_CUDA(cudaStreamSynchronize(s));
    return U;
}

void drop_unions(Ctx& c, const Op* o) {
    auto& v = c.unions;
    v.erase(std::remove_if(v.begin(), v.end(),
                           [o](const Ctx::Union& u) { return std::find(u.ops.begin(), u.ops.end(), o) != u.ops.end(); }),
            v.end());
}

namespace {

// The joined operator of `ops`: the cached one if the same operators (in the
// same order, with the same factors) were batched before, else a new one that
// replaces the least recently used of at most kUnionCache entries.  Its work
// lists and self-block copies are built once and reused across calls.
constexpr size_t kUnionCache = 4;

Op* get_union(const std::vector<Op*>& ops) {
    Ctx& c = *ops[0]->ctx;
    std::vector<const Op*> key(ops.begin(), ops.end());
    std::vector<uint64_t> gens;
    for (const Op* p : ops) gens.push_back(p->gen);
    for (Ctx::Union& u : c.unions)
        if (u.ops == key && u.gens == gens) {
            u.used = ++c.union_clock;
            return u.U.get();
        }
    std::unique_ptr<Op> U = make_union(ops);
    if (c.unions.size() >= kUnionCache) {
        auto lru = std::min_element(c.unions.begin(), c.unions.end(),
                                    [](const Ctx::Union& a, const Ctx::Union& b) { return a.used < b.used; });
        c.unions.erase(lru);
    }
    c.unions.push_back(Ctx::Union{std::move(key), std::move(gens), std::move(U), ++c.union_clock});
    return c.unions.back().U.get();
}

}  // namespace

int solve_batch(const std::vector<Op*>& ops, const vie_incident* incs, const int* nrhs, const vie_solve_opts* o,
                void** I_out, vie_solve_stats* st) {
    const int B = (int)ops.size();
    int K = 0;
    for (int p = 0; p < B; ++p) {
        if (nrhs[p] < 1) fail(VIE_ERR_INVALID_ARG, "every problem of a batch needs a right-hand side");
        check_solve_opts(*ops[p], o, nrhs[p]);
        if (o->method != 0) fail(VIE_ERR_INVALID_ARG, "batched solves use GMRES (method 0)");
        K += nrhs[p];
    }
    if (K > 1024) fail(VIE_ERR_INVALID_ARG, "a batch takes at most 1024 right-hand sides in total");
    if (o->precision == VIE_C128) fail(VIE_ERR_INVALID_ARG, "batched solves use VIE_C64 or VIE_BF16X3");
    const double t0 = now_s();
    Op* U = get_union(ops);
    cudaStream_t s = U->ctx->stream;
    const int64_t n = U->n();
    // columns grouped by problem; problem p owns rows [lo_p, lo_p + n_p)
    ColumnLayout lay;
    lay.nprob = B;
    std::vector<int> cbeg(B + 1, 0);
    std::vector<long long> lo(B);
    long long row = 0;
    for (int p = 0; p < B; ++p) {
        lo[p] = row;
        row += ops[p]->n();
        cbeg[p + 1] = cbeg[p] + nrhs[p];
        for (int c = 0; c < nrhs[p]; ++c) {
            lay.lo.push_back(lo[p]);
            lay.len.push_back(ops[p]->n());
            lay.prob.push_back(p);
        }
    }
    DevBuf b((size_t)n * K * sizeof(double2)), X((size_t)n * K * sizeof(double2));
    VIE_CUDA(cudaMemsetAsync(b.p, 0, b.bytes, s));
    for (int p = 0; p < B; ++p) {
        DevBuf kh(3 * nrhs[p] * sizeof(double)), pl(6 * nrhs[p] * sizeof(double));
        VIE_CUDA(cudaMemcpyAsync(kh.p, incs[p].khat, 3 * nrhs[p] * sizeof(double), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(pl.p, incs[p].pol, 6 * nrhs[p] * sizeof(double), cudaMemcpyHostToDevice, s));
        rhs_kernel_launch(*ops[p], kh.as<double>(), pl.as<double>(), nrhs[p],
                          b.as<double2>() + (int64_t)cbeg[p] * n + lo[p], n, s);
        VIE_CUDA(cudaStreamSynchronize(s));  // kh, pl go out of scope
    }
    const GmresOutcome r = run_gmres(*U, lay, b.as<double2>(), X.as<double2>(), *o, K);
    const double tol = o->tol > 0 ? o->tol : 1e-6;
    int status = VIE_OK;
    for (int p = 0; p < B; ++p) {
        const int64_t np_rows = ops[p]->n();
        VIE_CUDA(cudaMemcpy2DAsync(I_out[p], np_rows * sizeof(double2), X.as<double2>() + (int64_t)cbeg[p] * n + lo[p],
                                   n * sizeof(double2), np_rows * sizeof(double2), nrhs[p],
                                   o->out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        const int sp = fill_stats(r, cbeg[p], cbeg[p + 1], tol, t0, st ? &st[p] : nullptr);
        if (sp != VIE_OK) status = sp;
    }
    VIE_CUDA(cudaStreamSynchronize(s));
    if (st)
        for (int p = 0; p < B; ++p) st[p].t_solve_s = now_s() - t0;
    return status;
}

}  // namespace vie
