// C-ABI entry points of libvie (declared in include/vie.h).  Every function
// catches the library's internal errors and returns a vie_status; nothing is
// thrown across the interface.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <memory>

#include "common.h"
#include "krylov.h"

// A context stays alive while operators made from it exist: vie_destroy only
// marks it closed when operators remain, the last vie_op_destroy frees it.
struct vie_ctx {
    vie::Ctx c;
    std::atomic<int> ops{0};
    std::atomic<bool> closed{false};
};
struct vie_op {
    vie::Op o;
};

namespace vie {

// ------------------------------------------------------------------ applies
static void ensure_F(Op& op, size_t bytes) {
    if (op.d_F.bytes < bytes) op.d_F.alloc(bytes);
}

void op_apply_fused32(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "float32 applies need VIE_C64 factors");
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(float2));
    float2* F = op.d_F.as<float2>();
    far32(op, x, n, F, n, nrhs, VIE_C64, s);
    self_gemm<float2, float2>(op, op.d_inv32.as<float2>(), x, n, F, n, y, n, nrhs, 1, s);
}

void op_apply_plain32(Op& op, const float2* x, float2* y, int nrhs, int precision, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "float32 applies need VIE_C64 factors");
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(float2));
    float2* F = op.d_F.as<float2>();
    far32(op, x, n, F, n, nrhs, precision, s);
    self_gemm<float2, float2>(op, op.d_zself32.as<float2>(), x, n, F, n, y, n, nrhs, 0, s);
}

// E x = P^-1 Zs x - x = Z_D^-1 (far part) x in the inner precision: the fused
// apply without its identity term (the Arnoldi steps of the mixed-precision
// GMRES build the Krylov space of E, the same as that of I + E)
void op_apply_shift32(Op& op, const float2* x, float2* y, int nrhs, int precision, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "float32 applies need VIE_C64 factors");
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(float2));
    float2* F = op.d_F.as<float2>();
    far32(op, x, n, F, n, nrhs, precision, s);
    self_gemm<float2, float2>(op, op.d_inv32.as<float2>(), F, n, nullptr, 0, y, n, nrhs, 2, s);  // y = Z_D^-1 F
}

void op_apply_fused_bf16x3(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s) {
    if (op.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "VIE_BF16X3 applies need VIE_C64 factors");
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(float2));
    float2* F = op.d_F.as<float2>();
    far32(op, x, n, F, n, nrhs, VIE_BF16X3, s);
    self_gemm<float2, float2>(op, op.d_inv32.as<float2>(), x, n, F, n, y, n, nrhs, 1, s);
}

void op_apply64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s) {
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(double2));
    double2* F = op.d_F.as<double2>();
    if (op.fprec == VIE_C128) apply_far<double2, double2>(op, x, n, F, n, nrhs, s);
    else apply_far_df(op, x, n, F, n, nrhs, s);
    self_gemm<double2, double2>(op, op.d_zself64.as<double2>(), x, n, F, n, y, n, nrhs, 0, s);
}

void op_apply_fused64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s) {
    const int64_t n = op.n();
    ensure_F(op, (size_t)n * nrhs * sizeof(double2));
    double2* F = op.d_F.as<double2>();
    if (op.fprec == VIE_C128) apply_far<double2, double2>(op, x, n, F, n, nrhs, s);
    else apply_far_df(op, x, n, F, n, nrhs, s);
    self_gemm<double2, double2>(op, op.d_inv64.as<double2>(), x, n, F, n, y, n, nrhs, 1, s);
}

void op_reserve(Op& op, int nrhs, int precision, cudaStream_t s) {
    if (precision == VIE_BF16X3) {
        umma_prepare(op, s);
        umma_pack(op, s);  // any cycle's right-hand-side count may choose the packed variant
    }
    ensure_F(op, (size_t)op.n() * nrhs * sizeof(double2));
    const size_t need = (size_t)std::max<int64_t>(op.t_total, 1) * nrhs * sizeof(double2);
    if (op.d_t.bytes < need) op.d_t.alloc(need);
    const size_t need_x = (size_t)op.n() * nrhs * sizeof(float4);
    if (op.fprec == VIE_C64 && op.d_xs.bytes < need_x) op.d_xs.alloc(need_x);
    if (op.fprec == VIE_C64) shared_reserve(op);
}

void op_precond64(Op& op, const double2* x, double2* y, int nrhs, cudaStream_t s) {
    self_gemm<double2, double2>(op, op.d_inv64.as<double2>(), x, op.n(), nullptr, 0, y, op.n(), nrhs, 2, s);
}

}  // namespace vie

using namespace vie;

namespace {

template <class F>
int guarded(vie_ctx* ctx, F&& f) {
    cudaGetLastError();  // an earlier failure elsewhere is not this call's error
    AllocScope scope(ctx ? &ctx->c : nullptr);
    try {
        f();
        if (ctx) ctx->c.err.clear();
        return VIE_OK;
    } catch (const Error& e) {
        if (ctx) ctx->c.err = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->c.err = "host allocation failed";
        return VIE_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->c.err = e.what();
        return VIE_ERR_INVALID_ARG;
    }
}

vie_ctx* ctx_of(vie_op* op) { return op ? static_cast<vie_ctx*>(op->o.ctx->owner) : nullptr; }

}  // namespace

// server use: the cap of a slot context is the footprint its request was
// admitted with; the peak shows what the request really held
void ctx_set_cap(vie_ctx* ctx, int64_t cap) {
    ctx->c.cap = cap;
    ctx->c.peak = ctx->c.allocated.load();
}
int64_t ctx_peak(vie_ctx* ctx) { return ctx->c.peak.load(); }

namespace {

void set_device(Ctx& c) { VIE_CUDA(cudaSetDevice(c.device)); }

// Caller vectors: 16-byte aligned (the apply kernels read two complex float32
// entries as one 16-byte load) and, for an input / output pair of `bytes`
// bytes each, disjoint.  Checked before anything is launched.
void check_vectors(const char* who, const void* x, const void* y, size_t bytes) {
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
        fail(VIE_ERR_INVALID_ARG, std::string(who) + ": vectors must be 16-byte aligned");
    const char* a = static_cast<const char*>(x);
    const char* b = static_cast<const char*>(y);
    if (y && a < b + bytes && b < a + bytes) fail(VIE_ERR_INVALID_ARG, std::string(who) + ": x and y overlap");
}

size_t elem_bytes(int precision) { return (precision == VIE_C128 || precision == VIE_C64_ACC64) ? 16 : 8; }

}  // namespace

extern "C" {

int vie_create(vie_ctx** out, const vie_ctx_opts* opts) {
    if (!out) return VIE_ERR_INVALID_ARG;
    *out = nullptr;
    auto ctx = std::make_unique<vie_ctx>();
    int st = guarded(ctx.get(), [&] {
        Ctx& c = ctx->c;
        c.owner = ctx.get();
        c.device = opts ? opts->device : 0;
        c.verbose = opts ? opts->verbose : 0;
        c.no_sharing = opts ? opts->no_sharing : 0;
        int ndev = 0;
        VIE_CUDA(cudaGetDeviceCount(&ndev));
        if (c.device < 0 || c.device >= ndev) fail(VIE_ERR_INVALID_ARG, "no such CUDA device");
        set_device(c);
        cudaDeviceProp prop;
        VIE_CUDA(cudaGetDeviceProperties(&prop, c.device));
        c.n_sm = prop.multiProcessorCount;
        VIE_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        VIE_BLAS(cublasCreate(&c.blas));
        VIE_BLAS(cublasSetStream(c.blas, c.stream));
        size_t fr = 0, tot = 0;
        VIE_CUDA(cudaMemGetInfo(&fr, &tot));
        size_t reserve = (size_t)4 << 30;
        c.budget = (opts && opts->hbm_budget) ? opts->hbm_budget : (fr > 2 * reserve ? fr - reserve : fr / 2);
        c.cap = (opts && opts->hbm_budget) ? (int64_t)opts->hbm_budget : 0;
    });
    if (st != VIE_OK) {
        // keep the message readable through a stub context
        static thread_local std::string last;
        last = ctx->c.err;
        return st;
    }
    *out = ctx.release();
    return VIE_OK;
}

static void free_ctx(vie_ctx* ctx) {
    cudaSetDevice(ctx->c.device);
    if (ctx->c.blas) cublasDestroy(ctx->c.blas);
    if (ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
    delete ctx;
}

void vie_destroy(vie_ctx* ctx) {
    if (!ctx) return;
    ctx->closed = true;
    if (ctx->ops.load() == 0) free_ctx(ctx);
}

const char* vie_last_error(vie_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "no context"; }

int vie_assemble(vie_ctx* ctx, const vie_geometry* g, double wavelength, vie_op** out) {
    if (!ctx || !g || !out) return VIE_ERR_INVALID_ARG;
    *out = nullptr;
    auto op = std::make_unique<vie_op>();
    int st = guarded(ctx, [&] {
        set_device(ctx->c);
        Op& o = op->o;
        o.ctx = &ctx->c;
        double t0 = now_s();
        if (g->n_atoms < 1 || g->n_types < 1 || !g->centres || !g->types || !g->sides || !g->nv || !g->eps)
            fail(VIE_ERR_INVALID_ARG, "incomplete geometry");
        if (!(wavelength > 0) || !std::isfinite(wavelength)) fail(VIE_ERR_INVALID_ARG, "wavelength must be > 0");
        o.N = g->n_atoms;
        o.T = g->n_types;
        o.centres.assign(g->centres, g->centres + 3 * o.N);
        o.types.assign(g->types, g->types + o.N);
        o.sides.assign(g->sides, g->sides + o.T);
        o.nvs.assign(g->nv, g->nv + o.T);
        for (int t = 0; t < o.T; ++t) {
            o.eps.emplace_back(g->eps[2 * t], g->eps[2 * t + 1]);
            if (!(o.sides[t] > 0) || !std::isfinite(o.sides[t])) fail(VIE_ERR_INVALID_ARG, "cube side must be > 0");
            if (o.nvs[t] < 1 || o.nvs[t] > 16) fail(VIE_ERR_INVALID_ARG, "voxels per edge must be in 1..16");
            if (o.nvs[t] != o.nvs[0]) fail(VIE_ERR_INVALID_ARG, "all atom types must have the same nv");
            if (std::abs(o.eps[t] - cd(1.0)) < 1e-12) fail(VIE_ERR_INVALID_ARG, "eps_r = 1 (no scatterer)");
        }
        for (int a = 0; a < o.N; ++a) {
            if (o.types[a] < 0 || o.types[a] >= o.T) fail(VIE_ERR_INVALID_ARG, "atom type out of range");
            for (int d = 0; d < 3; ++d)
                if (!std::isfinite(o.centres[3 * a + d])) fail(VIE_ERR_INVALID_ARG, "non-finite atom centre");
        }
        // atoms must not touch: the rule between atoms assumes separated cubes
        for (int a = 0; a < o.N; ++a)
            for (int b = a + 1; b < o.N; ++b) {
                double dmax = 0;
                for (int d = 0; d < 3; ++d) dmax = std::max(dmax, std::fabs(o.centres[3 * a + d] - o.centres[3 * b + d]));
                if (dmax <= 0.5 * (o.sides[o.types[a]] + o.sides[o.types[b]]))
                    fail(VIE_ERR_INVALID_ARG, "atoms " + std::to_string(a) + " and " + std::to_string(b) + " overlap or touch");
            }
        o.wavelength = wavelength;
        o.k = 2.0 * M_PI / wavelength;
        o.mesh = build_mesh(1.0, o.nvs[0]);
        o.np = o.mesh.np;
        for (int t = 0; t < o.T; ++t) o.h.push_back(o.sides[t] / o.nvs[t]);
        // device geometry and mesh topology
        upload(o.d_centres, o.centres);
        upload(o.d_types, o.types);
        upload(o.d_sides, o.sides);
        std::vector<double2> ichi(o.T);
        for (int t = 0; t < o.T; ++t) {
            cd ic = 1.0 / (o.eps[t] - 1.0);
            ichi[t] = make_double2(ic.real(), ic.imag());
        }
        upload(o.d_inv_chi, ichi);
        std::vector<int4> face(o.np);
        for (int f = 0; f < o.np; ++f)
            face[f] = make_int4(o.mesh.face_dir[f], o.mesh.face_lo[f], o.mesh.face_hi[f], o.mesh.face_sheet[f]);
        upload(o.d_mesh_face, face);
        upload(o.d_mesh_sign, o.mesh.face_sheet_sign);
        upload(o.d_mesh_vox, o.mesh.vox_ijk);
        upload(o.d_mesh_surf, o.mesh.surf_face);
        std::vector<float4> voxc(o.mesh.nvox), surfc(o.mesh.nsurf);
        for (int v = 0; v < o.mesh.nvox; ++v)
            voxc[v] = make_float4(o.mesh.vox_ijk[3 * v] + 0.5f, o.mesh.vox_ijk[3 * v + 1] + 0.5f,
                                  o.mesh.vox_ijk[3 * v + 2] + 0.5f, 0.f);
        {
            // face (d, i, j, k) in its direction-major numbering
            const int nv = o.mesh.nv;
            for (int sidx = 0; sidx < o.mesh.nsurf; ++sidx) {
                int f = o.mesh.surf_face[sidx], d = o.mesh.face_dir[f];
                int g = f - d * (nv + 1) * nv * nv;
                int ijk[3];
                if (d == 0) { ijk[0] = g / (nv * nv); ijk[1] = (g / nv) % nv; ijk[2] = g % nv; }
                else if (d == 1) { ijk[0] = g / (nv * (nv + 1)); ijk[1] = (g / nv) % (nv + 1); ijk[2] = g % nv; }
                else { ijk[0] = g / (nv * (nv + 1)); ijk[1] = (g / (nv + 1)) % nv; ijk[2] = g % (nv + 1); }
                float c[3];
                for (int e = 0; e < 3; ++e) c[e] = e == d ? (float)ijk[e] : ijk[e] + 0.5f;
                surfc[sidx] = make_float4(c[0], c[1], c[2], (float)d);
            }
        }
        upload(o.d_mesh_voxc, voxc);
        upload(o.d_mesh_surfc, surfc);
        o.dmesh = DevMesh{o.mesh.nv, o.mesh.np, o.mesh.nvox, o.mesh.nsurf, o.d_mesh_face.as<int4>(),
                          o.d_mesh_sign.as<int>(), o.d_mesh_vox.as<int>(), o.d_mesh_surf.as<int>(),
                          o.d_mesh_voxc.as<float4>(), o.d_mesh_surfc.as<float4>()};
        o.atoms_of_type.assign(o.T, {});
        for (int a = 0; a < o.N; ++a) o.atoms_of_type[o.types[a]].push_back(a);
        std::vector<int> flat;
        o.type_atom_off.assign(o.T + 1, 0);
        for (int t = 0; t < o.T; ++t) {
            flat.insert(flat.end(), o.atoms_of_type[t].begin(), o.atoms_of_type[t].end());
            o.type_atom_off[t + 1] = (int)flat.size();
        }
        upload(o.d_atoms_by_type, flat);
        // grid hierarchy and far-block lists
        build_tree(o);
        // self blocks, their inverses (float64) and float32 copies
        assemble_self_blocks(o);
        invert_self_blocks(o);
        size_t ne = (size_t)o.T * o.np * o.np;
        o.d_zself32.alloc(ne * sizeof(float2));
        o.d_inv32.alloc(ne * sizeof(float2));
        convert_c128_to_c64(o.d_zself64.p, o.d_zself32.p, ne, ctx->c.stream);
        convert_c128_to_c64(o.d_inv64.p, o.d_inv32.p, ne, ctx->c.stream);
        VIE_CUDA(cudaStreamSynchronize(ctx->c.stream));
        o.t_assemble = now_s() - t0;
        if (ctx->c.verbose)
            fprintf(stderr, "[vie] assemble: N=%d np=%d levels=%d far blocks=%zu  %.3f s\n", o.N, o.np, o.L,
                    o.blocks.size(), o.t_assemble);
    });
    if (st == VIE_OK) {
        ctx->ops.fetch_add(1);
        *out = op.release();
    }
    return st;
}

static int compress_with(vie_op* op, double tol, int factor_precision, int method) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        set_device(*op->o.ctx);
        if (!(tol > 0 && tol < 1)) fail(VIE_ERR_INVALID_ARG, "tolerance must be in (0, 1)");
        if (factor_precision != VIE_C64 && factor_precision != VIE_C128)
            fail(VIE_ERR_INVALID_ARG, "factor precision must be VIE_C64 or VIE_C128");
        double t0 = now_s();
        drop_unions(*op->o.ctx, &op->o);
        ++op->o.gen;
        compress_operator(op->o, tol, factor_precision, method);
        op->o.t_compress = now_s() - t0;
        if (op->o.ctx->verbose)
            fprintf(stderr, "[vie] compress: %lld factor entries  %.3f s\n", (long long)op->o.factor_entries,
                    op->o.t_compress);
    });
}

int vie_compress(vie_op* op, double tol, int factor_precision) {
    return compress_with(op, tol, factor_precision, VIE_COMPRESS_RANGE_FINDER);
}

int vie_compress_cross(vie_op* op, double tol, int factor_precision) {
    return compress_with(op, tol, factor_precision, VIE_COMPRESS_CROSS);
}

void vie_op_destroy(vie_op* op) {
    if (!op) return;
    vie_ctx* ctx = ctx_of(op);
    cudaSetDevice(op->o.ctx->device);
    cudaStreamSynchronize(op->o.ctx->stream);
    {
        AllocScope scope(op->o.ctx);
        drop_unions(*op->o.ctx, &op->o);
    }
    delete op;
    if (ctx->ops.fetch_sub(1) == 1 && ctx->closed.load()) free_ctx(ctx);
}

int vie_op_get_info(const vie_op* op, vie_op_info* info) {
    if (!op || !info) return VIE_ERR_INVALID_ARG;
    const Op& o = op->o;
    std::memset(info, 0, sizeof(*info));
    info->n_atoms = o.N;
    info->np = o.np;
    info->n_types = o.T;
    info->levels = o.L;
    info->n = o.n();
    info->n_far_blocks = (int64_t)o.blocks.size();
    int rmin = 1 << 30, rmax = 0;
    double rsum = 0;
    for (const auto& b : o.blocks) {
        info->far_entries += (int64_t)b.m * b.n;
        rmin = std::min(rmin, b.rank);
        rmax = std::max(rmax, b.rank);
        rsum += b.rank;
    }
    info->rank_min = o.blocks.empty() ? 0 : rmin;
    info->rank_max = rmax;
    info->rank_mean = o.blocks.empty() ? 0 : rsum / o.blocks.size();
    info->factor_entries = o.factor_entries;
    info->self_entries = (int64_t)o.N * o.np * o.np;
    double nqr = (double)o.factor_entries + (double)info->self_entries;
    info->gain = o.fprec ? (double)o.n() * (double)o.n() / nqr : 0.0;
    info->factor_precision = o.fprec;
    info->tol = o.tol;
    // one single-RHS c64 apply: factors once, distinct self/inverse blocks once,
    // x read once, y written once
    info->apply_bytes = 8 * (o.factor_entries + (int64_t)o.T * o.np * o.np + 2 * o.n());
    info->t_assemble_s = o.t_assemble;
    info->t_compress_s = o.t_compress;
    info->stored_entries = o.stored_entries;
    info->packed_bytes = o.umma_packed ? (int64_t)umma_pack_bytes(o) : 0;
    info->compress_method = o.cmethod;
    info->cross_bytes = o.cross_bytes;
    info->t_cross_s = o.t_cross;
    return VIE_OK;
}

// y = Zs^H x.  Between atoms the rule is symmetric and each mirror block
// stores the transposed factors of its partner, so the compressed far part F
// is a symmetric matrix (F^T = F) and F^H x = conj(F conj(x)); the self part
// uses the conjugate-transposed self blocks (the touching-pair rule is not
// exactly symmetric).
static void apply_adjoint(Op& o, const void* x, void* y, int nrhs, int precision, cudaStream_t s) {
    const int64_t n = o.n(), len = n * nrhs;
    const bool wide = precision == VIE_C128 || precision == VIE_C64_ACC64;
    const size_t eb = wide ? sizeof(double2) : sizeof(float2);
    if (precision == VIE_C128 && o.fprec != VIE_C128) fail(VIE_ERR_INVALID_ARG, "VIE_C128 applies need VIE_C128 factors");
    if (precision != VIE_C128 && o.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "this precision needs VIE_C64 factors");
    DevBuf& H = wide ? o.d_zselfH64 : o.d_zselfH32;
    if (!H.p) {
        H.alloc((size_t)o.T * o.np * o.np * eb);
        conj_transpose_blocks(wide ? o.d_zself64.p : o.d_zself32.p, H.p, o.T, o.np, wide, s);
    }
    if (o.d_adj.bytes < (size_t)len * eb) o.d_adj.alloc((size_t)len * eb);
    ensure_F(o, (size_t)len * eb);
    conj_copy(x, o.d_adj.p, len, wide, s);
    if (wide) {
        double2* F = o.d_F.as<double2>();
        if (o.fprec == VIE_C128) apply_far<double2, double2>(o, o.d_adj.as<double2>(), n, F, n, nrhs, s);
        else apply_far_df(o, o.d_adj.as<double2>(), n, F, n, nrhs, s);
        conj_copy(F, F, len, true, s);
        self_gemm<double2, double2>(o, H.as<double2>(), (const double2*)x, n, F, n, (double2*)y, n, nrhs, 0, s);
    } else {
        float2* F = o.d_F.as<float2>();
        far32(o, o.d_adj.as<float2>(), n, F, n, nrhs, precision, s);
        conj_copy(F, F, len, false, s);
        self_gemm<float2, float2>(o, H.as<float2>(), (const float2*)x, n, F, n, (float2*)y, n, nrhs, 0, s);
    }
}

int vie_apply(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, int precision, int flags, vie_stream stream) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (!x || !y || nrhs < 1 || ld != o.n()) fail(VIE_ERR_INVALID_ARG, "vie_apply: bad vectors (ld must be n)");
        check_vectors("vie_apply", x, y, (size_t)o.n() * nrhs * elem_bytes(precision));
        if (o.fprec == 0 && !(flags & VIE_APPLY_DENSE)) fail(VIE_ERR_STATE, "operator is not compressed");
        cudaStream_t s = stream ? (cudaStream_t)stream : o.ctx->stream;
        const bool fuse = flags & VIE_APPLY_FUSE_PRECOND;
        if (flags & ~(VIE_APPLY_FUSE_PRECOND | VIE_APPLY_DENSE | VIE_APPLY_ADJOINT))
            fail(VIE_ERR_INVALID_ARG, "vie_apply: unknown flags");
        if (flags & VIE_APPLY_ADJOINT) {
            if (flags != VIE_APPLY_ADJOINT)
                fail(VIE_ERR_INVALID_ARG, "VIE_APPLY_ADJOINT cannot be combined with other flags");
            if (precision != VIE_C64 && precision != VIE_BF16X3 && precision != VIE_C128 && precision != VIE_C64_ACC64)
                fail(VIE_ERR_INVALID_ARG, "unsupported apply precision");
            apply_adjoint(o, x, y, nrhs, precision, s);
            return;
        }
        if (flags & VIE_APPLY_DENSE) {
            if (fuse) fail(VIE_ERR_INVALID_ARG, "VIE_APPLY_DENSE cannot be combined with the preconditioner");
            if (nrhs != 1) fail(VIE_ERR_INVALID_ARG, "VIE_APPLY_DENSE takes one right-hand side");
            if (precision == VIE_C64) dense_apply_c64(o, (const float2*)x, (float2*)y, s);
            else if (precision == VIE_C128) dense_apply_c128(o, (const double2*)x, (double2*)y, s);
            else fail(VIE_ERR_INVALID_ARG, "VIE_APPLY_DENSE needs VIE_C64 or VIE_C128");
            return;
        }
        if (precision == VIE_C64) {
            if (fuse) op_apply_fused32(o, (const float2*)x, (float2*)y, nrhs, s);
            else {
                if (o.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "VIE_C64 applies need VIE_C64 factors");
                ensure_F(o, (size_t)o.n() * nrhs * sizeof(float2));
                float2* F = o.d_F.as<float2>();
                far32(o, (const float2*)x, o.n(), F, o.n(), nrhs, VIE_C64, s);
                self_gemm<float2, float2>(o, o.d_zself32.as<float2>(), (const float2*)x, o.n(), F, o.n(),
                                          (float2*)y, o.n(), nrhs, 0, s);
            }
        } else if (precision == VIE_BF16X3) {
            if (fuse) op_apply_fused_bf16x3(o, (const float2*)x, (float2*)y, nrhs, s);
            else {
                if (o.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "VIE_BF16X3 applies need VIE_C64 factors");
                ensure_F(o, (size_t)o.n() * nrhs * sizeof(float2));
                float2* F = o.d_F.as<float2>();
                far32(o, (const float2*)x, o.n(), F, o.n(), nrhs, VIE_BF16X3, s);
                self_gemm<float2, float2>(o, o.d_zself32.as<float2>(), (const float2*)x, o.n(), F, o.n(),
                                          (float2*)y, o.n(), nrhs, 0, s);
            }
        } else if (precision == VIE_C128 || precision == VIE_C64_ACC64) {
            if (precision == VIE_C128 && o.fprec != VIE_C128) fail(VIE_ERR_INVALID_ARG, "VIE_C128 applies need VIE_C128 factors");
            if (precision == VIE_C64_ACC64 && o.fprec != VIE_C64) fail(VIE_ERR_INVALID_ARG, "VIE_C64_ACC64 needs VIE_C64 factors");
            if (fuse) op_apply_fused64(o, (const double2*)x, (double2*)y, nrhs, s);
            else op_apply64(o, (const double2*)x, (double2*)y, nrhs, s);
        } else {
            fail(VIE_ERR_INVALID_ARG, "unsupported apply precision");
        }
    });
}

int vie_apply_noalloc(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, vie_stream stream) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (!x || !y || nrhs < 1 || ld != o.n()) fail(VIE_ERR_INVALID_ARG, "vie_apply_noalloc: bad vectors (ld must be n)");
        check_vectors("vie_apply_noalloc", x, y, (size_t)o.n() * nrhs * sizeof(float2));
        if (o.fprec == 0) fail(VIE_ERR_STATE, "operator is not compressed");
        apply_static(o, (const float2*)x, (float2*)y, nrhs, stream ? (cudaStream_t)stream : o.ctx->stream);
    });
}

int vie_precond(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, int precision, vie_stream stream) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (!x || !y || nrhs < 1 || ld != o.n()) fail(VIE_ERR_INVALID_ARG, "vie_precond: bad vectors (ld must be n)");
        check_vectors("vie_precond", x, y, (size_t)o.n() * nrhs * elem_bytes(precision));
        cudaStream_t s = stream ? (cudaStream_t)stream : o.ctx->stream;
        if (precision == VIE_C64)
            self_gemm<float2, float2>(o, o.d_inv32.as<float2>(), (const float2*)x, o.n(), nullptr, 0, (float2*)y,
                                      o.n(), nrhs, 2, s);
        else if (precision == VIE_C128)
            op_precond64(o, (const double2*)x, (double2*)y, nrhs, s);
        else
            fail(VIE_ERR_INVALID_ARG, "unsupported precond precision");
    });
}

int vie_rhs(vie_op* op, const vie_incident* inc, int nrhs, void* b, int64_t ld, vie_stream stream) {
    if (!op || !inc || !b || nrhs < 1) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (ld < o.n()) fail(VIE_ERR_INVALID_ARG, "ld < n");
        check_vectors("vie_rhs", b, nullptr, 0);
        cudaStream_t s = stream ? (cudaStream_t)stream : o.ctx->stream;
        DevBuf kh(3 * nrhs * sizeof(double)), pl(6 * nrhs * sizeof(double));
        VIE_CUDA(cudaMemcpyAsync(kh.p, inc->khat, 3 * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(pl.p, inc->pol, 6 * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        rhs_kernel_launch(o, kh.as<double>(), pl.as<double>(), nrhs, b, ld, s);
        VIE_CUDA(cudaStreamSynchronize(s));
    });
}

int vie_solve(vie_op* op, const vie_incident* inc, int nrhs, const vie_solve_opts* opts, void* I_out,
              vie_solve_stats* stats) {
    if (!op || !inc || !opts || !I_out || nrhs < 1) return VIE_ERR_INVALID_ARG;
    int result = VIE_OK;
    int st = guarded(ctx_of(op), [&] {
        set_device(*op->o.ctx);
        if (opts->out_on_device) check_vectors("vie_solve", I_out, nullptr, 0);
        result = solve(op->o, inc, nrhs, opts, I_out, stats);
    });
    if (st != VIE_OK) return st;
    if (result != VIE_OK && ctx_of(op)) ctx_of(op)->c.err = "GMRES did not reach the tolerance";
    return result;
}

int vie_solve_batch(vie_op* const* ops, int count, const vie_incident* inc, const int* nrhs,
                    const vie_solve_opts* opts, void* const* I_out, vie_solve_stats* stats) {
    if (!ops || count < 1 || !inc || !nrhs || !opts || !I_out) return VIE_ERR_INVALID_ARG;
    for (int p = 0; p < count; ++p)
        if (!ops[p] || !I_out[p]) return VIE_ERR_INVALID_ARG;
    int result = VIE_OK;
    int st = guarded(ctx_of(ops[0]), [&] {
        set_device(*ops[0]->o.ctx);
        std::vector<Op*> v(count);
        std::vector<void*> outs(count);
        for (int p = 0; p < count; ++p) {
            v[p] = &ops[p]->o;
            outs[p] = I_out[p];
            if (opts->out_on_device) check_vectors("vie_solve_batch", I_out[p], nullptr, 0);
        }
        result = solve_batch(v, inc, nrhs, opts, outs.data(), stats);
    });
    if (st != VIE_OK) return st;
    if (result != VIE_OK && ctx_of(ops[0])) ctx_of(ops[0])->c.err = "GMRES did not reach the tolerance";
    return result;
}

int vie_fields(vie_op* op, const vie_incident* inc, const void* I, int nrhs, const double* dirs, int npts, int mode,
               void* E_out, double* sigma_out) {
    if (!op || !I || nrhs < 1) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (mode != 0 && mode != 1) fail(VIE_ERR_INVALID_ARG, "vie_fields: mode 0 (far field) or 1 (near field)");
        cudaStream_t s = o.ctx->stream;
        const int64_t n = o.n();
        DevBuf dI((size_t)n * nrhs * sizeof(double2));
        VIE_CUDA(cudaMemcpyAsync(dI.p, I, dI.bytes, cudaMemcpyHostToDevice, s));
        if (mode == 1) {
            if (!E_out || !dirs || npts < 1) fail(VIE_ERR_INVALID_ARG, "vie_fields: the near field needs points and E_out");
            for (int64_t i = 0; i < 3 * (int64_t)npts; ++i)
                if (!std::isfinite(dirs[i])) fail(VIE_ERR_INVALID_ARG, "vie_fields: non-finite point");
            DevBuf dp((size_t)3 * npts * sizeof(double)), out((size_t)npts * nrhs * 3 * sizeof(double2));
            VIE_CUDA(cudaMemcpyAsync(dp.p, dirs, dp.bytes, cudaMemcpyHostToDevice, s));
            near_field_launch(o, dI.p, nrhs, dp.as<double>(), npts, out.p, s);
            VIE_CUDA(cudaMemcpyAsync(E_out, out.p, out.bytes, cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            if (sigma_out) fail(VIE_ERR_INVALID_ARG, "vie_fields: cross sections come with mode 0");
            return;
        }
        auto far = [&](const std::vector<double>& d, std::vector<cd>& F) {
            int np_ = (int)(d.size() / 3);
            DevBuf dd(d.size() * sizeof(double)), out((size_t)np_ * nrhs * 3 * sizeof(double2));
            VIE_CUDA(cudaMemcpyAsync(dd.p, d.data(), dd.bytes, cudaMemcpyHostToDevice, s));
            far_field_launch(o, dI.p, nrhs, dd.as<double>(), np_, out.p, s);
            std::vector<cd> N((size_t)np_ * nrhs * 3);
            VIE_CUDA(cudaMemcpyAsync(N.data(), out.p, out.bytes, cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            // F = -j k / (4 pi) (N - rhat (rhat . N))
            F.resize(N.size());
            for (int c = 0; c < nrhs; ++c)
                for (int p = 0; p < np_; ++p) {
                    const double* r = &d[3 * p];
                    cd* v = &N[((size_t)c * np_ + p) * 3];
                    cd dot = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
                    for (int e = 0; e < 3; ++e)
                        F[((size_t)c * np_ + p) * 3 + e] = cd(0, -o.k / (4 * M_PI)) * (v[e] - r[e] * dot);
                }
        };
        if (E_out && dirs && npts > 0) {
            std::vector<double> d(dirs, dirs + 3 * npts);
            std::vector<cd> F;
            far(d, F);
            std::memcpy(E_out, F.data(), F.size() * sizeof(cd));
        }
        if (sigma_out) {
            if (!inc) fail(VIE_ERR_INVALID_ARG, "cross sections need the incident field");
            // 24-point Gauss-Legendre in cos(theta) x 48-point trapezoid in phi
            const int nt = 24, nph = 48;
            std::vector<double> x(nt), w(nt);
            for (int i = 0; i < nt; ++i) {  // Newton on P_n
                double z = std::cos(M_PI * (i + 0.75) / (nt + 0.5));
                for (int it = 0; it < 100; ++it) {
                    double p1 = 1, p2 = 0;
                    for (int j = 1; j <= nt; ++j) {
                        double p3 = p2;
                        p2 = p1;
                        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
                    }
                    double pp = nt * (z * p1 - p2) / (z * z - 1.0);
                    double z1 = z;
                    z = z1 - p1 / pp;
                    if (std::fabs(z - z1) < 1e-15) {
                        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
                        break;
                    }
                    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
                }
                x[i] = z;
            }
            std::vector<double> d, wt;
            for (int i = 0; i < nt; ++i)
                for (int j = 0; j < nph; ++j) {
                    double st_ = std::sqrt(1 - x[i] * x[i]), ph = 2 * M_PI * j / nph;
                    d.push_back(st_ * std::cos(ph));
                    d.push_back(st_ * std::sin(ph));
                    d.push_back(x[i]);
                    wt.push_back(w[i] * 2 * M_PI / nph);
                }
            std::vector<cd> F;
            far(d, F);
            // extinction Re(I^H v0), v0 = b / (j k)
            DevBuf b((size_t)n * nrhs * sizeof(double2)), kh(3 * nrhs * sizeof(double)), pl(6 * nrhs * sizeof(double));
            VIE_CUDA(cudaMemcpyAsync(kh.p, inc->khat, kh.bytes, cudaMemcpyHostToDevice, s));
            VIE_CUDA(cudaMemcpyAsync(pl.p, inc->pol, pl.bytes, cudaMemcpyHostToDevice, s));
            rhs_kernel_launch(o, kh.as<double>(), pl.as<double>(), nrhs, b.p, n, s);
            std::vector<cd> hb((size_t)n * nrhs);
            VIE_CUDA(cudaMemcpyAsync(hb.data(), b.p, b.bytes, cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            const cd* hI = static_cast<const cd*>(I);
            for (int c = 0; c < nrhs; ++c) {
                cd acc = 0;
                for (int64_t i = 0; i < n; ++i) acc += std::conj(hI[i + c * n]) * hb[i + c * n] / cd(0, o.k);
                double sca = 0;
                for (size_t p = 0; p < wt.size(); ++p)
                    for (int e = 0; e < 3; ++e) sca += wt[p] * std::norm(F[((size_t)c * wt.size() + p) * 3 + e]);
                sigma_out[2 * c] = acc.real();
                sigma_out[2 * c + 1] = sca;
            }
        }
    });
}

int vie_export_block(vie_op* op, int kind, int a, int b, int precision, void* out) {
    if (!op || !out) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        cudaStream_t s = o.ctx->stream;
        const size_t np2 = (size_t)o.np * o.np;
        if (kind == 0 || kind == 2) {
            if (a < 0 || a >= o.T) fail(VIE_ERR_INVALID_ARG, "type out of range");
            const DevBuf& src = kind == 0 ? o.d_zself64 : o.d_inv64;
            VIE_CUDA(cudaMemcpyAsync(out, src.as<double2>() + a * np2, np2 * sizeof(double2), cudaMemcpyDeviceToHost, s));
        } else if (kind == 1) {
            if (a < 0 || b < 0 || a >= o.N || b >= o.N || a == b) fail(VIE_ERR_INVALID_ARG, "need two different atoms");
            size_t esz = precision == VIE_C128 ? sizeof(double2) : sizeof(float2);
            DevBuf blk(np2 * esz);
            PairJob jb{a, b, 0, 0, 0};
            std::vector<PairJob> jobs{jb};
            std::vector<void*> dst{blk.p};
            std::vector<int64_t> ld{o.np};
            DevBuf dj, dd, dl;
            upload(dj, jobs);
            upload(dd, dst);
            upload(dl, ld);
            if (precision == VIE_C128)
                assemble_pairs<double>(o, dj.as<PairJob>(), 1, dd.as<void* const>(), dl.as<int64_t>(), s);
            else  // the complex float32 block the c64 compression forms
                assemble_pairs_f32_from_f64(o, dj.as<PairJob>(), 1, dd.as<void* const>(), dl.as<int64_t>(), s);
            VIE_CUDA(cudaMemcpyAsync(out, blk.p, np2 * esz, cudaMemcpyDeviceToHost, s));
        } else {
            fail(VIE_ERR_INVALID_ARG, "unknown block kind");
        }
        VIE_CUDA(cudaStreamSynchronize(s));
    });
}

int vie_far_block_info(vie_op* op, int64_t i, int* level, int* n_tatoms, int* n_satoms, int* rank) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        const Op& o = op->o;
        if (i < 0 || i >= (int64_t)o.blocks.size()) fail(VIE_ERR_INVALID_ARG, "block index out of range");
        const FarBlock& b = o.blocks[i];
        if (level) *level = b.level;
        if (n_tatoms) *n_tatoms = b.nt;
        if (n_satoms) *n_satoms = b.ns;
        if (rank) *rank = b.rank;
    });
}

int vie_export_far_block(vie_op* op, int64_t i, int* tatoms, int* satoms, void* Q, void* R) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        if (i < 0 || i >= (int64_t)o.blocks.size()) fail(VIE_ERR_INVALID_ARG, "block index out of range");
        const FarBlock& b = o.blocks[i];
        if (tatoms) std::memcpy(tatoms, &o.block_atoms[b.t_off], b.nt * sizeof(int));
        if (satoms) std::memcpy(satoms, &o.block_atoms[b.s_off], b.ns * sizeof(int));
        if (!Q && !R) return;
        if (o.fprec == 0) fail(VIE_ERR_STATE, "operator is not compressed");
        const size_t cnt = (size_t)b.rank * (b.m + b.n);
        std::vector<cd> h(cnt);
        cudaStream_t s = o.ctx->stream;
        if (o.fprec == VIE_C128) {
            VIE_CUDA(cudaMemcpyAsync(h.data(), o.d_factors.as<double2>() + b.q_off, cnt * sizeof(double2),
                                     cudaMemcpyDeviceToHost, s));
        } else {
            std::vector<std::complex<float>> f(cnt);
            VIE_CUDA(cudaMemcpyAsync(f.data(), o.d_factors.as<float2>() + b.q_off, cnt * sizeof(float2),
                                     cudaMemcpyDeviceToHost, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            for (size_t e = 0; e < cnt; ++e) h[e] = cd(f[e].real(), f[e].imag());
        }
        VIE_CUDA(cudaStreamSynchronize(s));
        cd* q = static_cast<cd*>(Q);
        cd* r = static_cast<cd*>(R);
        const size_t mq = (size_t)b.rank * b.m;
        if (q) std::memcpy(q, h.data(), mq * sizeof(cd));
        if (r)  // stored R^H (n x r col-major) -> R (r x n col-major)
            for (int k = 0; k < b.rank; ++k)
                for (int c = 0; c < b.n; ++c) r[k + (size_t)c * b.rank] = std::conj(h[mq + c + (size_t)k * b.n]);
    });
}

int64_t vie_kernel_launches(void) { return g_kernel_launches.load(); }

int vie_tune(vie_op* op, int precision, int nrhs, int force_variant, vie_tune_result* result) {
    if (!op) return VIE_ERR_INVALID_ARG;
    return guarded(ctx_of(op), [&] {
        Op& o = op->o;
        set_device(*o.ctx);
        tune_entry(o, precision, nrhs, force_variant, result, o.ctx->stream);
    });
}

int vie_plan_far_blocks(const double* xy, int n_atoms, int* levels, int64_t* n_blocks, int* out, int64_t out_len,
                        int64_t* out_needed) {
    if (!xy || n_atoms < 1 || !levels || !n_blocks) return VIE_ERR_INVALID_ARG;
    try {
        Op o;
        o.N = n_atoms;
        o.np = 1;
        o.centres.resize(3 * (size_t)n_atoms);
        for (int a = 0; a < n_atoms; ++a) {
            o.centres[3 * a] = xy[2 * a];
            o.centres[3 * a + 1] = xy[2 * a + 1];
            o.centres[3 * a + 2] = 0.0;
        }
        build_tree(o);
        *levels = o.L;
        *n_blocks = (int64_t)o.blocks.size();
        int64_t need = 0;
        for (const auto& b : o.blocks) need += 3 + b.nt + b.ns;
        if (out_needed) *out_needed = need;
        if (out && out_len >= need) {
            int64_t k = 0;
            for (const auto& b : o.blocks) {
                out[k++] = b.level;
                out[k++] = b.nt;
                out[k++] = b.ns;
                for (int i = 0; i < b.nt; ++i) out[k++] = o.block_atoms[b.t_off + i];
                for (int i = 0; i < b.ns; ++i) out[k++] = o.block_atoms[b.s_off + i];
            }
        }
        return VIE_OK;
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        return VIE_ERR_INVALID_ARG;
    }
}

int vie_lpt_assign(const double* w, int64_t n, int n_proc, int* owner, double* loads) {
    if (!w || n < 0 || n_proc < 1 || !owner || !loads) return VIE_ERR_INVALID_ARG;
    try {
        std::vector<double> wv(w, w + n), ld;
        std::vector<int> ow;
        lpt_assign(wv, n_proc, ow, ld);
        std::copy(ow.begin(), ow.end(), owner);
        std::copy(ld.begin(), ld.end(), loads);
        return VIE_OK;
    } catch (...) {
        return VIE_ERR_INVALID_ARG;
    }
}

int64_t vie_footprint_bytes(int64_t n, int np, int nrhs, int restart, int64_t factor_entries) {
    // factors (c64) + self/inverse blocks (c128 + c64, two per type upper bound 3 types)
    // + Krylov basis (restart + 1) n c128 per rhs in flight + solver vectors
    int64_t m = restart > 0 ? restart : 60;
    int64_t bytes = 8 * factor_entries;
    bytes += 3 * (int64_t)np * np * (16 + 16 + 8 + 8);
    bytes += (m + 1) * n * 16;
    bytes += n * (int64_t)nrhs * (16 * 3 + 8 * 2) + n * 16 * 6;
    return bytes;
}

}  // extern "C"
