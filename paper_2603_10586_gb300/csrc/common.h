// Internal declarations of libvie (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>

#include <atomic>
#include <complex>
#include <map>
#include <cstdint>
#include <cstdio>
#include <string>
#include <type_traits>
#include <memory>
#include <vector>

#include "../../include/vie.h"

namespace vie {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// errors: every internal failure throws vie::Error, caught at the C-ABI
// ---------------------------------------------------------------------------
struct Error {
    int status;
    std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg);

#define VIE_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            ::vie::fail(e_ == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA,         \
                        std::string(#call " -> ") + cudaGetErrorString(e_) + " at " __FILE__); \
    } while (0)

#define VIE_BLAS(call)                                                                   \
    do {                                                                                 \
        cublasStatus_t s_ = (call);                                                      \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                                 \
            ::vie::fail(VIE_ERR_CUDA, std::string(#call " -> cublas status ") +          \
                                          std::to_string((int)s_) + " at " __FILE__);    \
    } while (0)

// every launch site of a libvie kernel calls VIE_CHECK_LAUNCH (or VIE_COUNT_LAUNCH)
extern std::atomic<long long> g_kernel_launches;
#define VIE_COUNT_LAUNCH(k) (::vie::g_kernel_launches.fetch_add((k), std::memory_order_relaxed))
#define VIE_CHECK_LAUNCH()          \
    do {                            \
        VIE_COUNT_LAUNCH(1);        \
        VIE_CUDA(cudaGetLastError()); \
    } while (0)

// ---------------------------------------------------------------------------
// device buffer (RAII)
// ---------------------------------------------------------------------------
struct Ctx;
// Device allocation; charged to the context whose C-ABI call is running on
// this thread (see AllocScope), which may cap its total (VIE_ERR_OOM before
// cudaMalloc is asked).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    Ctx* owner = nullptr;
    DevBuf() = default;
    explicit DevBuf(size_t b) { alloc(b); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), owner(o.owner) { o.p = nullptr; o.bytes = 0; o.owner = nullptr; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; owner = o.owner;
            o.p = nullptr; o.bytes = 0; o.owner = nullptr;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t b);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

template <class T>
void upload(DevBuf& d, const std::vector<T>& h) {
    d.alloc(std::max<size_t>(1, h.size() * sizeof(T)));
    if (!h.empty()) VIE_CUDA(cudaMemcpy(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// mesh of one atom type (voxels, faces, boundary faces), Sec. 3 basis
// ---------------------------------------------------------------------------
struct MeshTables {
    int nv = 0, np = 0, nvox = 0, nsurf = 0;
    double side = 0, h = 0;
    std::vector<int> face_dir, face_lo, face_hi, face_sheet, face_sheet_sign;  // [np]
    std::vector<int> vox_ijk;   // [3 nvox]
    std::vector<int> surf_face; // [nsurf]
};
MeshTables build_mesh(double side, int nv);

// device copy, packed: for face f: dir, lo voxel, hi voxel, sheet, sign
struct DevMesh {
    int nv, np, nvox, nsurf;
    const int4* face;     // (dir, lo, hi, sheet)
    const int* sheet_sign;
    const int* vox_ijk;   // [3 nvox]
    const int* surf_face; // [nsurf]
    const float4* vox_c;  // voxel centres in units of h from the cube corner
    const float4* surf_c; // boundary-face centres in units of h, w = normal axis
};

// ---------------------------------------------------------------------------
// far block of the compressed operator (Sec. 5.2)
// ---------------------------------------------------------------------------
struct FarBlock {
    int level = 0;
    int nt = 0, ns = 0;        // atoms in target / source box
    int t_off = 0, s_off = 0;  // offsets into Op::block_atoms
    int m = 0, n = 0;          // unknowns
    int rank = 0;
    int64_t q_off = 0;         // element offset of Q (m x r col-major)
    int64_t rh_off = 0;        // element offset of R^H (n x r col-major) = conj(R) row-major
    int64_t t_off_vec = 0;     // offset of this block's R x in the t buffer (per RHS column)
    int dist = 0;              // Chebyshev distance of the two boxes at this level
    int dmin = 0;              // the smaller of the two box-offset components
    int mirror = -1;           // index of the block (source box, target box)
    bool derived = false;      // factors taken from the mirror's (transposed)
};

struct Ctx;

struct Op {
    Ctx* ctx = nullptr;
    uint64_t gen = 0;  // bumped by every compression (joined operators built from older factors are stale)
    // geometry
    int N = 0, T = 0, np = 0, L = 0;
    std::vector<double> centres;       // [3N]
    std::vector<int> types;            // [N]
    std::vector<double> sides;         // [T]
    std::vector<int> nvs;              // [T]
    std::vector<cd> eps;               // [T]
    double wavelength = 1, k = 0;
    MeshTables mesh;                   // topology shared by all types (same nv)
    std::vector<double> h;             // [T] voxel size per type
    // tree
    std::vector<FarBlock> blocks;
    std::vector<int> block_atoms;
    // device geometry
    DevBuf d_centres, d_types, d_sides, d_inv_chi;
    DevBuf d_mesh_face, d_mesh_sign, d_mesh_vox, d_mesh_surf, d_mesh_voxc, d_mesh_surfc;
    DevMesh dmesh{};                   // pointers into the buffers above
    // self blocks (per type, np x np col-major)
    DevBuf d_zself64, d_inv64, d_zself32, d_inv32;
    DevBuf d_zselfH64, d_zselfH32, d_adj;  // conjugate-transposed self blocks, conj(x) scratch (adjoint apply)
    std::vector<std::vector<int>> atoms_of_type;
    DevBuf d_atoms_by_type;            // atom indices grouped by type
    std::vector<int> type_atom_off;    // [T+1]
    // factors
    int fprec = 0;
    double tol = 0;
    DevBuf d_factors;
    // a batched operator does not copy its problems' factors: its block offsets
    // are relative to this base address (the lowest of their buffers)
    const void* factors_view = nullptr;
    template <class T> const T* fac() const {
        return static_cast<const T*>(factors_view ? factors_view : d_factors.p);
    }
    int64_t factor_entries = 0;         // sum over far blocks of (m + n) r (what an apply multiplies)
    int64_t stored_entries = 0;         // of those, held in memory (translated copies share storage)
    int64_t t_total = 0;               // sum of ranks
    // apply work lists (device)
    DevBuf d_blocks;                   // FarBlockDev[nb]
    DevBuf d_block_atoms;
    DevBuf d_p1_items, d_p1_cta;       // phase 1 items and per-CTA ranges
    DevBuf d_p2_items, d_p2_cta, d_p2_csr, d_p2_ent;
    int n_p1_items = 0, n_p2_items = 0, n_cta = 0;
    DevBuf d_t1_items, d_t1_cta, d_t2_items, d_t2_cta;  // warp-MMA tensor path (64-row items)
    int n_t1_items = 0, n_t2_items = 0, n_cta_tc = 0;
    // shared-factor path: blocks with the same factor storage (translated
    // copies) form a class; members of a class are listed together in
    // d_cmem and each item covers up to kShareGroup of them.  Phase 2 writes one
    // partial product per (block, target slot) at d_poff[block] + slot np.
    DevBuf d_cmem, d_c1_items, d_c1_cta, d_c2_items, d_c2_cta, d_poff, d_part;
    static constexpr int kShareGroup = 4;  // members per item (register tile of the kernels)
    int n_c1_items = 0, n_c2_items = 0, n_cta_c = 0;
    int64_t part_total = 0;             // complex entries of the partial products
    double share_mean = 1.0;            // far blocks per factor class (rank > 0)
    // tcgen05 tensor path (built on first use): phase 1 stacks the R rows of
    // all blocks with the same source atoms (one gathered x for up to 128
    // rows), phase 2 walks one virtual K axis over all blocks of an atom
    bool umma_ready = false;
    DevBuf d_u1_rowoff, d_u1_rowt, d_u1_items, d_u1_cta;
    DevBuf d_u2_qoff, d_u2_tidx, d_u2_kptr, d_u2_items, d_u2_cta;
    // packed variant: each item's A operand pre-split into bf16 planes in the
    // shared-memory stage layout (32 KiB per 32-wide K stage), copied by bulk TMA
    DevBuf d_u1_pk, d_u2_pk, d_u1_pack, d_u2_pack;  // stage offsets per item, planes
    // the SIMT lists mapped to two CTAs per SM (the multi-RHS SIMT kernels)
    int n_cta_m = 0;
    DevBuf d_p1m_items, d_p1m_cta, d_p2m_items, d_p2m_cta;
    DevBuf d_w1_items, d_w1_cta, d_w1_pk, d_w2_items, d_w2_cta, d_w2_pk;  // one CTA per SM (warp-specialised)
    // pairs of items that share their B operand (two M tiles per B tile), one CTA per SM: first and
    // second item (rows 0 when absent) and their packed stage offsets
    DevBuf d_x1_items, d_x1_items_b, d_x1_cta, d_x1_pk, d_x1_pk_b;
    DevBuf d_x2_items, d_x2_items_b, d_x2_cta, d_x2_pk, d_x2_pk_b;
    long long u1_stages = 0, u2_stages = 0;
    bool umma_packed = false, umma_pack_failed = false;
    int n_u1_items = 0, n_u2_items = 0, n_cta_u = 0;
    DevBuf d_err;  // set by a tensor-core kernel whose bounded wait gave up
    // batched operators (several problems as one block-diagonal operator,
    // batch.cpp): problem of every block, atom and type, and during a solve
    // the device table of each problem's right-hand-side columns [x, y)
    int nprob = 1;
    std::vector<int> block_prob, atom_prob, type_prob;
    const int2* colr = nullptr;
    // far-apply variant per (precision, log2 of the right-hand-side count),
    // chosen by the autotuner or set by the caller
    std::map<std::pair<int, int>, int> variant;
    // scratch
    DevBuf d_t, d_F;
    DevBuf d_xs;  // float64 vectors split into float32 head + tail (double-float apply)
    size_t t_cap = 0, F_cap = 0;
    double t_assemble = 0, t_compress = 0;
    // compression method of the stored factors (0: range finder, 1: cross
    // approximation) and, for the cross approximation, the bytes its residual
    // passes moved and the time of its step loops
    int cmethod = 0;
    double cross_bytes = 0, t_cross = 0;
    int64_t n() const { return (int64_t)N * np; }
};

struct Ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    cublasHandle_t blas = nullptr;
    std::string err;
    size_t budget = 0;
    int verbose = 0;
    int no_sharing = 0;
    void* owner = nullptr;  // the C-ABI handle holding this context
    // device bytes held by this context's buffers, the largest seen, and the cap
    // (0: none) above which an allocation is refused with VIE_ERR_OOM
    std::atomic<int64_t> allocated{0}, peak{0};
    std::atomic<int64_t> cap{0};
    // joined operators of recent vie_solve_batch calls (block-diagonal unions of
    // their problems), reused while the same operators with the same factors
    // come again; declared last so that they are freed first
    struct Union {
        std::vector<const Op*> ops;
        std::vector<uint64_t> gens;
        std::unique_ptr<Op> U;
        uint64_t used = 0;
    };
    std::vector<Union> unions;
    uint64_t union_clock = 0;
};

// The context charged for device allocations made by this thread while a
// C-ABI call of that context runs (set by the call's entry, restored on exit).
struct AllocScope {
    Ctx* prev;
    explicit AllocScope(Ctx* c);
    ~AllocScope();
};

// device-side block description used by the apply kernels
struct FarBlockDev {
    int m, n, rank, nt, ns, t_off, s_off, prob;  // prob: problem of a batched (union) operator
    long long q_off, rh_off, tvec_off;
};

// ---------------------------------------------------------------------------
// host algorithms
// ---------------------------------------------------------------------------
void build_tree(Op& op);   // fills op.L, op.blocks, op.block_atoms
void lpt_assign(const std::vector<double>& w, int nproc, std::vector<int>& owner,
                std::vector<double>& loads);
void build_apply_lists(Op& op);

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// assemble.cu
void assemble_self_blocks(Op& op);  // fills d_zself64 (float64)
// Interaction blocks between atom pairs, written into col-major destination
// matrices: pair p writes Zs_{a_p, b_p} at dst[p] + row_off + col_off * ld.
struct PairJob {
    int a, b;
    int dst;          // index into the destination pointer table
    int row_off, col_off;
};
// norm_out (optional, device): per job, the squared Frobenius norm of its block
template <class T>
void assemble_pairs(Op& op, const PairJob* d_jobs, int n_jobs, void* const* d_dst, const int64_t* d_ld,
                    cudaStream_t s, double* norm_out = nullptr);
// complex float32 entries from float64 tables.  The charge terms are second
// differences of voxel-pair potentials, and in float32 the rounding of each
// voxel pair's distance and phase survives the differencing: far blocks then
// carry noise near 1e-4 of their norm, which the compression must keep (ranks
// grow many times).  From float64 tables the entries are exact to their float32
// rounding.  The c64 compression forms its blocks this way.
void assemble_pairs_f32_from_f64(Op& op, const PairJob* d_jobs, int n_jobs, void* const* d_dst, const int64_t* d_ld,
                                 cudaStream_t s, double* norm_out = nullptr);
void dense_apply_c64(Op& op, const float2* x, float2* y, cudaStream_t s);
void dense_apply_c128(Op& op, const double2* x, double2* y, cudaStream_t s);
void rhs_kernel_launch(Op& op, const double* d_khat, const double* d_pol, int nrhs, void* b, int64_t ld,
                       cudaStream_t s);
void near_field_launch(Op& op, const void* d_I, int nrhs, const double* d_pts, int npts, void* d_out, cudaStream_t s);
void far_field_launch(Op& op, const void* d_I, int nrhs, const double* d_dirs, int npts, void* d_out,
                      cudaStream_t s);
void v0_dot_launch(Op& op, const void* d_I, const double* d_khat, const double* d_pol, int nrhs,
                   double* d_out, cudaStream_t s);

// linalg.cu
void invert_self_blocks(Op& op);   // d_inv64 from d_zself64 (Gauss-Jordan, partial pivoting)
void convert_c128_to_c64(const void* src, void* dst, int64_t n, cudaStream_t s);
void convert_c64_to_c128(const void* src, void* dst, int64_t n, cudaStream_t s);
// dst = conj(src) (n complex values; c128 selects double2, else float2)
void conj_copy(const void* src, void* dst, int64_t n, bool c128, cudaStream_t s);
// dst[t] = src[t]^H for T np x np column-major blocks
void conj_transpose_blocks(const void* src, void* dst, int T, int np, bool c128, cudaStream_t s);
template <class TM, class TX>
void self_gemm(Op& op, const TM* M, const TX* X, int64_t ldx, const TX* C, int64_t ldc, TX* Y, int64_t ldy,
               int nrhs, int mode, cudaStream_t s);

// apply.cu
template <class TF, class TX>
void apply_far(Op& op, const TX* x, int64_t ldx, TX* F, int64_t ldf, int nrhs, cudaStream_t s);

void apply_static(Op& op, const float2* x, float2* y, int nrhs, cudaStream_t s);
// complex float32 SIMT far apply with nr (1, 2, 4, 8) right-hand sides per factor read
void apply_far_simt32(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, int nr,
                      cudaStream_t s);
// far apply of float32 vectors by the variant chosen for (precision, nrhs)
void far32(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, int precision, cudaStream_t s);
int far_variant(const Op& op, int precision, int nrhs);
// time the admissible variants for (precision, nrhs), keep the fastest
int tune_far(Op& op, int precision, int nrhs, cudaStream_t s, std::vector<int>& cand, std::vector<double>& ms);
int tune_entry(Op& op, int precision, int nrhs, int force, vie_tune_result* res, cudaStream_t s);
bool tuned(const Op& op, int precision, int nrhs);
// work lists of the tcgen05 multi-RHS apply (host.cpp); idempotent
void build_umma_lists(Op& op);
// far part with c64 factors and c64 vectors, split-precision bf16 on tcgen05
void apply_far_umma(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);
// everything the tcgen05 apply allocates or configures, done ahead of graph capture
void umma_prepare(Op& op, cudaStream_t s);
// packed tcgen05 variant: split the factors once into bf16 planes in the stage
// layout (false when the free memory cannot hold them); the apply runs the
// unpacked kernel when packing is not possible
bool umma_pack(Op& op, cudaStream_t s);
size_t umma_pack_bytes(const Op& op);
void apply_far_umma_packed(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);
void apply_far_umma_ws(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);
void apply_far_umma_ws2(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);
// complex float32 far apply reading each shared factor once per group of up to
// Op::kShareGroup translated copies (one right-hand side at a time)
void apply_far_shared(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);
void shared_reserve(Op& op);
// far part with c64 factors and c128 vectors in double-float arithmetic
void apply_far_df(Op& op, const double2* x, int64_t ldx, double2* F, int64_t ldf, int nrhs, cudaStream_t s);
// apply_tc.cu: several right-hand sides on the tensor cores (BF16x3)
void apply_far_bf16x3(Op& op, const float2* x, int64_t ldx, float2* F, int64_t ldf, int nrhs, cudaStream_t s);

// compress.cu; method 0: adaptive randomised range finder, 1: cross
// approximation with full pivoting (cross.cu)
void compress_operator(Op& op, double tol, int prec, int method = 0);

// cross.cu: cross approximation with full pivoting of nb formed m x n blocks
// (column-major, E + q m n; overwritten by their residuals) to
// ||A - U V^T||_F <= tol ||A||_F with d_anorm2[q] = ||A_q||_F^2, at most rcap
// crosses (rcap <= rfull = min(m, n)).  Column k of block q goes to
// U + q us + k m (u_k) and VH + q vs + k n (conj(v_k)); rank[q] receives the
// block's rank.  flags: 1 a block needed more than rcap (< rfull) crosses,
// 2 a residual was not finite.
struct CrossStats {
    int flags = 0;
    double seconds = 0;    // step loop, device time between events
    double bytes = 0;      // residual bytes read and written
    int64_t passes = 0;    // residual passes (blocks x steps)
    std::vector<double> resid2;  // per block: ||E||_F^2 when it left the loop
};
template <class T2>
CrossStats cross_full_batch(T2* E, int nb, int m, int n, const double* d_anorm2, double tol, int rcap, int rfull,
                            T2* U, int64_t us, T2* VH, int64_t vs, std::vector<int>& rank, int n_sm,
                            cudaStream_t s);

// solve.cpp
// forget the joined operators that contain `o` (before it is destroyed or recompressed)
void drop_unions(Ctx& c, const Op* o);
int solve_batch(const std::vector<Op*>& ops, const vie_incident* incs, const int* nrhs, const vie_solve_opts* o,
                void** I_out, vie_solve_stats* st);
int solve(Op& op, const vie_incident* inc, int nrhs, const vie_solve_opts* o, void* I_out,
          vie_solve_stats* st);

double now_s();

}  // namespace vie
