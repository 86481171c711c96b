/*
 * libvie: QR-recursive compressed volume-integral-equation solver for arrays of
 * dielectric meta-atoms, on one NVIDIA GB300 (sm_103a).
 *
 * The problem (paper Sec. 2, eq. IntEq): the polarisation current J in the
 * dielectric region satisfies
 *     J / (j w eps0 chi) + j w mu0 int J g + (1/(j w eps0)) grad int (div J) g = E0,
 * g = exp(-j k R) / (4 pi R), e^{j w t} time convention, sigma = 0.
 * Galerkin discretisation (Sec. 3, eq. matrixeq / eq_vie) gives Z I = v0.  The
 * meta-atoms are axis-aligned cubes split into nv^3 voxels carrying one
 * div-conforming rooftop per voxel face (boundary faces included), so an atom
 * has Np = 3 (nv+1) nv^2 unknowns; unknowns are ordered atom by atom (Sec. 4,
 * eq. bp) and, inside an atom, x-faces, y-faces, z-faces, each lexicographic in
 * (i, j, k) with the normal index running 0..nv.
 *
 * The library works with the scaled system Zs I = b, Zs = j w eps0 Z,
 * b = j w eps0 v0, in units eps0 = mu0 = c = 1 (so w = k = 2 pi / lambda).  The
 * solution vector I is the same as for Z I = v0.
 *
 * Conventions for every function below:
 *  - Return value: VIE_OK (0) or a negative vie_status.  Nothing is thrown
 *    across this interface.  vie_last_error(ctx) gives a one-line message.
 *  - Complex numbers are interleaved (re, im) pairs: "c64" = 2 x float,
 *    "c128" = 2 x double.  Matrices of vectors are column-major n x nrhs with
 *    a leading dimension ld >= n (in elements).
 *  - Device pointers are owned by the caller and must stay valid until the
 *    call's work on `stream` has finished; host pointers are read or written
 *    before the call returns.  Objects (vie_ctx, vie_op, vie_server) own
 *    their internal device memory until the matching *_destroy.
 *  - Calls on one vie_ctx (and on the operators made from it) are not
 *    thread-safe; a vie_server is safe for concurrent submit/poll.
 *  - Every wait inside the library is bounded (VIE_ERR_TIMEOUT).
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vie_ctx vie_ctx;
typedef struct vie_op vie_op;
typedef struct vie_server vie_server;
typedef void* vie_stream; /* a cudaStream_t; NULL = the context's own stream */

enum vie_status {
    VIE_OK = 0,
    VIE_ERR_INVALID_ARG = -1,
    VIE_ERR_OOM = -2,
    VIE_ERR_CUDA = -3,
    VIE_ERR_NOT_CONVERGED = -4, /* result and stats are still written */
    VIE_ERR_BREAKDOWN = -5,
    VIE_ERR_NAN = -6,
    VIE_ERR_TIMEOUT = -7,
    VIE_ERR_ADMISSION = -8,
    VIE_ERR_STATE = -9
};

/* Precision of stored factors and of an apply. */
enum vie_precision {
    VIE_C64 = 1,    /* complex float32 storage and arithmetic */
    VIE_C128 = 2,   /* complex float64 storage and arithmetic */
    VIE_BF16X3 = 3, /* c64 operands split into bf16 hi/lo, three tensor-core
                       products (hi.hi + hi.lo + lo.hi), float32 accumulation */
    VIE_C64_ACC64 = 4 /* c64 factors, float64 vectors and accumulation (the
                         refinement residual) */
};

/* Implementations of the far part of a complex float32 apply (the paper's
 * method fixes what is computed, not how; these are the kernel variants the
 * autotuner chooses between).  The SIMT variants read every factor element
 * once per group of 1, 2, 4 or 8 right-hand sides; the tensor-core variants
 * compute in split bf16 (admissible for VIE_BF16X3 only). */
enum vie_variant {
    VIE_VAR_AUTO = 0,
    VIE_VAR_SIMT_R1 = 1,
    VIE_VAR_SIMT_R2 = 2,
    VIE_VAR_SIMT_R4 = 3,
    VIE_VAR_SIMT_R8 = 4,
    VIE_VAR_MMA_BF16X3 = 5,     /* warp-level mma.sync, 64-row tiles */
    VIE_VAR_TCGEN05_BF16X3 = 6, /* tcgen05 MMAs with tensor-memory accumulators, 128-row tiles */
    VIE_VAR_TCGEN05_PACKED_BF16X3 = 7, /* as 6, with the factors split once into bf16 planes in the
                                          shared-memory stage layout and moved by bulk TMA copies (needs
                                          ~1.1x the factor memory; runs as 6 when that is not free) */
    VIE_VAR_SIMT_SHARED = 8 /* complex float32, one right-hand side at a time: far blocks that share
                               their factors (translated copies) are applied together, each factor
                               element read once per group of up to 4 copies; partial products are
                               summed per target atom in a fixed order (default for one right-hand
                               side when the operator has translated copies) */,
    VIE_VAR_TCGEN05_WS_BF16X3 = 9 /* the planes of 7 in a warp-specialised persistent kernel (one CTA
                                     per SM): a warp moves the A planes by bulk TMA into a ring of 3 to
                                     5 stages (5 up to 16 right-hand sides, 4 up to 48), up to four warp
                                     pairs gather and split B into two stacked plane sets, one thread
                                     issues four wide MMAs per K step (each A plane read once), four
                                     warps drain two tensor-memory accumulator buffers; equal to 7 to
                                     float32 rounding (default for 8 to 16 right-hand sides; runs as 6
                                     when the planes do not fit) */,
    VIE_VAR_TCGEN05_WS2_BF16X3 = 10 /* 9 with two 128-row tiles of factor rows sharing each B tile (the
                                       two row tiles of a target atom, or two consecutive row tiles of
                                       a source group), 16 K values per stage: the B operand is gathered
                                       and split once for twice the rows; equal to 9 to float32
                                       rounding (default for more than 16 right-hand sides; runs as 6
                                       when the planes do not fit) */
};

/* vie_apply flags */
#define VIE_APPLY_FUSE_PRECOND 1 /* y = x + Z_D^-1 (far part of Zs x) = P^-1 Zs x */
#define VIE_APPLY_DENSE 2        /* y = Zs x with the uncompressed operator: every
                                    block regenerated on the device and never stored
                                    (accuracy reference; 1 RHS; C64 or C128) */
#define VIE_APPLY_ADJOINT 4      /* y = Zs^H x with the compressed operator (the Z^H I
                                    products of Sec. 4); alone, not with the other flags */

typedef struct vie_ctx_opts {
    int device;            /* CUDA device ordinal */
    size_t hbm_budget;     /* bytes the context may allocate: an allocation beyond it fails with
                              VIE_ERR_OOM before cudaMalloc is asked (0 = no cap; free memory - 4 GiB
                              sizes the compression batches) */
    int verbose;           /* 0 quiet, 1 stage timings on stderr */
    int no_sharing;        /* 0 (default): far blocks that are translated copies of one another
                              (same level, same atom types, same relative atom positions, as in a
                              periodic array of identical meta-atoms) are formed and compressed once
                              and share their factors; 1: every far block is compressed */
} vie_ctx_opts;

/* Metasurface geometry (host memory, copied by vie_assemble).
 * Paper Sec. 2: region Omega (the atoms), susceptibility chi = eps_r - 1 per
 * homogeneous component, angular frequency from `wavelength`. */
typedef struct vie_geometry {
    int n_atoms;               /* N >= 1 */
    const double* centres;     /* [3 N] atom centres (x, y, z); units of length */
    const int* types;          /* [N] type index in [0, n_types) */
    int n_types;               /* T >= 1 */
    const double* sides;       /* [T] cube side */
    const int* nv;             /* [T] voxels per edge, 1..16; all types must give
                                  the same Np (VIE_ERR_INVALID_ARG otherwise) */
    const double* eps;         /* [2 T] relative permittivity (re, im); lossy media
                                  have im < 0 under e^{j w t}; eps != 1 */
} vie_geometry;

typedef struct vie_op_info {
    int n_atoms, np, n_types, levels;
    int64_t n;                 /* unknowns = N Np */
    int64_t n_far_blocks;
    int64_t far_entries;       /* sum over far blocks of m n */
    int64_t factor_entries;    /* sum over far blocks of (m + n) r */
    int64_t self_entries;      /* N Np^2 (eq. eqn_cgain's near part) */
    double gain;               /* G = n^2 / N_QR (eq. eqn_cgain) */
    int rank_min, rank_max;
    double rank_mean;
    int factor_precision;      /* vie_precision of stored factors, 0 before compression */
    double tol;                /* compression tolerance */
    int64_t apply_bytes;       /* algorithmic bytes of one single-RHS c64 apply */
    double t_assemble_s, t_compress_s;
    int64_t stored_entries;    /* factor entries held in memory: translated copies of a far block
                                  share one set of factors (see vie_ctx_opts.no_sharing) */
    int64_t packed_bytes;      /* bytes of the bf16 planes the packed tensor-core apply streams per
                                  application (every far block's own planes, tiles padded to 128 rows
                                  and K to 32); 0 until a VIE_BF16X3 apply has built them */
    int compress_method;       /* vie_compress_method of the stored factors */
    double cross_bytes;        /* cross approximation: residual bytes its passes read and wrote */
    double t_cross_s;          /* cross approximation: device time of its step loops */
} vie_op_info;

/* How vie_compress / vie_compress_cross built the far-block factors. */
enum vie_compress_method {
    VIE_COMPRESS_RANGE_FINDER = 0, /* adaptive randomised range finder, Q orthonormal */
    VIE_COMPRESS_CROSS = 1         /* cross approximation with full pivoting (Sec. 6.5) */
};

/* Plane-wave incident fields E0 = p exp(-j k khat . r), one per right-hand side. */
typedef struct vie_incident {
    const double* khat;        /* [3 nrhs] unit propagation directions */
    const double* pol;         /* [6 nrhs] complex polarisation (re x, im x, re y, im y, re z, im z) */
} vie_incident;

typedef struct vie_solve_opts {
    double tol;                /* relative residual ||P^-1 (b - Zs I)|| / ||P^-1 b|| (1e-6) */
    int restart;               /* GMRES restart length m (e.g. 60); larger than 512 is taken as 512 */
    int max_iters;             /* iteration cap (e.g. 2000) */
    int precision;             /* VIE_C64: FP32 inner applies with FP64-accurate Krylov and FP64
                                  residual refinement (a cycle that ends while every residual is above
                                  100 x tol restarts from a residual in the inner precision; only a
                                  float64-accurate residual ends a solve); VIE_BF16X3: as VIE_C64 but the far part of
                                  the inner applies on the tensor cores (split bf16, FP32 accumulation);
                                  VIE_C128: all-FP64 (needs C128 factors) */
    int out_on_device;         /* 1: I_out is a device pointer, 0: host pointer */
    int precond;               /* 1: block-diagonal preconditioner (default), 0: none */
    int launch;                /* 0: each restart cycle is one CUDA graph (Arnoldi steps in a
                                  conditional while-node, no host round trip inside a cycle);
                                  1: the host launches every step and reads the continue flag */
    int autotune;              /* 1: run vie_tune for the first cycle's right-hand-side count
                                  (unless already tuned) before the solve */
    int method;                /* 0: restarted GMRES (Sec. 6, the paper's choice), each right-hand side
                                  in its own Krylov space, all advanced in lockstep; 1: BiCGStab, the
                                  method Sec. 6 compares it with (same preconditioner, precisions and
                                  stopping test; two applies per iteration; restart and launch are
                                  not used); 2: block GMRES, one Krylov space shared by all right-hand
                                  sides (float64 block Gram-Schmidt; restart counts block steps and is
                                  capped so that (restart + 1) nrhs <= 512; launch is not used).
                                  Methods 1 and 2: vie_solve only */
} vie_solve_opts;

/* Result of vie_tune. */
typedef struct vie_tune_result {
    int variant;               /* the variant now used for (precision, nrhs) */
    int n_candidates;
    int candidates[16];        /* vie_variant values that were timed */
    double ms[16];             /* best of three timed far applies per candidate */
} vie_tune_result;

typedef struct vie_solve_stats {
    int iterations;            /* Arnoldi steps of the slowest right-hand side */
    int applies;               /* operator applications (each on all right-hand sides still iterating) */
    int refinements;           /* FP64 residual recomputations */
    double residual;           /* final true preconditioned relative residual (max over RHS) */
    double true_residual;      /* ||b - Zs I|| / ||b|| with the compressed operator (max over RHS) */
    double t_solve_s;
    double history[512];       /* estimated residual after each iteration (first 512) */
    int n_history;
} vie_solve_stats;

/* ---- context ---------------------------------------------------------------- */
int vie_create(vie_ctx** out, const vie_ctx_opts* opts);
/* Releases the context; if operators made from it still exist it is freed
 * when the last of them is destroyed. */
void vie_destroy(vie_ctx* ctx);
const char* vie_last_error(vie_ctx* ctx);

/* ---- operator --------------------------------------------------------------
 * vie_assemble (paper Sec. 3 entries, Sec. 4 self blocks, Sec. 5 grid):
 * builds the quadtree and far-block lists (Sec. 5.1 Definition, eq. eq_rec01,
 * Sec. 5.4), assembles the distinct self blocks Z_ii in float64, factors them
 * (LU, Sec. 4 eq. diagprecond) and keeps the explicit inverses.  Far blocks
 * are not formed here.  wavelength > 0 in the units of the geometry. */
int vie_assemble(vie_ctx* ctx, const vie_geometry* g, double wavelength, vie_op** out);

/* vie_compress (Sec. 5.2 eq. eq_02, Sec. 5.3): forms every far block on the
 * device, in batches (VIE_C64: float64 quadrature tables, entries rounded to
 * complex float32), and replaces it by Q (m x r, orthonormal columns) and
 * R (r x n) with ||A - Q R||_F <= tol ||A||_F (randomised adaptive range
 * finder; the bound is enforced with a safety factor on a stochastic
 * estimate).  factor_precision: VIE_C64 or VIE_C128.  May be called again
 * with another tolerance or precision; the old factors are freed. */
int vie_compress(vie_op* op, double tol, int factor_precision);

/* vie_compress_cross (Sec. 6.5: local assembly of each far block, then its
 * "full-cross" approximation): forms every far block on the device, in
 * batches, and compresses it by cross approximation with full pivoting.  Step k
 * takes the entry of largest modulus of the residual E_k (ties: smallest
 * column, then smallest row) and subtracts the cross through it,
 * E_{k+1} = E_k - E_k[:, j] E_k[i, :] / E_k[i, j]; a block stops at the first
 * k with ||E_k||_F <= tol ||A||_F, a bound that holds on the formed block up to
 * the float rounding of the residual (no stochastic estimate).  The factors are
 * stored as Q = U (m x r, not orthonormal) and R = V^T (r x n) in the layout
 * vie_compress writes, so every apply, solve and export works unchanged.
 * Arguments, errors and reuse as for vie_compress; VIE_ERR_NAN if a formed
 * block has non-finite entries.  The residual passes cost r m n entries read
 * and written per block (vie_op_info.cross_bytes / t_cross_s). */
int vie_compress_cross(vie_op* op, double tol, int factor_precision);

void vie_op_destroy(vie_op* op);
int vie_op_get_info(const vie_op* op, vie_op_info* info);

/* vie_apply (Sec. 5.2: y = Z_D x + sum_far Q (R x)):
 * x, y: device pointers, n x nrhs, leading dimension ld (elements).
 * precision VIE_C64 (x, y c64), VIE_C128 (c128, needs C128 factors),
 * VIE_C64_ACC64 (x, y c128, c64 factors), VIE_BF16X3 (x, y c64, c64 factors;
 * the far part on the tensor cores, relative error ~1e-5).
 * flags: VIE_APPLY_FUSE_PRECOND returns P^-1 Zs x instead of Zs x;
 * VIE_APPLY_DENSE applies the uncompressed matrix (works before vie_compress;
 * at VIE_C64 its interaction blocks are the ones vie_compress forms).
 * x and y must be 16-byte aligned (cudaMalloc'd buffers are) and must not
 * overlap; either violation fails with VIE_ERR_INVALID_ARG before anything is
 * launched.  Asynchronous on `stream`. */
int vie_apply(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, int precision,
              int flags, vie_stream stream);

/* vie_apply_noalloc: y = Zs x, the same product as vie_apply(op, x, y, nrhs, ld,
 * VIE_C64, 0, stream) to float32 rounding (the summation order differs), but
 * without allocating any device memory.  It always runs the per-column SIMT
 * kernels, so for nrhs > 1 every factor is read once per column (up to nrhs
 * times the traffic of vie_apply, which reads a factor once for all columns).
 * The paper
 * has no counterpart: it is an interface for callers that cannot call
 * cudaMalloc between set-up and use, for instance code whose device memory is
 * all handed to its own pool allocator (a new cudaMalloc could fail or
 * fragment that pool), or loops in which the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  vie_apply may
 * allocate its scratch on first use; this entry point never does.
 *  - Scratch: a file-scope device array of VIE_NOALLOC_SCRATCH_ELEMS
 *    complex float32 elements (32 MiB), held by every GPU that loads the
 *    library until the process exits.  A call needs (sum of the far-block
 *    ranks) x nrhs elements; larger requests fail with VIE_ERR_INVALID_ARG
 *    before anything is launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: do not call this entry point again after cudaDeviceReset on
 *    that device (the reset destroys the context the address belongs to).
 *  - Every call on a device shares the one array and overwrites it; nothing
 *    in it has to start at zero.  Calls that overlap on the GPU (different
 *    streams, or different operators on one device) race on the array: order
 *    them on one stream or synchronise between them.
 *  - x, y: device pointers, c64, n x nrhs, ld = n, 16-byte aligned and not
 *    overlapping (VIE_ERR_INVALID_ARG otherwise); the
 *    operator must hold VIE_C64 factors.  Asynchronous on `stream` (NULL =
 *    the context's stream). */
#define VIE_NOALLOC_SCRATCH_ELEMS (1LL << 22)
int vie_apply_noalloc(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, vie_stream stream);

/* vie_precond (Sec. 4, eq. diagprecond): y = Z_D^-1 x atom by atom, with the
 * inverse of the atom's type.  Same pointer conventions as vie_apply;
 * precision VIE_C64 or VIE_C128. */
int vie_precond(vie_op* op, const void* x, void* y, int nrhs, int64_t ld, int precision,
                vie_stream stream);

/* vie_rhs: b = j k v0, v0_i = int w_i . E0 (eq. matrixeq), Gauss-Legendre 3 points
 * per voxel axis; b is a device pointer (16-byte aligned), c128, n x nrhs,
 * leading dimension ld. */
int vie_rhs(vie_op* op, const vie_incident* inc, int nrhs, void* b, int64_t ld, vie_stream stream);

/* vie_solve (Sec. 6: left-preconditioned GMRES, Sec. 4 preconditioner):
 * solves Zs I = b for the plane waves in `inc`; writes I (c128, n x nrhs,
 * column-major, ld = n) to I_out (host or device per opts->out_on_device; a
 * device I_out must be 16-byte aligned).
 * The right-hand sides iterate in lockstep: every Arnoldi step applies the
 * operator once to all of them still iterating (each keeps its own Krylov
 * space); the solve returns when all have converged or max_iters is hit.
 * Returns VIE_ERR_NOT_CONVERGED (I and stats still written) if max_iters is hit. */
int vie_solve(vie_op* op, const vie_incident* inc, int nrhs, const vie_solve_opts* opts,
              void* I_out, vie_solve_stats* stats);

/* vie_solve_batch (no paper counterpart; a batching of vie_solve): solves
 * `count` problems together, e.g. arrays of different size, wavelength or
 * permittivity made of meta-atoms with the same voxels per edge, all
 * compressed with VIE_C64 factors on one context.  The operators are joined
 * into one block-diagonal operator (no block couples two problems), so each
 * problem's result is what vie_solve would give it; what changes is that
 * every phase of the far apply is one persistent launch over all problems'
 * work and every Arnoldi step serves all of them.
 * inc[p], nrhs[p]: right-hand sides of problem p (sum at most 1024);
 * I_out[p]: its c128 n_p x nrhs[p] solution (host or device per
 * opts->out_on_device); stats[p] (may be NULL): its statistics (applies,
 * refinements and history are those of the shared lockstep).
 * opts->precision VIE_C64 or VIE_BF16X3.  The joined operator reads every
 * problem's factors in place (no copy); it holds the self blocks and the work
 * lists for the duration of the call. */
int vie_solve_batch(vie_op* const* ops, int count, const vie_incident* inc, const int* nrhs,
                    const vie_solve_opts* opts, void* const* I_out, vie_solve_stats* stats);

/* vie_fields: outputs from a solution I (host c128, n x nrhs, ld = n):
 * mode 0: far-field amplitude F(rhat) = -j k/(4 pi) (I - rhat rhat) int J exp(j k rhat.r) dV
 *         for the unit directions dirs[3 npts]; E_out host c128 [3 npts nrhs].
 * mode 1: scattered near field E_sca(r) = -j k int J g dV' + (1/(j k)) grad int q g dV' (Sec. 2,
 *         eq. IntEq: the field of the polarisation current J and its charge q = div J, boundary
 *         sheets included) at the points dirs[3 npts] (same units as the geometry), which must lie
 *         outside the atoms (the 3-point Gauss rule per voxel axis is accurate from about a voxel
 *         away); E_out host c128 [3 npts nrhs] in units of the incident amplitude.  sigma_out
 *         must be NULL in this mode.
 * sigma_out (host, may be NULL) [2 nrhs]: extinction Re(I^H v0) and scattering
 * cross section (closed surface integral of |F|^2, 24 x 48 rule) for |E0| = 1. */
int vie_fields(vie_op* op, const vie_incident* inc, const void* I, int nrhs, const double* dirs,
               int npts, int mode, void* E_out, double* sigma_out);

/* ---- debugging / verification ------------------------------------------------
 * vie_export_block: copies one operator block to host memory.
 * kind 0: self block of type `a` (c128 Np x Np, col-major);
 * kind 1: dense interaction block Zs_ab between atoms a != b, assembled on the
 *         device at `precision` (VIE_C64 -> c64, VIE_C128 -> c128), col-major;
 *         the c64 block is the one vie_compress forms: float64 quadrature
 *         tables, entries rounded to complex float32;
 * kind 2: explicit inverse of the self block of type `a` (c128).  */
int vie_export_block(vie_op* op, int kind, int a, int b, int precision, void* out);

/* vie_far_block_info: block `i` of the compressed operator: level, number of
 * target / source atoms, rank.  vie_export_far_block copies its atom lists
 * (int) and factors Q (m x r col-major) and R (r x n col-major) as c128. */
int vie_far_block_info(vie_op* op, int64_t i, int* level, int* n_tatoms, int* n_satoms, int* rank);
int vie_export_far_block(vie_op* op, int64_t i, int* tatoms, int* satoms, void* Q, void* R);

/* ---- host-only planning (no GPU needed) --------------------------------------
 * vie_plan_far_blocks: the grid hierarchy and far-block list that vie_assemble
 * builds (Sec. 5.1 Definition, eq. eq_rec01, Sec. 5.4), for atom centres
 * xy[2 n_atoms] (host).  Writes *levels and *n_blocks; if `out` is not NULL and
 * out_len is large enough it receives, per block in order, the record
 * (level, nt, ns, nt target atoms, ns source atoms) as ints; *out_needed
 * receives the length required.  VIE_ERR_INVALID_ARG for coincident atoms. */
int vie_plan_far_blocks(const double* xy, int n_atoms, int* levels, int64_t* n_blocks, int* out, int64_t out_len,
                        int64_t* out_needed);

/* vie_lpt_assign (App. C): greedy least-loaded assignment of n weights w[n] to
 * n_proc processes; owner[n] receives each weight's process, loads[n_proc]
 * the process totals (both host memory). */
int vie_lpt_assign(const double* w, int64_t n, int n_proc, int* owner, double* loads);

/* ---- serving (continuous batching) ------------------------------------------
 * Requests (geometry + plane waves) are admitted while the modelled HBM
 * footprint of their compressed operator, inverses and Krylov state fits
 * the budget; admitted requests run concurrently, each on its own CUDA stream.
 * A request's allocations are capped at its admitted footprint; one that
 * reaches the cap goes back to the head of the queue with twice the footprint
 * (at most the budget) and runs again when that much is free; one that fails
 * with the whole budget returns VIE_ERR_ADMISSION. */
typedef struct vie_serve_opts {
    int max_inflight;          /* concurrent requests (slots) */
    size_t hbm_budget;         /* bytes for all in-flight requests (0 = context budget) */
    double tol;                /* compression tolerance (1e-4) */
    vie_solve_opts solve;      /* solver options for every request */
} vie_serve_opts;

typedef struct vie_request {
    vie_geometry geometry;     /* copied at submit */
    double wavelength;
    int nrhs;
    vie_incident inc;          /* copied at submit */
} vie_request;

typedef struct vie_result {
    int status;                /* vie_status of the solve */
    int64_t n;                 /* unknowns */
    int nrhs;
    double* I;                 /* host c128 n x nrhs, owned by the server until vie_result_free */
    vie_solve_stats stats;
    double t_submit_s, t_start_s, t_done_s; /* server clock */
    int64_t footprint_bytes;   /* footprint the request finally ran with */
    int retries;               /* times it went back to the queue after its allocations met the
                                  admitted footprint (each retry doubles it) */
    int64_t peak_bytes;        /* device bytes the request held at most */
} vie_result;

int vie_serve(vie_server** out, vie_ctx* ctx, const vie_serve_opts* opts);
int vie_submit(vie_server* s, const vie_request* req, uint64_t* ticket);
/* Waits up to timeout_ms for the ticket; VIE_ERR_TIMEOUT if not done yet. */
int vie_poll(vie_server* s, uint64_t ticket, vie_result* out, int timeout_ms);
void vie_result_free(vie_result* r);
int vie_server_stop(vie_server* s); /* drains in-flight work, then frees the server */

/* Modelled footprint (bytes) of a request of n unknowns, nrhs right-hand sides,
 * restart m and the given factor-entry estimate: the admission rule. */
int64_t vie_footprint_bytes(int64_t n, int np, int nrhs, int restart, int64_t factor_entries);

/* Number of libvie kernels launched by this process so far (all contexts);
 * cuBLAS kernels are not counted.  Diagnostic, thread-safe. */
int64_t vie_kernel_launches(void);

/* vie_tune (no paper counterpart; a project-written autotuner): times every
 * far-apply variant admissible for `precision` (VIE_C64: the SIMT tiles;
 * VIE_BF16X3: those and the two tensor-core kernels) on nrhs right-hand sides
 * of this operator, with CUDA events on the context stream, and keeps the
 * fastest for every later apply and solve whose right-hand-side count has
 * the same floor(log2).  force_variant > 0 sets that variant without timing
 * (VIE_ERR_INVALID_ARG if it is not admissible).  Synchronises the context
 * stream; not callable during stream capture.  result may be NULL. */
int vie_tune(vie_op* op, int precision, int nrhs, int force_variant, vie_tune_result* result);

#ifdef __cplusplus
}
#endif
#endif /* VIE_H */
