/*
 * gbstokes.h -- C ABI of the GB300 solve-phase library for Stokes
 * saddle-point systems (Demidov, Mu, Wang, "Accelerating linear solvers
 * for Stokes problems with C++ metaprogramming").
 *
 * The library solves K x = b, K a square matrix stored as CSR or block
 * CSR (BSR) with bdim x bdim blocks, with a right-preconditioned Krylov
 * method (BiCGStab, restarted GMRES, or IDR(s) -- the paper's outer
 * solver, Section 4 Listings V1/V2) and one of two preconditioners:
 *   - a monolithic smoothed-aggregation AMG V-cycle with SPAI0 or damped
 *     Jacobi relaxation (Section 2.1, Listing "composition");
 *   - the Schur pressure-correction preconditioner of Section 4,
 *     Eq. SchurPC, with the pressure operator of Eq. SchurApprox; both
 *     inner solves are one AMG V-cycle (velocity: bdim-1 = nvel blocks;
 *     pressure: scalar).
 * The AMG hierarchy may be stored in FP64, FP32 or BF16 (the last two
 * accumulate in FP32); the outer Krylov vectors, dot products, norms and
 * true-residual replacement are always FP64 (Section 4, mixed precision,
 * Listing V4).
 *
 * Conventions shared by every entry point:
 *   - Return value: gbs_status.  On failure gbs_last_error() returns a
 *     thread-local message.  Invalid input is rejected before any device
 *     work is queued.
 *   - "host" pointers are read during the call only; the library copies
 *     what it keeps.  "device" pointers are caller-owned CUDA global
 *     memory on the current device, FP64, length n = n_brows * bdim,
 *     16-byte aligned (GBS_ERR_INVALID otherwise).
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is ordered on it; a call blocks
 *     only where it states so.
 *   - Vectors are interleaved per block row (for the Stokes systems:
 *     [u v w p] per node).
 */
#ifndef GBSTOKES_H
#define GBSTOKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbs_hierarchy gbs_hierarchy;   /* opaque, library-owned */

typedef enum {
  GBS_OK = 0,
  GBS_NOT_CONVERGED = 1,    /* x and info are still written */
  GBS_ERR_INVALID = -1,     /* bad argument or matrix (nothing queued) */
  GBS_ERR_CUDA = -2,        /* a CUDA call failed */
  GBS_ERR_OOM = -3,         /* device allocation failed */
  GBS_ERR_BREAKDOWN = -4,   /* Krylov breakdown (rho or (rhat,v) = 0) */
  GBS_ERR_NAN = -5          /* NaN/Inf in a norm */
} gbs_status;

enum { GBS_PC_AMG = 0, GBS_PC_SCHUR = 1 };
enum { GBS_BICGSTAB = 0, GBS_GMRES = 1, GBS_IDRS = 2 };
enum { GBS_FP64 = 0, GBS_FP32 = 1, GBS_BF16 = 2 };
enum { GBS_SPAI0 = 0, GBS_JACOBI = 1, GBS_ILUT = 2 };

/* A square or rectangular block-CSR matrix in HOST memory.
 * row_ptr: int32[n_brows + 1], monotone, row_ptr[0] = 0.
 * col_idx: int32[nnzb], strictly increasing within each block row,
 *          each < n_bcols.
 * vals:    double[nnzb * bdim * bdim], row-major blocks.
 * bdim = 1 is plain CSR.  bdim in {1, 2, 3, 4}. */
typedef struct {
  int32_t n_brows;
  int32_t n_bcols;
  int32_t bdim;
  int64_t nnzb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* vals;
} gbs_bsr;

/* Runtime parameters; mirrors the nested params of Listing "params"
 * (restart length, tolerance, strong-coupling threshold) as plain
 * fields.  Obtain defaults with gbs_params_default(). */
typedef struct {
  int32_t precond;        /* GBS_PC_AMG | GBS_PC_SCHUR */
  int32_t krylov;         /* GBS_BICGSTAB | GBS_GMRES | GBS_IDRS */
  int32_t restart;        /* GMRES restart length m (default 30, max 64) */
  double tol;             /* relative true residual ||b-Kx||/||b|| (1e-8) */
  int32_t maxiter;        /* default 1000 */
  int32_t replace_every;  /* BiCGStab true-residual replacement period (50) */
  int32_t precision;      /* hierarchy storage: GBS_FP64 | GBS_FP32 | GBS_BF16 */
  double eps_strong;      /* strength threshold at level 0 (0.08), halved per level */
  int32_t coarse_enough;  /* max scalar unknowns of the coarsest level (1000) */
  int32_t max_levels;     /* default 10 */
  int32_t npre, npost;    /* relaxation sweeps (1, 1); npost >= 1 */
  int32_t relax;          /* smoother of the monolithic / velocity AMG */
  int32_t relax_p;        /* smoother of the pressure AMG (Schur) */
  double jacobi_omega;    /* damped Jacobi weight (0.72) */
  int32_t smooth_P;       /* 1 smoothed aggregation, 0 plain aggregation */
  int32_t power_iters;    /* power iterations for rho(D^-1 A) (20) */
  int32_t nvel;           /* velocity unknowns per node for Schur (3) */
  int32_t use_graph;      /* 1: replay each Krylov iteration as a CUDA graph */
  int32_t enable_adjoint; /* 1: build transpose maps for solve_adjoint */
  int32_t setup_only;     /* 1: build the host hierarchy only (no device work,
                             no GPU needed); export/info work, solves do not */
  int32_t level_format;   /* 0: hierarchy levels (and K) whose stored blocks are
                             at most half nonzero run as scalar CSR of their
                             nonzeros (same operator, fewer bytes and FMAs);
                             hierarchy levels among them in 32-node component
                             slices where that pads at most 10%; 1: keep every
                             level in block form; 2: plain scalar CSR wherever
                             blocks are not 1x1; 3: as 2, hierarchy levels in
                             slices */
  int32_t schur_p;        /* Schur pressure solve: 0 one AMG V-cycle on S_hat;
                             1 one application of the relax_p smoother on S_hat
                             (Section 4: a single SPAI0 application) */
  int32_t schur_order;    /* 0 "full" Eq. SchurPC (two velocity solves);
                             1 "lower" factorisation (one velocity solve) */
  int32_t idr_s;          /* IDR(s) shadow-space dimension (5, as the paper's
                             solvers; 1..8).  The shadow space is SplitMix64
                             (seed idr_seed) orthonormalised by MGS */
  int32_t idr_seed;
  /* ILUT relaxation (relax or relax_p = GBS_ILUT; the velocity smoother of
   * Section 4, Listings V2-V4): Saad's dual-threshold incomplete LU of each
   * level's scalar nonzeros, keeping per row at most ilut_p times the
   * row's own lower and upper counts of entries above ilut_tau times the
   * row's 2-norm; each triangular solve is ilut_sweeps Jacobi sweeps; the
   * step is x += ilut_omega (LU)^-1 (f - A x). */
  double ilut_p;          /* fill factor (2) */
  double ilut_tau;        /* drop tolerance (1e-2) */
  int32_t ilut_sweeps;    /* Jacobi sweeps per triangular solve (2; 0..16) */
  double ilut_omega;      /* damping (1) */
  int32_t gmres_reorth;   /* GMRES orthogonalisation against the basis:
                             0 classical Gram-Schmidt, one pass (default); 1 a
                             second pass when ||w|| drops below ||w_before|| /
                             sqrt(2) (DGKS); 2 always two passes.  Every restart
                             begins from the true residual, so a less orthogonal
                             basis costs iterations, never accuracy */
  int32_t wait_log2;      /* each wait of the FP32/BF16 bulk-copy pipelines gives
                             up after 2^wait_log2 SM clocks (31: about a second;
                             0..40); the solve then returns GBS_ERR_CUDA.  Small
                             values exist to test that path: the copies still
                             land before the kernel returns */
  int32_t iso_blocks;     /* 1 (default): a hierarchy level whose every block --
                             of A_l, P_l, R_l and the smoother -- is a scalar
                             multiple of the identity (checked exactly; the
                             velocity hierarchy of a scalar-viscosity Stokes
                             system is, and every scalar level trivially) is
                             stored as the scalar matrix S with
                             A_l = S (x) I_B, one value and one column a block,
                             and each product applies S to the B interleaved
                             components at once, in 32-node slices or with
                             lane groups sized to the level (unless
                             level_format is 1); 0: such levels follow
                             level_format like any other */
} gbs_params;

typedef struct {
  int32_t iters;          /* Krylov iterations (GMRES: Arnoldi steps) */
  int32_t replacements;   /* true-residual replacements */
  int32_t converged;
  double rel_res;         /* final true ||b - K x|| / ||b|| in FP64 */
  float ms;               /* device time of the solve (CUDA events) */
  double* history;        /* optional caller host buffer of recurrence residuals */
  int32_t history_cap;
  int32_t history_len;
} gbs_info;

/* Fill *p with the defaults listed above. */
gbs_status gbs_params_default(gbs_params* p);

/* Build the preconditioner hierarchy on the host (smoothed aggregation,
 * Galerkin coarse operators, SPAI0/Jacobi blocks, dense coarse inverse;
 * Section 2: setup on builtin structures, then moved to the backend),
 * cast it to params->precision and upload it, together with K in FP64
 * and every work vector, to the current device.  After this call
 * gbs_solve allocates no device memory.
 * A: host BSR of K.  For GBS_PC_SCHUR, A->bdim must be nvel + 1 and
 * each block row is one node with the pressure unknown last.
 * stream: used for the uploads; the call synchronises it before return.
 * out: receives the handle; free with gbs_destroy. */
gbs_status gbs_build_hierarchy(const gbs_bsr* A, const gbs_params* params,
                               void* stream, gbs_hierarchy** out);

/* Solve K x = b.  b_dev: device FP64[n] (read only).  x_dev: device
 * FP64[n], initial guess on entry, solution on return.  Blocks until the
 * solve ends (one small device->host read per iteration decides
 * convergence).  info may be NULL.  Returns GBS_NOT_CONVERGED when
 * maxiter is reached (x still holds the last iterate). */
gbs_status gbs_solve(gbs_hierarchy* h, const double* b_dev, double* x_dev,
                     void* stream, gbs_info* info);

/* Adjoint solve K^T lam = g with the same Krylov method and the
 * transposed preconditioner (A_l^T through transpose maps, M_l^T, the
 * same P and R since R = P^T, transposed coarse inverse; for Schur the
 * same steps on K^T).  g_dev, lam_dev: device FP64[n]; lam is also the
 * initial guess.  Requires enable_adjoint and a structurally symmetric
 * block pattern at every level. */
gbs_status gbs_solve_adjoint(gbs_hierarchy* h, const double* g_dev, double* lam_dev,
                             void* stream, gbs_info* info);

/* Sampled outer product on the stored pattern of K:
 * grad[k*bdim*bdim + a*bdim + c] = alpha * lam[bdim*i + a] * x[bdim*j + c]
 * for stored block k = (i, j).  With alpha = -1 this is dL/dK for
 * x = K^-1 b and lam = K^-T dL/dx.  All pointers device FP64;
 * grad has nnzb * bdim^2 entries.  Asynchronous on stream. */
gbs_status gbs_sampled_outer(const gbs_hierarchy* h, const double* lam_dev,
                             const double* x_dev, double alpha, double* grad_dev,
                             void* stream);

/* Replace the values of K (same pattern, device FP64[nnzb*bdim^2]); the
 * preconditioner is kept as built.  Asynchronous on stream.  When K runs
 * as scalar CSR of its build-time nonzeros (level_format 0), the next
 * solve or spmv reads one device flag and switches K to its block form if
 * a new value outside that pattern is nonzero. */
gbs_status gbs_update_values(gbs_hierarchy* h, const double* vals_dev, void* stream);

/* y = K x (transpose != 0: y = K^T x) with the library's FP64 outer SpMV.
 * x_dev, y_dev: device FP64[n].  Asynchronous on stream (synchronises
 * once after a gbs_update_values, see there). */
gbs_status gbs_spmv(const gbs_hierarchy* h, const double* x_dev, double* y_dev,
                    int32_t transpose, void* stream);

/* One application of the preconditioner: z = M^-1 r (transpose != 0:
 * the transposed preconditioner).  r_dev, z_dev: device FP64[n].
 * Asynchronous on stream. */
gbs_status gbs_apply_precond(gbs_hierarchy* h, const double* r_dev, double* z_dev,
                             int32_t transpose, void* stream);

/* Hierarchy shape.  which: 0 monolithic / velocity AMG, 1 pressure AMG.
 * Writes the number of levels (coarsest included) to *nlevels and, if
 * the arrays are non-NULL, per level n_brows and nnzb of A_l (up to cap
 * entries).  bytes: device bytes held by the hierarchy (may be NULL). */
gbs_status gbs_hierarchy_info(const gbs_hierarchy* h, int32_t which, int32_t* nlevels,
                              int32_t* n_brows, int64_t* nnzb, int32_t cap,
                              int64_t* bytes);

/* Algorithmic bytes that one preconditioner application moves (values,
 * indices and vectors of every kernel it launches, from the formats the
 * hierarchy is stored in).  Used for bandwidth reporting. */
gbs_status gbs_precond_bytes(const gbs_hierarchy* h, double* bytes_per_apply);

/* Layout the FP64 outer SpMV of K runs in now (no counterpart in the
 * paper; the library's per-operator format choice): *format = 0 block
 * CSR, 1 scalar CSR of K's build-time nonzeros, 2 those nonzeros in
 * 32-node component slices (when at least 90% of the slices share their
 * rows' column offsets, as on a stencil).  *stored: value entries the
 * kernel streams (stored block values, nonzeros, or slice entries with
 * padding).  Host only; reflects a pending fall-back to blocks only after
 * the next solve or spmv. */
gbs_status gbs_outer_format(const gbs_hierarchy* h, int32_t* format, int64_t* stored);

/* Layout in which level `level` (below the coarsest) of AMG `which` (0
 * monolithic / velocity, 1 pressure) runs its forward products (no
 * counterpart in the paper; the library's per-level format choice, for
 * measurement): *format = 0 block CSR, 1 scalar CSR of the nonzeros, 2
 * those nonzeros in 32-node component slices, 3 block-row slices; plus 4
 * when the level fuses its zero-guess smoothing step with the residual
 * (x = M f, r = f - (A M) f in one pass); plus 8 when the level runs as
 * S (x) I_B (iso_blocks: the layout code then describes S, whose rows are
 * the nodes).  Host only. */
gbs_status gbs_level_format(const gbs_hierarchy* h, int32_t which, int32_t level,
                            int32_t* format);

/* One operation on level `level` (below the coarsest) of AMG `which` (0
 * monolithic / velocity, 1 pressure), launched exactly as the V-cycle
 * launches it (no counterpart in the paper; for measurement and tests):
 * op 0: y = f - A_l x (the residual of Section 2.3's primitives);
 * op 1: one relaxation sweep y = x + S (f - A_l x), S the level's SPAI0,
 * Jacobi or ILUT smoother.  x, f, y: device vectors of the level's scalar
 * size in the hierarchy's vector type (double for GBS_FP64, float for the
 * FP32/BF16 forms), 16-byte aligned; y aliases neither.  Asynchronous on
 * stream. */
gbs_status gbs_level_apply(gbs_hierarchy* h, int32_t which, int32_t level, int32_t op,
                           const void* x_dev, const void* f_dev, void* y_dev, void* stream);

/* Copy level l (0 = finest) of AMG `which` to host arrays.  part: 0 = A,
 * 1 = P, 2 = R, 3 = smoother blocks M (row_ptr/col_idx untouched),
 * 4 = aggregate ids (written to col_idx, n_brows entries), 5 = dense
 * coarse inverse (vals, n*n, row-major; level must be the coarsest);
 * for a level relaxed by ILUT, scalar CSR over the level's scalar
 * unknowns: 6 = L (strictly lower; the factor's diagonal is 1), 7 = U
 * (strictly upper), 8 = the diagonal of U (vals, n_brows entries).
 * Pass NULL arrays to query sizes: *n_brows, *n_bcols, *nnzb are always
 * written.  Values are the FP64 setup values (before any cast). */
gbs_status gbs_export_level(const gbs_hierarchy* h, int32_t which, int32_t level,
                            int32_t part, int32_t* n_brows, int32_t* n_bcols,
                            int64_t* nnzb, int32_t* row_ptr, int32_t* col_idx,
                            double* vals);

/* Build a monolithic-AMG hierarchy from caller-supplied levels instead of
 * running the setup: A[0..nlev-1] (A[0] = K), P[0..nlev-2], R[0..nlev-2],
 * M[0..nlev-2] smoother blocks (double[n_brows_l * bdim^2] each), and
 * the dense coarse inverse Ainv (double[n_L^2], row-major, n_L the
 * scalar size of A[nlev-1]).  With params->relax = GBS_ILUT, M may be
 * NULL: the ILUT factors are computed here from each A[l].  Other
 * arguments as gbs_build_hierarchy (params->precond must be GBS_PC_AMG). */
gbs_status gbs_import_hierarchy(const gbs_bsr* A, const gbs_bsr* P, const gbs_bsr* R,
                                const double* const* M, const double* Ainv, int32_t nlev,
                                const gbs_params* params, void* stream,
                                gbs_hierarchy** out);

/* One AMG hierarchy given level by level, as gbs_import_hierarchy takes
 * it: A[0..nlev-1], P[0..nlev-2], R[0..nlev-2], M[0..nlev-2] smoother
 * blocks (double[n_brows_l * bdim^2] each; may be NULL with ILUT
 * relaxation) and the dense coarse inverse Ainv (double[n_L^2]).  All
 * host memory, read during the call only. */
typedef struct {
  const gbs_bsr* A;
  const gbs_bsr* P;
  const gbs_bsr* R;
  const double* const* M;
  const double* Ainv;
  int32_t nlev;
} gbs_levels;

/* Build a Schur pressure-correction preconditioner (Section 4, Eq.
 * SchurPC) from caller-supplied inner hierarchies instead of running the
 * setup.  K: host BSR of the saddle-point system, bdim = nvel + 1, the
 * pressure unknown last in each block; its couplings G (velocity rows,
 * pressure column) and D (pressure row, velocity columns) are taken from
 * K's blocks as stored.  vel: the velocity AMG (bdim = params->nvel, level
 * 0 the velocity block of K).  pres: the pressure AMG on the operator of
 * Eq. SchurApprox (bdim 1), used when params->schur_p = 0 (may be NULL
 * otherwise).  pres_smoother: double[n_brows of K], the diagonal pressure
 * smoother applied once when params->schur_p = 1 (may be NULL otherwise).
 * params->precond must be GBS_PC_SCHUR; the other arguments are as in
 * gbs_build_hierarchy.  Shapes are checked before any device work. */
gbs_status gbs_import_schur(const gbs_bsr* K, const gbs_levels* vel, const gbs_levels* pres,
                            const double* pres_smoother, const gbs_params* params,
                            void* stream, gbs_hierarchy** out);

/* Number of CUDA kernels this library has launched in this process (a
 * replayed CUDA graph counts each of its kernel nodes).  Telemetry only. */
int64_t gbs_kernel_launches(void);

/* y = A x, dots[0] = w . y (0 if w is NULL) and dots[1] = y . y for an FP64
 * block-CSR matrix held in DEVICE memory, without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the operation -- code
 * running inside CUDA graph capture (allocation cannot be captured), or
 * applications whose own memory manager owns the device.  Its reduction
 * scratch (two doubles per CTA of a fixed 608-CTA grid plus a counter,
 * 9.7 KB) is a file-scope __device__ array that every GPU loading the
 * library holds until the process exits; the grid never grows with the
 * matrix, so any matrix fits, and sizes beyond the int32 index range
 * (nnzb, n_brows*bdim, n_bcols*bdim > 2^31-1) are rejected with
 * GBS_ERR_INVALID.
 * row_ptr int32[n_brows+1], col_idx int32[nnzb] (sorted, < n_bcols), vals
 * f64[nnzb*bdim*bdim] row-major blocks, x f64[n_bcols*bdim], y
 * f64[n_brows*bdim], w f64[n_brows*bdim] or NULL, dots f64[2]: all device
 * pointers, caller-owned; vals, x, y, w 16-byte aligned; w must not alias
 * y.  The structure is not validated (it lives on the device).
 * The first call on a device looks up the scratch address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture.
 * A cudaDeviceReset of that device (which also frees every hierarchy's
 * device memory) invalidates the kept address: call this entry point no
 * more in that process after such a reset.  Every call shares the one scratch array, so
 * calls that overlap on the GPU (different streams, no ordering) race;
 * each call clears the counter it needs.  Asynchronous on stream. */
gbs_status gbs_spmv_dots_noalloc(int32_t n_brows, int32_t n_bcols, int32_t bdim, int64_t nnzb,
                                 const int32_t* row_ptr, const int32_t* col_idx,
                                 const double* vals, const double* x, double* y,
                                 const double* w, double* dots, void* stream);

/* FP64 FMA throughput of the current device, measured: the best of four
 * CUDA-event-timed launches (after two warm-up launches) of a kernel that
 * issues only independent DFMA chains, all three operands in per-thread
 * registers as in the solve's products, from as many CTAs as stay
 * resident (SM count from the device properties).  No counterpart in the
 * paper: it
 * gives the roofline of the FP64 kernels, which on GB300 the FP64 pipe
 * bounds before HBM.  *tflops: 2 * FMAs / second / 1e12.  *sms: the
 * device's SM count.  sink_dev: device double[1], written only if the
 * chains reach an impossible value.  Blocks for about half a second. */
gbs_status gbs_fp64_peak(double* tflops, int32_t* sms, double* sink_dev, void* stream);

/* Free everything the handle owns.  Synchronises the device. */
gbs_status gbs_destroy(gbs_hierarchy* h);

/* Thread-local message of the last failure ("" if none). */
const char* gbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBSTOKES_H */
