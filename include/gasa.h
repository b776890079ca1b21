/*
 * gasa.h -- C ABI of the GB300 geometric adaptive smoothed aggregation
 * (alpha-SA) multigrid library for DG discretisations.
 *
 * Method: Pan, Lindsey & Persson, "Geometric adaptive smoothed aggregation
 * multigrid for discontinuous Galerkin discretisations" (2025).  The
 * paper's problem statement (Section 4.5) takes the system operator A and
 * the element graph G; the nested element aggregates (Section 4.1) are
 * passed in as well.  gasa_setup follows Alg. 5, gasa_solve applies the
 * V-cycle of Alg. 2 as a preconditioner of CG or GMRES (Section 6).
 *
 * Naming: the paper calls the tentative (orthonormal, block-diagonal)
 * prolongator P_{k+1}^k and the smoothed one T_{k+1}^k.  This library calls
 * the tentative one T and the smoothed one P = (I - w D^-1 A) T, R = P^T.
 *
 * Conventions for every entry point:
 *  - every function returns a gasa_status (0 = GASA_OK); nothing aborts,
 *    prints or throws; inputs are validated before any device work;
 *  - "device pointer" means memory of the CUDA device the call runs on;
 *    the caller keeps ownership of everything it passes in;
 *  - BSR matrices store one dense block per stored (block row, block
 *    column) pair, blocks row-major and contiguous, block columns sorted
 *    ascending within each block row;
 *  - indices are int32, values FP64 unless a name ends in _f32;
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef GASA_H
#define GASA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GASA_OK = 0,
  GASA_ERR_INVALID_ARG = 1,     /* malformed input, detected before device work */
  GASA_ERR_OOM = 2,             /* device allocation failed */
  GASA_ERR_CUDA = 3,            /* a CUDA call failed; text in gasa_last_error */
  GASA_ERR_SINGULAR_BLOCK = 4,  /* a diagonal block or the coarse matrix is singular */
  GASA_ERR_NOT_SPD = 5,         /* CG met p^T A p <= 0 */
  GASA_ERR_NOT_CONVERGED = 6,   /* max_iter reached; x and info hold the last iterate */
  GASA_ERR_BREAKDOWN = 7,       /* Krylov breakdown or rank-deficient candidate block */
  GASA_ERR_TIMEOUT = 8,
  GASA_ERR_BUDGET = 9,
  GASA_PENDING = 10,
  GASA_ERR_UNSUPPORTED = 11,    /* valid input this build does not handle */
  GASA_ERR_STATE = 12           /* call out of order (e.g. solve before setup) */
} gasa_status;

/* CG (SPD, Section 6), left-preconditioned GMRES (Section 6), or the V-cycle
 * of Alg. 2 as a stationary iteration x <- x + V(b - A x) */
enum { GASA_SOLVER_CG = 0, GASA_SOLVER_GMRES = 1, GASA_SOLVER_STATIONARY = 2 };
/* FP64: FP64 V-cycle.  MIXED32: FP32 V-cycle (FP32 storage and arithmetic)
 * inside FP64 flexible CG / FGMRES.  MIXED16: as MIXED32, with the level-0
 * operator and block inverses stored as FP16 blocks with one FP32 scale per
 * block (arithmetic FP32).  The coarsest solve is FP64 in every mode. */
enum { GASA_PREC_FP64 = 0, GASA_PREC_MIXED32 = 1, GASA_PREC_MIXED16 = 2 };
enum { GASA_CAND_R = 0, GASA_CAND_TT = 1 };
enum { GASA_MV_ASSIGN = 0, GASA_MV_RESIDUAL = 1, GASA_MV_ADD = 2 };

#define GASA_MAX_LEVELS 24

/* Level-0 operator A: n_blocks x n_blocks blocks of block x block entries
 * (one block per element pair, Section 2 / Eq. Auf).  The diagonal block of
 * every block row must be stored. */
typedef struct {
  int32_t n_blocks;          /* number of elements n_e */
  int32_t block;             /* dofs per element n_p */
  int32_t nnzb;              /* stored blocks */
  const int32_t *row_ptr;    /* n_blocks + 1 */
  const int32_t *col;        /* nnzb */
  const double *val;         /* nnzb * block * block */
  int32_t on_device;         /* 1: the three arrays are device pointers */
} gasa_bsr;

/* Nested aggregates (Section 4.1): levels L0..LN, N = n_levels - 1.
 * agg_of[k-1][i] (host memory) is the level-k aggregate containing level-(k-1)
 * unit i, for k = 1..N; level-0 units are elements.  Aggregate ids of each
 * level are 0..n-1 and every aggregate is non-empty. */
typedef struct {
  int32_t n_levels;
  const int32_t *const *agg_of;
} gasa_hierarchy;

typedef struct {
  int32_t dim;               /* spatial dimension d (sets n_cut default) */
  int32_t solver;            /* GASA_SOLVER_CG (SPD), GASA_SOLVER_GMRES or GASA_SOLVER_STATIONARY */
  int32_t restart;           /* GMRES restart length (default 30) */
  int32_t precision;         /* GASA_PREC_FP64 or GASA_PREC_MIXED32 */
  int32_t t_pre, t_post;     /* smoothing steps (Section 6: 3 and 3) */
  int32_t q_power;           /* Alg. 4 iterations (Section 4.4: q = 3) */
  int32_t n_cand;            /* r; 0 = median level-1 aggregate dofs (Section 4.2) */
  int32_t max_relax;         /* cap on Eq. bsmooth sweeps per candidate (default 100) */
  int32_t max_iter;          /* outer Krylov iterations (default 10000) */
  int32_t cand_init;         /* GASA_CAND_R: B^{k+1} = R B^k (Alg. 5); GASA_CAND_TT: T^T B^k (Eq. SA_Bk) */
  int32_t keep_setup_data;   /* 1: keep T and the candidates B^k for gasa_get_level */
  double gamma;              /* Eq. bsmooth tolerance (default 0.03) */
  double omega_factor;       /* Eq. omega numerator (default 4/3) */
  double n_cut;              /* Eq. sik cut factor; 0 = 2^d - (d - 1) */
  uint64_t seed;             /* splitmix64 seed of the power-iteration vectors */
  const double *init_candidates; /* optional host B^0, n x r column-major; NULL = N(0,1) drawn on device */
  int32_t bulk_staging;      /* 1: level-0 FP32 smoothing steps stage A and w D^-1 in shared
                                memory by bulk copies where the block size allows; 0 (default):
                                plain loads (faster on the measured workloads).  Both give the
                                same bits. */
  int32_t matrix_free_levels; /* kappa of Section 4.4: A_1 .. A_kappa (kappa < N) are not kept
                                after setup and are applied as R_{k-1} A_{k-1} P_{k-1}
                                (Eq. matfree2 with the transfers unrolled); their block
                                inverses are kept.  0 (default): every A_k stored. */
  int32_t hstar;             /* 1: one h*-multigrid step at the top (Section 4.3): level 0 and its
                                elements are duplicated, every element keeps the singular vectors
                                of its candidate rows above delta * sigma_1 (Eq. sik, h*-branch);
                                the given hierarchy follows one level lower.  0 (default): off */
  double delta;              /* h* threshold; 0 = the paper's 1e-3 */
  int32_t tail_kib;          /* bottom of the V-cycle of Alg. 2 as one thread-block-cluster
                                launch (kernels_tail.cu) instead of one launch per step: the
                                deepest run of levels k >= 1 whose A_k takes at most this many
                                KiB in the V-cycle's precision, with every coarser level and the
                                coarsest solve, while A_N^{-1} takes at most 2 MB; top levels
                                are left out until each CTA's rows and vectors fit its shared
                                memory.  Same arithmetic per row, so results agree with the
                                per-step launches to rounding.  0 (default): one launch per
                                step (measured faster inside the graph-captured CG loop). */
  int32_t grid_tail;         /* 1: the coarse levels of the V-cycle of Alg. 2 as one persistent
                                cooperative launch over the whole GPU (kernels_grid.cu): every level
                                k >= k0 >= 1 down to the coarsest, k0 the first level from which all
                                levels have one block size s <= 8 and are stored unpadded; its
                                steps are phases separated by bounded grid barriers.  Results agree
                                with the per-step launches to rounding.  0: one launch per step. */
  double wait_budget_s;      /* budget of one launch's bounded device-side waits (grid barriers of
                                the persistent coarse launch); a wait that runs out ends the launch
                                and the solve returns GASA_ERR_TIMEOUT.  0 = 1 second. */
  int32_t fused_restriction; /* 1 (default): setup also forms R_k A_k on every stored level where it
                                holds no more values than A_k, and there the V-cycle restricts as
                                b_{k+1} = R_k b_k - (R_k A_k) u_k, the same
                                vector as R_k (b_k - A_k u_k) of Alg. 2, in one product that on
                                the FP32 levels also takes level k+1's first smoothing step
                                u_{k+1} = w D_{k+1}^{-1} b_{k+1}; results agree with the two-step
                                form to rounding.  0: residual and restriction as two steps. */
  int32_t dense_tail_dofs;   /* bottom of the V-cycle of Alg. 2 as one dense operator: from the first
                                level k >= 1 holding at most this many (stored) dofs, with every
                                level below it stored (not matrix-free), the steps of levels
                                k .. N-1 and the coarsest solve, started from u_k = 0, form a fixed
                                linear map b_k -> u_k.  Setup forms it (FP64, n_k x n_k) by running
                                those steps on the unit vectors, and the V-cycle applies it as one
                                dense FP64 product (FP32 vectors in the FP32 cycle).  Results agree
                                with the per-step cycle to rounding.  Not built when tail_kib or
                                grid_tail is set.  0: off; default 2048; at most 8192. */
  int32_t folded_smoother;   /* 1 (default): level 0 also stores w D_0^{-1} A_0 in FP32 (block row i
                                multiplied by its block inverse, in A_0's pattern, formed in FP64),
                                and the FP32 cycle's smoothing steps of Alg. 1 after the first run as
                                u + c - (w D_0^{-1} A_0) u with c = w D_0^{-1} b, which the first
                                step u = c leaves: the same step, without re-reading the block
                                inverses (block sizes up to 16; the FP64 cycle and the FP16-block
                                level 0 keep the plain step, measured faster there).  Results agree
                                with the plain step to rounding.  0: the plain step
                                u + w D^{-1} (b - A u). */
} gasa_options;

typedef struct {
  int32_t n_levels;          /* N + 1 */
  int32_t n_cand;            /* r actually used */
  int64_t units[GASA_MAX_LEVELS];   /* elements or aggregates per level */
  int32_t block[GASA_MAX_LEVELS];   /* dofs per unit s_k (uniform per level) */
  int64_t dofs[GASA_MAX_LEVELS];
  int64_t nnzb[GASA_MAX_LEVELS];    /* stored blocks of A_k */
  int64_t nnz[GASA_MAX_LEVELS];     /* stored scalars of A_k */
  double omega[GASA_MAX_LEVELS];    /* w_k (0 on the coarsest level) */
  double rho[GASA_MAX_LEVELS];      /* Alg. 4 estimate */
  int32_t relax_sweeps_max[GASA_MAX_LEVELS];
  double seconds;
  int64_t device_bytes;      /* resident hierarchy size */
} gasa_setup_info;

typedef struct {
  int32_t iterations;        /* Krylov iterations (one V-cycle each) */
  int32_t converged;
  double rel_residual;       /* true ||b - A x|| / ||b|| at exit */
  double seconds;
} gasa_solve_info;

typedef struct gasa_ctx gasa_ctx;

/* ------------------------------------------------------------------ */
/* context API                                                          */
/* ------------------------------------------------------------------ */

/* Fill `opt` with the paper's defaults (Sections 4.2-4.4, 6). */
void gasa_default_options(gasa_options *opt);

/* Create a context on CUDA device `device`; `stream` (nullable) is used for
 * every launch of the context, else the context creates its own. */
gasa_status gasa_create(gasa_ctx **ctx, int32_t device, void *stream);

/* Alg. 5: build the hierarchy on the device.  A is copied; adj (element face
 * graph, CSR) and centroids (n_e x dim) are validated and kept for the
 * record; `hier` gives the aggregates (NULL is GASA_ERR_UNSUPPORTED in this
 * build).  Equal keep counts s_k per level are required
 * (GASA_ERR_UNSUPPORTED otherwise).  `info` is nullable. */
gasa_status gasa_setup(gasa_ctx *ctx, const gasa_bsr *A,
                       const int32_t *adj_ptr, const int32_t *adj_idx,
                       const double *centroids, const gasa_hierarchy *hier,
                       const gasa_options *opt, gasa_setup_info *info);

/* Solve A x = b to ||b - A x|| <= tol ||b|| from x = 0 with the V-cycle
 * (Alg. 2) preconditioning CG (opt.solver = CG) or left-preconditioned
 * GMRES(restart) (Section 6); precision MIXED32 runs the V-cycle in FP32
 * inside flexible CG / FGMRES.  b and x are n_e*n_p doubles, host memory if
 * on_device == 0, else device pointers.  x is written on GASA_OK and on
 * GASA_ERR_NOT_CONVERGED.  `info` is nullable. */
gasa_status gasa_solve(gasa_ctx *ctx, const double *b, double *x, double tol,
                       int32_t precision, int32_t on_device, gasa_solve_info *info);

/* One V-cycle z = M r (Alg. 2 from a zero initial guess), device pointers,
 * FP64 or MIXED32 (FP32 inside, FP64 in and out). */
gasa_status gasa_vcycle(gasa_ctx *ctx, const double *r, double *z, int32_t precision);

/* Level data, copied to host memory for inspection. */
enum {
  GASA_LV_A_ROWPTR = 0, GASA_LV_A_COL = 1, GASA_LV_A_VAL = 2,
  GASA_LV_P_ROWPTR = 3, GASA_LV_P_COL = 4, GASA_LV_P_VAL = 5,
  GASA_LV_R_ROWPTR = 6, GASA_LV_R_COL = 7, GASA_LV_R_VAL = 8,
  GASA_LV_T_VAL = 9,         /* units x s_k x s_{k+1}, unit i's block of T */
  GASA_LV_W = 10,            /* units x s_k x s_k: w_k D_k^{-1} */
  GASA_LV_CAND = 11,         /* relaxed B^k, dofs x r column-major */
  GASA_LV_SWEEPS = 12,       /* int32 r: Eq. bsmooth sweeps per column */
  GASA_LV_COARSE_INV = 13,   /* coarsest level: dense A_N^{-1}, row-major */
  GASA_LV_CAND_IN = 14,      /* B^k before relaxation */
  GASA_LV_SIZES = 15,        /* int32 units: real dofs of each unit */
  GASA_LV_RA_ROWPTR = 16,    /* R_k A_k (option fused_restriction), next-level rows x level-k units */
  GASA_LV_RA_COL = 17,
  GASA_LV_RA_VAL = 18,
  GASA_LV_DENSE_TAIL = 19,   /* first level k of the dense bottom (option dense_tail_dofs): its
                                n_k x n_k FP64 operator b_k -> u_k, row-major */
  GASA_LV_WA = 20            /* level 0 with folded_smoother and keep_setup_data: w D_0^{-1} A_0
                                in A_0's block pattern (nnzb x s x s, FP64; block row i
                                multiplied by its block inverse) */
};
/* shape[0..7] = units, s_k, nnzb(A), P nnzb, R nnzb, s_{k+1}, r, dofs.  On a
 * level whose aggregates keep different counts (h*-step, or unequal
 * aggregates) every unit is stored padded to s_k; GASA_LV_SIZES gives the
 * real dofs of each unit (the padding holds zeros, with 1 on the diagonal of
 * A_k so that the block inverses exist), and dofs counts real dofs only. */
gasa_status gasa_level_shape(gasa_ctx *ctx, int32_t level, int64_t shape[8]);

/* Fused bottom of the V-cycle of one precision (option grid_tail, else
 * tail_kib): out[0] = first level k0 run inside the fused launch
 * (n_levels - 1 when every level runs as its own launches), out[1] = CTAs of
 * the launch (the persistent grid's CTAs with grid_tail, the CTAs per
 * cluster with tail_kib; 0 when unfused), out[2] = 1 when the coarsest solve
 * runs inside the launch.
 * GASA_PREC_MIXED16 reports the FP32 tail it shares with MIXED32.
 * GASA_ERR_STATE before a successful gasa_setup, GASA_ERR_INVALID_ARG for an
 * unknown precision or a null pointer. */
gasa_status gasa_tail_info(gasa_ctx *ctx, int32_t precision, int32_t out[3]);

/* Layout of the V-cycle as set up: out[0] = first level k of the dense bottom
 * operator (option dense_tail_dofs; n_levels - 1 when there is none), out[1] =
 * n_k, its order (0 when there is none), out[2] = 1 when level 0's FP32 smoothing
 * steps run in the folded form (option folded_smoother), else 0.
 * GASA_ERR_STATE before a successful gasa_setup, GASA_ERR_INVALID_ARG for a
 * null pointer. */
gasa_status gasa_cycle_info(gasa_ctx *ctx, int32_t out[3]);
gasa_status gasa_get_level(gasa_ctx *ctx, int32_t level, int32_t what,
                           void *host_out, int64_t n_bytes);

/* Per-kernel timing over CUDA events on the context stream (for the
 * benchmark's roofline; a profiled solve runs the host-driven loop): class 0 =
 * level-0 smoothing steps after the first (x + w D^{-1}(b - A x), or the folded
 * x + c - (w D^{-1} A) x), 1 = level-0 residual and restriction (the fused
 * b_1 = R b - (R A) x where R A is stored, else the residual SpMV alone),
 * 2 = outer A*p SpMV, 3 = level-0 first pre-smoothing step x = w D^{-1} b,
 * 4 = level-0 prolongation x += P e.  Enable, run, then read total
 * milliseconds, launches and algorithmic bytes moved. */
gasa_status gasa_profile_enable(gasa_ctx *ctx, int32_t on);
gasa_status gasa_profile_read(gasa_ctx *ctx, int32_t kernel_class, double *ms,
                              int64_t *launches, double *bytes);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts and single operations), for launch accounting. */
int64_t gasa_kernel_launches(void);

gasa_status gasa_destroy(gasa_ctx *ctx);
const char *gasa_status_string(gasa_status s);
const char *gasa_last_error(const gasa_ctx *ctx);

/* ------------------------------------------------------------------ */
/* single operations on caller-owned device memory                      */
/* ------------------------------------------------------------------ */

/* Block-sparse matrix-vector product (Alg. 1 / Alg. 2 residuals, and the
 * transfers u += P u_c, b_c = R r of Alg. 2): A has n_brows block rows of
 * br x bc blocks.  mode ASSIGN: y = A x; RESIDUAL: y = b - A x;
 * ADD: y += A x.  x holds (max col + 1) * bc entries, y and b n_brows * br. */
gasa_status gasa_bsr_mv(int32_t mode, int32_t n_brows, int32_t br, int32_t bc,
                        const int32_t *row_ptr, const int32_t *col, const double *val,
                        const double *x, const double *b, double *y, void *stream);
gasa_status gasa_bsr_mv_f32(int32_t mode, int32_t n_brows, int32_t br, int32_t bc,
                            const int32_t *row_ptr, const int32_t *col, const float *val,
                            const float *x, const float *b, float *y, void *stream);

/* y = A x (FP64 result) of the outer Krylov product of the mixed-precision
 * solve (the Alg. 2 preconditioner runs in FP32; the paper fixes no
 * precision), in double-single arithmetic from exact two-term FP32 splits:
 * a = a_hi + a_lo per stored value and x = x_hi + x_lo per entry (hi the FP32
 * rounding, lo the FP32 rounding of the remainder).  Each product's leading
 * part is exact and joins the sum by an error-free two-sum; the low word
 * gathers the rest in FP32, so a row of n terms agrees with an FP64 product
 * to within n * 2^-47 of sum |a x| (an FP32 product: 2^-24).  Layout as
 * gasa_bsr_mv; all pointers device memory; errors as gasa_bsr_mv. */
gasa_status gasa_bsr_mv_ds(int32_t n_brows, int32_t br, int32_t bc, const int32_t *row_ptr,
                           const int32_t *col, const float *a_hi, const float *a_lo,
                           const float *x_hi, const float *x_lo, double *y, void *stream);

/* One block-Jacobi step of Alg. 1 with A~^{-1} = W = w D^{-1}
 * (Eq. smoother_choice): x_out = x + W (b - A x); first != 0 gives the
 * step from x = 0, x_out = W b (x unused).  W holds n_units blocks of
 * bs x bs.  x_out must not alias x. */
gasa_status gasa_jacobi_sweep(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                              const int32_t *col, const double *val, const double *W,
                              const double *x, const double *b, double *x_out,
                              int32_t first, void *stream);
gasa_status gasa_jacobi_sweep_f32(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                  const int32_t *col, const float *val, const float *W,
                                  const float *x, const float *b, float *x_out,
                                  int32_t first, void *stream);

/* W_out = scale * D^{-1} for the diagonal blocks D of a square BSR matrix
 * (block Jacobi, Section 4.4); LU with partial pivoting per block.
 * *n_singular (host) receives the number of singular blocks. */
gasa_status gasa_block_inverse(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                               const int32_t *col, const double *val, double scale,
                               double *W_out, int32_t *n_singular, void *stream);

/* Alg. 4: rho = ||D^{-1} A x_q|| after q normalised steps from x0
 * (device, n_units*bs; x0 need not be normalised).  Dinv from
 * gasa_block_inverse with scale 1.  *rho is written to host memory. */
gasa_status gasa_power_estimate(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                const int32_t *col, const double *val, const double *Dinv,
                                const double *x0, int32_t q, double *rho, void *stream);

/* Eq. bsmooth: relax every column of B (device, n x r column-major, in
 * place) with x <- x - W A x until ||x^(m-1)|| / ||x^(m)|| < 1 + gamma
 * (at least one and at most max_relax sweeps).  sweeps (host, r ints)
 * receives the sweep count per column. */
gasa_status gasa_relax_candidates(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                  const int32_t *col, const double *val, const double *W,
                                  double *B, int32_t r, double gamma, int32_t max_relax,
                                  int32_t *sweeps, void *stream);

/* Eq. splitB_dg + Eq. sik: per aggregate J, the left singular vectors of the
 * rows of B (device, n x r column-major, n = n_units * bs) owned by J's
 * units (increasing unit id, then dof), ordered by descending singular
 * value, the first s_next kept and signed so that each column's entry of
 * largest magnitude (lowest row on ties) is positive.  agg_of (device,
 * n_units) maps units to aggregates 0..n_agg-1.  T_out (device): n_units
 * blocks of bs x s_next, unit i's rows of its aggregate's kept vectors.
 * sigma_out (device, nullable): n_agg x r singular values, descending,
 * zero-padded. */
gasa_status gasa_tentative(int32_t n_units, int32_t bs, int32_t n_agg, const int32_t *agg_of,
                           const double *B, int32_t r, int32_t s_next, double *T_out,
                           double *sigma_out, void *stream);

/* Allocation-free variant of gasa_power_estimate, for callers that cannot
 * allocate device memory when they run this step (a fixed device-memory
 * budget after start-up, an allocator owned by a host framework, or serving
 * code that must not block on or fail in the allocator).  It computes the
 * same estimate with the same arguments, but its scratch (two vectors,
 * reduction partials, scalars) lives in a fixed device array inside the
 * library: about 4.2 MB on every device that loads the library, held until
 * the process exits.  The paper has no counterpart to this entry point.
 *  - n_units * bs must not exceed GASA_NOALLOC_MAX_DOFS, else
 *    GASA_ERR_INVALID_ARG is returned before any device work;
 *  - it calls no cudaMalloc, cudaFree or other allocating routine;
 *  - the array's device address is looked up once per device, with that
 *    device current: by gasa_create for its device, else by the first call
 *    on the device.  Under CUDA's lazy module loading that lookup, and the
 *    first launch of each of the library's kernels on the device, load the
 *    library's device code there, which is when the array (and the code)
 *    take device memory.  So make a first call, or create a context, on each
 *    device before the stretch in which nothing may allocate, and before any
 *    stream capture on that device;
 *  - failures are reported as gasa_power_estimate reports them (the same
 *    arithmetic runs on the scratch it allocates);
 *  - all calls on a device share the array; calls that overlap on the GPU
 *    (different streams or host threads) race on it and must be avoided. */
#define GASA_NOALLOC_MAX_DOFS 262144
gasa_status gasa_power_estimate_noalloc(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                        const int32_t *col, const double *val,
                                        const double *Dinv, const double *x0, int32_t q,
                                        double *rho, void *stream);

/* Dense inverse (Gauss-Jordan, partial pivoting) of the n x n row-major
 * device matrix A into Ainv (device); the coarsest solve u_N = A_N^{-1} b_N
 * of Alg. 2.  *singular (host) is set to 1 if a pivot vanishes. */
gasa_status gasa_dense_inverse(int32_t n, const double *A, double *Ainv, int32_t *singular,
                               void *stream);

/* ------------------------------------------------------------------ */
/* request server: continuous batching of solves on resident hierarchies */
/* ------------------------------------------------------------------ */
/* The paper solves one system at a time; this server is not in it.  It keeps
 * the hierarchies of several set-up contexts (meshes) resident and runs the
 * solves submitted for them in batches: for each (mesh, precision) an engine
 * holds K slots whose right-hand sides are stored interleaved, so every
 * matrix block of the V-cycle (Alg. 2) and of the outer A x is read once for
 * the whole batch.  One engine step is a CUDA graph launch: for CG a
 * conditional loop of whole iterations, for GMRES one restart cycle.
 * Requests join free slots between launches (CG: between iterations; GMRES:
 * between cycles) and leave when they converge, so the batch changes while
 * others are in flight.  Engines of different meshes run on their own
 * streams and overlap on the device.  Every result depends only on its own
 * column (per-column reductions of fixed shape), so a solve gives the same
 * bits alone and in any mix.  Device memory for hierarchies and engines is
 * admitted against the budget given at creation; a request whose engine does
 * not fit waits until idle engines are released.
 * Precisions: GASA_PREC_FP64, GASA_PREC_MIXED32 and GASA_PREC_MIXED16 (level 0
 * read from its FP16 blocks, the other levels as in MIXED32). */
typedef struct gasa_server gasa_server;

typedef struct {
  int64_t submitted, completed, queued, running;
  int64_t engines, engines_created, engines_released;
  int64_t budget_bytes, used_bytes, peak_bytes;
  int64_t peak_running;        /* most slots iterating at the same time */
  int64_t graph_launches;
} gasa_server_stats;

/* max_batch: slots per engine, 1, 2, 4 or 8 (an engine takes fewer when the
 * budget does not hold max_batch).  Starts no work until a request arrives. */
gasa_status gasa_server_create(gasa_server **srv, int32_t device, int64_t hbm_budget_bytes,
                               int32_t max_batch);
/* Register a set-up context.  The server reads its hierarchy (solver, restart,
 * max_iter and tolerances come from its options and the request); the caller
 * keeps the context alive and unchanged until gasa_server_destroy.  The
 * hierarchy's bytes count against the budget: GASA_ERR_BUDGET if it does not
 * fit. */
gasa_status gasa_server_add_mesh(gasa_server *srv, gasa_ctx *ctx, int32_t *mesh_id);
/* Queue a solve of A x = b (b: host, copied before return) to relative
 * residual tol from x = 0 in `precision` (GASA_PREC_FP64, MIXED32 or
 * MIXED16; another value is GASA_ERR_INVALID_ARG).  Returns at once with a
 * ticket. */
gasa_status gasa_server_submit(gasa_server *srv, int32_t mesh_id, const double *b, double tol,
                               int32_t precision, uint64_t *ticket);
/* GASA_PENDING while the solve is queued or running.  Once finished: copies
 * x to x_out (host, nullable) and the solve's info (seconds = latency from
 * submit to completion), releases the ticket and returns the solve's status
 * (GASA_OK, GASA_ERR_NOT_CONVERGED with the last iterate, or an error). */
gasa_status gasa_server_poll(gasa_server *srv, uint64_t ticket, double *x_out,
                             gasa_solve_info *info);
/* Block until no request is queued or running, or timeout_s elapses
 * (GASA_ERR_TIMEOUT). */
gasa_status gasa_server_drain(gasa_server *srv, double timeout_s);
gasa_status gasa_server_stats_read(gasa_server *srv, gasa_server_stats *out);
/* Stop the engines (requests still queued or running end with
 * GASA_ERR_STATE) and free the server's device memory. */
gasa_status gasa_server_destroy(gasa_server *srv);
const char *gasa_server_last_error(const gasa_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* GASA_H */
