// Host-side launchers shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gasa {

// ---- kernels_tma.cu: level-0 sweep with bulk-copy staging -------------------
// plan for n_units block rows of bs x bs blocks of wbytes-byte values whose
// rows hold at most max_row blocks; false when the staged kernel does not apply
bool tma_plan(int n_units, int bs, int wbytes, int max_row, int *TR, int *stageA, int *stageW,
              int *smem, int *grid);
template <typename T>
cudaError_t launch_jacobi_tma(int n_units, int bs, int TR, int stageA, int stageW, int smem,
                              int grid, const int *rp, const int *col, const T *val, const T *W,
                              const T *x, const T *b, T *xo, int *err, cudaStream_t s);

// ---- kernels_h16.cu: FP16 blocks with one FP32 scale per block -------------
cudaError_t launch_to_h16_blocks(int64_t nblocks, int bsz, const double *v, __half *h,
                                 float *scale, cudaStream_t s);
cudaError_t launch_bsr_mv_h16(int mode, int n_brows, int br, int bc, const int *rp,
                              const int *col, const __half *val, const float *scale,
                              const float *x, const float *b, float *y, cudaStream_t s);
cudaError_t launch_jacobi_h16(int mode, int n_units, int bs, const int *rp, const int *col,
                              const __half *val, const float *ascale, const __half *W,
                              const float *wscale, const float *x, const float *b, float *xo,
                              cudaStream_t s);

// ---- Alg. 4 on caller-provided scratch (gasa_api.cu) -------------------------
// The power-iteration estimate shared by gasa_power_estimate (scratch from the
// stream-ordered allocator) and gasa_power_estimate_noalloc (scratch in a
// static device array).  a and b hold n_units * bs doubles each, part
// kRedBlocks doubles, sc two doubles; nnzb is row_ptr[n_units].  On success
// *rho holds ||D^-1 A x|| after q normalised steps from x0.
cudaError_t power_estimate_on(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                              const int32_t *col, const double *val, const double *Dinv,
                              const double *x0, int32_t q, int64_t nnzb, double *a, double *b,
                              double *part, double *sc, double *rho, cudaStream_t s);
// stored blocks of a device BSR matrix (row_ptr[n], read with a synchronous
// copy on s); -1 when it cannot be read
int64_t op_nnzb(const int32_t *row_ptr, int32_t n, cudaStream_t s);
// a CUDA error as the single-operation entry points report it
int op_status_code(cudaError_t e);
// ---- noalloc.cu --------------------------------------------------------------
// looks up (and caches) the device address of the static scratch array on the
// current device; gasa_create calls it so that the lookup, and the loading of
// the module that holds the array, happen outside allocation-free calls
cudaError_t noalloc_scratch_on_current_device(double **out);

// kernel launches issued by this library (process-wide counter)
void note_launch();
long long launch_count();

enum JacobiMode { JAC_SWEEP = 0, JAC_FIRST = 1, JAC_APPLY = 2, JAC_RELAX = 3 };

// ---- kernels_wide.cu: FP32 blocks wider than 8, a team of warps per block row
// true for blocks with more than 8 rows or columns (at most 40 of either) and
// at least 8 blocks per block row on average
bool wide_applies(int br, int bc, int n_brows, int64_t nnzb);
// fused residual + restriction y = R b - (R A) x (br x bc blocks of R and R A)
// with the next level's first step xn = Wn y (square br x br) when Wn is given;
// nnzb: blocks of R and R A together
cudaError_t launch_wide_restrict(int n_brows, int br, int bc, int64_t nnzb, const int *rrp,
                                 const int *rcol, const float *rval, const int *arp,
                                 const int *acol, const float *aval, const float *b,
                                 const float *x, float *y, const float *Wn, float *xn,
                                 cudaStream_t s);
// op: 0 y = A x, 1 y = b - A x, 2 y += A x, 3 y = x + W (b - A x) (square)
cudaError_t launch_wide(int op, int n_brows, int br, int bc, int64_t nnzb, const int *rp,
                        const int *col, const float *val, const float *W, const float *x,
                        const float *b, float *y, cudaStream_t s);

// ---- kernels_blk.cu: small square blocks, one lane per block ---------------
// true when square s x s blocks (2 <= s <= 8) average at least 6 per block row;
// launch_blk then takes FP32 operands (FP64 returns cudaErrorNotSupported)
bool blk_applies(int bs, int n_brows, int64_t nnzb);
// fused residual + restriction y = R b - (R A) x (FP32, s x s blocks, s <= 8)
// with the next level's first step xn = Wn y when Wn is given; nnzb: blocks
// of R and R A together
cudaError_t launch_blk_restrict(int n_brows, int bs, int64_t nnzb, const int *rrp,
                                const int *rcol, const float *rval, const int *arp,
                                const int *acol, const float *aval, const float *b,
                                const float *x, float *y, const float *Wn, float *xn,
                                cudaStream_t s);
// the same with br x bc blocks from the finest level (br 4 or 8 coarse rows,
// bc 9 or 10 fine columns); cudaErrorNotSupported for other shapes
bool blk_restrict_rect_applies(int br, int bc, int n_brows, int64_t nnzb);
cudaError_t launch_blk_restrict_rect(int n_brows, int br, int bc, int64_t nnzb, const int *rrp,
                                     const int *rcol, const float *rval, const int *arp,
                                     const int *acol, const float *aval, const float *b,
                                     const float *x, float *y, const float *Wn, float *xn,
                                     cudaStream_t s);
// op 0/1/2: y = A x, y = b - A x, y += A x; op 3: y = x + W (b - A x).
// cudaErrorNotSupported when the shape or the alignment does not fit.
template <typename T>
cudaError_t launch_blk(int op, int n_brows, int bs, int64_t nnzb, const int *rp, const int *col,
                       const T *val, const T *W, const T *x, const T *b, T *y, cudaStream_t s);

// ---- kernels_mv.cu ---------------------------------------------------------
// nnzb >= 0 lets the launcher pick a warp per block row when rows are long
// (>= 12 blocks on average); nnzb < 0 always uses one thread per scalar row.
template <typename T>
cudaError_t launch_bsr_mv(int mode, int n_brows, int br, int bc, const int *rp, const int *col,
                          const T *val, const T *x, const T *b, T *y, cudaStream_t s,
                          int64_t nnzb = -1);

template <typename T>
cudaError_t launch_jacobi(int mode, int n_units, int bs, const int *rp, const int *col,
                          const T *val, const T *W, const T *x, const T *b, T *xo,
                          cudaStream_t s, int64_t nnzb = -1);

// The first level-0 FP32 smoothing step of the mixed-precision V-cycle,
// x = W b from x = 0, reading the FP64 b; b32 receives its FP32 rounding for
// the later steps (cudaErrorNotSupported when the block size or the
// alignment does not fit).
int jacobi_grid(int n_units, int bs);
cudaError_t launch_jacobi_first_conv(int n_units, int bs, const double *bd, float *b32,
                                     const float *W, float *xo, cudaStream_t s,
                                     float *c_out = nullptr);

// Smoothing step of Alg. 1 with the block inverse folded into the operator:
// xo = x + c - (W A) x, where WA holds W_i A_ij in A's block pattern and
// c = W b (one thread per scalar row, no exchange between the rows of a unit)
constexpr int kMvFolded = 3;   // internal product mode next to GASA_MV_*
template <typename T>
cudaError_t launch_folded_sweep(int n_units, int bs, const int *rp, const int *col, const T *WA,
                                const T *x, const T *c, T *xo, cudaStream_t s);
// WA = W A block row by block row: block k of block row i becomes W_i A_k (FP64)
cudaError_t launch_fold_block_rows(int n_units, int bs, const int *rp, const double *W,
                                   const double *A, double *WA, cudaStream_t s);

// multi-column relaxation x_c <- x_c - W A x_c for `nc` columns given by
// device tables of column base pointers (each column n_units*bs long).
cudaError_t launch_relax_multi(int n_units, int bs, const int *rp, const int *col,
                               const double *val, const double *W, const double *const *xin,
                               double *const *xout, int nc, cudaStream_t s);

// Y(:, c) = R * X(:, c) for r columns (column-major, leading dims ldx / ldy)
cudaError_t launch_bsr_mm(int n_brows, int br, int bc, const int *rp, const int *col,
                          const double *val, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int ncols, cudaStream_t s);

// y = A x (FP64 out) in double-single arithmetic from exact two-term FP32
// splits of A (hi, lo) and x (hi, lo); with xd and partials also the
// bsr_mv_ds_grid(n_brows, br) partial sums of xd . y (16-byte aligned
// operands only, else cudaErrorNotSupported)
cudaError_t launch_bsr_mv_ds(int n_brows, int br, int bc, const int *rp, const int *col,
                             const float *ahi, const float *alo, const float *xhi,
                             const float *xlo, double *y, cudaStream_t s,
                             const double *xd = nullptr, double *partials = nullptr);
int bsr_mv_ds_grid(int n_brows, int br);

// y = A x for a dense row-major n x n matrix with row pitch ld (>= n; 0 = n)
template <typename T>
cudaError_t launch_dense_mv(int n, const double *A, const T *x, T *y, cudaStream_t s, int ld = 0);
// the same in double-single arithmetic on FP32 units from the exact two-term
// FP32 split (Mh, Ml) of A (row pitch ld), FP32 x and y
cudaError_t launch_dense_mv_ds(int n, int ld, const float *Mh, const float *Ml, const float *x,
                               float *y, cudaStream_t s);

// ---- kernels_red.cu --------------------------------------------------------
// partials[kRedBlocks] of sum_i x_i y_i (y == nullptr: sum x_i^2)
cudaError_t launch_dot_partials(int64_t n, const double *x, const double *y, double *partials,
                                cudaStream_t s);
// multi-column squared norms: partials[c * kRedBlocks + blk]
cudaError_t launch_colnorm_partials(int64_t n, const double *const *cols, int nc,
                                    double *partials, cudaStream_t s);
// out[c] = sum of partials of column c (one block per column)
cudaError_t launch_finalize(const double *partials, int nc, double *out, cudaStream_t s);
// out[0] = sum of n partials
cudaError_t launch_finalize_n(const double *partials, int n, double *out, cudaStream_t s);
cudaError_t launch_scale_by_inv_sqrt(int64_t n, double *x, const double *sumsq, cudaStream_t s);
cudaError_t launch_uniform_pm1(int64_t n, uint64_t seed, uint64_t stream, double *x,
                               cudaStream_t s);
cudaError_t launch_normal(int64_t n, uint64_t seed, uint64_t stream, double *x, cudaStream_t s);
// uniform(-1,1) draws of the real dofs of a padded level, zero on padding
cudaError_t launch_uniform_pm1_padded(int n_units, int s_pad, const int *usize,
                                      const int64_t *uoff, uint64_t seed, uint64_t stream,
                                      double *x, cudaStream_t s);
// 1 on the diagonal of a padded level's padding dofs
cudaError_t launch_pad_identity(int n_units, int s_pad, const int *usize, const int *rp,
                                const int *col, double *val, cudaStream_t s);
template <typename Tin, typename Tout>
cudaError_t launch_convert(int64_t n, const Tin *in, Tout *out, cudaStream_t s);
cudaError_t launch_fill(int64_t n, double v, double *x, cudaStream_t s);
// y[i] += x[i]
template <typename T>
cudaError_t launch_add(int64_t n, const T *x, T *y, cudaStream_t s);

// CG pieces (device scalars; partial arrays of kRedBlocks entries)
cudaError_t launch_cg_update_xr(int64_t n, double *x, double *r, const double *p,
                                const double *q, const double *rz, const double *pq_partials,
                                double *rr_partials, double *alpha_out, cudaStream_t s,
                                int n_pq);
cudaError_t launch_cg_update_p(int64_t n, double *p, const double *z, const double *rz_old,
                               const double *rz_partials, const double *rzold_partials,
                               double *rz_out, int flexible, cudaStream_t s,
                               double *zold_out, float *p_hi, float *p_lo, int n_rz);
// mixed-precision CG with z, zold in FP32 (exact in FP64): partials of r . z
// and r . zold in one pass (the sums of launch_dot_partials on FP64 copies),
// and the flexible p update reading z from FP32, copying it to zold_out and
// splitting p (8-byte aligned FP32 and 16-byte aligned FP64 arrays, else
// cudaErrorNotSupported)
cudaError_t launch_cg_dots_f32(int64_t n, const double *r, const float *z, const float *zold,
                               double *part_rz, double *part_rzo, cudaStream_t s);
cudaError_t launch_cg_update_p_f32(int64_t n, double *p, const float *z, const double *rz_old,
                                   const double *rz_partials, const double *rzold_partials,
                                   double *rz_out, float *zold_out, float *p_hi, float *p_lo,
                                   int n_rz, cudaStream_t s);
// exact two-term FP32 split v = hi + lo of an FP64 vector
cudaError_t launch_split(int64_t n, const double *v, float *hi, float *lo, cudaStream_t s);
cudaError_t launch_cg_check(const double *rr_partials, double *scal, int *iters, int max_iter,
                            cudaGraphConditionalHandle handle, cudaStream_t s);
void note_launches(long long n);
cudaError_t launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s);
cudaError_t launch_copy(int64_t n, const double *x, double *y, cudaStream_t s);
cudaError_t launch_sub(int64_t n, const double *a, const double *b, double *out, cudaStream_t s);

// GMRES pieces
cudaError_t launch_multi_dot(int64_t n, const double *V, int64_t ldv, int k, const double *w,
                             double *partials, cudaStream_t s);
cudaError_t launch_multi_dot_finalize(const double *partials, int k, double *h,
                                      double *hacc, cudaStream_t s);
cudaError_t launch_gs_update(int64_t n, const double *V, int64_t ldv, int k, const double *h,
                             double *w, cudaStream_t s);
cudaError_t launch_normalize_into(int64_t n, const double *w, const double *sumsq, double *v,
                                  double *hout, cudaStream_t s);
cudaError_t launch_gmres_givens(double *H, int ldh, int j, double *cs, double *sn, double *g,
                                cudaStream_t s);
cudaError_t launch_gmres_backsolve(const double *H, int ldh, int j, const double *g, double *y,
                                   cudaStream_t s);
cudaError_t launch_combine(int64_t n, const double *V, int64_t ldv, int k, const double *y,
                           double *x, cudaStream_t s);

// ---- kernels_setup.cu ------------------------------------------------------
cudaError_t launch_block_inverse(int n_units, int bs, const int *rp, const int *col,
                                 const double *val, double scale, double *W, int *n_singular,
                                 cudaStream_t s);
cudaError_t launch_scale(int64_t n, double a, double *x, cudaStream_t s);
// T (padded to s_next columns per aggregate); unit_size (nullable): real dofs
// of each unit of a padded level; keep (nullable): kept columns per aggregate
// (default s_next); T may be null with s_next = 0 to compute sigma only
cudaError_t launch_tentative(int bs, int n_agg, int max_children, const int *child_ptr,
                             const int *child_idx, const double *B, int64_t ldb, int r,
                             int s_next, double *T, double *sigma, int *status, cudaStream_t s,
                             const int *unit_size = nullptr, const int *keep = nullptr);
// children lists of aggregates (counting sort of agg_of, stable by unit id)
cudaError_t build_children(int n_units, int n_agg, const int *agg_of, int *child_ptr,
                           int *child_idx, int *scratch, cudaStream_t s);

// structural products; all produce sorted unique block-column lists
// cand_count[i] is written for every row (candidates before de-duplication)
cudaError_t launch_pattern_P(int n, const int *Arp, const int *Acol, const int *agg,
                             int *count_or_null, const int *Prp_or_null, int *Pcol_or_null,
                             int max_cand, int ncols, cudaStream_t s);
cudaError_t launch_pattern_AB(int n, const int *Arp, const int *Acol, const int *Brp,
                              const int *Bcol, int *count_or_null, const int *Crp_or_null,
                              int *Ccol_or_null, int max_cand, int ncols, cudaStream_t s);
cudaError_t launch_cand_count_AB(int n, const int *Arp, const int *Acol, const int *Brp,
                                 int *cand, cudaStream_t s);
cudaError_t launch_numeric_P(int n, int sk, int sn, const int *Arp, const int *Acol,
                             const double *Aval, const double *W, const double *T,
                             const int *agg, const int *Prp, const int *Pcol, double *Pval,
                             cudaStream_t s);
cudaError_t launch_numeric_AB(int n, int br, int bm, int bc, const int *Arp, const int *Acol,
                              const double *Aval, const int *Brp, const int *Bcol,
                              const double *Bval, const int *Crp, const int *Ccol,
                              double *Cval, cudaStream_t s);
cudaError_t launch_transpose(int n_rows, int n_cols, int br, int bc, const int *Prp,
                             const int *Pcol, const double *Pval, int *Rrp, int *Rcol,
                             double *Rval, int *scratch_pos, int *scratch_cnt, cudaStream_t s);
cudaError_t launch_bsr_to_dense(int n, int bs, const int *rp, const int *col, const double *val,
                                double *D, cudaStream_t s);
cudaError_t launch_dense_inverse(int n, const double *A, double *Ainv, double *work,
                                 int *singular, cudaStream_t s);
cudaError_t launch_max_int(int n, const int *x, int *out, cudaStream_t s);
cudaError_t launch_exclusive_scan(int n, const int *in, int *out, int *scratch, cudaStream_t s);

}  // namespace gasa
