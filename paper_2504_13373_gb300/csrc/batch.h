// Batched kernels over K interleaved right-hand sides (entry i of column c at
// i * K + c) used by the request server.  Per-column solver state lives in
// two device arrays: doubles sc[BD_* * K + c] and ints st[BI_* * K + c].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace gasa {

enum BatchState {
  BS_EMPTY = 0,       // slot free
  BS_RUNNING = 1,     // iterating
  BS_CONVERGED = 2,   // stopping test passed (the host confirms with the true residual)
  BS_MAXIT = 3,       // iteration limit reached
  BS_BREAKDOWN = 4,   // non-finite value
  BS_NOT_SPD = 5,     // CG: p^T A p <= 0
};

enum BatchDouble {
  BD_RZ_OLD = 0, BD_RZ = 1, BD_BETA = 2, BD_PQ = 3, BD_ALPHA = 4, BD_RR = 5, BD_BN = 6,
  BD_TOL = 7, BD_INNER = 8, BD_BETA0 = 9, BD_COUNT = 10
};

enum BatchInt {
  BI_STATE = 0, BI_FRESH = 1, BI_ITERS = 2, BI_MAXIT = 3, BI_CYCLE = 4, BI_JDONE = 5,
  BI_COUNT = 6
};

// level 0 of the FP16-block V-cycle: A and w D^-1 in FP16 blocks with one
// FP32 scale per block (square bs x bs blocks), FP32 vectors
cudaError_t launch_bmv_h16(int mode, int n_brows, int bs, const int *rp, const int *col,
                           const __half *val, const float *scale, const float *X, const float *B,
                           float *Y, int K, cudaStream_t s);
cudaError_t launch_bjacobi_h16(int mode, int n, int bs, const int *rp, const int *col,
                               const __half *A, const float *ascale, const __half *W,
                               const float *wscale, const float *X, const float *B, float *Xo,
                               int K, cudaStream_t s);

// nnzb: stored blocks of the matrix (picks the long-row variant)
template <typename T>
cudaError_t launch_bmv(int mode, int n_brows, int br, int bc, const int *rp, const int *col,
                       const T *val, const T *X, const T *B, T *Y, int K, cudaStream_t s,
                       int64_t nnzb);
template <typename T>
cudaError_t launch_bjacobi(int mode, int n, int bs, const int *rp, const int *col, const T *A,
                           const T *W, const T *X, const T *B, T *Xo, int K, cudaStream_t s,
                           int64_t nnzb);
// X = Ainv B for a dense row-major nc x nc Ainv with row pitch ld (>= nc; 0 = nc)
template <typename T>
cudaError_t launch_bdense(int nc, const double *Ainv, const T *B, T *X, int K, cudaStream_t s,
                          int ld = 0);

cudaError_t launch_bdot(int64_t n, const double *X, const double *Y, double *part, int K,
                        cudaStream_t s);
cudaError_t launch_bfinalize(const double *part, double *out, int K, cudaStream_t s);
cudaError_t launch_bnorm(const double *part, double *out, int K, cudaStream_t s);
cudaError_t launch_bnormalize(int64_t n, const double *w, const double *nrm, double *v, int K,
                              cudaStream_t s);

cudaError_t launch_bcg_beta(const double *part_rz, const double *part_rzo, double *sc,
                            const int *st, int flex, int K, cudaStream_t s);
cudaError_t launch_bcg_update_p(int64_t n, double *p, const double *z, double *zold,
                                const double *sc, int K, cudaStream_t s);
cudaError_t launch_bcg_alpha(const double *part_pq, double *sc, const int *st, int K,
                             cudaStream_t s);
cudaError_t launch_bcg_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                                 const double *sc, double *part_rr, int K, cudaStream_t s);
cudaError_t launch_bcg_check(const double *part_rr, double *sc, int *st, int *ctl, int flex,
                             cudaGraphConditionalHandle h, int K, cudaStream_t s);

// GMRES: the Arnoldi step j is read from device memory (*dj)
cudaError_t launch_bgm_load(int64_t nk, const double *base, int64_t ld, const int *dj, int off,
                            double *dst, cudaStream_t s);
cudaError_t launch_bgm_store(int64_t nk, const double *src, double *base, int64_t ld, const int *dj,
                             int off, cudaStream_t s);
cudaError_t launch_bmulti_dot(int64_t n, const double *V, int64_t ldv, int max_k, const int *dj,
                              const double *w, double *part, int K, cudaStream_t s);
cudaError_t launch_bmulti_finalize(const double *part, int m, const int *dj, double *h, double *H,
                                   int accumulate, int K, cudaStream_t s);
cudaError_t launch_bgs_update(int64_t n, const double *V, int64_t ldv, const int *dj, const double *h,
                              double *w, int K, cudaStream_t s);
cudaError_t launch_bgm_norm(const double *part, int m, const int *dj, double *H, int K,
                            cudaStream_t s);
cudaError_t launch_bgm_normalize(int64_t n, const double *w, const double *H, int m, const int *dj,
                                 double *V, int K, cudaStream_t s);
cudaError_t launch_bgm_start(int m, const double *beta, double *g, double *sc, int *st, int flex,
                             int *dj, int K, cudaStream_t s);
cudaError_t launch_bgm_givens(int m, double *H, double *cs, double *sn, double *g, double *sc,
                              int *st, int *dj, cudaGraphConditionalHandle h, int K, cudaStream_t s);
cudaError_t launch_bgm_backsolve(int m, const double *H, const double *g, double *y, const int *st,
                                 int K, cudaStream_t s);
cudaError_t launch_bgm_combine(int64_t n, const double *Bv, int64_t ldb, const double *y,
                               const int *st, double *x, int K, cudaStream_t s);
cudaError_t launch_bgm_check(const double *part_rr, double *sc, int *st, int K, cudaStream_t s);

template <typename T>
cudaError_t launch_bscatter(int64_t n, int K, int c, const T *src, T *dst, cudaStream_t s);
template <typename T>
cudaError_t launch_bgather(int64_t n, int K, int c, const T *src, T *dst, cudaStream_t s);
cudaError_t launch_bcolcopy(int64_t n, int K, int c, const double *src, double *dst,
                            cudaStream_t s);
// B (n x K interleaved) = columns c0 .. c0 + K - 1 of the n x n identity
cudaError_t launch_bunit_columns(int n, int K, int c0, double *B, cudaStream_t s);

}  // namespace gasa
