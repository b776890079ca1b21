// Kernels over a batch of K right-hand sides stored interleaved: entry i of
// column c lives at i * K + c (K = 1, 2, 4 or 8).  Used by the request server
// to run the V-cycle (Alg. 2) and the outer Krylov loop on several solves of
// one mesh at once, so every matrix block is read once per batch.
//
// Determinism: every output of column c is computed from column c's data
// alone, in an order that depends neither on the other columns nor on c, and
// reductions use a fixed grid and a fixed tree per column.  A solve therefore
// gives the same bits whether it runs alone or in a batch, in any slot and at
// any batch width K.
#include <algorithm>

#include "batch.h"
#include "common.cuh"

namespace gasa {

namespace {

constexpr int kThreads = 256;

// K consecutive values (one entry of every column) as vector loads
template <typename T, int K>
__device__ __forceinline__ void load_k(const T *p, T (&v)[K]) {
  constexpr int W = (K * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : K;
  using V = typename VecOf<T, W>::type;
#pragma unroll
  for (int c = 0; c < K; c += W) {
    const V t = __ldg(reinterpret_cast<const V *>(p + c));
    const T *tt = reinterpret_cast<const T *>(&t);
#pragma unroll
    for (int w = 0; w < W; ++w) v[c + w] = tt[w];
  }
}

// sum over the blocks [beg, end) of scalar row r of A X, all K columns, in
// block order; one thread
template <typename T, int K>
__device__ __forceinline__ void row_dot_k(int beg, int end, int r, int br, int bc,
                                          const int *__restrict__ col, const T *__restrict__ val,
                                          const T *__restrict__ X, T (&acc)[K]) {
  for (int kb = beg; kb < end; ++kb) {
    const int j = __ldg(col + kb);
    const T *a = val + ((size_t)kb * br + r) * bc;
    const T *x = X + (size_t)j * bc * K;
    for (int q = 0; q < bc; ++q) {
      const T av = __ldg(a + q);
      T xv[K];
      load_k<T, K>(x + (size_t)q * K, xv);
#pragma unroll
      for (int c = 0; c < K; ++c) acc[c] = fma(av, xv[c], acc[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// block SpMV over K columns: Y = A X, Y += A X or Y = B - A X.  Short rows:
// one thread per scalar row computes all K columns (each matrix value is
// read once per batch); long rows (coarse levels): one warp per scalar row.
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void store_row(int mode, size_t row, const T (&acc)[K],
                                          const T *__restrict__ B, T *__restrict__ Y) {
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const size_t e = row * K + c;
    T out;
    if (mode == GASA_MV_RESIDUAL) out = B[e] - acc[c];
    else if (mode == GASA_MV_ADD) out = Y[e] + acc[c];
    else out = acc[c];
    Y[e] = out;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads)
bmv_kernel(int mode, int64_t n_rows, int br, int bc, const int *__restrict__ rp,
           const int *__restrict__ col, const T *__restrict__ val, const T *__restrict__ X,
           const T *__restrict__ B, T *__restrict__ Y) {
  const int64_t row = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (row >= n_rows) return;
  const int i = (int)(row / br);
  const int r = (int)(row - (int64_t)i * br);
  T acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = T(0);
  row_dot_k<T, K>(__ldg(rp + i), __ldg(rp + i + 1), r, br, bc, col, val, X, acc);
  store_row<T, K>(mode, (size_t)row, acc, B, Y);
}

template <typename T, int K>
__device__ __forceinline__ void row_dot_k_strided(int beg, int end, int r, int br, int bc,
                                                  int lane, const int *__restrict__ col,
                                                  const T *__restrict__ val,
                                                  const T *__restrict__ X, T (&acc)[K]) {
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = T(0);
  for (int kb = beg + lane; kb < end; kb += 32) {
    const int j = __ldg(col + kb);
    const T *a = val + ((size_t)kb * br + r) * bc;
    const T *x = X + (size_t)j * bc * K;
    for (int q = 0; q < bc; ++q) {
      const T av = __ldg(a + q);
      T xv[K];
      load_k<T, K>(x + (size_t)q * K, xv);
#pragma unroll
      for (int c = 0; c < K; ++c) acc[c] = fma(av, xv[c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = warp_sum(acc[c]);
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads)
bmv_warp_kernel(int mode, int64_t n_rows, int br, int bc, const int *__restrict__ rp,
                const int *__restrict__ col, const T *__restrict__ val, const T *__restrict__ X,
                const T *__restrict__ B, T *__restrict__ Y) {
  const int64_t row = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int i = (int)(row / br);
  const int r = (int)(row - (int64_t)i * br);
  T acc[K];
  row_dot_k_strided<T, K>(__ldg(rp + i), __ldg(rp + i + 1), r, br, bc, lane, col, val, X, acc);
  if (lane == 0) store_row<T, K>(mode, (size_t)row, acc, B, Y);
}

// ---------------------------------------------------------------------------
// block-Jacobi step over K columns (Alg. 1): Xo = X + W (B - A X), or
// Xo = W B for the first step from zero.  A CTA owns whole block rows; the
// residuals of a block row (all K columns) go through shared memory.  Short
// rows: one thread per scalar row; long rows: one warp per scalar row.
// ---------------------------------------------------------------------------
template <typename T, int K, bool WARP>
__global__ void __launch_bounds__(kThreads)
bjacobi_kernel(int mode, int n, int bs, int rows_cta, const int *__restrict__ rp,
               const int *__restrict__ col, const T *__restrict__ A, const T *__restrict__ W,
               const T *__restrict__ X, const T *__restrict__ B, T *__restrict__ Xo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *res = reinterpret_cast<T *>(smem_raw);          // [rows_cta * bs][K]
  const int i0 = blockIdx.x * rows_cta;
  const int nrow = rows_cta * bs;
  const int lane = threadIdx.x & 31;
  const int step = WARP ? (int)(blockDim.x >> 5) : (int)blockDim.x;
  for (int t = WARP ? (int)(threadIdx.x >> 5) : (int)threadIdx.x; t < nrow; t += step) {
    const int li = t / bs, r = t - li * bs;
    const int i = i0 + li;
    T v[K];
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = T(0);
    if (i < n) {
      const size_t g = ((size_t)i * bs + r) * K;
      if (mode == JAC_SWEEP) {
        T acc[K];
        if (WARP) {
          row_dot_k_strided<T, K>(__ldg(rp + i), __ldg(rp + i + 1), r, bs, bs, lane, col, A, X, acc);
        } else {
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c] = T(0);
          row_dot_k<T, K>(__ldg(rp + i), __ldg(rp + i + 1), r, bs, bs, col, A, X, acc);
        }
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = B[g + c] - acc[c];
      } else {
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = B[g + c];
      }
    }
    if (!WARP || lane == 0) {
#pragma unroll
      for (int c = 0; c < K; ++c) res[(size_t)t * K + c] = v[c];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) {
    const int li = t / bs, r = t - li * bs;
    const int i = i0 + li;
    if (i >= n) continue;
    const T *w = W + ((size_t)i * bs + r) * bs;
    const T *rl = res + (size_t)li * bs * K;
    T out[K];
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = T(0);
    for (int q = 0; q < bs; ++q) {
      const T wv = __ldg(w + q);
#pragma unroll
      for (int c = 0; c < K; ++c) out[c] = fma(wv, rl[q * K + c], out[c]);
    }
    const size_t g = ((size_t)i * bs + r) * K;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      T o = out[c];
      if (mode == JAC_SWEEP) o += X[g + c];
      Xo[g + c] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// Level 0 of the FP16-block V-cycle over K columns: every stored block of A
// and of w D^{-1} holds FP16 values v / s with one FP32 scale s per block.
// Values are widened on load, each block's partial row sum is formed in
// FP32 and joins the row by fma(s, partial, acc), in block order, as in the
// single-solve FP16 kernels; every column is summed on its own.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void row_dot_k_h16(int beg, int end, int r, int bs,
                                              const int *__restrict__ col,
                                              const __half *__restrict__ val,
                                              const float *__restrict__ scale,
                                              const float *__restrict__ X, float (&acc)[K]) {
  for (int kb = beg; kb < end; ++kb) {
    const int j = __ldg(col + kb);
    const __half *a = val + ((size_t)kb * bs + r) * bs;
    const float *x = X + (size_t)j * bs * K;
    float part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.f;
    for (int q = 0; q < bs; ++q) {
      const float av = __half2float(a[q]);
      float xv[K];
      load_k<float, K>(x + (size_t)q * K, xv);
#pragma unroll
      for (int c = 0; c < K; ++c) part[c] = fmaf(av, xv[c], part[c]);
    }
    const float sc = __ldg(scale + kb);
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = fmaf(sc, part[c], acc[c]);
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
bmv_h16_kernel(int mode, int64_t n_rows, int bs, const int *__restrict__ rp,
               const int *__restrict__ col, const __half *__restrict__ val,
               const float *__restrict__ scale, const float *__restrict__ X,
               const float *__restrict__ B, float *__restrict__ Y) {
  const int64_t row = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (row >= n_rows) return;
  const int i = (int)(row / bs);
  const int r = (int)(row - (int64_t)i * bs);
  float acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.f;
  row_dot_k_h16<K>(__ldg(rp + i), __ldg(rp + i + 1), r, bs, col, val, scale, X, acc);
  store_row<float, K>(mode, (size_t)row, acc, B, Y);
}

template <int K>
__global__ void __launch_bounds__(kThreads)
bjacobi_h16_kernel(int mode, int n, int bs, int rows_cta, const int *__restrict__ rp,
                   const int *__restrict__ col, const __half *__restrict__ A,
                   const float *__restrict__ ascale, const __half *__restrict__ W,
                   const float *__restrict__ wscale, const float *__restrict__ X,
                   const float *__restrict__ B, float *__restrict__ Xo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *res = reinterpret_cast<float *>(smem_raw);     // [rows_cta * bs][K]
  const int i0 = blockIdx.x * rows_cta;
  const int nrow = rows_cta * bs;
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) {
    const int li = t / bs, r = t - li * bs;
    const int i = i0 + li;
    float v[K];
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = 0.f;
    if (i < n) {
      const size_t g = ((size_t)i * bs + r) * K;
      if (mode == JAC_SWEEP) {
        float acc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = 0.f;
        row_dot_k_h16<K>(__ldg(rp + i), __ldg(rp + i + 1), r, bs, col, A, ascale, X, acc);
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = B[g + c] - acc[c];
      } else {
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = B[g + c];
      }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) res[(size_t)t * K + c] = v[c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) {
    const int li = t / bs, r = t - li * bs;
    const int i = i0 + li;
    if (i >= n) continue;
    const __half *w = W + ((size_t)i * bs + r) * bs;
    const float *rl = res + (size_t)li * bs * K;
    float out[K];
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = 0.f;
    for (int q = 0; q < bs; ++q) {
      const float wv = __half2float(w[q]);
#pragma unroll
      for (int c = 0; c < K; ++c) out[c] = fmaf(wv, rl[q * K + c], out[c]);
    }
    const float ws = __ldg(wscale + i);
    const size_t g = ((size_t)i * bs + r) * K;
    // explicit roundings: a multiply and add the compiler could fuse in some
    // instantiations of K and not in others would make a column's bits
    // depend on the batch width
#pragma unroll
    for (int c = 0; c < K; ++c) {
      float o = __fmul_rn(out[c], ws);
      if (mode == JAC_SWEEP) o = __fadd_rn(o, X[g + c]);
      Xo[g + c] = o;
    }
  }
}

// coarsest level: X = A^{-1} B with the FP64 inverse, FP64 accumulation
template <typename T, int K>
__global__ void __launch_bounds__(kThreads)
bdense_kernel(int nc, int ld, const double *__restrict__ Ainv, const T *__restrict__ B,
              T *__restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= (int64_t)nc * K) return;
  const int i = (int)(e / K), c = (int)(e - (int64_t)i * K);
  const double *a = Ainv + (size_t)i * ld;
  double acc = 0.0;
  for (int j = 0; j < nc; ++j) acc = fma(__ldg(a + j), (double)B[(size_t)j * K + c], acc);
  X[e] = (T)acc;
}

// ---------------------------------------------------------------------------
// per-column reductions on a fixed grid of kRedBlocks CTAs.  Thread t of CTA
// blk takes rows blk * 256 + t, + kRedBlocks * 256, ... for all K columns,
// then a fixed tree over the 256 threads: the partial sums of a column do not
// depend on K, on the slot or on the other columns.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void column_tree(const double (&acc)[K], double *part) {
  __shared__ double sh[K][kThreads];
#pragma unroll
  for (int c = 0; c < K; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int c = 0; c < K; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < K) part[(size_t)threadIdx.x * kRedBlocks + blockIdx.x] = sh[threadIdx.x][0];
}

// part[c * kRedBlocks + blk]: partial sums of x_c . y_c (y null: x_c . x_c)
template <int K>
__global__ void __launch_bounds__(kThreads)
bdot_kernel(int64_t n, const double *__restrict__ X, const double *__restrict__ Y,
            double *__restrict__ part) {
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double x = X[i * K + c];
      acc[c] = fma(x, Y ? Y[i * K + c] : x, acc[c]);
    }
  }
  column_tree<K>(acc, part);
}

// out[c] = sum of the kRedBlocks partials of column c, in index order
__device__ __forceinline__ double sum_partials(const double *p) {
  double v = 0.0;
  for (int b = 0; b < kRedBlocks; ++b) v += p[b];
  return v;
}

template <int K>
__global__ void bfinalize_kernel(const double *__restrict__ part, double *__restrict__ out) {
  const int c = threadIdx.x;
  if (c < K) out[c] = sum_partials(part + (size_t)c * kRedBlocks);
}

// out[c] = sqrt(sum of the partials of column c)
template <int K>
__global__ void bnorm_kernel(const double *__restrict__ part, double *__restrict__ out) {
  const int c = threadIdx.x;
  if (c < K) out[c] = sqrt(sum_partials(part + (size_t)c * kRedBlocks));
}

// v_c = w_c / nrm[c] (zero when the norm is zero)
template <int K>
__global__ void __launch_bounds__(kThreads)
bnormalize_kernel(int64_t nk, const double *__restrict__ w, const double *__restrict__ nrm,
                  double *__restrict__ v) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= nk) return;
  const double d = nrm[e % K];
  v[e] = d > 0.0 ? w[e] / d : 0.0;
}

// ---------------------------------------------------------------------------
// batched CG (flexible when flex = 1): one iteration in the order
//   z = M r; rz; beta; p = z + beta p; q = A p; pq; alpha; x, r update; check
// ---------------------------------------------------------------------------
template <int K>
__global__ void bcg_beta_kernel(const double *__restrict__ part_rz, const double *__restrict__ part_rzo,
                                double *__restrict__ sc, const int *__restrict__ st, int flex) {
  const int c = threadIdx.x;
  if (c >= K) return;
  const double rz = sum_partials(part_rz + (size_t)c * kRedBlocks);
  double beta = 0.0;
  if (st[BI_STATE * K + c] == BS_RUNNING && !st[BI_FRESH * K + c]) {
    const double num = flex ? rz - sum_partials(part_rzo + (size_t)c * kRedBlocks) : rz;
    beta = num / sc[BD_RZ_OLD * K + c];
  }
  sc[BD_RZ * K + c] = rz;
  sc[BD_BETA * K + c] = beta;
}

template <int K>
__global__ void __launch_bounds__(kThreads)
bcg_update_p_kernel(int64_t nk, double *__restrict__ p, const double *__restrict__ z,
                    double *__restrict__ zold, const double *__restrict__ sc) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= nk) return;
  const int c = (int)(e % K);
  const double zv = z[e];
  p[e] = fma(sc[BD_BETA * K + c], p[e], zv);
  if (zold) zold[e] = zv;
}

template <int K>
__global__ void bcg_alpha_kernel(const double *__restrict__ part_pq, double *__restrict__ sc,
                                 const int *__restrict__ st) {
  const int c = threadIdx.x;
  if (c >= K) return;
  const double pq = sum_partials(part_pq + (size_t)c * kRedBlocks);
  sc[BD_PQ * K + c] = pq;
  const bool run = st[BI_STATE * K + c] == BS_RUNNING;
  sc[BD_ALPHA * K + c] = (run && pq != 0.0 && isfinite(pq)) ? sc[BD_RZ * K + c] / pq : 0.0;
}

// x += alpha p; r -= alpha q; partial sums of r_c . r_c
template <int K>
__global__ void __launch_bounds__(kThreads)
bcg_update_xr_kernel(int64_t n, double *__restrict__ x, double *__restrict__ r,
                     const double *__restrict__ p, const double *__restrict__ q,
                     const double *__restrict__ sc, double *__restrict__ part_rr) {
  double a[K], acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    a[c] = sc[BD_ALPHA * K + c];
    acc[c] = 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const int64_t e = i * K + c;
      x[e] = fma(a[c], p[e], x[e]);
      const double rv = fma(-a[c], q[e], r[e]);
      r[e] = rv;
      acc[c] = fma(rv, rv, acc[c]);
    }
  }
  column_tree<K>(acc, part_rr);
}

// per-column stopping test; ctl[0] counts iterations of this launch, ctl[1]
// caps them, ctl[2] is set when a column leaves the running state
template <int K>
__global__ void bcg_check_kernel(const double *__restrict__ part_rr, double *__restrict__ sc,
                                 int *__restrict__ st, int *__restrict__ ctl, int flex,
                                 cudaGraphConditionalHandle h) {
  __shared__ int changed, running;
  if (threadIdx.x == 0) {
    changed = 0;
    running = 0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < K) {
    const double rr = sum_partials(part_rr + (size_t)c * kRedBlocks);
    sc[BD_RR * K + c] = rr;
    int s = st[BI_STATE * K + c];
    if (s == BS_RUNNING) {
      const int it = ++st[BI_ITERS * K + c];
      st[BI_FRESH * K + c] = 0;
      sc[BD_RZ_OLD * K + c] = sc[BD_RZ * K + c];
      const double pq = sc[BD_PQ * K + c];
      if (!isfinite(rr) || !isfinite(pq)) s = BS_BREAKDOWN;
      else if (!flex && !(pq > 0.0)) s = BS_NOT_SPD;
      else if (sqrt(rr) <= sc[BD_TOL * K + c] * sc[BD_BN * K + c]) s = BS_CONVERGED;
      else if (it >= st[BI_MAXIT * K + c]) s = BS_MAXIT;
      if (s != BS_RUNNING) {
        st[BI_STATE * K + c] = s;
        atomicExch(&changed, 1);
      } else {
        atomicExch(&running, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int loops = ++ctl[0];
    if (changed) ctl[2] = 1;
    const bool more = !changed && running && loops < ctl[1];
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// batched GMRES pieces (classical Gram-Schmidt twice, Givens rotations).  The
// Arnoldi step j lives in device memory (*dj) so that one captured step,
// repeated by a conditional while node, serves every j.  H is (m+1) x m per
// column, entry (i, j) at (j * (m + 1) + i) * K + c; basis vector i at
// V + i * ldv.
// ---------------------------------------------------------------------------
// dst = src_base + (*dj + off) * ld  (copy of one basis vector)
__global__ void __launch_bounds__(kThreads)
bgm_load_kernel(int64_t nk, const double *__restrict__ base, int64_t ld, const int *__restrict__ dj,
                int off, double *__restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e < nk) dst[e] = base[(size_t)(*dj + off) * ld + e];
}

__global__ void __launch_bounds__(kThreads)
bgm_store_kernel(int64_t nk, const double *__restrict__ src, double *__restrict__ base, int64_t ld,
                 const int *__restrict__ dj, int off) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e < nk) base[(size_t)(*dj + off) * ld + e] = src[e];
}

// part[(i * K + c) * kRedBlocks + blk] for basis vectors i <= j
template <int K>
__global__ void __launch_bounds__(kThreads)
bmulti_dot_kernel(int64_t n, const double *__restrict__ V, int64_t ldv, const int *__restrict__ dj,
                  const double *__restrict__ w, double *__restrict__ part) {
  const int i = blockIdx.y;
  if (i > *dj) return;
  const double *v = V + (size_t)i * ldv;
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = fma(v[t * K + c], w[t * K + c], acc[c]);
  }
  column_tree<K>(acc, part + (size_t)i * K * kRedBlocks);
}

// h[i * K + c] = sum of partials; H(i, j) = h (pass 0) or += h (pass 1)
template <int K>
__global__ void bmulti_finalize_kernel(const double *__restrict__ part, int m, const int *__restrict__ dj,
                                       double *__restrict__ h, double *__restrict__ H, int accumulate) {
  const int j = *dj;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (j + 1) * K) return;
  const double v = sum_partials(part + (size_t)t * kRedBlocks);
  h[t] = v;
  double *Hj = H + (size_t)j * (m + 1) * K;
  Hj[t] = accumulate ? Hj[t] + v : v;
}

// w_c -= sum_{i <= j} h[i, c] v_i,c (i in index order)
template <int K>
__global__ void __launch_bounds__(kThreads)
bgs_update_kernel(int64_t nk, const double *__restrict__ V, int64_t ldv, const int *__restrict__ dj,
                  const double *__restrict__ h, double *__restrict__ w) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= nk) return;
  const int c = (int)(e % K);
  const int k = *dj + 1;
  double acc = w[e];
  for (int i = 0; i < k; ++i) acc = fma(-h[i * K + c], V[(size_t)i * ldv + e], acc);
  w[e] = acc;
}

// H(j+1, j) = ||w_c||
template <int K>
__global__ void bgm_norm_kernel(const double *__restrict__ part, int m, const int *__restrict__ dj,
                                double *__restrict__ H) {
  const int c = threadIdx.x;
  if (c >= K) return;
  const int j = *dj;
  H[((size_t)j * (m + 1) + j + 1) * K + c] = sqrt(sum_partials(part + (size_t)c * kRedBlocks));
}

// v_{j+1} = w / H(j+1, j) (zero when the norm is zero)
template <int K>
__global__ void __launch_bounds__(kThreads)
bgm_normalize_kernel(int64_t nk, const double *__restrict__ w, const double *__restrict__ H, int m,
                     const int *__restrict__ dj, double *__restrict__ V) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= nk) return;
  const int j = *dj;
  const int c = (int)(e % K);
  const double d = H[((size_t)j * (m + 1) + j + 1) * K + c];
  V[(size_t)(j + 1) * nk + e] = d > 0.0 ? w[e] / d : 0.0;
}

// Cycle start (one thread per column): g = (beta, 0, ...), the inner
// tolerance on a fresh start, whether the column takes part, j = 0.
template <int K>
__global__ void bgm_start_kernel(int m, const double *__restrict__ beta, double *__restrict__ g,
                                 double *__restrict__ sc, int *__restrict__ st, int flex,
                                 int *__restrict__ dj) {
  const int c = threadIdx.x;
  if (c == 0) *dj = 0;
  if (c >= K) return;
  for (int i = 0; i <= m; ++i) g[i * K + c] = 0.0;
  const bool run = st[BI_STATE * K + c] == BS_RUNNING;
  int cyc = run ? 1 : 0;     // 1: iterating, 0: not in this cycle, 2: done with it
  st[BI_JDONE * K + c] = 0;
  if (run) {
    const double b = beta[c];
    g[c] = b;
    if (st[BI_FRESH * K + c]) {
      sc[BD_INNER * K + c] = sc[BD_TOL * K + c] * (flex ? sc[BD_BN * K + c] : b);
      st[BI_FRESH * K + c] = 0;
    }
    if (!(b > 0.0)) cyc = 0;
  }
  st[BI_CYCLE * K + c] = cyc;
}

// Givens step j for every column still iterating; advances j and sets the
// while condition (some column iterating and j < m)
template <int K>
__global__ void bgm_givens_kernel(int m, double *__restrict__ H, double *__restrict__ cs,
                                  double *__restrict__ sn, double *__restrict__ g,
                                  double *__restrict__ sc, int *__restrict__ st, int *__restrict__ dj,
                                  cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int j = *dj;
  const int c = threadIdx.x;
  if (c < K && st[BI_CYCLE * K + c] == 1) {
    const int ld = m + 1;
    double *Hj = H + (size_t)j * ld * K;
    for (int i = 0; i < j; ++i) {
      const double a = Hj[i * K + c], b = Hj[(i + 1) * K + c];
      const double ci = cs[i * K + c], si = sn[i * K + c];
      Hj[i * K + c] = ci * a + si * b;
      Hj[(i + 1) * K + c] = -si * a + ci * b;
    }
    const double a = Hj[j * K + c], b = Hj[(j + 1) * K + c];
    const double d = hypot(a, b);
    const double cj = d > 0.0 ? a / d : 1.0, sj = d > 0.0 ? b / d : 0.0;
    cs[j * K + c] = cj;
    sn[j * K + c] = sj;
    Hj[j * K + c] = d;
    Hj[(j + 1) * K + c] = 0.0;
    const double gj = g[j * K + c];
    g[j * K + c] = cj * gj;
    g[(j + 1) * K + c] = -sj * gj;
    const int it = ++st[BI_ITERS * K + c];
    // a zero pivot (exact breakdown) keeps the step out of the update
    st[BI_JDONE * K + c] = d > 0.0 ? j + 1 : j;
    const double gres = fabs(g[(j + 1) * K + c]);
    if (!isfinite(gres)) {
      st[BI_CYCLE * K + c] = 0;
      st[BI_STATE * K + c] = BS_BREAKDOWN;
    } else if (gres <= sc[BD_INNER * K + c] || it >= st[BI_MAXIT * K + c] || !(d > 0.0)) {
      st[BI_CYCLE * K + c] = 2;
    } else {
      atomicExch(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *dj = j + 1;
    cudaGraphSetConditional(h, (any && j + 1 < m) ? 1u : 0u);
  }
}

// y = R^{-1} g over the column's own step count
template <int K>
__global__ void bgm_backsolve_kernel(int m, const double *__restrict__ H, const double *__restrict__ g,
                                     double *__restrict__ y, const int *__restrict__ st) {
  const int c = threadIdx.x;
  if (c >= K) return;
  const int jd = st[BI_CYCLE * K + c] ? st[BI_JDONE * K + c] : 0;
  const int ld = m + 1;
  for (int i = jd - 1; i >= 0; --i) {
    double v = g[i * K + c];
    for (int l = i + 1; l < jd; ++l) v -= H[((size_t)l * ld + i) * K + c] * y[l * K + c];
    y[i * K + c] = v / H[((size_t)i * ld + i) * K + c];
  }
}

// x_c += sum_{i < jdone_c} y_i B_i,c
template <int K>
__global__ void __launch_bounds__(kThreads)
bgm_combine_kernel(int64_t nk, const double *__restrict__ Bv, int64_t ldb,
                   const double *__restrict__ y, const int *__restrict__ st, double *__restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= nk) return;
  const int c = (int)(e % K);
  const int jd = st[BI_CYCLE * K + c] ? st[BI_JDONE * K + c] : 0;
  double acc = x[e];
  for (int i = 0; i < jd; ++i) acc = fma(y[i * K + c], Bv[(size_t)i * ldb + e], acc);
  x[e] = acc;
}

// after the cycle: the true residual decides (one thread per column)
template <int K>
__global__ void bgm_check_kernel(const double *__restrict__ part_rr, double *__restrict__ sc,
                                 int *__restrict__ st) {
  const int c = threadIdx.x;
  if (c >= K) return;
  const double rr = sum_partials(part_rr + (size_t)c * kRedBlocks);
  sc[BD_RR * K + c] = rr;
  if (st[BI_STATE * K + c] != BS_RUNNING) return;
  if (!isfinite(rr)) st[BI_STATE * K + c] = BS_BREAKDOWN;
  else if (sqrt(rr) <= sc[BD_TOL * K + c] * sc[BD_BN * K + c]) st[BI_STATE * K + c] = BS_CONVERGED;
  else if (st[BI_ITERS * K + c] >= st[BI_MAXIT * K + c]) st[BI_STATE * K + c] = BS_MAXIT;
}

// ---------------------------------------------------------------------------
// slot traffic: scatter a contiguous vector into column c, gather it back,
// fill a column
// ---------------------------------------------------------------------------
template <typename T>
__global__ void bscatter_kernel(int64_t n, int K, int c, const T *__restrict__ src, T *__restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) dst[i * K + c] = src ? src[i] : T(0);
}

template <typename T>
__global__ void bgather_kernel(int64_t n, int K, int c, const T *__restrict__ src, T *__restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) dst[i] = src[i * K + c];
}

template <typename T>
__global__ void bcolcopy_kernel(int64_t n, int K, int c, const T *__restrict__ src, T *__restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) dst[i * K + c] = src[i * K + c];
}

// B (n x K interleaved) = columns c0 .. c0 + K - 1 of the n x n identity
// (columns past n are zero)
__global__ void bunit_columns_kernel(int n, int K, int c0, double *__restrict__ B) {
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= (int64_t)n * K) return;
  const int64_t i = t / K, c = t - i * K;
  B[t] = (i == c0 + c) ? 1.0 : 0.0;
}

// X = A B for a dense row-major n x n FP64 A and K interleaved columns, FP64
// arithmetic: a warp per row, lane l takes columns j = l, l + 32, ... of the
// row in order (four rows of B in flight), then an xor-shuffle tree; a
// column's sum does not depend on K
template <typename T, int K>
__global__ void __launch_bounds__(kThreads)
bdense_warp_kernel(int n, int ld, const double *__restrict__ A, const T *__restrict__ B,
                   T *__restrict__ X) {
  const int row = (int)(((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double *a = A + (size_t)row * ld;
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  int j = lane;
  for (; j + 96 < n; j += 128) {
    const double a0 = __ldg(a + j), a1 = __ldg(a + j + 32), a2 = __ldg(a + j + 64),
                 a3 = __ldg(a + j + 96);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      acc[c] = fma(a0, (double)__ldg(B + (size_t)j * K + c), acc[c]);
      acc[c] = fma(a1, (double)__ldg(B + (size_t)(j + 32) * K + c), acc[c]);
      acc[c] = fma(a2, (double)__ldg(B + (size_t)(j + 64) * K + c), acc[c]);
      acc[c] = fma(a3, (double)__ldg(B + (size_t)(j + 96) * K + c), acc[c]);
    }
  }
  for (; j < n; j += 32) {
    const double a0 = __ldg(a + j);
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = fma(a0, (double)__ldg(B + (size_t)j * K + c), acc[c]);
  }
#pragma unroll
  for (int c = 0; c < K; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) X[(size_t)row * K + c] = (T)acc[c];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define GASA_KSWITCH(K, ...)                       \
  switch (K) {                                     \
    case 1: { constexpr int KK = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int KK = 2; __VA_ARGS__; } break; \
    case 4: { constexpr int KK = 4; __VA_ARGS__; } break; \
    case 8: { constexpr int KK = 8; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;         \
  }

// long rows (coarse levels, >= 16 blocks per block row on average) take the
// warp variants; the choice depends on the matrix only, never on K, so a
// column's bits do not depend on the batch width
static bool long_rows(int n_brows, int64_t nnzb) { return nnzb >= 16 * (int64_t)n_brows; }

template <typename T>
cudaError_t launch_bmv(int mode, int n_brows, int br, int bc, const int *rp, const int *col,
                       const T *val, const T *X, const T *B, T *Y, int K, cudaStream_t s,
                       int64_t nnzb) {
  const int64_t rows = (int64_t)n_brows * br;
  if (rows == 0) return cudaSuccess;
  if (long_rows(n_brows, nnzb)) {
    GASA_KSWITCH(K, launch_k(bmv_warp_kernel<T, KK>, div_up(rows * 32, kThreads), kThreads, 0, s,
                             mode, rows, br, bc, rp, col, val, X, B, Y));
  } else {
    GASA_KSWITCH(K, launch_k(bmv_kernel<T, KK>, div_up(rows, kThreads), kThreads, 0, s,
                             mode, rows, br, bc, rp, col, val, X, B, Y));
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bjacobi(int mode, int n, int bs, const int *rp, const int *col, const T *A,
                           const T *W, const T *X, const T *B, T *Xo, int K, cudaStream_t s,
                           int64_t nnzb) {
  if (n == 0) return cudaSuccess;
  const bool warp = mode == JAC_SWEEP && long_rows(n, nnzb);
  const int rows_cta = warp ? 1 : std::max(1, kThreads / bs);
  const size_t smem = (size_t)rows_cta * bs * K * sizeof(T);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  if (warp) {
    GASA_KSWITCH(K, launch_k(bjacobi_kernel<T, KK, true>, div_up(n, rows_cta), kThreads, smem, s,
                             mode, n, bs, rows_cta, rp, col, A, W, X, B, Xo));
  } else {
    GASA_KSWITCH(K, launch_k(bjacobi_kernel<T, KK, false>, div_up(n, rows_cta), kThreads, smem, s,
                             mode, n, bs, rows_cta, rp, col, A, W, X, B, Xo));
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bmv_h16(int mode, int n_brows, int bs, const int *rp, const int *col,
                           const __half *val, const float *scale, const float *X, const float *B,
                           float *Y, int K, cudaStream_t s) {
  const int64_t rows = (int64_t)n_brows * bs;
  if (rows == 0) return cudaSuccess;
  GASA_KSWITCH(K, launch_k(bmv_h16_kernel<KK>, div_up(rows, kThreads), kThreads, 0, s, mode, rows,
                           bs, rp, col, val, scale, X, B, Y));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bjacobi_h16(int mode, int n, int bs, const int *rp, const int *col,
                               const __half *A, const float *ascale, const __half *W,
                               const float *wscale, const float *X, const float *B, float *Xo,
                               int K, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int rows_cta = std::max(1, kThreads / bs);
  const size_t smem = (size_t)rows_cta * bs * K * sizeof(float);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  GASA_KSWITCH(K, launch_k(bjacobi_h16_kernel<KK>, div_up(n, rows_cta), kThreads, smem, s, mode,
                           n, bs, rows_cta, rp, col, A, ascale, W, wscale, X, B, Xo));
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bdense(int nc, const double *Ainv, const T *B, T *X, int K, cudaStream_t s,
                          int ld) {
  const int64_t tot = (int64_t)nc * K;
  if (ld < nc) ld = nc;
  // orders of 128 and more (the dense bottom of the V-cycle) take a warp per row
  if (nc >= 128) {
    GASA_KSWITCH(K, launch_k(bdense_warp_kernel<T, KK>, div_up((int64_t)nc * 32, kThreads),
                             kThreads, 0, s, nc, ld, Ainv, B, X));
  } else {
    GASA_KSWITCH(K, launch_k(bdense_kernel<T, KK>, div_up(tot, kThreads), kThreads, 0, s, nc, ld,
                             Ainv, B, X));
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bdot(int64_t n, const double *X, const double *Y, double *part, int K,
                        cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bdot_kernel<KK>, kRedBlocks, kThreads, 0, s, n, X, Y, part));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bfinalize(const double *part, double *out, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bfinalize_kernel<KK>, 1, 32, 0, s, part, out));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bnorm(const double *part, double *out, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bnorm_kernel<KK>, 1, 32, 0, s, part, out));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bnormalize(int64_t n, const double *w, const double *nrm, double *v, int K,
                              cudaStream_t s) {
  const int64_t nk = n * K;
  GASA_KSWITCH(K, launch_k(bnormalize_kernel<KK>, div_up(nk, kThreads), kThreads, 0, s, nk, w, nrm, v));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcg_beta(const double *part_rz, const double *part_rzo, double *sc,
                            const int *st, int flex, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bcg_beta_kernel<KK>, 1, 32, 0, s, part_rz, part_rzo, sc, st, flex));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcg_update_p(int64_t n, double *p, const double *z, double *zold,
                                const double *sc, int K, cudaStream_t s) {
  const int64_t nk = n * K;
  GASA_KSWITCH(K, launch_k(bcg_update_p_kernel<KK>, div_up(nk, kThreads), kThreads, 0, s, nk, p, z, zold, sc));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcg_alpha(const double *part_pq, double *sc, const int *st, int K,
                             cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bcg_alpha_kernel<KK>, 1, 32, 0, s, part_pq, sc, st));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcg_update_xr(int64_t n, double *x, double *r, const double *p, const double *q,
                                 const double *sc, double *part_rr, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bcg_update_xr_kernel<KK>, kRedBlocks, kThreads, 0, s, n, x, r, p, q, sc, part_rr));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcg_check(const double *part_rr, double *sc, int *st, int *ctl, int flex,
                             cudaGraphConditionalHandle h, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bcg_check_kernel<KK>, 1, 32, 0, s, part_rr, sc, st, ctl, flex, h));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_load(int64_t nk, const double *base, int64_t ld, const int *dj, int off,
                            double *dst, cudaStream_t s) {
  launch_k(bgm_load_kernel, div_up(nk, kThreads), kThreads, 0, s, nk, base, ld, dj, off, dst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_store(int64_t nk, const double *src, double *base, int64_t ld, const int *dj,
                             int off, cudaStream_t s) {
  launch_k(bgm_store_kernel, div_up(nk, kThreads), kThreads, 0, s, nk, src, base, ld, dj, off);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bmulti_dot(int64_t n, const double *V, int64_t ldv, int max_k, const int *dj,
                              const double *w, double *part, int K, cudaStream_t s) {
  dim3 grid(kRedBlocks, max_k);
  GASA_KSWITCH(K, launch_k(bmulti_dot_kernel<KK>, grid, kThreads, 0, s, n, V, ldv, dj, w, part));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bmulti_finalize(const double *part, int m, const int *dj, double *h, double *H,
                                   int accumulate, int K, cudaStream_t s) {
  const int tot = (m + 1) * K;
  GASA_KSWITCH(K, launch_k(bmulti_finalize_kernel<KK>, div_up(tot, 64), 64, 0, s, part, m, dj, h, H, accumulate));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgs_update(int64_t n, const double *V, int64_t ldv, const int *dj, const double *h,
                              double *w, int K, cudaStream_t s) {
  const int64_t nk = n * K;
  GASA_KSWITCH(K, launch_k(bgs_update_kernel<KK>, div_up(nk, kThreads), kThreads, 0, s, nk, V, ldv, dj, h, w));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_norm(const double *part, int m, const int *dj, double *H, int K,
                            cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bgm_norm_kernel<KK>, 1, 32, 0, s, part, m, dj, H));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_normalize(int64_t n, const double *w, const double *H, int m, const int *dj,
                                 double *V, int K, cudaStream_t s) {
  const int64_t nk = n * K;
  GASA_KSWITCH(K, launch_k(bgm_normalize_kernel<KK>, div_up(nk, kThreads), kThreads, 0, s, nk, w, H, m, dj, V));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_start(int m, const double *beta, double *g, double *sc, int *st, int flex,
                             int *dj, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bgm_start_kernel<KK>, 1, 32, 0, s, m, beta, g, sc, st, flex, dj));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_givens(int m, double *H, double *cs, double *sn, double *g, double *sc,
                              int *st, int *dj, cudaGraphConditionalHandle h, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bgm_givens_kernel<KK>, 1, 32, 0, s, m, H, cs, sn, g, sc, st, dj, h));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_backsolve(int m, const double *H, const double *g, double *y, const int *st,
                                 int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bgm_backsolve_kernel<KK>, 1, 32, 0, s, m, H, g, y, st));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_combine(int64_t n, const double *Bv, int64_t ldb, const double *y,
                               const int *st, double *x, int K, cudaStream_t s) {
  const int64_t nk = n * K;
  GASA_KSWITCH(K, launch_k(bgm_combine_kernel<KK>, div_up(nk, kThreads), kThreads, 0, s, nk, Bv, ldb, y, st, x));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bgm_check(const double *part_rr, double *sc, int *st, int K, cudaStream_t s) {
  GASA_KSWITCH(K, launch_k(bgm_check_kernel<KK>, 1, 32, 0, s, part_rr, sc, st));
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bscatter(int64_t n, int K, int c, const T *src, T *dst, cudaStream_t s) {
  launch_k(bscatter_kernel<T>, div_up(n, kThreads), kThreads, 0, s, n, K, c, src, dst);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bgather(int64_t n, int K, int c, const T *src, T *dst, cudaStream_t s) {
  launch_k(bgather_kernel<T>, div_up(n, kThreads), kThreads, 0, s, n, K, c, src, dst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bunit_columns(int n, int K, int c0, double *B, cudaStream_t s) {
  if (n <= 0 || K <= 0) return cudaSuccess;
  launch_k(bunit_columns_kernel, div_up((int64_t)n * K, kThreads), kThreads, 0, s, n, K, c0, B);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bcolcopy(int64_t n, int K, int c, const double *src, double *dst,
                            cudaStream_t s) {
  launch_k(bcolcopy_kernel<double>, div_up(n, kThreads), kThreads, 0, s, n, K, c, src, dst);
  note_launch();
  return cudaGetLastError();
}

#define GASA_INST_T(T)                                                                          \
  template cudaError_t launch_bmv<T>(int, int, int, int, const int *, const int *, const T *,   \
                                     const T *, const T *, T *, int, cudaStream_t, int64_t);    \
  template cudaError_t launch_bjacobi<T>(int, int, int, const int *, const int *, const T *,    \
                                         const T *, const T *, const T *, T *, int,             \
                                         cudaStream_t, int64_t);                                \
  template cudaError_t launch_bdense<T>(int, const double *, const T *, T *, int, cudaStream_t,  \
                                        int);                                                   \
  template cudaError_t launch_bscatter<T>(int64_t, int, int, const T *, T *, cudaStream_t);     \
  template cudaError_t launch_bgather<T>(int64_t, int, int, const T *, T *, cudaStream_t);
GASA_INST_T(double)
GASA_INST_T(float)
#undef GASA_INST_T

}  // namespace gasa
