// Setup kernels of Alg. 5: block-Jacobi inverses (Section 4.4), per-aggregate
// SVD building the tentative prolongator (Eq. splitB_dg, Eq. sik), the
// smoothed prolongator P = T - w D^{-1} A T and R = P^T (Eq. TR0), the
// Galerkin product A_{k+1} = R (A P), and the coarsest dense inverse.
//
// Every product is a gather over a sorted structural pattern: one CTA owns
// one output block row, each thread owns fixed entries of the output block,
// and the summation order over the inner index is the pattern order, so the
// results are reproducible run to run and need no atomics on values.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gasa {

// ----------------------------------------------------------------------------
// small helpers: max, exclusive scan (single CTA, chunked), block flag scan
// ----------------------------------------------------------------------------
__global__ void max_int_kernel(int n, const int *__restrict__ x, int *out) {
  int v = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v = max(v, x[i]);
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

cudaError_t launch_max_int(int n, const int *x, int *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (e != cudaSuccess || n == 0) return e;
  max_int_kernel<<<kNumSM, 256, 0, s>>>(n, x, out); note_launch();
  return cudaGetLastError();
}

// returns the exclusive prefix of `flag` over the block, `total` the block sum
__device__ int block_scan_flag(int flag, int *sh, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  const int pre = __popc(m & ((1u << lane) - 1u));
  __syncthreads();
  if (lane == 0) sh[wid] = __popc(m);
  __syncthreads();
  if (wid == 0) {
    int v = lane < nw ? sh[lane] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane < nw) sh[lane] = inc - v;
    if (lane == 31) sh[32] = inc;
  }
  __syncthreads();
  const int res = sh[wid] + pre;
  total = sh[32];
  __syncthreads();
  return res;
}

// out[i] = sum_{k<i} in[k], out[n] = total (single CTA, 1024 threads)
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(int n, const int *__restrict__ in,
                                                              int *__restrict__ out) {
  __shared__ int sh[33];
  __shared__ int sv[1024];
  int base = 0;
  for (int c = 0; c < n; c += 1024) {
    const int i = c + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    sv[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan in shared memory
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? sv[threadIdx.x - o] : 0;
      __syncthreads();
      sv[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) out[i] = base + sv[threadIdx.x] - v;
    const int tot = sv[1023];
    __syncthreads();
    base += tot;
  }
  if (threadIdx.x == 0) out[n] = base;
  (void)sh;
}

cudaError_t launch_exclusive_scan(int n, const int *in, int *out, int *scratch, cudaStream_t s) {
  (void)scratch;
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(n, in, out); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// block-Jacobi inverses: W = scale * D^{-1}, Gauss-Jordan with partial
// pivoting on [D | I] in shared memory, one CTA per diagonal block.
// ----------------------------------------------------------------------------
__global__ void block_inverse_kernel(int n_units, int bs, const int *__restrict__ rp,
                                     const int *__restrict__ col, const double *__restrict__ val,
                                     double scale, double *__restrict__ W, int *n_singular) {
  extern __shared__ double M[];   // bs x 2bs, then bs factors
  __shared__ int piv;
  __shared__ int sing;
  const int u = blockIdx.x;
  if (u >= n_units) return;
  const int w2 = 2 * bs;
  double *f = M + (size_t)bs * w2;
  // locate the diagonal block (columns sorted)
  if (threadIdx.x == 0) {
    int lo = rp[u], hi = rp[u + 1] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = col[mid];
      if (c == u) { pos = mid; break; }
      if (c < u) lo = mid + 1; else hi = mid - 1;
    }
    piv = pos;
    sing = 0;
  }
  __syncthreads();
  const int pos = piv;
  double amax = 0.0;
  for (int e = threadIdx.x; e < bs * w2; e += blockDim.x) {
    const int i = e / w2, j = e - i * w2;
    double v;
    if (j < bs) v = pos >= 0 ? val[(size_t)pos * bs * bs + i * bs + j] : 0.0;
    else v = (j - bs == i) ? 1.0 : 0.0;
    M[e] = v;
    if (j < bs) amax = fmax(amax, fabs(v));
  }
  __shared__ double shm[32];
  amax = warp_max(amax);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmax(m, shm[w]);
    shm[0] = m;
  }
  __syncthreads();
  const double thresh = shm[0] * 1e-14 + 1e-300;
  for (int k = 0; k < bs; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(M[k * w2 + k]);
      for (int i = k + 1; i < bs; ++i) {
        const double a = fabs(M[i * w2 + k]);
        if (a > best) { best = a; p = i; }
      }
      piv = p;
      if (best <= thresh) sing = 1;
    }
    __syncthreads();
    if (sing) break;
    const int p = piv;
    if (p != k) {
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const double t = M[k * w2 + j];
        M[k * w2 + j] = M[p * w2 + j];
        M[p * w2 + j] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / M[k * w2 + k];
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) M[k * w2 + j] *= inv;
    for (int i = threadIdx.x; i < bs; i += blockDim.x) f[i] = (i == k) ? 0.0 : M[i * w2 + k];
    __syncthreads();
    for (int e = threadIdx.x; e < bs * w2; e += blockDim.x) {
      const int i = e / w2, j = e - i * w2;
      if (i != k) M[e] = fma(-f[i], M[k * w2 + j], M[e]);
    }
    __syncthreads();
  }
  double *out = W + (size_t)u * bs * bs;
  if (sing) {
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) out[e] = 0.0;
    if (threadIdx.x == 0) atomicAdd(n_singular, 1);
    return;
  }
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int i = e / bs, j = e - i * bs;
    out[e] = scale * M[i * w2 + bs + j];
  }
}

cudaError_t launch_block_inverse(int n_units, int bs, const int *rp, const int *col,
                                 const double *val, double scale, double *W, int *n_singular,
                                 cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
  const size_t sm = ((size_t)bs * 2 * bs + bs) * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(block_inverse_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int th = bs <= 8 ? 64 : (bs <= 24 ? 128 : 256);
  block_inverse_kernel<<<n_units, th, sm, s>>>(n_units, bs, rp, col, val, scale, W, n_singular); note_launch();
  return cudaGetLastError();
}

__global__ void scale_kernel(int64_t n, double a, double *x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] *= a;
}
// WA = W A with W block diagonal: block k of block row i becomes W_i A_k
// (bs x bs times bs x bs, FP64); one CTA per block row, threads over the
// row's block entries
__global__ void __launch_bounds__(256)
fold_block_rows_kernel(int bs, const int *__restrict__ rp, const double *__restrict__ W,
                       const double *__restrict__ A, double *__restrict__ WA) {
  const int i = blockIdx.x;
  const int beg = rp[i], end = rp[i + 1];
  const int bb = bs * bs;
  const double *w = W + (size_t)i * bb;
  const int64_t tot = (int64_t)(end - beg) * bb;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int64_t k = beg + e / bb;
    const int rc = (int)(e % bb), r = rc / bs, c = rc - r * bs;
    const double *a = A + (size_t)k * bb;
    double acc = 0.0;
    for (int q = 0; q < bs; ++q) acc = fma(w[r * bs + q], a[q * bs + c], acc);
    WA[(size_t)k * bb + rc] = acc;
  }
}

cudaError_t launch_fold_block_rows(int n_units, int bs, const int *rp, const double *W,
                                   const double *A, double *WA, cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
  launch_k(fold_block_rows_kernel, n_units, 256, 0, s, bs, rp, W, A, WA);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(int64_t n, double a, double *x, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  scale_kernel<<<kRedBlocks * 2, 256, 0, s>>>(n, a, x); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// children of every aggregate, sorted by unit id
// ----------------------------------------------------------------------------
__global__ void count_children_kernel(int n_units, const int *__restrict__ agg, int *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_units; i += gridDim.x * blockDim.x)
    atomicAdd(cnt + agg[i], 1);
}
__global__ void fill_children_kernel(int n_units, const int *__restrict__ agg,
                                     const int *__restrict__ ptr, int *fillc, int *idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_units; i += gridDim.x * blockDim.x) {
    const int a = agg[i];
    const int slot = atomicAdd(fillc + a, 1);
    idx[ptr[a] + slot] = i;
  }
}
__global__ void sort_segments_kernel(int n_seg, const int *__restrict__ ptr, int *idx) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_seg; a += gridDim.x * blockDim.x) {
    const int b = ptr[a], e = ptr[a + 1];
    for (int i = b + 1; i < e; ++i) {
      const int v = idx[i];
      int j = i - 1;
      while (j >= b && idx[j] > v) { idx[j + 1] = idx[j]; --j; }
      idx[j + 1] = v;
    }
  }
}

cudaError_t build_children(int n_units, int n_agg, const int *agg_of, int *child_ptr,
                           int *child_idx, int *scratch, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * n_agg, s);
  if (e != cudaSuccess) return e;
  count_children_kernel<<<kRedBlocks, 256, 0, s>>>(n_units, agg_of, scratch); note_launch();
  if ((e = launch_exclusive_scan(n_agg, scratch, child_ptr, nullptr, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(scratch, 0, sizeof(int) * n_agg, s)) != cudaSuccess) return e;
  fill_children_kernel<<<kRedBlocks, 256, 0, s>>>(n_units, agg_of, child_ptr, scratch, child_idx); note_launch();
  sort_segments_kernel<<<div_up(n_agg, 128), 128, 0, s>>>(n_agg, child_ptr, child_idx); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// tentative prolongator: one-sided (Hestenes) Jacobi SVD of each aggregate's
// rows of B.  Column pairs are visited in round-robin order, one warp per
// pair; a sweep repeats until no pair needs a rotation.  Left singular
// vectors are the converged columns divided by their norms.
// ----------------------------------------------------------------------------
__global__ void tentative_kernel(int bs, const int *__restrict__ child_ptr,
                                 const int *__restrict__ child_idx, const double *__restrict__ B,
                                 int64_t ldb, int r, int s_next, double *__restrict__ T,
                                 double *__restrict__ sigma, int *status,
                                 const int *__restrict__ unit_size, const int *__restrict__ keep) {
  extern __shared__ double G[];    // rows x r, column-major (ld = rows)
  __shared__ int rotated;
  __shared__ int order[256];
  __shared__ double sv[256];
  __shared__ int rows_real_s;
  const int J = blockIdx.x;
  const int c0 = child_ptr[J], nch = child_ptr[J + 1] - c0;
  const int rows = nch * bs;
  // padded levels: unit u holds unit_size[u] real dofs followed by zeros, and
  // this aggregate keeps keep[J] columns of its s_next (the rest are zero)
  if (threadIdx.x == 0) {
    int rr = rows;
    if (unit_size) {
      rr = 0;
      for (int ch = 0; ch < nch; ++ch) rr += unit_size[child_idx[c0 + ch]];
    }
    rows_real_s = rr;
  }
  const int sJ = keep ? keep[J] : s_next;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  // gather B rows of the aggregate
  for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
    const int c = e / rows, q = e - c * rows;
    const int ch = q / bs, d = q - ch * bs;
    const int unit = child_idx[c0 + ch];
    G[e] = B[(size_t)c * ldb + (size_t)unit * bs + d];
  }
  __syncthreads();
  const int rows_real = rows_real_s;
  const int m = (r + 1) & ~1;        // even number of players (one dummy if r is odd)
  const double tol = 2.220446049250313e-16 * (double)rows;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int t = 0; t < m - 1; ++t) {
      for (int k = wid; k < m / 2; k += nwarps) {
        const int a = (k == 0) ? 0 : ((k - 1 + t) % (m - 1)) + 1;
        const int b = ((m - 1 - k - 1 + t) % (m - 1)) + 1;
        int p = min(a, b), q = max(a, b);
        if (q >= r) continue;   // dummy player
        double *gp = G + (size_t)p * rows, *gq = G + (size_t)q * rows;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < rows; i += 32) {
          const double x = gp[i], y = gq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt);
          const double sn = cs * tt;
          for (int i = lane; i < rows; i += 32) {
            const double x = gp[i], y = gq[i];
            gp[i] = cs * x - sn * y;
            gq[i] = sn * x + cs * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // singular values (column norms) and descending order, ties by column index
  for (int c = wid; c < r; c += nwarps) {
    double a = 0.0;
    const double *gc = G + (size_t)c * rows;
    for (int i = lane; i < rows; i += 32) a = fma(gc[i], gc[i], a);
    a = warp_sum(a);
    if (lane == 0) sv[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    int rank = 0;
    const double s0 = sv[c];
    for (int d = 0; d < r; ++d) {
      const double s1 = sv[d];
      if (s1 > s0 || (s1 == s0 && d < c)) ++rank;
    }
    order[rank] = c;
  }
  __syncthreads();
  if (sigma) {
    for (int l = threadIdx.x; l < r; l += blockDim.x)
      sigma[(size_t)J * r + l] = (l < rows_real) ? sv[order[l]] : 0.0;
  }
  // Singular values at or below kNullSigma * sigma_1 are numerically zero:
  // their vectors carry rounding noise, not candidate information.
  constexpr double kNullSigma = 1e-10;
  const double snull = kNullSigma * sv[order[0]];
  // normalise the kept columns with nonzero singular value
  for (int l = wid; l < sJ; l += nwarps) {
    const int c = order[l];
    const double sc = sv[c];
    if (l < rows_real && sc > snull) {
      const double inv = 1.0 / sc;
      double *gc = G + (size_t)c * rows;
      for (int i = lane; i < rows; i += 32) gc[i] *= inv;
    }
  }
  __syncthreads();
  // the others (candidate block of lower numerical rank than the kept count)
  // are replaced, in order, by unit vectors e_t (t = l, l+1, ... cyclically)
  // orthogonalised twice against the columns already fixed, the first with
  // norm above 1/2 being kept
  if (wid == 0) {
    for (int l = 0; l < sJ && l < rows_real; ++l) {
      const int c = order[l];
      if (sv[c] > snull) continue;
      double *gc = G + (size_t)c * rows;
      bool done = false;
      for (int t = 0; t < rows_real && !done; ++t) {
        // the (l + t)-th real row, in the aggregate's padded row numbering
        int e = (l + t) % rows_real;
        if (unit_size) {
          int ch = 0;
          while (e >= unit_size[child_idx[c0 + ch]]) e -= unit_size[child_idx[c0 + ch++]];
          e += ch * bs;
        }
        for (int i = lane; i < rows; i += 32) gc[i] = (i == e) ? 1.0 : 0.0;
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int m = 0; m < l; ++m) {
            const double *gm = G + (size_t)order[m] * rows;
            double d = 0.0;
            for (int i = lane; i < rows; i += 32) d = fma(gm[i], gc[i], d);
            d = warp_sum(d);
            for (int i = lane; i < rows; i += 32) gc[i] = fma(-d, gm[i], gc[i]);
            __syncwarp();
          }
        }
        double nn = 0.0;
        for (int i = lane; i < rows; i += 32) nn = fma(gc[i], gc[i], nn);
        nn = warp_sum(nn);
        if (nn > 0.25) {
          const double inv = 1.0 / sqrt(nn);
          for (int i = lane; i < rows; i += 32) gc[i] *= inv;
          done = true;
        }
        __syncwarp();
      }
      if (!done && lane == 0) atomicExch(status, 1);
      if (lane == 0) sv[c] = -1.0;   // marks a completed column (kept as zero singular value)
      __syncwarp();
    }
  }
  __syncthreads();
  // sign so that the largest |entry| (lowest row on ties) is positive, then write
  for (int l = wid; l < s_next; l += nwarps) {
    if (l >= sJ) {   // padding column of this aggregate
      for (int i = lane; i < rows; i += 32) {
        const int ch = i / bs, d = i - ch * bs;
        T[((size_t)child_idx[c0 + ch] * bs + d) * s_next + l] = 0.0;
      }
      continue;
    }
    const int c = order[l];
    const bool ok = (l < rows_real);
    double best = -1.0;
    int bi = INT_MAX;
    const double *gc = G + (size_t)c * rows;
    for (int i = lane; i < rows; i += 32) {
      const double a = fabs(gc[i]);
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const double sgn = (ok && bi < rows && gc[bi] < 0.0) ? -1.0 : 1.0;
    const double scl = ok ? sgn : 0.0;
    for (int i = lane; i < rows; i += 32) {
      const int ch = i / bs, d = i - ch * bs;
      const int unit = child_idx[c0 + ch];
      T[((size_t)unit * bs + d) * s_next + l] = gc[i] * scl;
    }
    if (!ok && lane == 0) atomicExch(status, 1);
  }
}

// Padded level: the Galerkin product leaves the padding rows and columns of
// A zero; put 1 on their diagonal so that the block inverses exist.  The
// padding then stays exactly zero through every smoothing step.
__global__ void pad_identity_kernel(int n_units, int s, const int *__restrict__ usize,
                                    const int *__restrict__ rp, const int *__restrict__ col,
                                    double *__restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_units) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    if (col[k] != i) continue;
    double *d = val + (size_t)k * s * s;
    for (int l = usize[i]; l < s; ++l) d[(size_t)l * s + l] = 1.0;
  }
}

cudaError_t launch_pad_identity(int n_units, int s_pad, const int *usize, const int *rp,
                                const int *col, double *val, cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
  pad_identity_kernel<<<div_up(n_units, 128), 128, 0, s>>>(n_units, s_pad, usize, rp, col, val);
  note_launch();
  return cudaGetLastError();
}

// shared memory holds the largest aggregate's rows x r block of B
cudaError_t launch_tentative(int bs, int n_agg, int max_children, const int *child_ptr,
                                   const int *child_idx, const double *B, int64_t ldb, int r,
                                   int s_next, double *T, double *sigma, int *status,
                                   cudaStream_t s, const int *unit_size, const int *keep) {
  if (n_agg == 0) return cudaSuccess;
  const size_t sm = (size_t)max_children * bs * r * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(tentative_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int pairs = (r + 1) / 2;
  int th = 32 * (pairs < 8 ? (pairs < 1 ? 1 : pairs) : 8);
  tentative_kernel<<<n_agg, th, sm, s>>>(bs, child_ptr, child_idx, B, ldb, r, s_next, T, sigma,
                                         status, unit_size, keep); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// structural patterns: sorted unique candidate lists per row (bitonic sort in
// shared memory, flag-scan compaction)
// ----------------------------------------------------------------------------
__device__ int sort_unique(int *buf, int ncap, int *shscan) {
  for (int k = 2; k <= ncap; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < ncap; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const int a = buf[i], b = buf[ixj];
          if ((a > b) == up) { buf[i] = b; buf[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  // compaction in place, chunk by chunk (writes never overtake reads)
  int base = 0;
  for (int c = 0; c < ncap; c += blockDim.x) {
    const int i = c + threadIdx.x;
    int v = INT_MAX;
    int flag = 0;
    if (i < ncap) {
      v = buf[i];
      flag = (v != INT_MAX) && (i == 0 || buf[i - 1] != v);
    }
    int total;
    const int pre = block_scan_flag(flag, shscan, total);
    if (flag) buf[base + pre] = v;
    base += total;
    __syncthreads();
  }
  return base;
}

__device__ __forceinline__ int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// P pattern: row i -> unique agg[j], j in A(i)
__global__ void pattern_P_kernel(int n, const int *__restrict__ Arp, const int *__restrict__ Acol,
                                 const int *__restrict__ agg, int *count,
                                 const int *__restrict__ Prp, int *Pcol, int ncap) {
  extern __shared__ int buf[];
  __shared__ int shscan[33];
  const int i = blockIdx.x;
  const int b = Arp[i], e = Arp[i + 1];
  for (int t = threadIdx.x; t < ncap; t += blockDim.x) buf[t] = (t < e - b) ? agg[Acol[b + t]] : INT_MAX;
  __syncthreads();
  const int u = sort_unique(buf, ncap, shscan);
  if (count && threadIdx.x == 0) count[i] = u;
  if (Pcol) for (int t = threadIdx.x; t < u; t += blockDim.x) Pcol[Prp[i] + t] = buf[t];
}

// C = A B pattern: row i -> unique B(col) for col in A(i)
__global__ void pattern_AB_kernel(int n, const int *__restrict__ Arp, const int *__restrict__ Acol,
                                  const int *__restrict__ Brp, const int *__restrict__ Bcol,
                                  int *count, const int *__restrict__ Crp, int *Ccol, int ncap) {
  extern __shared__ int buf[];
  __shared__ int shscan[33];
  __shared__ int fill;
  const int i = blockIdx.x;
  if (threadIdx.x == 0) fill = 0;
  for (int t = threadIdx.x; t < ncap; t += blockDim.x) buf[t] = INT_MAX;
  __syncthreads();
  const int b = Arp[i], e = Arp[i + 1];
  int off = 0;
  for (int k = b; k < e; ++k) {
    const int j = Acol[k];
    const int bb = Brp[j], be = Brp[j + 1];
    for (int t = threadIdx.x; t < be - bb; t += blockDim.x) buf[off + t] = Bcol[bb + t];
    off += be - bb;
  }
  __syncthreads();
  (void)fill;
  const int u = sort_unique(buf, ncap, shscan);
  if (count && threadIdx.x == 0) count[i] = u;
  if (Ccol) for (int t = threadIdx.x; t < u; t += blockDim.x) Ccol[Crp[i] + t] = buf[t];
}

// ----------------------------------------------------------------------------
// Long candidate lists (coarse Galerkin rows can collect tens of thousands of
// candidates): a bitmap over the ncols output columns in shared memory; set
// bits are then written out in column order, which sorts and de-duplicates
// at once.  mode 0: C = pattern(A) x agg (P's pattern); mode 1: C = A B.
// ----------------------------------------------------------------------------
__device__ int block_scan_int(int v, int *sh, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int w = lane < nw ? sh[lane] : 0;
    int winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    if (lane < nw) sh[lane] = winc - w;
    if (lane == 31) sh[32] = winc;
  }
  __syncthreads();
  const int res = sh[wid] + inc - v;
  total = sh[32];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(256)
pattern_bitmap_kernel(int n, int mode, int ncols, const int *__restrict__ Arp,
                      const int *__restrict__ Acol, const int *__restrict__ Brp,
                      const int *__restrict__ Bcol_or_agg, int *count,
                      const int *__restrict__ Crp, int *Ccol) {
  extern __shared__ unsigned bits[];
  __shared__ int sh[33];
  const int nwords = (ncols + 31) >> 5;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  const int i = blockIdx.x;
  const int b = Arp[i], e = Arp[i + 1];
  if (mode == 0) {
    for (int k = b + threadIdx.x; k < e; k += blockDim.x) {
      const int c = Bcol_or_agg[Acol[k]];
      atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
  } else {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int k = b + wid; k < e; k += nwarp) {
      const int j = Acol[k];
      for (int q = Brp[j] + lane; q < Brp[j + 1]; q += 32) {
        const int c = Bcol_or_agg[q];
        atomicOr(&bits[c >> 5], 1u << (c & 31));
      }
    }
  }
  __syncthreads();
  int base = 0;
  for (int w0 = 0; w0 < nwords; w0 += blockDim.x) {
    const int w = w0 + threadIdx.x;
    unsigned word = w < nwords ? bits[w] : 0u;
    int total;
    const int pre = block_scan_int(__popc(word), sh, total);
    if (Ccol) {
      int pos = Crp[i] + base + pre;
      while (word) {
        const int bit = __ffs(word) - 1;
        Ccol[pos++] = (w << 5) + bit;
        word &= word - 1u;
      }
    }
    base += total;
  }
  if (count && threadIdx.x == 0) count[i] = base;
}

static cudaError_t launch_pattern_bitmap(int n, int mode, int ncols, const int *Arp,
                                         const int *Acol, const int *Brp, const int *Bcol_or_agg,
                                         int *count, const int *Crp, int *Ccol, cudaStream_t s) {
  const size_t sm = (size_t)((ncols + 31) / 32) * sizeof(unsigned);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(pattern_bitmap_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sm, 1));
  if (e != cudaSuccess) return e;
  pattern_bitmap_kernel<<<n, 256, sm, s>>>(n, mode, ncols, Arp, Acol, Brp, Bcol_or_agg, count, Crp, Ccol); note_launch();
  return cudaGetLastError();
}

__global__ void cand_count_AB_kernel(int n, const int *__restrict__ Arp, const int *__restrict__ Acol,
                                     const int *__restrict__ Brp, int *cand) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = 0;
    for (int k = Arp[i]; k < Arp[i + 1]; ++k) {
      const int j = Acol[k];
      c += Brp[j + 1] - Brp[j];
    }
    cand[i] = c;
  }
}

cudaError_t launch_cand_count_AB(int n, const int *Arp, const int *Acol, const int *Brp, int *cand,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cand_count_AB_kernel<<<div_up(n, 256), 256, 0, s>>>(n, Arp, Acol, Brp, cand); note_launch();
  return cudaGetLastError();
}

static cudaError_t set_smem(const void *f, size_t sm) {
  if (sm <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

static int host_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// candidate lists up to kSortCap entries are sorted in shared memory, longer
// ones go through the column bitmap
constexpr int kSortCap = 4096;

cudaError_t launch_pattern_P(int n, const int *Arp, const int *Acol, const int *agg, int *count,
                             const int *Prp, int *Pcol, int max_cand, int ncols, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (max_cand > kSortCap)
    return launch_pattern_bitmap(n, 0, ncols, Arp, Acol, nullptr, agg, count, Prp, Pcol, s);
  const int ncap = host_pow2(max_cand < 1 ? 1 : max_cand);
  const size_t sm = (size_t)ncap * sizeof(int);
  cudaError_t e = set_smem((const void *)pattern_P_kernel, sm);
  if (e != cudaSuccess) return e;
  pattern_P_kernel<<<n, 128, sm, s>>>(n, Arp, Acol, agg, count, Prp, Pcol, ncap); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pattern_AB(int n, const int *Arp, const int *Acol, const int *Brp,
                              const int *Bcol, int *count, const int *Crp, int *Ccol, int max_cand,
                              int ncols, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (max_cand > kSortCap)
    return launch_pattern_bitmap(n, 1, ncols, Arp, Acol, Brp, Bcol, count, Crp, Ccol, s);
  const int ncap = host_pow2(max_cand < 1 ? 1 : max_cand);
  const size_t sm = (size_t)ncap * sizeof(int);
  cudaError_t e = set_smem((const void *)pattern_AB_kernel, sm);
  if (e != cudaSuccess) return e;
  const int th = ncap >= 1024 ? 512 : 128;
  pattern_AB_kernel<<<n, th, sm, s>>>(n, Arp, Acol, Brp, Bcol, count, Crp, Ccol, ncap); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// numeric products
// ----------------------------------------------------------------------------
__device__ __forceinline__ int find_col(const int *__restrict__ cols, int b, int e, int key) {
  int lo = b, hi = e - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = cols[mid];
    if (c == key) return mid;
    if (c < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// P_iJ = [agg(i) = J] T_i - W_i sum_{j in A(i), agg(j) = J} A_ij T_j
__global__ void numeric_P_kernel(int n, int sk, int sn, const int *__restrict__ Arp,
                                 const int *__restrict__ Acol, const double *__restrict__ Aval,
                                 const double *__restrict__ Wm, const double *__restrict__ T,
                                 const int *__restrict__ agg, const int *__restrict__ Prp,
                                 const int *__restrict__ Pcol, double *__restrict__ Pval) {
  extern __shared__ double AT[];   // sk x sn
  const int i = blockIdx.x;
  const int ab = Arp[i], ae = Arp[i + 1];
  const int ne = sk * sn;
  const int gi = agg[i];
  for (int pk = Prp[i]; pk < Prp[i + 1]; ++pk) {
    const int J = Pcol[pk];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int rr = e / sn, cc = e - rr * sn;
      double acc = 0.0;
      for (int k = ab; k < ae; ++k) {
        const int j = Acol[k];
        if (agg[j] != J) continue;
        const double *a = Aval + ((size_t)k * sk + rr) * sk;
        const double *tj = T + (size_t)j * sk * sn + cc;
        for (int m = 0; m < sk; ++m) acc = fma(a[m], tj[(size_t)m * sn], acc);
      }
      AT[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int rr = e / sn, cc = e - rr * sn;
      const double *w = Wm + ((size_t)i * sk + rr) * sk;
      double acc = 0.0;
      for (int m = 0; m < sk; ++m) acc = fma(w[m], AT[m * sn + cc], acc);
      const double tv = (gi == J) ? T[(size_t)i * sk * sn + e] : 0.0;
      Pval[(size_t)pk * ne + e] = tv - acc;
    }
    __syncthreads();
  }
}

cudaError_t launch_numeric_P(int n, int sk, int sn, const int *Arp, const int *Acol,
                             const double *Aval, const double *W, const double *T, const int *agg,
                             const int *Prp, const int *Pcol, double *Pval, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t sm = (size_t)sk * sn * sizeof(double);
  cudaError_t e = set_smem((const void *)numeric_P_kernel, sm);
  if (e != cudaSuccess) return e;
  const int th = sk * sn <= 64 ? 64 : (sk * sn <= 256 ? 128 : 256);
  numeric_P_kernel<<<n, th, sm, s>>>(n, sk, sn, Arp, Acol, Aval, W, T, agg, Prp, Pcol, Pval); note_launch();
  return cudaGetLastError();
}

// C_iJ = sum_{k in A(i)} A_k B_{col(k), J}, blocks br x bm times bm x bc
__global__ void numeric_AB_kernel(int n, int br, int bm, int bc, const int *__restrict__ Arp,
                                  const int *__restrict__ Acol, const double *__restrict__ Aval,
                                  const int *__restrict__ Brp, const int *__restrict__ Bcol,
                                  const double *__restrict__ Bval, const int *__restrict__ Crp,
                                  const int *__restrict__ Ccol, double *__restrict__ Cval) {
  __shared__ int bpos[1024];
  const int i = blockIdx.x;
  const int ab = Arp[i], ae = Arp[i + 1];
  const int na = ae - ab;
  const int ne = br * bc;
  for (int ck = Crp[i]; ck < Crp[i + 1]; ++ck) {
    const int J = Ccol[ck];
    // locate B_{j, J} for every j in A(i) (chunks of 1024)
    for (int c0 = 0; c0 < na; c0 += 1024) {
      const int cn = min(1024, na - c0);
      for (int t = threadIdx.x; t < cn; t += blockDim.x) {
        const int j = Acol[ab + c0 + t];
        bpos[t] = find_col(Bcol, Brp[j], Brp[j + 1], J);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int rr = e / bc, cc = e - rr * bc;
        double acc = (c0 == 0) ? 0.0 : Cval[(size_t)ck * ne + e];
        for (int t = 0; t < cn; ++t) {
          const int bp = bpos[t];
          if (bp < 0) continue;
          const double *a = Aval + ((size_t)(ab + c0 + t) * br + rr) * bm;
          const double *bv = Bval + (size_t)bp * bm * bc + cc;
          for (int m = 0; m < bm; ++m) acc = fma(a[m], bv[(size_t)m * bc], acc);
        }
        Cval[(size_t)ck * ne + e] = acc;
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_numeric_AB(int n, int br, int bm, int bc, const int *Arp, const int *Acol,
                              const double *Aval, const int *Brp, const int *Bcol,
                              const double *Bval, const int *Crp, const int *Ccol, double *Cval,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int ne = br * bc;
  const int th = ne <= 64 ? 64 : (ne <= 128 ? 128 : 256);
  numeric_AB_kernel<<<n, th, 0, s>>>(n, br, bm, bc, Arp, Acol, Aval, Brp, Bcol, Bval, Crp, Ccol,
                                     Cval); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// R = P^T (explicit): counting by block column, rows sorted by source row
// ----------------------------------------------------------------------------
__global__ void tr_count_kernel(int nnzb, const int *__restrict__ Pcol, int *cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnzb; k += gridDim.x * blockDim.x)
    atomicAdd(cnt + Pcol[k], 1);
}
__global__ void tr_fill_kernel(int n_rows, const int *__restrict__ Prp, const int *__restrict__ Pcol,
                               const int *__restrict__ Rrp, int *fillc, int *Rcol, int *src) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_rows; i += gridDim.x * blockDim.x) {
    for (int k = Prp[i]; k < Prp[i + 1]; ++k) {
      const int J = Pcol[k];
      const int slot = Rrp[J] + atomicAdd(fillc + J, 1);
      Rcol[slot] = i;
      src[slot] = k;
    }
  }
}
__global__ void tr_sort_kernel(int n_seg, const int *__restrict__ ptr, int *key, int *src) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_seg; a += gridDim.x * blockDim.x) {
    const int b = ptr[a], e = ptr[a + 1];
    for (int i = b + 1; i < e; ++i) {
      const int v = key[i], w = src[i];
      int j = i - 1;
      while (j >= b && key[j] > v) { key[j + 1] = key[j]; src[j + 1] = src[j]; --j; }
      key[j + 1] = v;
      src[j + 1] = w;
    }
  }
}
__global__ void tr_values_kernel(int nnzb, int br, int bc, const int *__restrict__ src,
                                 const double *__restrict__ Pval, double *__restrict__ Rval) {
  const int ne = br * bc;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)nnzb * ne;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t / ne), e = (int)(t - (long long)k * ne);
    const int rr = e / br, cc = e - rr * br;      // R block is bc x br
    Rval[t] = Pval[(size_t)src[k] * ne + cc * bc + rr];
  }
}

cudaError_t launch_transpose(int n_rows, int n_cols, int br, int bc, const int *Prp, const int *Pcol,
                             const double *Pval, int *Rrp, int *Rcol, double *Rval, int *src,
                             int *cnt, cudaStream_t s) {
  int nnzb = 0;
  cudaError_t e = cudaMemcpyAsync(&nnzb, Prp + n_rows, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * n_cols, s)) != cudaSuccess) return e;
  if (nnzb > 0) tr_count_kernel<<<kRedBlocks, 256, 0, s>>>(nnzb, Pcol, cnt); note_launch();
  if ((e = launch_exclusive_scan(n_cols, cnt, Rrp, nullptr, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * n_cols, s)) != cudaSuccess) return e;
  tr_fill_kernel<<<div_up(n_rows, 256), 256, 0, s>>>(n_rows, Prp, Pcol, Rrp, cnt, Rcol, src); note_launch();
  tr_sort_kernel<<<div_up(n_cols, 128), 128, 0, s>>>(n_cols, Rrp, Rcol, src); note_launch();
  if (nnzb > 0)
    tr_values_kernel<<<kRedBlocks * 4, 256, 0, s>>>(nnzb, br, bc, src, Pval, Rval); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// coarsest level: BSR -> dense row-major, Gauss-Jordan inverse on [A | I]
// ----------------------------------------------------------------------------
__global__ void bsr_to_dense_kernel(int n, int bs, const int *__restrict__ rp,
                                    const int *__restrict__ col, const double *__restrict__ val,
                                    double *__restrict__ D) {
  const int i = blockIdx.x;
  const int N = n * bs;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
      const int rr = e / bs, cc = e - rr * bs;
      D[(size_t)(i * bs + rr) * N + j * bs + cc] = val[(size_t)k * bs * bs + e];
    }
  }
}

cudaError_t launch_bsr_to_dense(int n, int bs, const int *rp, const int *col, const double *val,
                                double *D, cudaStream_t s) {
  const size_t N = (size_t)n * bs;
  cudaError_t e = cudaMemsetAsync(D, 0, N * N * sizeof(double), s);
  if (e != cudaSuccess || n == 0) return e;
  bsr_to_dense_kernel<<<n, 128, 0, s>>>(n, bs, rp, col, val, D); note_launch();
  return cudaGetLastError();
}

__global__ void gj_init_kernel(int n, const double *__restrict__ A, double *__restrict__ M) {
  const long long w = 2LL * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * w;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / w, j = t - i * w;
    M[t] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  }
}

// pivot search, row swap, row scaling and multiplier capture for column k
__global__ void __launch_bounds__(1024) gj_pivot_kernel(int n, double *M, int k, double *colk,
                                                        double thresh, int *singular) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int piv;
  const long long w = 2LL * n;
  double best = -1.0;
  int idx = INT_MAX;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(M[i * w + k]);
    if (a > best) { best = a; idx = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int p = INT_MAX;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
      if (bv[q] > b || (bv[q] == b && bi[q] < p)) { b = bv[q]; p = bi[q]; }
    piv = p;
    if (!(b > thresh)) *singular = 1;
  }
  __syncthreads();
  const int p = piv;
  if (p >= n) return;
  if (p != k) {
    for (long long j = k + threadIdx.x; j < w; j += blockDim.x) {
      const double t = M[k * w + j];
      M[k * w + j] = M[p * w + j];
      M[p * w + j] = t;
    }
    __syncthreads();
  }
  const double inv = 1.0 / M[k * w + k];
  __syncthreads();
  for (long long j = k + threadIdx.x; j < w; j += blockDim.x) M[k * w + j] *= inv;
  __syncthreads();
  if (threadIdx.x == 0) M[k * w + k] = 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : M[i * w + k];
}

__global__ void gj_elim_kernel(int n, double *__restrict__ M, int k, const double *__restrict__ colk) {
  const long long w = 2LL * n;
  const long long ncol = w - k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * ncol;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / ncol);
    const long long j = k + (t - (long long)i * ncol);
    if (i == k) continue;
    const double f = colk[i];
    if (f == 0.0) continue;
    M[i * w + j] = fma(-f, M[k * w + j], M[i * w + j]);
  }
}

__global__ void gj_extract_kernel(int n, const double *__restrict__ M, double *__restrict__ Ainv) {
  const long long w = 2LL * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / n, j = t - i * n;
    Ainv[t] = M[i * w + n + j];
  }
}

cudaError_t launch_dense_inverse(int n, const double *A, double *Ainv, double *work, int *singular,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  double *M = work;                         // n x 2n
  double *colk = work + (size_t)2 * n * n;  // n
  cudaError_t e = cudaMemsetAsync(singular, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  gj_init_kernel<<<kRedBlocks * 4, 256, 0, s>>>(n, A, M); note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const double thresh = 1e-300;
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, s>>>(n, M, k, colk, thresh, singular); note_launch();
    const long long work_items = (long long)n * (2LL * n - k);
    int grid = div_up(work_items, 256);
    if (grid > kRedBlocks * 8) grid = kRedBlocks * 8;
    gj_elim_kernel<<<grid, 256, 0, s>>>(n, M, k, colk); note_launch();
  }
  gj_extract_kernel<<<kRedBlocks * 4, 256, 0, s>>>(n, M, Ainv); note_launch();
  return cudaGetLastError();
}

}  // namespace gasa
