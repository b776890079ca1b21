// Vector kernels of the outer Krylov loop and of setup: deterministic
// reductions (fixed grid, fixed order: partial sums per CTA, then one CTA
// sums the partials), fused CG updates, GMRES Arnoldi pieces, counter-based
// random vectors and precision conversions.
#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"

namespace gasa {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }


// ----------------------------------------------------------------------------
// reductions
// ----------------------------------------------------------------------------
// Streaming vector kernels read 16-byte pairs when both arrays are 16-byte
// aligned (VEC), four pairs per array in flight per thread; the pair index
// runs over a grid-stride loop and the odd last entry (if any) goes to
// thread 0 of CTA 0, so each partial sums a fixed set of entries in a fixed
// order.
__device__ __forceinline__ double2 ld2(const double *p, int64_t k) {
  return __ldg(reinterpret_cast<const double2 *>(p) + k);
}

template <bool VEC>
__global__ void __launch_bounds__(kRedThreads)
dot_partials_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                    double *__restrict__ partials) {
  __shared__ double sh[32];
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!y) y = x;
  if (VEC) {
    const int64_t m = n >> 1;
    for (; i + 3 * stride < m; i += 4 * stride) {
      const double2 a0 = ld2(x, i), a1 = ld2(x, i + stride), a2 = ld2(x, i + 2 * stride),
                    a3 = ld2(x, i + 3 * stride);
      const double2 b0 = ld2(y, i), b1 = ld2(y, i + stride), b2 = ld2(y, i + 2 * stride),
                    b3 = ld2(y, i + 3 * stride);
      v0 = fma(a0.y, b0.y, fma(a0.x, b0.x, v0));
      v1 = fma(a1.y, b1.y, fma(a1.x, b1.x, v1));
      v2 = fma(a2.y, b2.y, fma(a2.x, b2.x, v2));
      v3 = fma(a3.y, b3.y, fma(a3.x, b3.x, v3));
    }
    for (; i < m; i += stride) {
      const double2 a0 = ld2(x, i), b0 = ld2(y, i);
      v0 = fma(a0.y, b0.y, fma(a0.x, b0.x, v0));
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) v0 = fma(x[n - 1], y[n - 1], v0);
  } else {
    for (; i + 3 * stride < n; i += 4 * stride) {
      v0 = fma(x[i], y[i], v0);
      v1 = fma(x[i + stride], y[i + stride], v1);
      v2 = fma(x[i + 2 * stride], y[i + 2 * stride], v2);
      v3 = fma(x[i + 3 * stride], y[i + 3 * stride], v3);
    }
    for (; i < n; i += stride) v0 = fma(x[i], y[i], v0);
  }
  double v = (v0 + v1) + (v2 + v3);
  v = block_sum(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t launch_dot_partials(int64_t n, const double *x, const double *y, double *partials,
                                cudaStream_t s) {
  if (al16(x) && (!y || al16(y)))
    launch_k(dot_partials_kernel<true>, kRedBlocks, kRedThreads, 0, s, n, x, y, partials);
  else
    launch_k(dot_partials_kernel<false>, kRedBlocks, kRedThreads, 0, s, n, x, y, partials);
  note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
colnorm_partials_kernel(int64_t n, const double *const *__restrict__ cols,
                        double *__restrict__ partials) {
  __shared__ double sh[32];
  const double *x = cols[blockIdx.y];
  double v = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    v = fma(x[i], x[i], v);
  v = block_sum(v, sh);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = v;
}

cudaError_t launch_colnorm_partials(int64_t n, const double *const *cols, int nc,
                                    double *partials, cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  launch_k(colnorm_partials_kernel, dim3(kRedBlocks, nc), kRedThreads, 0, s, n, cols, partials); note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
finalize_kernel(const double *__restrict__ partials, double *__restrict__ out) {
  __shared__ double sh[32];
  double v = block_sum_partials(partials + (size_t)blockIdx.x * kRedBlocks, kRedBlocks, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// one sum of n partials (same order as block_sum_partials elsewhere)
__global__ void __launch_bounds__(kRedThreads)
finalize_n_kernel(const double *__restrict__ partials, int n, double *__restrict__ out) {
  __shared__ double sh[32];
  const double v = block_sum_partials(partials, n, sh);
  if (threadIdx.x == 0) out[0] = v;
}

cudaError_t launch_finalize_n(const double *partials, int n, double *out, cudaStream_t s) {
  launch_k(finalize_n_kernel, 1, kRedThreads, 0, s, partials, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int nc, double *out, cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  launch_k(finalize_kernel, nc, kRedThreads, 0, s, partials, out); note_launch();
  return cudaGetLastError();
}

__global__ void scale_inv_sqrt_kernel(int64_t n, double *x, const double *sumsq) {
  const double a = 1.0 / sqrt(sumsq[0]);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] *= a;
}

cudaError_t launch_scale_by_inv_sqrt(int64_t n, double *x, const double *sumsq, cudaStream_t s) {
  launch_k(scale_inv_sqrt_kernel, kRedBlocks, 256, 0, s, n, x, sumsq); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood 2014): draw i of (seed, stream) is
// mix(key + (i+1) * GOLDEN), key = seed ^ (stream * GOLDEN); uniform =
// (z >> 11) * 2^-53.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix_draw(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double splitmix_uniform(uint64_t key, uint64_t i) {
  return (double)(splitmix_draw(key, i) >> 11) * 0x1.0p-53;
}

__global__ void uniform_pm1_kernel(int64_t n, uint64_t key, double *x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    x[i] = 2.0 * splitmix_uniform(key, (uint64_t)i) - 1.0;
}

cudaError_t launch_uniform_pm1(int64_t n, uint64_t seed, uint64_t stream, double *x,
                               cudaStream_t s) {
  const uint64_t key = seed ^ (stream * 0x9E3779B97F4A7C15ull);
  launch_k(uniform_pm1_kernel, kRedBlocks, 256, 0, s, n, key, x); note_launch();
  return cudaGetLastError();
}

// the same vector on a padded level (unit u: usize[u] real dofs, then zeros):
// real dof number uoff[u] + l gets draw uoff[u] + l, padding gets 0
__global__ void uniform_pm1_padded_kernel(int n_units, int s, const int *__restrict__ usize,
                                          const int64_t *__restrict__ uoff, uint64_t key,
                                          double *x) {
  const int64_t n = (int64_t)n_units * s;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int u = (int)(i / s), l = (int)(i - (int64_t)u * s);
    x[i] = l < usize[u] ? 2.0 * splitmix_uniform(key, (uint64_t)(uoff[u] + l)) - 1.0 : 0.0;
  }
}

cudaError_t launch_uniform_pm1_padded(int n_units, int s_pad, const int *usize,
                                      const int64_t *uoff, uint64_t seed, uint64_t stream,
                                      double *x, cudaStream_t s) {
  const uint64_t key = seed ^ (stream * 0x9E3779B97F4A7C15ull);
  launch_k(uniform_pm1_padded_kernel, kRedBlocks, 256, 0, s, n_units, s_pad, usize, uoff, key, x);
  note_launch();
  return cudaGetLastError();
}

// Box-Muller over pairs of uniforms: u1 = 1 - U[2m], u2 = U[2m+1]
__global__ void normal_kernel(int64_t n, uint64_t key, double *x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t m = i >> 1;
    const double u1 = 1.0 - splitmix_uniform(key, (uint64_t)(2 * m));
    const double u2 = splitmix_uniform(key, (uint64_t)(2 * m + 1));
    const double rr = sqrt(-2.0 * log(u1));
    double sv, cv;
    sincospi(2.0 * u2, &sv, &cv);
    x[i] = (i & 1) ? rr * sv : rr * cv;
  }
}

cudaError_t launch_normal(int64_t n, uint64_t seed, uint64_t stream, double *x, cudaStream_t s) {
  const uint64_t key = seed ^ (stream * 0x9E3779B97F4A7C15ull);
  launch_k(normal_kernel, kRedBlocks, 256, 0, s, n, key, x); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// elementwise
// ----------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void convert_kernel(int64_t n, const Tin *__restrict__ in, Tout *__restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (Tout)in[i];
}

template <typename Tin, typename Tout>
cudaError_t launch_convert(int64_t n, const Tin *in, Tout *out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int grid = div_up(n, 256);
  if (grid > 8 * kNumSM) grid = 8 * kNumSM;
  launch_k(convert_kernel<Tin, Tout>, grid, 256, 0, s, n, in, out); note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(int64_t, const double *, float *, cudaStream_t);
template cudaError_t launch_convert<float, double>(int64_t, const float *, double *, cudaStream_t);

__global__ void fill_kernel(int64_t n, double v, double *x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = v;
}
cudaError_t launch_fill(int64_t n, double v, double *x, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_k(fill_kernel, kRedBlocks, 256, 0, s, n, v, x); note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void add_kernel(int64_t n, const T *__restrict__ x, T *__restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = y[i] + x[i];
}
template <typename T>
cudaError_t launch_add(int64_t n, const T *x, T *y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_k(add_kernel<T>, std::min<int64_t>(div_up(n, 256), kRedBlocks * 4), 256, 0, s, n, x, y);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_add<double>(int64_t, const double *, double *, cudaStream_t);
template cudaError_t launch_add<float>(int64_t, const float *, float *, cudaStream_t);

__global__ void axpy_kernel(int64_t n, double a, const double *__restrict__ x,
                            double *__restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = fma(a, x[i], y[i]);
}
cudaError_t launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_k(axpy_kernel, kRedBlocks * 2, 256, 0, s, n, a, x, y); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_copy(int64_t n, const double *x, double *y, cudaStream_t s) {
  return cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

__global__ void sub_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ o) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    o[i] = a[i] - b[i];
}
cudaError_t launch_sub(int64_t n, const double *a, const double *b, double *out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_k(sub_kernel, kRedBlocks * 2, 256, 0, s, n, a, b, out); note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// CG: x += alpha p, r -= alpha q with alpha = rz / (p.q); partial ||r||^2
// ----------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(kRedThreads)
cg_update_xr_kernel(int64_t n, double *__restrict__ x, double *__restrict__ r,
                    const double *__restrict__ p, const double *__restrict__ q,
                    const double *__restrict__ rz, const double *__restrict__ pq_partials,
                    double *__restrict__ rr_partials, double *__restrict__ alpha_out, int n_pq) {
  __shared__ double sh[32];
  const double pq = block_sum_partials(pq_partials, n_pq, sh);
  const double alpha = rz[0] / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha_out[0] = alpha;
    alpha_out[1] = pq;
  }
  double v0 = 0.0, v1 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    // pairs: two pairs of each of x, r, p, q in flight per thread
    const int64_t m = n >> 1;
    double2 *x2 = reinterpret_cast<double2 *>(x), *r2 = reinterpret_cast<double2 *>(r);
    for (; i < m; i += 2 * stride) {
      const int64_t i2 = i + stride;
      const bool two = i2 < m;
      const double2 p0 = ld2(p, i), q0 = ld2(q, i), x0 = x2[i], r0 = r2[i];
      double2 p1 = p0, q1 = q0, x1 = x0, r1 = r0;
      if (two) {
        p1 = ld2(p, i2);
        q1 = ld2(q, i2);
        x1 = x2[i2];
        r1 = r2[i2];
      }
      x2[i] = make_double2(fma(alpha, p0.x, x0.x), fma(alpha, p0.y, x0.y));
      const double2 ra = make_double2(fma(-alpha, q0.x, r0.x), fma(-alpha, q0.y, r0.y));
      r2[i] = ra;
      v0 = fma(ra.y, ra.y, fma(ra.x, ra.x, v0));
      if (two) {
        x2[i2] = make_double2(fma(alpha, p1.x, x1.x), fma(alpha, p1.y, x1.y));
        const double2 rb = make_double2(fma(-alpha, q1.x, r1.x), fma(-alpha, q1.y, r1.y));
        r2[i2] = rb;
        v1 = fma(rb.y, rb.y, fma(rb.x, rb.x, v1));
      }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      x[n - 1] = fma(alpha, p[n - 1], x[n - 1]);
      const double ri = fma(-alpha, q[n - 1], r[n - 1]);
      r[n - 1] = ri;
      v0 = fma(ri, ri, v0);
    }
  } else {
    for (; i + stride < n; i += 2 * stride) {
      const int64_t i2 = i + stride;
      const double p0 = p[i], p1 = p[i2], q0 = q[i], q1 = q[i2];
      const double x0 = x[i], x1 = x[i2], r0 = r[i], r1 = r[i2];
      x[i] = fma(alpha, p0, x0);
      x[i2] = fma(alpha, p1, x1);
      const double ra = fma(-alpha, q0, r0), rb = fma(-alpha, q1, r1);
      r[i] = ra;
      r[i2] = rb;
      v0 = fma(ra, ra, v0);
      v1 = fma(rb, rb, v1);
    }
    for (; i < n; i += stride) {
      x[i] = fma(alpha, p[i], x[i]);
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      v0 = fma(ri, ri, v0);
    }
  }
  double v = v0 + v1;
  v = block_sum(v, sh);
  if (threadIdx.x == 0) rr_partials[blockIdx.x] = v;
}

cudaError_t launch_cg_update_xr(int64_t n, double *x, double *r, const double *p,
                                const double *q, const double *rz, const double *pq_partials,
                                double *rr_partials, double *alpha_out, cudaStream_t s, int n_pq) {
  if (al16(x) && al16(r) && al16(p) && al16(q))
    launch_k(cg_update_xr_kernel<true>, kRedBlocks, kRedThreads, 0, s, n, x, r, p, q, rz,
             pq_partials, rr_partials, alpha_out, n_pq);
  else
    launch_k(cg_update_xr_kernel<false>, kRedBlocks, kRedThreads, 0, s, n, x, r, p, q, rz,
             pq_partials, rr_partials, alpha_out, n_pq);
  note_launch();
  return cudaGetLastError();
}

// exact two-term FP32 split v = hi + lo (hi the FP32 rounding of v, lo the
// FP32 rounding of v - hi)
__device__ __forceinline__ void split_f32(double v, float *hi, float *lo, int64_t i) {
  const float h = __double2float_rn(v);
  hi[i] = h;
  lo[i] = __double2float_rn(v - (double)h);
}

__global__ void split_kernel(int64_t n, const double *__restrict__ v, float *__restrict__ hi,
                             float *__restrict__ lo) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    split_f32(v[i], hi, lo, i);
}

cudaError_t launch_split(int64_t n, const double *v, float *hi, float *lo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 8 * kNumSM);
  launch_k(split_kernel, grid, 256, 0, s, n, v, hi, lo);
  note_launch();
  return cudaGetLastError();
}

// p = z + beta p, beta = rz_new / rz_old (flexible: (rz_new - r.z_old) / rz_old);
// with zold_out the new z is also copied there for the next flexible step
template <bool VEC>
__global__ void __launch_bounds__(kRedThreads)
cg_update_p_kernel(int64_t n, double *__restrict__ p, const double *__restrict__ z,
                   const double *__restrict__ rz_old, const double *__restrict__ rz_partials,
                   const double *__restrict__ rzold_partials, double *__restrict__ rz_out,
                   int flexible, double *__restrict__ zold_out, float *__restrict__ p_hi,
                   float *__restrict__ p_lo, int n_rz) {
  __shared__ double sh[32];
  const double rz_new = block_sum_partials(rz_partials, n_rz, sh);
  double num = rz_new;
  if (flexible) num -= block_sum_partials(rzold_partials, n_rz, sh);
  const double beta = num / rz_old[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) rz_out[0] = rz_new;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (VEC) {
    const int64_t m = n >> 1;
    double2 *p2 = reinterpret_cast<double2 *>(p);
    double2 *zo2 = reinterpret_cast<double2 *>(zold_out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
      const double2 zi = ld2(z, i), pi = p2[i];
      const double2 pn = make_double2(fma(beta, pi.x, zi.x), fma(beta, pi.y, zi.y));
      p2[i] = pn;
      if (zold_out) zo2[i] = zi;
      if (p_hi) {
        split_f32(pn.x, p_hi, p_lo, 2 * i);
        split_f32(pn.y, p_hi, p_lo, 2 * i + 1);
      }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const double zi = z[n - 1];
      const double pn = fma(beta, p[n - 1], zi);
      p[n - 1] = pn;
      if (zold_out) zold_out[n - 1] = zi;
      if (p_hi) split_f32(pn, p_hi, p_lo, n - 1);
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const double zi = z[i];
      const double pn = fma(beta, p[i], zi);
      p[i] = pn;
      if (zold_out) zold_out[i] = zi;
      if (p_hi) split_f32(pn, p_hi, p_lo, i);
    }
  }
}

cudaError_t launch_cg_update_p(int64_t n, double *p, const double *z, const double *rz_old,
                               const double *rz_partials, const double *rzold_partials,
                               double *rz_out, int flexible, cudaStream_t s, double *zold_out,
                               float *p_hi, float *p_lo, int n_rz) {
  if (al16(p) && al16(z) && (!zold_out || al16(zold_out)))
    launch_k(cg_update_p_kernel<true>, kRedBlocks, kRedThreads, 0, s, n, p, z, rz_old,
             rz_partials, rzold_partials, rz_out, flexible, zold_out, p_hi, p_lo, n_rz);
  else
    launch_k(cg_update_p_kernel<false>, kRedBlocks, kRedThreads, 0, s, n, p, z, rz_old,
             rz_partials, rzold_partials, rz_out, flexible, zold_out, p_hi, p_lo, n_rz);
  note_launch();
  return cudaGetLastError();
}

// The mixed-precision CG step with z and zold left in FP32 by the V-cycle
// (their FP64 values are exact): the partial sums of r . z and r . zold in
// one pass, over the same pairs, in the same order and tree as
// dot_partials_kernel<true>, so they equal those of FP64 copies bit for bit
__global__ void __launch_bounds__(kRedThreads)
cg_dots_f32_kernel(int64_t n, const double *__restrict__ r, const float *__restrict__ z,
                   const float *__restrict__ zo, double *__restrict__ part_rz,
                   double *__restrict__ part_rzo) {
  __shared__ double sh[32];
  double a[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t m = n >> 1;
  const float2 *z2 = reinterpret_cast<const float2 *>(z);
  const float2 *o2 = reinterpret_cast<const float2 *>(zo);
  for (; i + 3 * stride < m; i += 4 * stride) {
    double2 rv[4];
    float2 zv[4], ov[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rv[u] = ld2(r, i + u * stride);
      zv[u] = __ldg(z2 + i + u * stride);
      ov[u] = __ldg(o2 + i + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = fma(rv[u].y, (double)zv[u].y, fma(rv[u].x, (double)zv[u].x, a[u]));
      c[u] = fma(rv[u].y, (double)ov[u].y, fma(rv[u].x, (double)ov[u].x, c[u]));
    }
  }
  for (; i < m; i += stride) {
    const double2 rv = ld2(r, i);
    const float2 zv = __ldg(z2 + i), ov = __ldg(o2 + i);
    a[0] = fma(rv.y, (double)zv.y, fma(rv.x, (double)zv.x, a[0]));
    c[0] = fma(rv.y, (double)ov.y, fma(rv.x, (double)ov.x, c[0]));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    a[0] = fma(r[n - 1], (double)z[n - 1], a[0]);
    c[0] = fma(r[n - 1], (double)zo[n - 1], c[0]);
  }
  const double va = block_sum((a[0] + a[1]) + (a[2] + a[3]), sh);
  const double vc = block_sum((c[0] + c[1]) + (c[2] + c[3]), sh);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = va;
    part_rzo[blockIdx.x] = vc;
  }
}

cudaError_t launch_cg_dots_f32(int64_t n, const double *r, const float *z, const float *zold,
                               double *part_rz, double *part_rzo, cudaStream_t s) {
  if (!al16(r) || ((uintptr_t)z & 7u) || ((uintptr_t)zold & 7u)) return cudaErrorNotSupported;
  launch_k(cg_dots_f32_kernel, kRedBlocks, kRedThreads, 0, s, n, r, z, zold, part_rz, part_rzo);
  note_launch();
  return cudaGetLastError();
}

// flexible p = z + beta p, beta = (rz_new - r . zold) / rz_old, with z read
// from its FP32 copy (exact in FP64) and copied to zold_out for the next step,
// and the two-term FP32 split of the new p: the values of cg_update_p_kernel
__global__ void __launch_bounds__(kRedThreads)
cg_update_p_f32_kernel(int64_t n, double *__restrict__ p, const float *__restrict__ z,
                       const double *__restrict__ rz_old, const double *__restrict__ rz_partials,
                       const double *__restrict__ rzold_partials, double *__restrict__ rz_out,
                       float *__restrict__ zold_out, float *__restrict__ p_hi,
                       float *__restrict__ p_lo, int n_rz) {
  __shared__ double sh[32];
  const double rz_new = block_sum_partials(rz_partials, n_rz, sh);
  const double num = rz_new - block_sum_partials(rzold_partials, n_rz, sh);
  const double beta = num / rz_old[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) rz_out[0] = rz_new;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t m = n >> 1;
  double2 *p2 = reinterpret_cast<double2 *>(p);
  const float2 *z2 = reinterpret_cast<const float2 *>(z);
  float2 *zo2 = reinterpret_cast<float2 *>(zold_out);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const float2 zi = __ldg(z2 + i);
    const double2 pi = p2[i];
    const double2 pn = make_double2(fma(beta, pi.x, (double)zi.x), fma(beta, pi.y, (double)zi.y));
    p2[i] = pn;
    zo2[i] = zi;
    split_f32(pn.x, p_hi, p_lo, 2 * i);
    split_f32(pn.y, p_hi, p_lo, 2 * i + 1);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const float zi = z[n - 1];
    const double pn = fma(beta, p[n - 1], (double)zi);
    p[n - 1] = pn;
    zold_out[n - 1] = zi;
    split_f32(pn, p_hi, p_lo, n - 1);
  }
}

cudaError_t launch_cg_update_p_f32(int64_t n, double *p, const float *z, const double *rz_old,
                                   const double *rz_partials, const double *rzold_partials,
                                   double *rz_out, float *zold_out, float *p_hi, float *p_lo,
                                   int n_rz, cudaStream_t s) {
  if (!al16(p) || ((uintptr_t)z & 7u) || ((uintptr_t)zold_out & 7u)) return cudaErrorNotSupported;
  launch_k(cg_update_p_f32_kernel, kRedBlocks, kRedThreads, 0, s, n, p, z, rz_old, rz_partials,
           rzold_partials, rz_out, zold_out, p_hi, p_lo, n_rz);
  note_launch();
  return cudaGetLastError();
}

// End of one graph-resident CG step: ||r||^2 from the partials, iteration
// count, and the loop condition (continue while the recurrence residual is
// above tol * ||b||, p^T A p > 0 and fewer than max_iter steps were taken).
// scal: [0] r.r  [2] p.Ap  [3] rz (old)  [4] rz (new)  [9] ||b||  [10] tol
__global__ void __launch_bounds__(kRedThreads)
cg_check_kernel(const double *__restrict__ rr_partials, double *__restrict__ scal, int *iters,
                int max_iter, cudaGraphConditionalHandle handle) {
  __shared__ double sh[32];
  const double rr = block_sum_partials(rr_partials, kRedBlocks, sh);
  if (threadIdx.x == 0) {
    scal[0] = rr;
    const int k = ++iters[0];
    const double pq = scal[2];
    const double rel = sqrt(rr) / scal[9];
    const bool cont = (rel > scal[10]) && (k < max_iter) && (pq > 0.0) && isfinite(rel);
    scal[3] = scal[4];
    cudaGraphSetConditional(handle, cont ? 1u : 0u);
  }
}

cudaError_t launch_cg_check(const double *rr_partials, double *scal, int *iters, int max_iter,
                            cudaGraphConditionalHandle handle, cudaStream_t s) {
  launch_k(cg_check_kernel, 1, kRedThreads, 0, s, rr_partials, scal, iters, max_iter, handle); note_launch();
  return cudaGetLastError();
}

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ----------------------------------------------------------------------------
// GMRES (classical Gram-Schmidt applied twice; basis V column-major)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads)
multi_dot_kernel(int64_t n, const double *__restrict__ V, int64_t ldv,
                 const double *__restrict__ w, double *__restrict__ partials) {
  __shared__ double sh[32];
  const double *v = V + (size_t)blockIdx.y * ldv;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    acc = fma(v[i], w[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * kRedBlocks + blockIdx.x] = acc;
}

cudaError_t launch_multi_dot(int64_t n, const double *V, int64_t ldv, int k, const double *w,
                             double *partials, cudaStream_t s) {
  if (k == 0) return cudaSuccess;
  launch_k(multi_dot_kernel, dim3(kRedBlocks, k), kRedThreads, 0, s, n, V, ldv, w, partials); note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
multi_dot_finalize_kernel(const double *__restrict__ partials, double *__restrict__ h,
                          double *__restrict__ hacc) {
  __shared__ double sh[32];
  const double v = block_sum_partials(partials + (size_t)blockIdx.x * kRedBlocks, kRedBlocks, sh);
  if (threadIdx.x == 0) {
    h[blockIdx.x] = v;
    if (hacc) hacc[blockIdx.x] += v;
  }
}

cudaError_t launch_multi_dot_finalize(const double *partials, int k, double *h, double *hacc,
                                      cudaStream_t s) {
  if (k == 0) return cudaSuccess;
  launch_k(multi_dot_finalize_kernel, k, kRedThreads, 0, s, partials, h, hacc); note_launch();
  return cudaGetLastError();
}

__global__ void gs_update_kernel(int64_t n, const double *__restrict__ V, int64_t ldv, int k,
                                 const double *__restrict__ h, double *__restrict__ w) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc = w[i];
    for (int c = 0; c < k; ++c) acc = fma(-h[c], V[(size_t)c * ldv + i], acc);
    w[i] = acc;
  }
}

cudaError_t launch_gs_update(int64_t n, const double *V, int64_t ldv, int k, const double *h,
                             double *w, cudaStream_t s) {
  if (k == 0 || n == 0) return cudaSuccess;
  launch_k(gs_update_kernel, kRedBlocks * 2, 256, 0, s, n, V, ldv, k, h, w); note_launch();
  return cudaGetLastError();
}

__global__ void normalize_into_kernel(int64_t n, const double *__restrict__ w,
                                      const double *__restrict__ sumsq, double *__restrict__ v,
                                      double *__restrict__ hout) {
  const double nr = sqrt(sumsq[0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) hout[0] = nr;
  const double a = nr > 0.0 ? 1.0 / nr : 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    v[i] = w[i] * a;
}

cudaError_t launch_normalize_into(int64_t n, const double *w, const double *sumsq, double *v,
                                  double *hout, cudaStream_t s) {
  launch_k(normalize_into_kernel, kRedBlocks * 2, 256, 0, s, n, w, sumsq, v, hout); note_launch();
  return cudaGetLastError();
}

// H column-major with leading dimension ldh (= restart + 1); column j complete
// in rows 0..j+1.  Applies rotations 0..j-1, forms rotation j, updates g.
__global__ void gmres_givens_kernel(double *H, int ldh, int j, double *cs, double *sn,
                                    double *g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *h = H + (size_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
    h[i] = t;
  }
  const double a = h[j], b = h[j + 1];
  double c = 1.0, s = 0.0;
  if (b != 0.0) {
    const double hh = hypot(a, b);
    c = a / hh;
    s = b / hh;
  }
  cs[j] = c;
  sn[j] = s;
  h[j] = c * a + s * b;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
}

cudaError_t launch_gmres_givens(double *H, int ldh, int j, double *cs, double *sn, double *g,
                                cudaStream_t s) {
  launch_k(gmres_givens_kernel, 1, 32, 0, s, H, ldh, j, cs, sn, g); note_launch();
  return cudaGetLastError();
}

__global__ void gmres_backsolve_kernel(const double *H, int ldh, int j, const double *g,
                                       double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = j - 1; i >= 0; --i) {
    double acc = g[i];
    for (int c = i + 1; c < j; ++c) acc -= H[(size_t)c * ldh + i] * y[c];
    y[i] = acc / H[(size_t)i * ldh + i];
  }
}

cudaError_t launch_gmres_backsolve(const double *H, int ldh, int j, const double *g, double *y,
                                   cudaStream_t s) {
  launch_k(gmres_backsolve_kernel, 1, 32, 0, s, H, ldh, j, g, y); note_launch();
  return cudaGetLastError();
}

__global__ void combine_kernel(int64_t n, const double *__restrict__ V, int64_t ldv, int k,
                               const double *__restrict__ y, double *__restrict__ x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc = x[i];
    for (int c = 0; c < k; ++c) acc = fma(y[c], V[(size_t)c * ldv + i], acc);
    x[i] = acc;
  }
}

cudaError_t launch_combine(int64_t n, const double *V, int64_t ldv, int k, const double *y,
                           double *x, cudaStream_t s) {
  if (k == 0 || n == 0) return cudaSuccess;
  launch_k(combine_kernel, kRedBlocks * 2, 256, 0, s, n, V, ldv, k, y, x); note_launch();
  return cudaGetLastError();
}

}  // namespace gasa
