// FP16 block storage for the level-0 operators of the mixed-precision
// V-cycle: every dense block holds FP16 values v/s with one FP32 scale
// s = max |v| of the block, so the stored values lie in [-1, 1] and keep
// FP16's 11-bit significand.  Arithmetic stays FP32 (values are widened
// and scaled on load), halving the matrix bytes of the FP32 path.
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace gasa {

// ----------------------------------------------------------------------------
// setup: FP64 blocks -> FP16 blocks + FP32 per-block scales (warp per block)
// ----------------------------------------------------------------------------
__global__ void to_h16_blocks_kernel(int64_t nblocks, int bsz, const double *__restrict__ v,
                                     __half *__restrict__ h, float *__restrict__ scale) {
  const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (blk >= nblocks) return;
  const double *src = v + blk * bsz;
  double m = 0.0;
  for (int e = lane; e < bsz; e += 32) m = fmax(m, fabs(src[e]));
  m = warp_max(m);
  const float s = m > 0.0 ? (float)m : 1.0f;
  for (int e = lane; e < bsz; e += 32) h[blk * bsz + e] = __double2half(src[e] / (double)s);
  if (lane == 0) scale[blk] = s;
}

cudaError_t launch_to_h16_blocks(int64_t nblocks, int bsz, const double *v, __half *h,
                                 float *scale, cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  launch_k(to_h16_blocks_kernel, div_up(nblocks * 32, 256), 256, 0, s, nblocks, bsz, v, h, scale); note_launch();
  return cudaGetLastError();
}

// widen a row of BC FP16 values (half2 loads when the row is 4-byte aligned)
template <int BC>
__device__ __forceinline__ void load_h_row(const __half *p, float *out) {
  if constexpr (BC % 2 == 0) {
#pragma unroll
    for (int c = 0; c < BC; c += 2) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p + c));
      out[c] = f.x;
      out[c + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < BC; ++c) out[c] = __half2float(p[c]);
  }
}

// ----------------------------------------------------------------------------
// y = A x | y = b - A x | y += A x, A in FP16 blocks, FP32 vectors
// ----------------------------------------------------------------------------
template <int BC, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_h16_kernel(int n_brows, int br, const int *__restrict__ rp, const int *__restrict__ col,
                  const __half *__restrict__ val, const float *__restrict__ scale,
                  const float *__restrict__ x, const float *__restrict__ b, float *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  constexpr int W = RowVec<float, BC>::value;
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  float acc = 0.f;
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    float av[BC], xv[BC];
    load_h_row<BC>(val + ((size_t)k * br + r) * BC, av);
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec<float, W>(x + (size_t)j * BC + c, xv + c);
    float part = 0.f;
#pragma unroll
    for (int c = 0; c < BC; ++c) part = fmaf(av[c], xv[c], part);
    acc = fmaf(__ldg(scale + k), part, acc);
  }
  if (MODE == GASA_MV_ASSIGN) y[t] = acc;
  else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - acc;
  else y[t] += acc;
}

template <int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_h16_generic(int n_brows, int br, int bc, const int *__restrict__ rp,
                   const int *__restrict__ col, const __half *__restrict__ val,
                   const float *__restrict__ scale, const float *__restrict__ x,
                   const float *__restrict__ b, float *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  float acc = 0.f;
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    const __half *a = val + ((size_t)k * br + r) * bc;
    float part = 0.f;
    for (int c = 0; c < bc; ++c) part = fmaf(__half2float(a[c]), __ldg(x + (size_t)j * bc + c), part);
    acc = fmaf(__ldg(scale + k), part, acc);
  }
  if (MODE == GASA_MV_ASSIGN) y[t] = acc;
  else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - acc;
  else y[t] += acc;
}

template <int MODE>
static cudaError_t mv_h16_dispatch(int n_brows, int br, int bc, const int *rp, const int *col,
                                   const __half *val, const float *scale, const float *x,
                                   const float *b, float *y, cudaStream_t s) {
  const long long rows = (long long)n_brows * br;
  if (rows == 0) return cudaSuccess;
  const int grid = div_up(rows, 256);
#define GASA_H16_MV(BC)                                                                          \
  case BC:                                                                                       \
    launch_k(bsr_mv_h16_kernel<BC, MODE>, grid, 256, 0, s, n_brows, br, rp, col, val, scale, x, b, y); \
    note_launch();                                                                               \
    return cudaGetLastError();
  switch (bc) {
    GASA_H16_MV(1) GASA_H16_MV(2) GASA_H16_MV(3) GASA_H16_MV(4) GASA_H16_MV(6) GASA_H16_MV(8)
    GASA_H16_MV(9) GASA_H16_MV(10) GASA_H16_MV(12) GASA_H16_MV(16)
    default: break;
  }
#undef GASA_H16_MV
  launch_k(bsr_mv_h16_generic<MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, scale, x, b, y); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bsr_mv_h16(int mode, int n_brows, int br, int bc, const int *rp, const int *col,
                              const __half *val, const float *scale, const float *x,
                              const float *b, float *y, cudaStream_t s) {
  switch (mode) {
    case GASA_MV_ASSIGN:
      return mv_h16_dispatch<GASA_MV_ASSIGN>(n_brows, br, bc, rp, col, val, scale, x, b, y, s);
    case GASA_MV_RESIDUAL:
      return mv_h16_dispatch<GASA_MV_RESIDUAL>(n_brows, br, bc, rp, col, val, scale, x, b, y, s);
    default:
      return mv_h16_dispatch<GASA_MV_ADD>(n_brows, br, bc, rp, col, val, scale, x, b, y, s);
  }
}

// ----------------------------------------------------------------------------
// block-Jacobi step with A and W = w D^{-1} in FP16 blocks (modes as in
// jacobi_kernel: SWEEP x + W(b - Ax), FIRST W b)
// ----------------------------------------------------------------------------
template <int BS, int MODE>
__global__ void __launch_bounds__(256)
jacobi_h16_kernel(int n_units, const int *__restrict__ rp, const int *__restrict__ col,
                  const __half *__restrict__ val, const float *__restrict__ ascale,
                  const __half *__restrict__ Wm, const float *__restrict__ wscale,
                  const float *__restrict__ x, const float *__restrict__ b,
                  float *__restrict__ xo) {
  __shared__ float res[256];
  constexpr int RPB = 256 / BS;
  constexpr int W = RowVec<float, BS>::value;
  const int li = threadIdx.x / BS;
  const int r = threadIdx.x - li * BS;
  const int i = blockIdx.x * RPB + li;
  const bool active = (li < RPB) && (i < n_units);
  const size_t row = (size_t)i * BS + r;
  float v = 0.f;
  if (active) {
    if (MODE == JAC_FIRST) {
      v = b[row];
    } else {
      const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
      float acc = 0.f;
      for (int k = beg; k < end; ++k) {
        const int j = __ldg(col + k);
        float av[BS], xv[BS];
        load_h_row<BS>(val + ((size_t)k * BS + r) * BS, av);
#pragma unroll
        for (int c = 0; c < BS; c += W) load_vec<float, W>(x + (size_t)j * BS + c, xv + c);
        float part = 0.f;
#pragma unroll
        for (int c = 0; c < BS; ++c) part = fmaf(av[c], xv[c], part);
        acc = fmaf(__ldg(ascale + k), part, acc);
      }
      v = b[row] - acc;
    }
  }
  res[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  float wv[BS];
  load_h_row<BS>(Wm + row * BS, wv);
  float out = 0.f;
#pragma unroll
  for (int c = 0; c < BS; ++c) out = fmaf(wv[c], res[li * BS + c], out);
  out *= __ldg(wscale + i);
  if (MODE == JAC_SWEEP) out += x[row];
  xo[row] = out;
}

template <int MODE>
__global__ void __launch_bounds__(256)
jacobi_h16_generic(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
                   const __half *__restrict__ val, const float *__restrict__ ascale,
                   const __half *__restrict__ Wm, const float *__restrict__ wscale,
                   const float *__restrict__ x, const float *__restrict__ b,
                   float *__restrict__ xo) {
  extern __shared__ float resg[];
  const int rpb = blockDim.x / bs;
  const int li = threadIdx.x / bs;
  const int r = threadIdx.x - li * bs;
  const int i = blockIdx.x * rpb + li;
  const bool active = (li < rpb) && (i < n_units);
  const size_t row = (size_t)i * bs + r;
  float v = 0.f;
  if (active) {
    if (MODE == JAC_FIRST) {
      v = b[row];
    } else {
      const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
      float acc = 0.f;
      for (int k = beg; k < end; ++k) {
        const int j = __ldg(col + k);
        const __half *a = val + ((size_t)k * bs + r) * bs;
        float part = 0.f;
        for (int c = 0; c < bs; ++c) part = fmaf(__half2float(a[c]), __ldg(x + (size_t)j * bs + c), part);
        acc = fmaf(__ldg(ascale + k), part, acc);
      }
      v = b[row] - acc;
    }
  }
  resg[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  const __half *w = Wm + row * bs;
  float out = 0.f;
  for (int c = 0; c < bs; ++c) out = fmaf(__half2float(w[c]), resg[li * bs + c], out);
  out *= __ldg(wscale + i);
  if (MODE == JAC_SWEEP) out += x[row];
  xo[row] = out;
}

template <int MODE>
static cudaError_t jac_h16_dispatch(int n_units, int bs, const int *rp, const int *col,
                                    const __half *val, const float *ascale, const __half *W,
                                    const float *wscale, const float *x, const float *b,
                                    float *xo, cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
#define GASA_H16_JAC(BS)                                                                        \
  case BS: {                                                                                    \
    constexpr int rpb = 256 / BS;                                                               \
    launch_k(jacobi_h16_kernel<BS, MODE>, div_up(n_units, rpb), 256, 0, s, n_units, rp, col, val,     \
                                                                    ascale, W, wscale, x, b,    \
                                                                    xo);                        \
    note_launch();                                                                              \
    return cudaGetLastError();                                                                  \
  }
  switch (bs) {
    GASA_H16_JAC(1) GASA_H16_JAC(2) GASA_H16_JAC(3) GASA_H16_JAC(4) GASA_H16_JAC(6)
    GASA_H16_JAC(8) GASA_H16_JAC(9) GASA_H16_JAC(10) GASA_H16_JAC(12) GASA_H16_JAC(16)
    default: break;
  }
#undef GASA_H16_JAC
  int rpb = 256 / bs;
  if (rpb < 1) rpb = 1;
  const int th = rpb * bs;
  if (th > 1024) return cudaErrorInvalidValue;
  launch_k(jacobi_h16_generic<MODE>, div_up(n_units, rpb), th, th * sizeof(float), s, 
      n_units, bs, rp, col, val, ascale, W, wscale, x, b, xo); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_jacobi_h16(int mode, int n_units, int bs, const int *rp, const int *col,
                              const __half *val, const float *ascale, const __half *W,
                              const float *wscale, const float *x, const float *b, float *xo,
                              cudaStream_t s) {
  if (mode == JAC_FIRST)
    return jac_h16_dispatch<JAC_FIRST>(n_units, bs, rp, col, val, ascale, W, wscale, x, b, xo, s);
  return jac_h16_dispatch<JAC_SWEEP>(n_units, bs, rp, col, val, ascale, W, wscale, x, b, xo, s);
}

}  // namespace gasa
