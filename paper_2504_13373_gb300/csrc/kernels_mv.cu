// Block-sparse products on the V-cycle hot path (Alg. 1, Alg. 2).
//
// Layout: BSR, one dense br x bc block per stored pair, blocks row-major and
// contiguous in block-row order.  One thread owns one scalar row (block row
// i, row r of the block): it streams row r of every block of block row i
// (bc contiguous values, loaded with the widest aligned vector) and gathers
// the matching bc entries of x, which stay L2-resident.  The threads of one
// block row read one contiguous br*bc span per block, so a warp's requests
// cover whole 32-byte sectors and every matrix byte crosses HBM once per
// pass.  The block-Jacobi step additionally exchanges the block row's
// residual through shared memory and applies the precomputed w D^{-1}.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace gasa {

// ----------------------------------------------------------------------------
// y = A x | y = b - A x | y += A x
// ----------------------------------------------------------------------------
template <typename T, int BC, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_kernel(int n_brows, int br, const int *__restrict__ rp, const int *__restrict__ col,
              const T *__restrict__ val, const T *__restrict__ x, const T *__restrict__ b,
              T *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  constexpr int W = RowVec<T, BC>::value;
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  T acc = T(0);
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    const T *a = val + ((size_t)k * br + r) * BC;
    const T *xj = x + (size_t)j * BC;
    T av[BC], xv[BC];
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec_stream<T, W>(a + c, av + c);
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec<T, W>(xj + c, xv + c);
#pragma unroll
    for (int c = 0; c < BC; ++c) acc = fma(av[c], xv[c], acc);
  }
  if (MODE == GASA_MV_ASSIGN) y[t] = acc;
  else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - acc;
  else if (MODE == kMvFolded) y[t] = x[t] + (b[t] - acc);
  else y[t] += acc;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_generic(int n_brows, int br, int bc, const int *__restrict__ rp,
               const int *__restrict__ col, const T *__restrict__ val, const T *__restrict__ x,
               const T *__restrict__ b, T *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  T acc = T(0);
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    const T *a = val + ((size_t)k * br + r) * bc;
    const T *xj = x + (size_t)j * bc;
    for (int c = 0; c < bc; ++c) acc = fma(__ldg(a + c), __ldg(xj + c), acc);
  }
  if (MODE == GASA_MV_ASSIGN) y[t] = acc;
  else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - acc;
  else if (MODE == kMvFolded) y[t] = x[t] + (b[t] - acc);
  else y[t] += acc;
}

// Folded smoothing step y = x + (c - A x) for the FP32 level 0, taking the
// blocks of a row two at a time: both column indices, both matrix rows and
// both x segments are requested before the first FMA, so each thread keeps
// two blocks' loads in flight, and the FMAs still run in block order (the
// same bits as bsr_mv_kernel).  MINB caps the registers so that MINB CTAs of
// 256 threads stay resident per SM.  On the 1.31M-dof P3 pattern (10 x 10
// blocks, about 4 per row) MINB = 6 took a step from 49.1 to 43.2 us on
// GB300; unrolling four blocks, or two without the register cap, was slower
// (fewer resident warps).
template <int BC, int MINB>
__global__ void __launch_bounds__(256, MINB)
folded_pair_kernel(int n_brows, int br, const int *__restrict__ rp, const int *__restrict__ col,
                   const float *__restrict__ val, const float *__restrict__ x,
                   const float *__restrict__ c, float *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  constexpr int W = RowVec<float, BC>::value;
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  float acc = 0.f;
  int k = beg;
  for (; k + 2 <= end; k += 2) {
    const int j0 = __ldg(col + k), j1 = __ldg(col + k + 1);
    float a0[BC], a1[BC], x0[BC], x1[BC];
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec_stream<float, W>(val + ((size_t)k * br + r) * BC + q, a0 + q);
#pragma unroll
    for (int q = 0; q < BC; q += W)
      load_vec_stream<float, W>(val + ((size_t)(k + 1) * br + r) * BC + q, a1 + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec<float, W>(x + (size_t)j0 * BC + q, x0 + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec<float, W>(x + (size_t)j1 * BC + q, x1 + q);
#pragma unroll
    for (int q = 0; q < BC; ++q) acc = fmaf(a0[q], x0[q], acc);
#pragma unroll
    for (int q = 0; q < BC; ++q) acc = fmaf(a1[q], x1[q], acc);
  }
  if (k < end) {
    const int j = __ldg(col + k);
    float av[BC], xv[BC];
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec_stream<float, W>(val + ((size_t)k * br + r) * BC + q, av + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec<float, W>(x + (size_t)j * BC + q, xv + q);
#pragma unroll
    for (int q = 0; q < BC; ++q) acc = fmaf(av[q], xv[q], acc);
  }
  y[t] = x[t] + (c[t] - acc);
}

// ----------------------------------------------------------------------------
// Coarse levels: few block rows, each with tens to hundreds of blocks (the
// Galerkin products widen the stencil level by level).  One warp owns one
// block row; lane l takes blocks l, l+32, ... and keeps br partial sums; an
// xor-shuffle reduction leaves every sum in every lane.
// ----------------------------------------------------------------------------
template <typename T, int BRMAX>
__device__ __forceinline__ void warp_row_product(int beg, int end, int br, int bc, int lane,
                                                 const int *__restrict__ col,
                                                 const T *__restrict__ val,
                                                 const T *__restrict__ x, T (&acc)[BRMAX]) {
#pragma unroll
  for (int r = 0; r < BRMAX; ++r) acc[r] = T(0);
  for (int k = beg + lane; k < end; k += 32) {
    const int j = __ldg(col + k);
    const T *a = val + (size_t)k * br * bc;
    const T *xj = x + (size_t)j * bc;
    for (int c = 0; c < bc; ++c) {
      const T xv = __ldg(xj + c);
#pragma unroll
      for (int r = 0; r < BRMAX; ++r)
        if (r < br) acc[r] = fma(__ldg(a + r * bc + c), xv, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < BRMAX; ++r)
    if (r < br) acc[r] = warp_sum(acc[r]);
}

template <typename T, int BRMAX>
__device__ __forceinline__ T pick(const T (&acc)[BRMAX], int r) {
  T v = T(0);
#pragma unroll
  for (int q = 0; q < BRMAX; ++q)
    if (q == r) v = acc[q];
  return v;
}

template <typename T, int BRMAX, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_warp_kernel(int n_brows, int br, int bc, const int *__restrict__ rp,
                   const int *__restrict__ col, const T *__restrict__ val, const T *__restrict__ x,
                   const T *__restrict__ b, T *__restrict__ y) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n_brows) return;
  T acc[BRMAX];
  warp_row_product<T, BRMAX>(__ldg(rp + i), __ldg(rp + i + 1), br, bc, lane, col, val, x, acc);
  for (int r = lane; r < br; r += 32) {
    const size_t t = (size_t)i * br + r;
    const T v = pick<T, BRMAX>(acc, r);
    if (MODE == GASA_MV_ASSIGN) y[t] = v;
    else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - v;
    else y[t] += v;
  }
}

// Power-of-two block heights: the warp's lanes form 32/br groups of br
// lanes; lane (g, r) takes row r of blocks g, g + 32/br, ... of the block row,
// so a block's br rows are read by br neighbouring lanes at once; the groups'
// partial sums meet in an xor-shuffle over the group bits.
template <typename T>
__device__ __forceinline__ T group_row_dot(int beg, int end, int br, int bc, int lane,
                                           const int *__restrict__ col,
                                           const T *__restrict__ val,
                                           const T *__restrict__ x) {
  const int r = lane & (br - 1);
  const int g = lane / br;
  const int G = 32 / br;
  T acc = T(0);
  for (int k = beg + g; k < end; k += G) {
    const int j = __ldg(col + k);
    const T *a = val + ((size_t)k * br + r) * bc;
    const T *xj = x + (size_t)j * bc;
#pragma unroll 4
    for (int c = 0; c < bc; ++c) acc = fma(__ldg(a + c), __ldg(xj + c), acc);
  }
  for (int o = br; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;   // every lane holds the sum of row (lane & (br - 1))
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_group_kernel(int n_brows, int br, int bc, const int *__restrict__ rp,
                    const int *__restrict__ col, const T *__restrict__ val,
                    const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ y) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n_brows) return;
  const T v = group_row_dot<T>(__ldg(rp + i), __ldg(rp + i + 1), br, bc, lane, col, val, x);
  if (lane < br) {
    const size_t t = (size_t)i * br + lane;
    if (MODE == GASA_MV_ASSIGN) y[t] = v;
    else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - v;
    else y[t] += v;
  }
}

static inline bool pow2_le32(int v) { return v > 0 && v <= 32 && (v & (v - 1)) == 0; }

// The coarsest levels hold a few thousand block rows or less, each with up
// to several hundred blocks: one CTA of 256 threads owns a block row.  The
// threads form G = 256 / br groups of br; thread (g, r) takes row r of blocks
// g, g + G, ...; the groups' partial sums are added in a fixed order from
// shared memory.  Returns the row sums in red[0..br).
template <typename T>
__device__ __forceinline__ void cta_row_dot(int beg, int end, int br, int bc,
                                            const int *__restrict__ col,
                                            const T *__restrict__ val,
                                            const T *__restrict__ x, T *red) {
  const int G = blockDim.x / br;
  const int t = threadIdx.x;
  const int g = t / br, r = t - g * br;
  T acc = T(0);
  if (g < G) {
    for (int k = beg + g; k < end; k += G) {
      const int j = __ldg(col + k);
      const T *a = val + ((size_t)k * br + r) * bc;
      const T *xj = x + (size_t)j * bc;
#pragma unroll 4
      for (int c = 0; c < bc; ++c) acc = fma(__ldg(a + c), __ldg(xj + c), acc);
    }
  }
  red[t] = acc;
  __syncthreads();
  if (t < br) {
    T s = T(0);
    for (int q = 0; q < G; ++q) s += red[q * br + t];
    red[blockDim.x + t] = s;
  }
  __syncthreads();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
bsr_mv_cta_kernel(int n_brows, int br, int bc, const int *__restrict__ rp,
                  const int *__restrict__ col, const T *__restrict__ val,
                  const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ y) {
  extern __shared__ unsigned char cta_smem[];
  T *red = reinterpret_cast<T *>(cta_smem);
  const int i = blockIdx.x;
  cta_row_dot<T>(__ldg(rp + i), __ldg(rp + i + 1), br, bc, col, val, x, red);
  for (int r = threadIdx.x; r < br; r += blockDim.x) {
    const size_t t = (size_t)i * br + r;
    const T v = red[blockDim.x + r];
    if (MODE == GASA_MV_ASSIGN) y[t] = v;
    else if (MODE == GASA_MV_RESIDUAL) y[t] = b[t] - v;
    else y[t] += v;
  }
}

// CTA per block row for few, long rows
static inline bool cta_rows(int n_brows, int br) { return n_brows <= 4096 && br <= 256; }

// A warp per block row pays when the thread-per-row grid would fill less
// than about half of the GPU, or when rows are very long.
static inline bool warp_rows(int n_brows, int br, int64_t nnzb) {
  if (nnzb < 0 || br > 64) return false;
  const long long threads = (long long)n_brows * br;
  return (threads < 65536 && nnzb >= 4LL * n_brows) || nnzb >= 64LL * n_brows;
}

static inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T, int MODE>
static cudaError_t mv_warp_dispatch(int n_brows, int br, int bc, const int *rp, const int *col,
                                    const T *val, const T *x, const T *b, T *y, cudaStream_t s) {
  const int grid = div_up((long long)n_brows * 32, 256);
  if (cta_rows(n_brows, br)) {
    launch_k(bsr_mv_cta_kernel<T, MODE>, n_brows, 256, (256 + br) * sizeof(T), s, n_brows, br, bc, rp, col, val, x, b, y);
    note_launch();
    return cudaGetLastError();
  }
  if (pow2_le32(br)) launch_k(bsr_mv_group_kernel<T, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  else if (br <= 4) launch_k(bsr_mv_warp_kernel<T, 4, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  else if (br <= 8) launch_k(bsr_mv_warp_kernel<T, 8, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  else if (br <= 16) launch_k(bsr_mv_warp_kernel<T, 16, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  else if (br <= 32) launch_k(bsr_mv_warp_kernel<T, 32, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  else launch_k(bsr_mv_warp_kernel<T, 64, MODE>, grid, 256, 0, s, n_brows, br, bc, rp, col, val, x, b, y);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t mv_dispatch(int n_brows, int br, int bc, const int *rp, const int *col,
                               const T *val, const T *x, const T *b, T *y, cudaStream_t s) {
  const long long rows = (long long)n_brows * br;
  if (rows == 0) return cudaSuccess;
  const int th = 256;
  const int grid = div_up(rows, th);
  const bool al = aligned16(val) && aligned16(x);
#define GASA_MV_CASE(BC)                                                                   \
  case BC:                                                                                 \
    launch_k(bsr_mv_kernel<T, BC, MODE>, grid, th, 0, s, n_brows, br, rp, col, val, x, b, y); note_launch();    \
    return cudaGetLastError();
  if (al) {
    switch (bc) {
      GASA_MV_CASE(1) GASA_MV_CASE(2) GASA_MV_CASE(3) GASA_MV_CASE(4) GASA_MV_CASE(5)
      GASA_MV_CASE(6) GASA_MV_CASE(7) GASA_MV_CASE(8) GASA_MV_CASE(9) GASA_MV_CASE(10)
      GASA_MV_CASE(11) GASA_MV_CASE(12) GASA_MV_CASE(13) GASA_MV_CASE(14) GASA_MV_CASE(15)
      GASA_MV_CASE(16)
      default: break;
    }
  }
#undef GASA_MV_CASE
  launch_k(bsr_mv_generic<T, MODE>, grid, th, 0, s, n_brows, br, bc, rp, col, val, x, b, y); note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bsr_mv(int mode, int n_brows, int br, int bc, const int *rp, const int *col,
                          const T *val, const T *x, const T *b, T *y, cudaStream_t s,
                          int64_t nnzb) {
  if (br == bc && mode >= GASA_MV_ASSIGN && mode <= GASA_MV_ADD && blk_applies(br, n_brows, nnzb)) {
    const cudaError_t e = launch_blk<T>(mode, n_brows, br, nnzb, rp, col, val, nullptr, x, b, y, s);
    if (e != cudaErrorNotSupported) return e;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (mode >= GASA_MV_ASSIGN && mode <= GASA_MV_ADD && wide_applies(br, bc, n_brows, nnzb)) {
      const int op = mode == GASA_MV_ASSIGN ? 0 : mode == GASA_MV_RESIDUAL ? 1 : 2;
      const cudaError_t e = launch_wide(op, n_brows, br, bc, nnzb, rp, col, val, nullptr, x, b, y, s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  if (n_brows > 0 && warp_rows(n_brows, br, nnzb)) {
    switch (mode) {
      case GASA_MV_ASSIGN:
        return mv_warp_dispatch<T, GASA_MV_ASSIGN>(n_brows, br, bc, rp, col, val, x, b, y, s);
      case GASA_MV_RESIDUAL:
        return mv_warp_dispatch<T, GASA_MV_RESIDUAL>(n_brows, br, bc, rp, col, val, x, b, y, s);
      default:
        return mv_warp_dispatch<T, GASA_MV_ADD>(n_brows, br, bc, rp, col, val, x, b, y, s);
    }
  }
  switch (mode) {
    case GASA_MV_ASSIGN:
      return mv_dispatch<T, GASA_MV_ASSIGN>(n_brows, br, bc, rp, col, val, x, b, y, s);
    case GASA_MV_RESIDUAL:
      return mv_dispatch<T, GASA_MV_RESIDUAL>(n_brows, br, bc, rp, col, val, x, b, y, s);
    default:
      return mv_dispatch<T, GASA_MV_ADD>(n_brows, br, bc, rp, col, val, x, b, y, s);
  }
}
template cudaError_t launch_bsr_mv<double>(int, int, int, int, const int *, const int *,
                                           const double *, const double *, const double *,
                                           double *, cudaStream_t, int64_t);
template cudaError_t launch_bsr_mv<float>(int, int, int, int, const int *, const int *,
                                          const float *, const float *, const float *, float *,
                                          cudaStream_t, int64_t);

template <typename T>
cudaError_t launch_folded_sweep(int n_units, int bs, const int *rp, const int *col, const T *WA,
                                const T *x, const T *c, T *xo, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (bs == 10 && n_units > 0 && aligned16(WA) && aligned16(x)) {
      launch_k(folded_pair_kernel<10, 6>, div_up((long long)n_units * bs, 256), 256, 0, s,
               n_units, bs, rp, col, WA, x, c, xo);
      note_launch();
      return cudaGetLastError();
    }
  }
  return mv_dispatch<T, kMvFolded>(n_units, bs, bs, rp, col, WA, x, c, xo, s);
}
template cudaError_t launch_folded_sweep<double>(int, int, const int *, const int *, const double *,
                                                 const double *, const double *, double *,
                                                 cudaStream_t);
template cudaError_t launch_folded_sweep<float>(int, int, const int *, const int *, const float *,
                                                const float *, const float *, float *,
                                                cudaStream_t);

// ----------------------------------------------------------------------------
// y = A x in double-single arithmetic (the outer Krylov product of the
// mixed-precision solve).  A and x arrive as exact two-term FP32 splits,
// a = a_hi + a_lo and x = x_hi + x_lo (a_hi the FP32 rounding of a, a_lo the
// FP32 rounding of a - a_hi, so each pair holds a to 2^-48 relative).  Per
// product: a_hi x_hi = p + e exactly (p rounded, e = fma(a_hi, x_hi, -p)),
// the cross terms a_hi x_lo + a_lo x_hi in FP32 (a_lo x_lo, below 2^-48, is
// dropped); p joins the running sum s by an error-free two-sum and every
// error and cross term joins the low word t.  The row result is s + t in
// FP64.  Every step uses FP32 units: on GB300 FP64 FMAs run at a small
// fraction of the FP32 rate, and an FP64 SpMV needs one FMA per 8 bytes of
// matrix, more than that rate feeds at full HBM bandwidth.  The __f*_rn
// intrinsics keep the compiler from contracting the two-sum into FMAs.
// ----------------------------------------------------------------------------
// One product of the recurrence above joined to the running pair (s, lo).
__device__ __forceinline__ void ds_product_add(float ah, float al, float xh, float xl, float &s,
                                               float &lo) {
  const float pr = __fmul_rn(ah, xh);
  const float e = __fmaf_rn(ah, xh, -pr);
  const float cross = __fmaf_rn(ah, xl, __fmul_rn(al, xh));
  const float s1 = __fadd_rn(s, pr);
  const float bp = __fsub_rn(s1, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bp)), __fsub_rn(pr, bp));
  s = s1;
  lo = __fadd_rn(lo, __fadd_rn(err, __fadd_rn(e, cross)));
}

// One block row segment: BC products joined in column order.
template <int BC>
__device__ __forceinline__ void ds_row_accumulate(const float *ah, const float *al,
                                                  const float *xh, const float *xl, float &s,
                                                  float &lo) {
#pragma unroll
  for (int c = 0; c < BC; ++c) ds_product_add(ah[c], al[c], xh[c], xl[c], s, lo);
}

// With DOT the kernel also leaves per-CTA partial sums of x . y (x given in
// FP64 as xd) in partials[blockIdx.x], summed in a fixed order.
template <int BC, bool DOT>
__global__ void __launch_bounds__(256)
bsr_mv_ds_kernel(int n_brows, int br, const int *__restrict__ rp, const int *__restrict__ col,
                 const float *__restrict__ ahi, const float *__restrict__ alo,
                 const float *__restrict__ xhi, const float *__restrict__ xlo,
                 double *__restrict__ y, const double *__restrict__ xd,
                 double *__restrict__ partials) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = t < (long long)n_brows * br;
  const int i = act ? (int)(t / br) : 0;
  const int r = act ? (int)(t - (long long)i * br) : 0;
  constexpr int W = RowVec<float, BC>::value;
  const int beg = act ? __ldg(rp + i) : 0, end = act ? __ldg(rp + i + 1) : 0;
  const double xt = (DOT && act) ? xd[t] : 0.0;
  float s = 0.0f, lo = 0.0f;
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    const size_t off = ((size_t)k * br + r) * BC;
    float ah[BC], al[BC], xh[BC], xl[BC];
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec_stream<float, W>(ahi + off + c, ah + c);
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec_stream<float, W>(alo + off + c, al + c);
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec<float, W>(xhi + (size_t)j * BC + c, xh + c);
#pragma unroll
    for (int c = 0; c < BC; c += W) load_vec<float, W>(xlo + (size_t)j * BC + c, xl + c);
    ds_row_accumulate<BC>(ah, al, xh, xl, s, lo);
  }
  const double yt = (double)s + (double)lo;
  if (act) y[t] = yt;
  if (DOT) {
    __shared__ double sh[32];
    const double v = block_sum(xt * yt, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// The same double-single product taking the blocks of a row two at a time:
// both blocks' hi and lo rows and x segments are requested before the first
// product, and the products join s and t in block order (the same bits as
// bsr_mv_ds_kernel).  MINB = 4 caps the registers at 64.  On the 1.31M-dof
// P3 pattern it took q = A p with p.q from 116.8 to 83.6 us on GB300.
template <int BC, bool DOT, int MINB>
__global__ void __launch_bounds__(256, MINB)
bsr_mv_ds_pair_kernel(int n_brows, int br, const int *__restrict__ rp, const int *__restrict__ col,
                      const float *__restrict__ ahi, const float *__restrict__ alo,
                      const float *__restrict__ xhi, const float *__restrict__ xlo,
                      double *__restrict__ y, const double *__restrict__ xd,
                      double *__restrict__ partials) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = t < (long long)n_brows * br;
  const int i = act ? (int)(t / br) : 0;
  const int r = act ? (int)(t - (long long)i * br) : 0;
  constexpr int W = RowVec<float, BC>::value;
  const int beg = act ? __ldg(rp + i) : 0, end = act ? __ldg(rp + i + 1) : 0;
  const double xt = (DOT && act) ? xd[t] : 0.0;
  float s = 0.0f, lo = 0.0f;
  int k = beg;
  for (; k + 2 <= end; k += 2) {
    const int j0 = __ldg(col + k), j1 = __ldg(col + k + 1);
    const size_t o0 = ((size_t)k * br + r) * BC, o1 = ((size_t)(k + 1) * br + r) * BC;
    float ah0[BC], al0[BC], ah1[BC], al1[BC], xh0[BC], xl0[BC], xh1[BC], xl1[BC];
#pragma unroll
    for (int q = 0; q < BC; q += W) {
      load_vec_stream<float, W>(ahi + o0 + q, ah0 + q);
      load_vec_stream<float, W>(alo + o0 + q, al0 + q);
    }
#pragma unroll
    for (int q = 0; q < BC; q += W) {
      load_vec_stream<float, W>(ahi + o1 + q, ah1 + q);
      load_vec_stream<float, W>(alo + o1 + q, al1 + q);
    }
#pragma unroll
    for (int q = 0; q < BC; q += W) {
      load_vec<float, W>(xhi + (size_t)j0 * BC + q, xh0 + q);
      load_vec<float, W>(xlo + (size_t)j0 * BC + q, xl0 + q);
    }
#pragma unroll
    for (int q = 0; q < BC; q += W) {
      load_vec<float, W>(xhi + (size_t)j1 * BC + q, xh1 + q);
      load_vec<float, W>(xlo + (size_t)j1 * BC + q, xl1 + q);
    }
    ds_row_accumulate<BC>(ah0, al0, xh0, xl0, s, lo);
    ds_row_accumulate<BC>(ah1, al1, xh1, xl1, s, lo);
  }
  if (k < end) {
    const int j = __ldg(col + k);
    const size_t off = ((size_t)k * br + r) * BC;
    float ah[BC], al[BC], xh[BC], xl[BC];
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec_stream<float, W>(ahi + off + q, ah + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec_stream<float, W>(alo + off + q, al + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec<float, W>(xhi + (size_t)j * BC + q, xh + q);
#pragma unroll
    for (int q = 0; q < BC; q += W) load_vec<float, W>(xlo + (size_t)j * BC + q, xl + q);
    ds_row_accumulate<BC>(ah, al, xh, xl, s, lo);
  }
  const double yt = (double)s + (double)lo;
  if (act) y[t] = yt;
  if (DOT) {
    __shared__ double sh[32];
    const double v = block_sum(xt * yt, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256)
bsr_mv_ds_generic(int n_brows, int br, int bc, const int *__restrict__ rp,
                  const int *__restrict__ col, const float *__restrict__ ahi,
                  const float *__restrict__ alo, const float *__restrict__ xhi,
                  const float *__restrict__ xlo, double *__restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_brows * br) return;
  const int i = (int)(t / br);
  const int r = (int)(t - (long long)i * br);
  const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
  float s = 0.0f, lo = 0.0f;
  for (int k = beg; k < end; ++k) {
    const int j = __ldg(col + k);
    const size_t off = ((size_t)k * br + r) * bc;
    for (int c = 0; c < bc; ++c) {
      const float ah = __ldg(ahi + off + c), al = __ldg(alo + off + c);
      const float xh = __ldg(xhi + (size_t)j * bc + c), xl = __ldg(xlo + (size_t)j * bc + c);
      ds_product_add(ah, al, xh, xl, s, lo);
    }
  }
  y[t] = (double)s + (double)lo;
}

int bsr_mv_ds_grid(int n_brows, int br) { return div_up((long long)n_brows * br, 256); }

cudaError_t launch_bsr_mv_ds(int n_brows, int br, int bc, const int *rp, const int *col,
                             const float *ahi, const float *alo, const float *xhi,
                             const float *xlo, double *y, cudaStream_t s, const double *xd,
                             double *partials) {
  const long long rows = (long long)n_brows * br;
  if (rows == 0) return cudaSuccess;
  const int grid = div_up(rows, 256);
  const bool al = aligned16(ahi) && aligned16(alo) && aligned16(xhi) && aligned16(xlo);
  const bool dot = xd && partials;
#define GASA_DS_CASE(BC)                                                                    \
  case BC:                                                                                  \
    if (dot)                                                                                \
      launch_k(bsr_mv_ds_kernel<BC, true>, grid, 256, 0, s, n_brows, br, rp, col, ahi, alo, xhi, \
               xlo, y, xd, partials);                                                       \
    else                                                                                    \
      launch_k(bsr_mv_ds_kernel<BC, false>, grid, 256, 0, s, n_brows, br, rp, col, ahi, alo, xhi, \
               xlo, y, xd, partials);                                                       \
    note_launch();                                                                          \
    return cudaGetLastError();
  if (dot && !al) return cudaErrorNotSupported;
  if (al && bc == 10) {
    if (dot)
      launch_k(bsr_mv_ds_pair_kernel<10, true, 4>, grid, 256, 0, s, n_brows, br, rp, col, ahi,
               alo, xhi, xlo, y, xd, partials);
    else
      launch_k(bsr_mv_ds_pair_kernel<10, false, 4>, grid, 256, 0, s, n_brows, br, rp, col, ahi,
               alo, xhi, xlo, y, xd, partials);
    note_launch();
    return cudaGetLastError();
  }
  if (al) {
    switch (bc) {
      GASA_DS_CASE(1) GASA_DS_CASE(2) GASA_DS_CASE(3) GASA_DS_CASE(4) GASA_DS_CASE(5)
      GASA_DS_CASE(6) GASA_DS_CASE(7) GASA_DS_CASE(8) GASA_DS_CASE(9)
      GASA_DS_CASE(11) GASA_DS_CASE(12) GASA_DS_CASE(13) GASA_DS_CASE(14) GASA_DS_CASE(15)
      GASA_DS_CASE(16)
      default: break;
    }
  }
#undef GASA_DS_CASE
  launch_k(bsr_mv_ds_generic, grid, 256, 0, s, n_brows, br, bc, rp, col, ahi, alo, xhi, xlo, y);
  note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// block Jacobi step (Alg. 1 with A~^{-1} = w D^{-1}):
//   SWEEP: xo = x + W (b - A x)   FIRST: xo = W b
//   APPLY: xo = W (A x)           RELAX: xo = x - W A x
// A CTA owns whole block rows; thread (li, r) computes the residual entry,
// the block row's residual meets in shared memory, then thread (li, r)
// applies row r of W_i.
// ----------------------------------------------------------------------------
template <typename T, int BS, int MODE>
__global__ void __launch_bounds__(256)
jacobi_kernel(int n_units, const int *__restrict__ rp, const int *__restrict__ col,
              const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
              const T *__restrict__ b, T *__restrict__ xo) {
  __shared__ T res[256];
  constexpr int RPB = 256 / BS;
  constexpr int W = RowVec<T, BS>::value;
  const int li = threadIdx.x / BS;
  const int r = threadIdx.x - li * BS;
  const int i = blockIdx.x * RPB + li;
  const bool active = (li < RPB) && (i < n_units);
  const size_t row = (size_t)i * BS + r;
  T v = T(0);
  if (active) {
    if (MODE == JAC_FIRST) {
      v = b[row];
    } else {
      const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
      T acc = T(0);
      for (int k = beg; k < end; ++k) {
        const int j = __ldg(col + k);
        const T *a = val + ((size_t)k * BS + r) * BS;
        const T *xj = x + (size_t)j * BS;
        T av[BS], xv[BS];
#pragma unroll
        for (int c = 0; c < BS; c += W) load_vec_stream<T, W>(a + c, av + c);
#pragma unroll
        for (int c = 0; c < BS; c += W) load_vec<T, W>(xj + c, xv + c);
#pragma unroll
        for (int c = 0; c < BS; ++c) acc = fma(av[c], xv[c], acc);
      }
      if (MODE == JAC_SWEEP) v = b[row] - acc;
      else if (MODE == JAC_RELAX) v = -acc;
      else v = acc;
    }
  }
  res[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  const T *w = Wm + row * BS;
  T wv[BS];
#pragma unroll
  for (int c = 0; c < BS; c += W) load_vec_stream<T, W>(w + c, wv + c);
  T out = T(0);
#pragma unroll
  for (int c = 0; c < BS; ++c) out = fma(wv[c], res[li * BS + c], out);
  if (MODE == JAC_SWEEP || MODE == JAC_RELAX) out += x[row];
  xo[row] = out;
}

// First smoothing step of the mixed-precision V-cycle, x = W b from x = 0,
// reading the FP64 right-hand side: it also leaves the FP32 rounding of b
// (read by the later steps and the residual) in b32, so the precision
// conversion needs no launch of its own.  Same arithmetic as jacobi_kernel
// in FIRST mode on the converted b.
template <int BS>
__global__ void __launch_bounds__(256)
jacobi_first_conv_kernel(int n_units, const double *__restrict__ bd, float *__restrict__ b32,
                         const float *__restrict__ Wm, float *__restrict__ xo,
                         float *__restrict__ c_out) {
  __shared__ float res[256];
  constexpr int RPB = 256 / BS;
  constexpr int W = RowVec<float, BS>::value;
  const int li = threadIdx.x / BS;
  const int r = threadIdx.x - li * BS;
  const int i = blockIdx.x * RPB + li;
  const bool active = (li < RPB) && (i < n_units);
  const size_t row = (size_t)i * BS + r;
  float v = 0.0f;
  if (active) {
    v = __double2float_rn(bd[row]);
    b32[row] = v;
  }
  res[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  const float *w = Wm + row * BS;
  float wv[BS];
#pragma unroll
  for (int c = 0; c < BS; c += W) load_vec_stream<float, W>(w + c, wv + c);
  float out = 0.0f;
#pragma unroll
  for (int c = 0; c < BS; ++c) out = fmaf(wv[c], res[li * BS + c], out);
  xo[row] = out;
  if (c_out) c_out[row] = out;
}

int jacobi_grid(int n_units, int bs) { return div_up(n_units, 256 / bs); }

cudaError_t launch_jacobi_first_conv(int n_units, int bs, const double *bd, float *b32,
                                     const float *W, float *xo, cudaStream_t s, float *c_out) {
  if (n_units == 0) return cudaSuccess;
  if (!aligned16(W) || bs < 1 || bs > 16) return cudaErrorNotSupported;
  const int grid = jacobi_grid(n_units, bs);
#define GASA_FC_CASE(BS)                                                                      \
  case BS:                                                                                    \
    launch_k(jacobi_first_conv_kernel<BS>, grid, 256, 0, s, n_units, bd, b32, W, xo, c_out);  \
    break;
  switch (bs) {
    GASA_FC_CASE(1) GASA_FC_CASE(2) GASA_FC_CASE(3) GASA_FC_CASE(4) GASA_FC_CASE(5)
    GASA_FC_CASE(6) GASA_FC_CASE(7) GASA_FC_CASE(8) GASA_FC_CASE(9) GASA_FC_CASE(10)
    GASA_FC_CASE(11) GASA_FC_CASE(12) GASA_FC_CASE(13) GASA_FC_CASE(14) GASA_FC_CASE(15)
    GASA_FC_CASE(16)
  }
#undef GASA_FC_CASE
  note_launch();
  return cudaGetLastError();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
jacobi_generic(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
               const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
               const T *__restrict__ b, T *__restrict__ xo) {
  extern __shared__ unsigned char smem_raw[];
  T *res = reinterpret_cast<T *>(smem_raw);
  const int rpb = blockDim.x / bs;
  const int li = threadIdx.x / bs;
  const int r = threadIdx.x - li * bs;
  const int i = blockIdx.x * rpb + li;
  const bool active = (li < rpb) && (i < n_units);
  const size_t row = (size_t)i * bs + r;
  T v = T(0);
  if (active) {
    if (MODE == JAC_FIRST) {
      v = b[row];
    } else {
      const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
      T acc = T(0);
      for (int k = beg; k < end; ++k) {
        const int j = __ldg(col + k);
        const T *a = val + ((size_t)k * bs + r) * bs;
        const T *xj = x + (size_t)j * bs;
        for (int c = 0; c < bs; ++c) acc = fma(__ldg(a + c), __ldg(xj + c), acc);
      }
      if (MODE == JAC_SWEEP) v = b[row] - acc;
      else if (MODE == JAC_RELAX) v = -acc;
      else v = acc;
    }
  }
  res[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  const T *w = Wm + row * bs;
  T out = T(0);
  for (int c = 0; c < bs; ++c) out = fma(__ldg(w + c), res[li * bs + c], out);
  if (MODE == JAC_SWEEP || MODE == JAC_RELAX) out += x[row];
  xo[row] = out;
}

// warp per block row: the reduced residual of the block row is in every lane,
// lane r then applies row r of W_i
template <typename T, int BRMAX, int MODE>
__global__ void __launch_bounds__(256)
jacobi_warp_kernel(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
                   const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
                   const T *__restrict__ b, T *__restrict__ xo) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n_units) return;
  T acc[BRMAX];
  warp_row_product<T, BRMAX>(__ldg(rp + i), __ldg(rp + i + 1), bs, bs, lane, col, val, x, acc);
#pragma unroll
  for (int r = 0; r < BRMAX; ++r) {
    if (r < bs) {
      if (MODE == JAC_SWEEP) acc[r] = b[(size_t)i * bs + r] - acc[r];
      else if (MODE == JAC_RELAX) acc[r] = -acc[r];
    }
  }
  for (int r = lane; r < bs; r += 32) {
    const T *w = Wm + ((size_t)i * bs + r) * bs;
    T out = T(0);
#pragma unroll
    for (int c = 0; c < BRMAX; ++c)
      if (c < bs) out = fma(__ldg(w + c), acc[c], out);
    const size_t row = (size_t)i * bs + r;
    if (MODE == JAC_SWEEP || MODE == JAC_RELAX) out += x[row];
    xo[row] = out;
  }
}

// CTA per block row (few, long rows): the block row's residual meets in
// shared memory, thread r < bs applies row r of W_i
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
jacobi_cta_kernel(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
                  const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
                  const T *__restrict__ b, T *__restrict__ xo) {
  extern __shared__ unsigned char cta_smem_j[];
  T *red = reinterpret_cast<T *>(cta_smem_j);
  const int i = blockIdx.x;
  cta_row_dot<T>(__ldg(rp + i), __ldg(rp + i + 1), bs, bs, col, val, x, red);
  T *res = red + blockDim.x;
  for (int r = threadIdx.x; r < bs; r += blockDim.x) {
    const size_t row = (size_t)i * bs + r;
    if (MODE == JAC_SWEEP) res[r] = b[row] - res[r];
    else if (MODE == JAC_RELAX) res[r] = -res[r];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < bs; r += blockDim.x) {
    const size_t row = (size_t)i * bs + r;
    const T *w = Wm + row * bs;
    T out = T(0);
    for (int c = 0; c < bs; ++c) out = fma(__ldg(w + c), res[c], out);
    if (MODE == JAC_SWEEP || MODE == JAC_RELAX) out += x[row];
    xo[row] = out;
  }
}

// power-of-two block size: lane groups as in bsr_mv_group_kernel; lane c
// then holds row c's residual and lane r < bs applies row r of W_i
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
jacobi_group_kernel(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
                    const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
                    const T *__restrict__ b, T *__restrict__ xo) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n_units) return;
  T v = group_row_dot<T>(__ldg(rp + i), __ldg(rp + i + 1), bs, bs, lane, col, val, x);
  const int r = lane & (bs - 1);
  const size_t row = (size_t)i * bs + r;
  if (MODE == JAC_SWEEP) v = b[row] - v;
  else if (MODE == JAC_RELAX) v = -v;
  const T *w = Wm + row * bs;
  T out = T(0);
  for (int c = 0; c < bs; ++c) {
    const T rc = __shfl_sync(0xffffffffu, v, c);
    out = fma(__ldg(w + c), rc, out);
  }
  if (lane < bs) {
    if (MODE == JAC_SWEEP || MODE == JAC_RELAX) out += x[row];
    xo[row] = out;
  }
}

template <typename T, int MODE>
static cudaError_t jac_warp_dispatch(int n_units, int bs, const int *rp, const int *col,
                                     const T *val, const T *W, const T *x, const T *b, T *xo,
                                     cudaStream_t s) {
  const int grid = div_up((long long)n_units * 32, 256);
  if (cta_rows(n_units, bs)) {
    launch_k(jacobi_cta_kernel<T, MODE>, n_units, 256, (256 + bs) * sizeof(T), s, n_units, bs, rp, col, val, W, x, b, xo);
    note_launch();
    return cudaGetLastError();
  }
  if (pow2_le32(bs)) launch_k(jacobi_group_kernel<T, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  else if (bs <= 4) launch_k(jacobi_warp_kernel<T, 4, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  else if (bs <= 8) launch_k(jacobi_warp_kernel<T, 8, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  else if (bs <= 16) launch_k(jacobi_warp_kernel<T, 16, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  else if (bs <= 32) launch_k(jacobi_warp_kernel<T, 32, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  else launch_k(jacobi_warp_kernel<T, 64, MODE>, grid, 256, 0, s, n_units, bs, rp, col, val, W, x, b, xo);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t jac_dispatch(int n_units, int bs, const int *rp, const int *col,
                                const T *val, const T *W, const T *x, const T *b, T *xo,
                                cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
  const bool al = aligned16(val) && aligned16(W) && (MODE == JAC_FIRST || aligned16(x));
#define GASA_JAC_CASE(BS)                                                                   \
  case BS: {                                                                                \
    constexpr int rpb = 256 / BS;                                                           \
    launch_k(jacobi_kernel<T, BS, MODE>, div_up(n_units, rpb), 256, 0, s, n_units, rp, col, val,  \
                                                                    W, x, b, xo); note_launch();           \
    return cudaGetLastError();                                                              \
  }
  if (al && bs <= 16) {
    switch (bs) {
      GASA_JAC_CASE(1) GASA_JAC_CASE(2) GASA_JAC_CASE(3) GASA_JAC_CASE(4) GASA_JAC_CASE(5)
      GASA_JAC_CASE(6) GASA_JAC_CASE(7) GASA_JAC_CASE(8) GASA_JAC_CASE(9) GASA_JAC_CASE(10)
      GASA_JAC_CASE(11) GASA_JAC_CASE(12) GASA_JAC_CASE(13) GASA_JAC_CASE(14)
      GASA_JAC_CASE(15) GASA_JAC_CASE(16)
      default: break;
    }
  }
#undef GASA_JAC_CASE
  // generic path: one or more whole block rows per CTA
  int rpb = 256 / bs;
  if (rpb < 1) rpb = 1;
  const int th = rpb * bs;
  if (th > 1024) return cudaErrorInvalidValue;
  launch_k(jacobi_generic<T, MODE>, div_up(n_units, rpb), th, th * sizeof(T), s, n_units, bs, rp, col,
                                                                           val, W, x, b, xo); note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi(int mode, int n_units, int bs, const int *rp, const int *col,
                          const T *val, const T *W, const T *x, const T *b, T *xo,
                          cudaStream_t s, int64_t nnzb) {
  if (mode == JAC_SWEEP && blk_applies(bs, n_units, nnzb)) {
    const cudaError_t e = launch_blk<T>(3, n_units, bs, nnzb, rp, col, val, W, x, b, xo, s);
    if (e != cudaErrorNotSupported) return e;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (mode == JAC_SWEEP && wide_applies(bs, bs, n_units, nnzb)) {
      const cudaError_t e = launch_wide(3, n_units, bs, bs, nnzb, rp, col, val, W, x, b, xo, s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  if (n_units > 0 && mode != JAC_FIRST && warp_rows(n_units, bs, nnzb)) {
    switch (mode) {
      case JAC_SWEEP: return jac_warp_dispatch<T, JAC_SWEEP>(n_units, bs, rp, col, val, W, x, b, xo, s);
      case JAC_APPLY: return jac_warp_dispatch<T, JAC_APPLY>(n_units, bs, rp, col, val, W, x, b, xo, s);
      default: return jac_warp_dispatch<T, JAC_RELAX>(n_units, bs, rp, col, val, W, x, b, xo, s);
    }
  }
  switch (mode) {
    case JAC_SWEEP: return jac_dispatch<T, JAC_SWEEP>(n_units, bs, rp, col, val, W, x, b, xo, s);
    case JAC_FIRST: return jac_dispatch<T, JAC_FIRST>(n_units, bs, rp, col, val, W, x, b, xo, s);
    case JAC_APPLY: return jac_dispatch<T, JAC_APPLY>(n_units, bs, rp, col, val, W, x, b, xo, s);
    default: return jac_dispatch<T, JAC_RELAX>(n_units, bs, rp, col, val, W, x, b, xo, s);
  }
}
template cudaError_t launch_jacobi<double>(int, int, int, const int *, const int *,
                                           const double *, const double *, const double *,
                                           const double *, double *, cudaStream_t, int64_t);
template cudaError_t launch_jacobi<float>(int, int, int, const int *, const int *,
                                          const float *, const float *, const float *,
                                          const float *, float *, cudaStream_t, int64_t);

// ----------------------------------------------------------------------------
// multi-column relaxation x_c <- x_c - W A x_c (Eq. bsmooth), column per
// blockIdx.y, columns given by device pointer tables
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
relax_multi_kernel(int n_units, int bs, const int *__restrict__ rp, const int *__restrict__ col,
                   const double *__restrict__ val, const double *__restrict__ Wm,
                   const double *const *__restrict__ xin, double *const *__restrict__ xout) {
  extern __shared__ double res_m[];
  const double *x = xin[blockIdx.y];
  double *xo = xout[blockIdx.y];
  const int rpb = blockDim.x / bs;
  const int li = threadIdx.x / bs;
  const int r = threadIdx.x - li * bs;
  const int i = blockIdx.x * rpb + li;
  const bool active = (li < rpb) && (i < n_units);
  const size_t row = (size_t)i * bs + r;
  double v = 0.0;
  if (active) {
    const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
    double acc = 0.0;
    for (int k = beg; k < end; ++k) {
      const int j = __ldg(col + k);
      const double *a = val + ((size_t)k * bs + r) * bs;
      const double *xj = x + (size_t)j * bs;
      for (int c = 0; c < bs; ++c) acc = fma(__ldg(a + c), xj[c], acc);
    }
    v = -acc;
  }
  res_m[threadIdx.x] = v;
  __syncthreads();
  if (!active) return;
  const double *w = Wm + row * bs;
  double out = 0.0;
  for (int c = 0; c < bs; ++c) out = fma(__ldg(w + c), res_m[li * bs + c], out);
  xo[row] = x[row] + out;
}

cudaError_t launch_relax_multi(int n_units, int bs, const int *rp, const int *col,
                               const double *val, const double *W, const double *const *xin,
                               double *const *xout, int nc, cudaStream_t s) {
  if (n_units == 0 || nc == 0) return cudaSuccess;
  int rpb = 256 / bs;
  if (rpb < 1) rpb = 1;
  const int th = rpb * bs;
  if (th > 1024) return cudaErrorInvalidValue;
  dim3 grid(div_up(n_units, rpb), nc);
  launch_k(relax_multi_kernel, grid, th, th * sizeof(double), s, n_units, bs, rp, col, val, W, xin,
                                                           xout); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bsr_mm(int n_brows, int br, int bc, const int *rp, const int *col,
                          const double *val, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int ncols, cudaStream_t s) {
  for (int c = 0; c < ncols; ++c) {
    cudaError_t e = launch_bsr_mv<double>(GASA_MV_ASSIGN, n_brows, br, bc, rp, col, val,
                                          X + (size_t)c * ldx, nullptr, Y + (size_t)c * ldy, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ----------------------------------------------------------------------------
// dense y = A x (coarsest level A = A_N^{-1}, or the dense bottom operator of
// the V-cycle; A row-major FP64, FP64 arithmetic): a CTA of 256 threads per
// row, thread t sums columns t, t + 256, ... in order (eight in flight), then
// a warp tree and the eight warp sums in order
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
dense_mv_kernel(int n, int ld, const double *__restrict__ A, const T *__restrict__ x,
                T *__restrict__ y) {
  __shared__ double sh[8];
  const int row = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double *a = A + (size_t)row * ld;
  double acc = 0.0;
  int j = threadIdx.x;
  for (; j + 7 * 256 < n; j += 8 * 256) {
    double av[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      av[u] = __ldg(a + j + u * 256);
      xv[u] = (double)__ldg(x + j + u * 256);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = fma(av[u], xv[u], acc);
  }
  for (; j < n; j += 256) acc = fma(__ldg(a + j), (double)__ldg(x + j), acc);
  acc = warp_sum(acc);
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += sh[w];
    y[row] = (T)v;
  }
}

// y = M x for the FP32 cycle's dense bottom operator: M as exact two-term
// FP32 splits (Mh the FP32 rounding of M, Ml that of M - Mh), FP32 x,
// products and sums in double-single arithmetic on FP32 units (the scheme of
// bsr_mv_ds_kernel with x exact in FP32), so each row agrees with the FP64
// product to about 2^-47 of sum |m x|; GB300's FP64 pipe would take n^2 FMAs
// at a small fraction of the FP32 rate.  A CTA of 256 threads per row, thread
// t over columns t, t + 256, ... (eight in flight), its (s, lo) pair to FP64,
// then a warp tree and the eight warp sums in order.
__global__ void __launch_bounds__(256)
dense_mv_ds_kernel(int n, int ld, const float *__restrict__ Mh, const float *__restrict__ Ml,
                   const float *__restrict__ x, float *__restrict__ y) {
  __shared__ double sh[8];
  const int row = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float *h = Mh + (size_t)row * ld;
  const float *l = Ml + (size_t)row * ld;
  float s = 0.0f, lo = 0.0f;
  auto add = [&](float ah, float al, float xh) {
    const float pr = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -pr);
    const float cross = __fmul_rn(al, xh);
    const float s1 = __fadd_rn(s, pr);
    const float bp = __fsub_rn(s1, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bp)), __fsub_rn(pr, bp));
    s = s1;
    lo = __fadd_rn(lo, __fadd_rn(err, __fadd_rn(e, cross)));
  };
  int j = threadIdx.x;
  for (; j + 7 * 256 < n; j += 8 * 256) {
    float hv[8], lv[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      hv[u] = __ldg(h + j + u * 256);
      lv[u] = __ldg(l + j + u * 256);
      xv[u] = __ldg(x + j + u * 256);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) add(hv[u], lv[u], xv[u]);
  }
  for (; j < n; j += 256) add(__ldg(h + j), __ldg(l + j), __ldg(x + j));
  double v = (double)s + (double)lo;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w];
    y[row] = (float)t;
  }
}

cudaError_t launch_dense_mv_ds(int n, int ld, const float *Mh, const float *Ml, const float *x,
                               float *y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_k(dense_mv_ds_kernel, n, 256, 0, s, n, ld, Mh, Ml, x, y);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dense_mv(int n, const double *A, const T *x, T *y, cudaStream_t s, int ld) {
  if (n == 0) return cudaSuccess;
  if (ld < n) ld = n;
  launch_k(dense_mv_kernel<T>, n, 256, 0, s, n, ld, A, x, y); note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_dense_mv<double>(int, const double *, const double *, double *,
                                             cudaStream_t, int);
template cudaError_t launch_dense_mv<float>(int, const double *, const float *, float *,
                                            cudaStream_t, int);

}  // namespace gasa
