// Shared device helpers of the GB300 alpha-SA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gasa.h"

namespace gasa {

constexpr int kNumSM = 152;          // GB300: 2 dies x 76 SMs
constexpr int kRedBlocks = 2 * kNumSM; // fixed grid of the deterministic reductions
constexpr int kRedThreads = 256;

// ----------------------------------------------------------------------------
// warp / block reductions (fixed order => deterministic)
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// block-wide sum; every thread gets the result.  `sh` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// Sum of `n` partials in a fixed order by one block; every thread gets it.
__device__ __forceinline__ double block_sum_partials(const double *p, int n, double *sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
  return block_sum(v, sh);
}

// ----------------------------------------------------------------------------
// vector load helpers
// ----------------------------------------------------------------------------
template <typename T, int N>
struct VecOf;
template <> struct VecOf<double, 1> { using type = double; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 4> { using type = float4; };

// widest vector (in elements) that keeps a row of BC elements aligned
template <typename T, int BC>
struct RowVec {
  static constexpr int bytes = BC * (int)sizeof(T);
  static constexpr int w16 = (bytes % 16 == 0) ? 16 / (int)sizeof(T) : 0;
  static constexpr int w8 = (bytes % 8 == 0 && sizeof(T) <= 8) ? 8 / (int)sizeof(T) : 1;
  static constexpr int value = w16 ? w16 : w8;
};

template <typename T, int W>
__device__ __forceinline__ void load_vec(const T *p, T *out) {
  if constexpr (W == 1) {
    out[0] = __ldg(p);
  } else {
    using V = typename VecOf<T, W>::type;
    V v = __ldg(reinterpret_cast<const V *>(p));
    const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int i = 0; i < W; ++i) out[i] = s[i];
  }
}

// streaming (evict-first) vector load for matrix values read once per pass
template <typename T, int W>
__device__ __forceinline__ void load_vec_stream(const T *p, T *out) {
  if constexpr (W == 1) {
    out[0] = __ldcs(p);
  } else {
    using V = typename VecOf<T, W>::type;
    V v = __ldcs(reinterpret_cast<const V *>(p));
    const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int i = 0; i < W; ++i) out[i] = s[i];
  }
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// plain kernel launch through the extended API (one place to change launch
// attributes); programmatic dependent launch was measured here and removed:
// the graph launches already hide the gaps between kernels (0.341 vs 0.342
// solves/s for the FP32 V-cycle on the P3 256x256 solve, 7 % slower for FP64)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace gasa
