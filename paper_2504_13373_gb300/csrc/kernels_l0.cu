// Level-0 block-Jacobi smoothing step with two blocks of the block row in
// flight per thread (option, for A/B timing against jacobi_kernel).
//
// Same operation and the same arithmetic order as jacobi_kernel in SWEEP
// mode, x_out = x + W (b - A x): thread (li, r) owns scalar row r of block
// row i and adds the products of row r of each block to one accumulator in
// the block row's order, so results are bit-identical.  The loads of two
// consecutive blocks (their column indices, A rows and x segments) are
// issued before their products, which doubles the bytes each thread has in
// flight at the cost of registers.
#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"

namespace gasa {

namespace {

template <typename T, int BS>
__global__ void __launch_bounds__(256)
jacobi_u2_kernel(int n_units, const int *__restrict__ rp, const int *__restrict__ col,
                 const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
                 const T *__restrict__ b, T *__restrict__ xo) {
  pdl_entry();
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
    const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
    T acc = T(0);
    int k = beg;
    for (; k + 1 < end; k += 2) {
      const int j0 = __ldg(col + k), j1 = __ldg(col + k + 1);
      const T *a0 = val + ((size_t)k * BS + r) * BS;
      const T *a1 = val + ((size_t)(k + 1) * BS + r) * BS;
      T av0[BS], av1[BS], xv0[BS], xv1[BS];
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec_stream<T, W>(a0 + c, av0 + c);
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec_stream<T, W>(a1 + c, av1 + c);
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec<T, W>(x + (size_t)j0 * BS + c, xv0 + c);
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec<T, W>(x + (size_t)j1 * BS + c, xv1 + c);
#pragma unroll
      for (int c = 0; c < BS; ++c) acc = fma(av0[c], xv0[c], acc);
#pragma unroll
      for (int c = 0; c < BS; ++c) acc = fma(av1[c], xv1[c], acc);
    }
    if (k < end) {
      const int j = __ldg(col + k);
      const T *a = val + ((size_t)k * BS + r) * BS;
      T av[BS], xv[BS];
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec_stream<T, W>(a + c, av + c);
#pragma unroll
      for (int c = 0; c < BS; c += W) load_vec<T, W>(x + (size_t)j * BS + c, xv + c);
#pragma unroll
      for (int c = 0; c < BS; ++c) acc = fma(av[c], xv[c], acc);
    }
    v = b[row] - acc;
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
  out += x[row];
  xo[row] = out;
}

std::atomic<int> g_u2{-1};

bool aligned16_l0(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

// off unless GASA_L0_U2=1 in the environment
bool jacobi_u2_enabled() {
  int v = g_u2.load(std::memory_order_relaxed);
  if (v < 0) {
    const char *e = std::getenv("GASA_L0_U2");
    v = (e && e[0] == '1') ? 1 : 0;
    g_u2.store(v, std::memory_order_relaxed);
  }
  return v != 0;
}

template <typename T>
cudaError_t launch_jacobi_u2(int n_units, int bs, const int *rp, const int *col, const T *val,
                             const T *W, const T *x, const T *b, T *xo, cudaStream_t s) {
  if (n_units == 0) return cudaSuccess;
  if (!aligned16_l0(val) || !aligned16_l0(W) || !aligned16_l0(x)) return cudaErrorNotSupported;
#define GASA_U2_CASE(BS)                                                                     \
  case BS:                                                                                   \
    launch_k(jacobi_u2_kernel<T, BS>, div_up(n_units, 256 / BS), 256, 0, s, n_units, rp, col, \
             val, W, x, b, xo);                                                              \
    note_launch();                                                                           \
    return cudaGetLastError();
  switch (bs) {
    GASA_U2_CASE(3) GASA_U2_CASE(4) GASA_U2_CASE(9) GASA_U2_CASE(10) GASA_U2_CASE(13)
    default: return cudaErrorNotSupported;
  }
#undef GASA_U2_CASE
}
template cudaError_t launch_jacobi_u2<float>(int, int, const int *, const int *, const float *,
                                             const float *, const float *, const float *, float *,
                                             cudaStream_t);
template cudaError_t launch_jacobi_u2<double>(int, int, const int *, const int *, const double *,
                                              const double *, const double *, const double *,
                                              double *, cudaStream_t);

}  // namespace gasa
