// Coarse-level block-sparse products with small square blocks (s <= 8) in
// FP32: one lane per block.
//
// Below level 0 every unit is an aggregate with s = a handful of dofs, and
// each Galerkin product widens the stencil (tens to over a hundred blocks
// per block row).  A thread per scalar row would walk that row's blocks one
// after another with s-wide loads; here a team of TL lanes owns a block row
// and lane l takes whole blocks beg + l, beg + l + TL, ...: it reads the
// s x s block (s*s contiguous values) with the widest aligned vector loads
// and the matching s entries of x, two blocks at a time, and keeps s
// partial row sums.  The team's sums meet in an xor-shuffle (and, for teams
// wider than a warp, in shared memory in a fixed order), so every row is
// summed in an order that depends only on the matrix.
//
// Operations: y = A x, y = b - A x, y += A x, and the block-Jacobi step
// x_out = x + W (b - A x) of Alg. 1 with W = w D^{-1}.
#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"

namespace gasa {

namespace {

enum { BLK_ASSIGN = 0, BLK_RESID = 1, BLK_ADD = 2, BLK_SWEEP = 3 };

template <typename T, int N>
struct BlkVec {
  // widest load (in elements) that keeps a run of N values aligned
  static constexpr int bytes = N * (int)sizeof(T);
  static constexpr int value = (bytes % 16 == 0) ? 16 / (int)sizeof(T)
                               : (bytes % 8 == 0 && sizeof(T) <= 8) ? 8 / (int)sizeof(T)
                                                                    : 1;
};

template <typename T, int N>
__device__ __forceinline__ void load_run(const T *p, T (&out)[N]) {
  constexpr int W = BlkVec<T, N>::value;
#pragma unroll
  for (int i = 0; i < N; i += W) load_vec<T, W>(p + i, out + i);
}

template <typename T, int S, int TL, int OP>
__global__ void __launch_bounds__(256)
bsr_blk_kernel(int n_brows, const int *__restrict__ rp, const int *__restrict__ col,
               const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
               const T *__restrict__ b, T *__restrict__ y) {
  constexpr int TW = TL < 32 ? TL : 32;          // lanes of a team inside one warp
  constexpr int WPT = TL > 32 ? TL / 32 : 1;     // warps per team
  __shared__ T red[(256 / 32) * S];
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int u = (int)(gt / TL);
  const int l = (int)(gt % TL);
  T acc[S];
#pragma unroll
  for (int r = 0; r < S; ++r) acc[r] = T(0);
  // the epilogue's operands (row l of W_u, b_u, x_t) do not depend on the
  // product: lanes l < S load them first so that their latency overlaps the
  // block loop instead of following it
  const bool writer = u < n_brows && l < S;
  const size_t t = (size_t)u * S + l;
  T bv[S], wv[S], xt = T(0), bt = T(0), yt = T(0);
  if (OP == BLK_SWEEP && writer) {
    load_run<T, S>(b + (size_t)u * S, bv);
    load_run<T, S>(Wm + t * S, wv);
    xt = x[t];
  }
  if (OP == BLK_RESID && writer) bt = b[t];
  if (OP == BLK_ADD && writer) yt = y[t];
  if (u < n_brows) {
    const int beg = __ldg(rp + u), end = __ldg(rp + u + 1);
    int k = beg + l;
    // two blocks in flight per lane while they fit in registers
    for (; S * S <= 25 && k + TL < end; k += 2 * TL) {
      T a0[S * S], a1[S * S], x0[S], x1[S];
      const int j0 = __ldg(col + k), j1 = __ldg(col + k + TL);
      load_run<T, S * S>(val + (size_t)k * S * S, a0);
      load_run<T, S * S>(val + (size_t)(k + TL) * S * S, a1);
      load_run<T, S>(x + (size_t)j0 * S, x0);
      load_run<T, S>(x + (size_t)j1 * S, x1);
#pragma unroll
      for (int r = 0; r < S; ++r) {
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int c = 0; c < S; ++c) {
          s0 = fma(a0[r * S + c], x0[c], s0);
          s1 = fma(a1[r * S + c], x1[c], s1);
        }
        acc[r] += s0 + s1;
      }
    }
    for (; k < end; k += TL) {
      T a0[S * S], x0[S];
      const int j0 = __ldg(col + k);
      load_run<T, S * S>(val + (size_t)k * S * S, a0);
      load_run<T, S>(x + (size_t)j0 * S, x0);
#pragma unroll
      for (int r = 0; r < S; ++r) {
        T s0 = T(0);
#pragma unroll
        for (int c = 0; c < S; ++c) s0 = fma(a0[r * S + c], x0[c], s0);
        acc[r] += s0;
      }
    }
  }
  // team sum: xor-shuffle inside the warp, then the warps of a wide team in
  // a fixed order through shared memory
#pragma unroll
  for (int o = 1; o < TW; o <<= 1) {
#pragma unroll
    for (int r = 0; r < S; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  }
  if constexpr (WPT > 1) {
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int r = 0; r < S; ++r) red[wid * S + r] = acc[r];
    }
    __syncthreads();
    const int w0 = wid - wid % WPT;   // first warp of this team
#pragma unroll
    for (int r = 0; r < S; ++r) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < WPT; ++q) v += red[(w0 + q) * S + r];
      acc[r] = v;
    }
  }
  if (!writer) return;
  // lane l < S of the team writes row l
  if (OP == BLK_SWEEP) {
    T out = T(0);
#pragma unroll
    for (int c = 0; c < S; ++c) out = fma(wv[c], bv[c] - acc[c], out);
    y[t] = xt + out;
    return;
  }
  T v = T(0);
#pragma unroll
  for (int r = 0; r < S; ++r)
    if (r == l) v = acc[r];
  if (OP == BLK_ASSIGN) y[t] = v;
  else if (OP == BLK_RESID) y[t] = bt - v;
  else y[t] = yt + v;
}

// Fused residual and restriction of Alg. 2 with S x SC blocks (S coarse
// rows, SC fine columns; SC = S on the coarse levels, SC up to 16 from the
// finest level): for coarse unit u, y_u = sum_j R_uj b_j - sum_j (R A)_uj x_j,
// the vector R (b - A x) formed without the fine residual; with Wn also the
// next level's first smoothing step xn_u = Wn_u y_u from zero (every lane of
// the team holds all S entries of y_u after the team sum).  One block per
// lane at a time, team sums as in bsr_blk_kernel.
template <typename T, int S, int SC, int TL>
__global__ void __launch_bounds__(256)
blk_restrict_kernel(int n_brows, const int *__restrict__ rrp, const int *__restrict__ rcol,
                    const T *__restrict__ rval, const int *__restrict__ arp,
                    const int *__restrict__ acol, const T *__restrict__ aval,
                    const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ y,
                    const T *__restrict__ Wn, T *__restrict__ xn) {
  constexpr int TW = TL < 32 ? TL : 32;
  constexpr int WPT = TL > 32 ? TL / 32 : 1;
  __shared__ T red[(256 / 32) * S];
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int u = (int)(gt / TL);
  const int l = (int)(gt % TL);
  T acc[S];
#pragma unroll
  for (int r = 0; r < S; ++r) acc[r] = T(0);
  if (u < n_brows) {
    for (int k = __ldg(rrp + u) + l; k < __ldg(rrp + u + 1); k += TL) {
      T a0[S * SC], v0[SC];
      load_run<T, S * SC>(rval + (size_t)k * S * SC, a0);
      load_run<T, SC>(b + (size_t)__ldg(rcol + k) * SC, v0);
#pragma unroll
      for (int r = 0; r < S; ++r) {
        T s0 = T(0);
#pragma unroll
        for (int c = 0; c < SC; ++c) s0 = fma(a0[r * SC + c], v0[c], s0);
        acc[r] += s0;
      }
    }
    for (int k = __ldg(arp + u) + l; k < __ldg(arp + u + 1); k += TL) {
      T a0[S * SC], v0[SC];
      load_run<T, S * SC>(aval + (size_t)k * S * SC, a0);
      load_run<T, SC>(x + (size_t)__ldg(acol + k) * SC, v0);
#pragma unroll
      for (int r = 0; r < S; ++r) {
        T s0 = T(0);
#pragma unroll
        for (int c = 0; c < SC; ++c) s0 = fma(a0[r * SC + c], v0[c], s0);
        acc[r] -= s0;
      }
    }
  }
#pragma unroll
  for (int o = 1; o < TW; o <<= 1) {
#pragma unroll
    for (int r = 0; r < S; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  }
  if constexpr (WPT > 1) {
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int r = 0; r < S; ++r) red[wid * S + r] = acc[r];
    }
    __syncthreads();
    const int w0 = wid - wid % WPT;
#pragma unroll
    for (int r = 0; r < S; ++r) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < WPT; ++q) v += red[(w0 + q) * S + r];
      acc[r] = v;
    }
  }
  if (u >= n_brows || l >= S) return;
  const size_t t = (size_t)u * S + l;
  T v = T(0);
#pragma unroll
  for (int r = 0; r < S; ++r)
    if (r == l) v = acc[r];
  y[t] = v;
  if (Wn) {
    T wv[S];
    load_run<T, S>(Wn + t * S, wv);
    T out = T(0);
#pragma unroll
    for (int c = 0; c < S; ++c) out = fma(wv[c], acc[c], out);
    xn[t] = out;
  }
}

// Lanes per block row: about 2.5 blocks per lane (two in flight, a short
// tail), a power of two in [4, 64] and at least s, so that lanes 0..s-1 of
// the team can write the s rows.
int blk_team(int bs, int n_brows, int64_t nnzb) {
  const double avg = (double)nnzb / (double)(n_brows > 0 ? n_brows : 1);
  int tl = 4;
  while (tl < 64 && tl * 2.5 < avg) tl *= 2;
  while (tl < bs) tl *= 2;
  return tl;
}

template <typename T, int S, int OP>
cudaError_t blk_launch_s(int n_brows, int64_t nnzb, const int *rp, const int *col, const T *val,
                         const T *W, const T *x, const T *b, T *y, cudaStream_t s) {
  const int TL = blk_team(S, n_brows, nnzb);
  const int grid = div_up((long long)n_brows * TL, 256);
#define GASA_BLK_TL(V)                                                                       \
  case V:                                                                                    \
    launch_k(bsr_blk_kernel<T, S, (V < S ? 8 : V), OP>, grid, 256, 0, s, n_brows, rp, col, val, W, \
             x, b, y);                                                                       \
    break;
  switch (TL) {
    GASA_BLK_TL(4) GASA_BLK_TL(8) GASA_BLK_TL(16) GASA_BLK_TL(32)
    default: launch_k(bsr_blk_kernel<T, S, 64, OP>, grid, 256, 0, s, n_brows, rp, col, val, W, x, b, y); break;
  }
#undef GASA_BLK_TL
  note_launch();
  return cudaGetLastError();
}

template <typename T, int OP>
cudaError_t blk_launch(int n_brows, int bs, int64_t nnzb, const int *rp, const int *col,
                       const T *val, const T *W, const T *x, const T *b, T *y, cudaStream_t s) {
  switch (bs) {
    case 2: return blk_launch_s<T, 2, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 3: return blk_launch_s<T, 3, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 4: return blk_launch_s<T, 4, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 5: return blk_launch_s<T, 5, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 6: return blk_launch_s<T, 6, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 7: return blk_launch_s<T, 7, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    case 8: return blk_launch_s<T, 8, OP>(n_brows, nnzb, rp, col, val, W, x, b, y, s);
    default: return cudaErrorNotSupported;
  }
}

template <int S, int SC = S>
cudaError_t blk_restrict_s(int n_brows, int64_t nnzb, const int *rrp, const int *rcol,
                           const float *rval, const int *arp, const int *acol, const float *aval,
                           const float *b, const float *x, float *y, const float *Wn, float *xn,
                           cudaStream_t s) {
  const int TL = blk_team(S, n_brows, nnzb);
  const int grid = div_up((long long)n_brows * TL, 256);
#define GASA_BLK_RTL(V)                                                                     \
  case V:                                                                                   \
    launch_k(blk_restrict_kernel<float, S, SC, (V < S ? 8 : V)>, grid, 256, 0, s, n_brows,  \
             rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn);                            \
    break;
  switch (TL) {
    GASA_BLK_RTL(4) GASA_BLK_RTL(8) GASA_BLK_RTL(16) GASA_BLK_RTL(32)
    default:
      launch_k(blk_restrict_kernel<float, S, SC, 64>, grid, 256, 0, s, n_brows, rrp, rcol, rval,
               arp, acol, aval, b, x, y, Wn, xn);
      break;
  }
#undef GASA_BLK_RTL
  note_launch();
  return cudaGetLastError();
}

bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

bool blk_applies(int bs, int n_brows, int64_t nnzb) {
  return bs >= 2 && bs <= 8 && n_brows > 0 && nnzb >= 6LL * n_brows;
}

// rectangular blocks from the finest level: br coarse rows (4 or 8) by bc
// fine columns (9 or 10), with at least six blocks of R and R A per row
bool blk_restrict_rect_applies(int br, int bc, int n_brows, int64_t nnzb) {
  return (br == 4 || br == 8) && (bc == 9 || bc == 10) && n_brows > 0 && nnzb >= 6LL * n_brows;
}

cudaError_t launch_blk_restrict_rect(int n_brows, int br, int bc, int64_t nnzb, const int *rrp,
                                     const int *rcol, const float *rval, const int *arp,
                                     const int *acol, const float *aval, const float *b,
                                     const float *x, float *y, const float *Wn, float *xn,
                                     cudaStream_t s) {
  // 16-byte block runs and 8-byte x runs (bc = 10), else 4-byte loads
  if (!blk_restrict_rect_applies(br, bc, n_brows, nnzb)) return cudaErrorNotSupported;
  if (br == 4 && bc == 10)
    return blk_restrict_s<4, 10>(n_brows, nnzb, rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn, s);
  if (br == 4 && bc == 9)
    return blk_restrict_s<4, 9>(n_brows, nnzb, rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn, s);
  if (br == 8 && bc == 10)
    return blk_restrict_s<8, 10>(n_brows, nnzb, rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn, s);
  return blk_restrict_s<8, 9>(n_brows, nnzb, rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn, s);
}

cudaError_t launch_blk_restrict(int n_brows, int bs, int64_t nnzb, const int *rrp,
                                const int *rcol, const float *rval, const int *arp,
                                const int *acol, const float *aval, const float *b,
                                const float *x, float *y, const float *Wn, float *xn,
                                cudaStream_t s) {
  switch (bs) {
#define GASA_BLK_RS(SV) \
  case SV: return blk_restrict_s<SV>(n_brows, nnzb, rrp, rcol, rval, arp, acol, aval, b, x, y, Wn, xn, s);
    GASA_BLK_RS(2) GASA_BLK_RS(3) GASA_BLK_RS(4) GASA_BLK_RS(5) GASA_BLK_RS(6) GASA_BLK_RS(7)
    GASA_BLK_RS(8)
#undef GASA_BLK_RS
    default: return cudaErrorNotSupported;
  }
}

// FP32 only: the team sums add s * log2(team) additions per lane, which the
// FP32 pipe absorbs; on GB300's narrow FP64 pipe they cost more than the
// loads they hide (measured: FP64 V-cycle 1.69 -> 2.36 ms per iteration), so
// FP64 keeps the thread-, warp- and CTA-per-row kernels.
template <>
cudaError_t launch_blk<double>(int, int, int, int64_t, const int *, const int *, const double *,
                               const double *, const double *, const double *, double *,
                               cudaStream_t) {
  return cudaErrorNotSupported;
}

template <>
cudaError_t launch_blk<float>(int op, int n_brows, int bs, int64_t nnzb, const int *rp,
                              const int *col, const float *val, const float *W, const float *x,
                              const float *b, float *y, cudaStream_t s) {
  if (!blk_applies(bs, n_brows, nnzb)) return cudaErrorNotSupported;
  // vector loads need the arrays aligned like their runs (cudaMalloc gives 256 bytes)
  for (const void *p : {(const void *)val, (const void *)W, (const void *)x, (const void *)b})
    if (p && !aligned_to(p, 16)) return cudaErrorNotSupported;
  using T = float;
  switch (op) {
    case BLK_ASSIGN: return blk_launch<T, BLK_ASSIGN>(n_brows, bs, nnzb, rp, col, val, W, x, b, y, s);
    case BLK_RESID: return blk_launch<T, BLK_RESID>(n_brows, bs, nnzb, rp, col, val, W, x, b, y, s);
    case BLK_ADD: return blk_launch<T, BLK_ADD>(n_brows, bs, nnzb, rp, col, val, W, x, b, y, s);
    case BLK_SWEEP: return blk_launch<T, BLK_SWEEP>(n_brows, bs, nnzb, rp, col, val, W, x, b, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gasa
