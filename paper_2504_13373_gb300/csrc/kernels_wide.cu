// Coarse-level block-sparse products with wide blocks (more than 8 rows or
// columns) in FP32.
//
// The Galerkin operators below level 0 of the 3-D and convection-diffusion
// workloads have blocks of 12 to 36 rows and tens to hundreds of blocks per
// block row, and at these sizes they hold more bytes than the level-0
// operator.  A lane per whole block (kernels_blk.cu) would need s*s
// registers; a thread per scalar row reads its row's blocks one after
// another with little memory-level parallelism.  Here a team of NW warps
// owns a block row; the lanes of a warp form G = 32 / br groups of br lanes
// (one group of up to 64 rows when br > 32) and group g of warp w takes the
// blocks beg + w*G + g, beg + (w + NW)*G + g, ...; lane r of a group reads row
// r of its block (the group's lanes together read the block's contiguous
// br*bc values) and the block's bc entries of x.  Each lane keeps one partial
// sum per row it owns; the team's partial sums meet in shared memory and are
// added in a fixed order (warp, then group), so every row is summed in an
// order that depends only on the matrix and NW.
//
// Operations: y = A x, y = b - A x, y += A x for any br x bc blocks, and the
// block-Jacobi step x_out = x + W (b - A x) of Alg. 1 (W = w D^{-1}, square
// blocks).
#include "common.cuh"
#include "internal.h"

namespace gasa {

namespace {

constexpr int kWideThreads = 256;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideMaxRows = 64;

enum { WIDE_ASSIGN = 0, WIDE_RESID = 1, WIDE_ADD = 2, WIDE_SWEEP = 3 };

template <int OP>
__global__ void __launch_bounds__(kWideThreads)
bsr_wide_kernel(int n_brows, int br, int bc, int nw, const int *__restrict__ rp,
                const int *__restrict__ col, const float *__restrict__ val,
                const float *__restrict__ Wm, const float *__restrict__ x,
                const float *__restrict__ b, float *__restrict__ y) {
  // red[warp][slot]: each lane's partial row sums (slot = lane, lane + 32)
  __shared__ float red[kWideWarps][kWideMaxRows];
  __shared__ float res[kWideWarps][kWideMaxRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int teams = kWideWarps / nw;
  const int team = warp / nw, wt = warp - team * nw;
  const int u = blockIdx.x * teams + team;
  const int G = br <= 32 ? 32 / br : 1;          // block groups per warp
  const int g = br <= 32 ? lane / br : 0;
  const int r0 = br <= 32 ? lane - g * br : lane;
  const bool lane_on = g < G && r0 < br;
  const bool two = br > 32 && lane + 32 < br;   // second row of this lane
  float a0 = 0.f, a1 = 0.f;
  if (u < n_brows && lane_on) {
    const int beg = __ldg(rp + u), end = __ldg(rp + u + 1);
    const int step = nw * G;
    for (int k = beg + wt * G + g; k < end; k += step) {
      const int j = __ldg(col + k);
      const float *a = val + (size_t)k * br * bc;
      const float *xj = x + (size_t)j * bc;
      const float *ar0 = a + (size_t)r0 * bc;
      const float *ar1 = a + (size_t)(r0 + 32) * bc;
      float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
      int c = 0;
      for (; c + 1 < bc; c += 2) {
        const float x0 = __ldg(xj + c), x1 = __ldg(xj + c + 1);
        s0 = fmaf(__ldg(ar0 + c), x0, s0);
        s1 = fmaf(__ldg(ar0 + c + 1), x1, s1);
        if (two) {
          t0 = fmaf(__ldg(ar1 + c), x0, t0);
          t1 = fmaf(__ldg(ar1 + c + 1), x1, t1);
        }
      }
      if (c < bc) {
        const float xc = __ldg(xj + c);
        s0 = fmaf(__ldg(ar0 + c), xc, s0);
        if (two) t0 = fmaf(__ldg(ar1 + c), xc, t0);
      }
      a0 += s0 + s1;
      a1 += t0 + t1;
    }
  }
  // partial sums to shared memory: slot = g * br + r0 (br <= 32), else r0, r0 + 32
  if (lane_on) red[warp][br <= 32 ? g * br + r0 : r0] = a0;
  if (two) red[warp][lane + 32] = a1;
  __syncthreads();
  if (u >= n_brows || wt != 0) return;
  // the team's first warp adds the partial sums of row r: warps in order, then groups
  const int w0 = team * nw;
  for (int r = lane; r < br; r += 32) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) {
      if (br <= 32) {
        for (int q = 0; q < G; ++q) v += red[w0 + w][q * br + r];
      } else {
        v += red[w0 + w][r];
      }
    }
    const size_t t = (size_t)u * br + r;
    if (OP == WIDE_ASSIGN) y[t] = v;
    else if (OP == WIDE_RESID) y[t] = b[t] - v;
    else if (OP == WIDE_ADD) y[t] = y[t] + v;
    else res[w0][r] = b[t] - v;
  }
  if (OP != WIDE_SWEEP) return;
  __syncwarp();
  // x_out = x + W (b - A x), W row r against the unit's residual
  for (int r = lane; r < br; r += 32) {
    const float *w = Wm + ((size_t)u * br + r) * br;
    float o0 = 0.f, o1 = 0.f;
    int c = 0;
    for (; c + 1 < br; c += 2) {
      o0 = fmaf(__ldg(w + c), res[w0][c], o0);
      o1 = fmaf(__ldg(w + c + 1), res[w0][c + 1], o1);
    }
    if (c < br) o0 = fmaf(__ldg(w + c), res[w0][c], o0);
    const size_t t = (size_t)u * br + r;
    y[t] = x[t] + (o0 + o1);
  }
}

// warps per block row: about four blocks per group, at most a CTA
int wide_team(int br, double avg) {
  const int G = br <= 32 ? 32 / br : 1;
  int nw = 1;
  while (nw < kWideWarps && nw * G * 4 < avg) nw *= 2;
  return nw;
}

}  // namespace

bool wide_applies(int br, int bc, int n_brows, int64_t nnzb) {
  return (br > 8 || bc > 8) && br <= kWideMaxRows && n_brows > 0 && nnzb >= 8LL * n_brows;
}

cudaError_t launch_wide(int op, int n_brows, int br, int bc, int64_t nnzb, const int *rp,
                        const int *col, const float *val, const float *W, const float *x,
                        const float *b, float *y, cudaStream_t s) {
  if (n_brows == 0) return cudaSuccess;
  if (br > kWideMaxRows || (op == WIDE_SWEEP && br != bc)) return cudaErrorNotSupported;
  const int nw = wide_team(br, (double)nnzb / (double)n_brows);
  const int teams = kWideWarps / nw;
  const int grid = div_up(n_brows, teams);
  switch (op) {
    case WIDE_ASSIGN:
      launch_k(bsr_wide_kernel<WIDE_ASSIGN>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col,
               val, W, x, b, y);
      break;
    case WIDE_RESID:
      launch_k(bsr_wide_kernel<WIDE_RESID>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col,
               val, W, x, b, y);
      break;
    case WIDE_ADD:
      launch_k(bsr_wide_kernel<WIDE_ADD>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col,
               val, W, x, b, y);
      break;
    default:
      launch_k(bsr_wide_kernel<WIDE_SWEEP>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col,
               val, W, x, b, y);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace gasa
