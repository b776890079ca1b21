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
// (one group, two rows per lane, when br > 32) and group g of warp w takes
// the blocks beg + w*G + g, beg + (w + NW)*G + g, ...; lane r of a group
// reads row r of its block (the group's lanes together read the block's
// contiguous br*bc values) with 16- or 8-byte loads where bc and the
// pointers allow, and the block's bc entries of x.  Each lane keeps one
// partial sum per row it owns (even and odd columns apart, in column order,
// whatever the load width); the team's partial sums meet in shared memory
// and are added in a fixed order (warp, then group), so every row is summed
// in an order that depends only on the matrix and NW.
//
// Operations: y = A x, y = b - A x, y += A x for any br x bc blocks (at most
// 40 x 40), the block-Jacobi step x_out = x + W (b - A x) of Alg. 1
// (W = w D^{-1}, square blocks), and the fused residual and restriction
// y = R b - (R A) x of Alg. 2 with the next level's first step W y.
#include "common.cuh"
#include "internal.h"

namespace gasa {

namespace {

constexpr int kWideThreads = 256;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideMaxRows = 40;    // rows and columns of a block at most

enum { WIDE_ASSIGN = 0, WIDE_RESID = 1, WIDE_ADD = 2, WIDE_SWEEP = 3, WIDE_RFUSED = 4 };

// one lane's rows (r0 and, with two, r0 + 32) over the blocks kbeg, kbeg +
// step, ... < end of one block row: adds sign * (row . x_col) to a0, a1
template <int VW>
__device__ __forceinline__ void lane_rows(int kbeg, int end, int step, int br, int bc, int r0,
                                          bool two, const int *__restrict__ col,
                                          const float *__restrict__ val,
                                          const float *__restrict__ x, float sign, float &a0,
                                          float &a1) {
  for (int k = kbeg; k < end; k += step) {
    const int j = __ldg(col + k);
    const float *ar0 = val + ((size_t)k * br + r0) * bc;
    const float *ar1 = ar0 + (size_t)32 * bc;
    const float *xj = x + (size_t)j * bc;
    float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
    if constexpr (VW == 4) {
      for (int c = 0; c < bc; c += 4) {
        const float4 xv = __ldg(reinterpret_cast<const float4 *>(xj + c));
        const float4 av = __ldg(reinterpret_cast<const float4 *>(ar0 + c));
        s0 = fmaf(av.x, xv.x, s0);
        s1 = fmaf(av.y, xv.y, s1);
        s0 = fmaf(av.z, xv.z, s0);
        s1 = fmaf(av.w, xv.w, s1);
        if (two) {
          const float4 bv = __ldg(reinterpret_cast<const float4 *>(ar1 + c));
          t0 = fmaf(bv.x, xv.x, t0);
          t1 = fmaf(bv.y, xv.y, t1);
          t0 = fmaf(bv.z, xv.z, t0);
          t1 = fmaf(bv.w, xv.w, t1);
        }
      }
    } else if constexpr (VW == 2) {
      for (int c = 0; c < bc; c += 2) {
        const float2 xv = __ldg(reinterpret_cast<const float2 *>(xj + c));
        const float2 av = __ldg(reinterpret_cast<const float2 *>(ar0 + c));
        s0 = fmaf(av.x, xv.x, s0);
        s1 = fmaf(av.y, xv.y, s1);
        if (two) {
          const float2 bv = __ldg(reinterpret_cast<const float2 *>(ar1 + c));
          t0 = fmaf(bv.x, xv.x, t0);
          t1 = fmaf(bv.y, xv.y, t1);
        }
      }
    } else {
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
    }
    a0 += sign * (s0 + s1);
    a1 += sign * (t0 + t1);
  }
}

// OP WIDE_ASSIGN / RESID / ADD / SWEEP on (rp, col, val); WIDE_RFUSED: the
// fused residual and restriction y = R b - (R A) x with R = (rp, col, val),
// R A = (rp2, col2, val2), and, with Wm (the next level's w D^{-1}), its first
// smoothing step x2o = Wm y
template <int OP, int VW>
__global__ void __launch_bounds__(kWideThreads)
bsr_wide_kernel(int n_brows, int br, int bc, int nw, const int *__restrict__ rp,
                const int *__restrict__ col, const float *__restrict__ val,
                const float *__restrict__ Wm, const float *__restrict__ x,
                const float *__restrict__ b, float *__restrict__ y, const int *__restrict__ rp2,
                const int *__restrict__ col2, const float *__restrict__ val2,
                float *__restrict__ x2o) {
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
    const int step = nw * G, off = wt * G + g;
    if (OP == WIDE_RFUSED) {
      lane_rows<VW>(__ldg(rp + u) + off, __ldg(rp + u + 1), step, br, bc, r0, two, col, val, b,
                    1.f, a0, a1);
      lane_rows<VW>(__ldg(rp2 + u) + off, __ldg(rp2 + u + 1), step, br, bc, r0, two, col2, val2, x,
                    -1.f, a0, a1);
    } else {
      lane_rows<VW>(__ldg(rp + u) + off, __ldg(rp + u + 1), step, br, bc, r0, two, col, val, x,
                    1.f, a0, a1);
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
    else if (OP == WIDE_RFUSED) {
      y[t] = v;
      res[w0][r] = v;
    } else {
      res[w0][r] = b[t] - v;
    }
  }
  if (OP == WIDE_RFUSED && !Wm) return;
  if (OP != WIDE_SWEEP && OP != WIDE_RFUSED) return;
  __syncwarp();
  // SWEEP: x_out = x + W (b - A x); RFUSED: x2o = Wm y (W row r against res)
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
    if (OP == WIDE_SWEEP) y[t] = x[t] + (o0 + o1);
    else x2o[t] = o0 + o1;
  }
}

// warps per block row: about four blocks per group, at most a CTA
int wide_team(int br, double avg) {
  const int G = br <= 32 ? 32 / br : 1;
  int nw = 1;
  while (nw < kWideWarps && nw * G * 4 < avg) nw *= 2;
  return nw;
}

bool al(const void *p, size_t a) { return p == nullptr || ((uintptr_t)p % a) == 0; }

// widest row load the block width and every row pointer allow
int wide_vec(int bc, const void *v1, const void *x1, const void *v2, const void *x2) {
  if (bc % 4 == 0 && al(v1, 16) && al(x1, 16) && al(v2, 16) && al(x2, 16)) return 4;
  if (bc % 2 == 0 && al(v1, 8) && al(x1, 8) && al(v2, 8) && al(x2, 8)) return 2;
  return 1;
}

template <int OP>
void wide_go(int vw, int grid, cudaStream_t s, int n_brows, int br, int bc, int nw, const int *rp,
             const int *col, const float *val, const float *W, const float *x, const float *b,
             float *y, const int *rp2, const int *col2, const float *val2, float *x2o) {
  if (vw == 4)
    launch_k(bsr_wide_kernel<OP, 4>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col, val, W,
             x, b, y, rp2, col2, val2, x2o);
  else if (vw == 2)
    launch_k(bsr_wide_kernel<OP, 2>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col, val, W,
             x, b, y, rp2, col2, val2, x2o);
  else
    launch_k(bsr_wide_kernel<OP, 1>, grid, kWideThreads, 0, s, n_brows, br, bc, nw, rp, col, val, W,
             x, b, y, rp2, col2, val2, x2o);
}

}  // namespace

bool wide_applies(int br, int bc, int n_brows, int64_t nnzb) {
  return (br > 8 || bc > 8) && br <= kWideMaxRows && bc <= kWideMaxRows && n_brows > 0 &&
         nnzb >= 8LL * n_brows;
}

cudaError_t launch_wide(int op, int n_brows, int br, int bc, int64_t nnzb, const int *rp,
                        const int *col, const float *val, const float *W, const float *x,
                        const float *b, float *y, cudaStream_t s) {
  if (n_brows == 0) return cudaSuccess;
  if (br > kWideMaxRows || bc > kWideMaxRows || (op == WIDE_SWEEP && br != bc))
    return cudaErrorNotSupported;
  const int nw = wide_team(br, (double)nnzb / (double)n_brows);
  const int grid = div_up(n_brows, kWideWarps / nw);
  const int vw = wide_vec(bc, val, x, nullptr, nullptr);
  switch (op) {
    case WIDE_ASSIGN:
      wide_go<WIDE_ASSIGN>(vw, grid, s, n_brows, br, bc, nw, rp, col, val, W, x, b, y, nullptr,
                           nullptr, nullptr, nullptr);
      break;
    case WIDE_RESID:
      wide_go<WIDE_RESID>(vw, grid, s, n_brows, br, bc, nw, rp, col, val, W, x, b, y, nullptr,
                          nullptr, nullptr, nullptr);
      break;
    case WIDE_ADD:
      wide_go<WIDE_ADD>(vw, grid, s, n_brows, br, bc, nw, rp, col, val, W, x, b, y, nullptr,
                        nullptr, nullptr, nullptr);
      break;
    default:
      wide_go<WIDE_SWEEP>(vw, grid, s, n_brows, br, bc, nw, rp, col, val, W, x, b, y, nullptr,
                          nullptr, nullptr, nullptr);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_wide_restrict(int n_brows, int br, int bc, int64_t nnzb, const int *rrp,
                                 const int *rcol, const float *rval, const int *arp,
                                 const int *acol, const float *aval, const float *b,
                                 const float *x, float *y, const float *Wn, float *xn,
                                 cudaStream_t s) {
  if (n_brows == 0) return cudaSuccess;
  if (br > kWideMaxRows || bc > kWideMaxRows) return cudaErrorNotSupported;
  const int nw = wide_team(br, (double)nnzb / (double)n_brows);
  const int grid = div_up(n_brows, kWideWarps / nw);
  const int vw = wide_vec(bc, rval, b, aval, x);
  wide_go<WIDE_RFUSED>(vw, grid, s, n_brows, br, bc, nw, rrp, rcol, rval, Wn, x, b, y, arp, acol,
                       aval, xn);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gasa
