// The coarse levels of the V-cycle (Alg. 2) as one persistent launch.
//
// Below level 0 the operators are small (the benchmark's levels 1-7 hold
// 60 MB of FP32 operators together, all of it L2-resident), but a V-cycle
// still takes about nine dependent steps per level: the first smoothing
// step x = w D^{-1} b, t_pre - 1 further steps, the residual, the
// restriction, and on the way up the prolongation and t_post steps.  Launched
// one by one, each step costs a launch and a grid drain, which on these
// levels is most of the step's time.  Here one cooperative launch of every
// resident CTA runs the whole range k0 .. N: the steps are phases separated
// by a grid barrier, each phase spreads its block rows over every warp of
// the grid, and the restriction also takes the next level's first step
// (its team holds all s entries of the coarse unit's new right-hand side).
//
// Arithmetic per block row: a team of TL lanes (a power of two, at most a
// warp) owns the row; lane l takes blocks beg + l, beg + l + TL, ... and keeps
// s partial sums; the team's sums meet in an xor-shuffle; lanes 0..s-1 write
// rows 0..s-1.  The order of every sum depends only on the matrix and TL,
// so repeated launches give the same bits.
//
// Memory ordering: vectors written in one phase and read in a later one
// are read with ld.global.cg (through L2, never a stale L1 line); the
// barrier is the cooperative-groups pattern (CTA barrier, one thread's
// gpu-scope fence and arrival, an acquire spin, CTA barrier).  Every wait is
// bounded by a %globaltimer budget: a CTA that runs out sets the error flag
// and returns, and every other CTA leaves at its next barrier, so a lost
// arrival ends the launch with an error instead of a hang.
#include <cuda_runtime.h>

#include "common.cuh"
#include "grid.h"
#include "internal.h"

namespace gasa {

namespace {

enum { GOP_SWEEP = 0, GOP_RESID = 1, GOP_RESTRICT = 2, GOP_PROLONG = 3 };

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// widest load (elements) that keeps a run of N values of T aligned
template <typename T, int N>
struct RunVec {
  static constexpr int bytes = N * (int)sizeof(T);
  static constexpr int value = (bytes % 16 == 0) ? 16 / (int)sizeof(T)
                               : (bytes % 8 == 0) ? 8 / (int)sizeof(T)
                                                  : 1;
};

// read-only operands (matrices): the non-coherent path is safe
template <typename T, int N>
__device__ __forceinline__ void ld_const(const T *p, T (&out)[N]) {
  constexpr int W = RunVec<T, N>::value;
#pragma unroll
  for (int i = 0; i < N; i += W) load_vec<T, W>(p + i, out + i);
}

// vectors written earlier in the same launch: through L2 only
template <typename T, int W>
__device__ __forceinline__ void ld_cg_vec(const T *p, T *out) {
  if constexpr (W == 1) {
    out[0] = __ldcg(p);
  } else {
    using V = typename VecOf<T, W>::type;
    V v = __ldcg(reinterpret_cast<const V *>(p));
    const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int i = 0; i < W; ++i) out[i] = s[i];
  }
}
template <typename T, int N>
__device__ __forceinline__ void ld_fresh(const T *p, T (&out)[N]) {
  constexpr int W = RunVec<T, N>::value;
#pragma unroll
  for (int i = 0; i < N; i += W) ld_cg_vec<T, W>(p + i, out + i);
}

// Grid barrier number `nb` (1-based) of the launch: true when every CTA
// arrived, false when this CTA gave up (budget spent, or another CTA set the
// error flag).  The counter counts arrivals from zero.
__device__ bool grid_sync(unsigned int *bar, unsigned int nb, int *err,
                          unsigned long long deadline) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = nb * gridDim.x;
    int ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    for (;;) {
      if (ld_acquire_u32(bar) >= target) break;
      if (*(volatile int *)err) {
        ok = 0;
        break;
      }
      if (global_ns() > deadline) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One team phase over the n block rows of an s x s block matrix (S = s):
//  SWEEP:    y = x + W (b - M x)
//  RESID:    y = b - M x
//  RESTRICT: y = M x and, when W is given, y2 = W y (the next level's first
//            smoothing step from zero)
//  PROLONG:  y += M x
template <typename T, int S, int OP>
__device__ void team_phase(int tl, int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const T *__restrict__ val, const T *__restrict__ Wm, const T *x,
                           const T *b, T *y, T *y2) {
  const int lane = threadIdx.x & 31;
  const int tpw = 32 / tl;                      // teams per warp
  const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int l = lane & (tl - 1);
  const int tw = lane / tl;
  for (int base = gwarp * tpw; base < n; base += nwarps * tpw) {
    const int u = base + tw;
    const bool act = u < n;
    T acc[S];
#pragma unroll
    for (int r = 0; r < S; ++r) acc[r] = T(0);
    if (act) {
      const int beg = __ldg(rp + u), end = __ldg(rp + u + 1);
      for (int k = beg + l; k < end; k += tl) {
        const int j = __ldg(col + k);
        T a[S * S], xv[S];
        ld_const<T, S * S>(val + (size_t)k * S * S, a);
        ld_fresh<T, S>(x + (size_t)j * S, xv);
#pragma unroll
        for (int r = 0; r < S; ++r) {
          T s0 = T(0);
#pragma unroll
          for (int c = 0; c < S; ++c) s0 = fma(a[r * S + c], xv[c], s0);
          acc[r] += s0;
        }
      }
    }
    for (int o = 1; o < tl; o <<= 1) {
#pragma unroll
      for (int r = 0; r < S; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
    if (!act || l >= S) continue;
    const size_t t = (size_t)u * S + l;
    T v = T(0);
#pragma unroll
    for (int r = 0; r < S; ++r)
      if (r == l) v = acc[r];
    if (OP == GOP_SWEEP) {
      T bv[S], wv[S];
      ld_fresh<T, S>(b + (size_t)u * S, bv);
      ld_const<T, S>(Wm + t * S, wv);
      T out = T(0);
#pragma unroll
      for (int c = 0; c < S; ++c) out = fma(wv[c], bv[c] - acc[c], out);
      y[t] = __ldcg(x + t) + out;
    } else if (OP == GOP_RESID) {
      y[t] = __ldcg(b + t) - v;
    } else if (OP == GOP_RESTRICT) {
      y[t] = v;
      if (Wm) {
        T wv[S];
        ld_const<T, S>(Wm + t * S, wv);
        T out = T(0);
#pragma unroll
        for (int c = 0; c < S; ++c) out = fma(wv[c], acc[c], out);
        y2[t] = out;
      }
    } else {
      y[t] = __ldcg(y + t) + v;
    }
  }
}

// x = W b (first smoothing step from zero), one thread per scalar row
template <typename T, int S>
__device__ void first_phase(int n, const T *__restrict__ Wm, const T *b, T *x) {
  const int64_t rows = (int64_t)n * S;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows; t += stride) {
    const int64_t u = t / S;
    T bv[S], wv[S];
    ld_fresh<T, S>(b + u * S, bv);
    ld_const<T, S>(Wm + t * S, wv);
    T out = T(0);
#pragma unroll
    for (int c = 0; c < S; ++c) out = fma(wv[c], bv[c], out);
    x[t] = out;
  }
}

// x_N = A_N^{-1} b_N with FP64 arithmetic: a warp per row
template <typename T>
__device__ void coarse_phase(int nc, const double *__restrict__ cinv, const T *bN, T *xN) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int i = gwarp; i < nc; i += nwarps) {
    const double *a = cinv + (size_t)i * nc;
    double acc = 0.0;
    for (int j = lane; j < nc; j += 32) acc = fma(__ldg(a + j), (double)__ldcg(bN + j), acc);
    acc = warp_sum(acc);
    if (lane == 0) xN[i] = (T)acc;
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(kGridThreads)
grid_tail_kernel(const GridPlan<T> *__restrict__ plan) {
  const GridPlan<T> &P = *plan;
  const unsigned long long deadline = global_ns() + P.budget_ns;
  unsigned int nb = 0;
  const int nlev = P.nlev;
  // the first step of every level writes the buffer that makes the last
  // post-smoothing step land in x: (t_pre - 1) + t_post swaps follow it
  const bool first_in_x2 = (((P.tpre - 1) + P.tpost) & 1) != 0;
  T *cur[GASA_MAX_LEVELS];
  // ---- down: pre-smoothing, residual, restriction ----
  for (int q = 0; q < nlev; ++q) {
    const GridLevel<T> &L = P.lv[q];
    T *xa = first_in_x2 ? L.x2 : L.x;
    T *xb = first_in_x2 ? L.x : L.x2;
    if (q == 0) {
      first_phase<T, S>(L.n, L.W, L.b, xa);
      if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
    }
    for (int t = 1; t < P.tpre; ++t) {
      team_phase<T, S, GOP_SWEEP>(L.tlA, L.n, L.arp, L.acol, L.aval, L.W, xa, L.b, xb, nullptr);
      T *tmp = xa;
      xa = xb;
      xb = tmp;
      if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
    }
    cur[q] = xa;
    team_phase<T, S, GOP_RESID>(L.tlA, L.n, L.arp, L.acol, L.aval, nullptr, xa, L.b, L.r, nullptr);
    if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
    const bool last = q + 1 == nlev;
    const GridLevel<T> &Nx = P.lv[q + 1];
    T *b_next = last ? P.bN : Nx.b;
    T *x_next = last ? nullptr : (first_in_x2 ? Nx.x2 : Nx.x);
    team_phase<T, S, GOP_RESTRICT>(L.tlR, L.n_next, L.rrp, L.rcol, L.rval, last ? nullptr : Nx.W,
                                   L.r, nullptr, b_next, x_next);
    if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
  }
  // ---- coarsest solve ----
  coarse_phase<T>(P.nc, P.cinv, P.bN, P.xN);
  if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
  // ---- up: prolongation and post-smoothing ----
  for (int q = nlev - 1; q >= 0; --q) {
    const GridLevel<T> &L = P.lv[q];
    T *xa = cur[q];
    T *xb = (xa == L.x) ? L.x2 : L.x;
    const T *u = (q + 1 == nlev) ? P.xN : cur[q + 1];
    team_phase<T, S, GOP_PROLONG>(L.tlP, L.n, L.prp, L.pcol, L.pval, nullptr, u, nullptr, xa,
                                  nullptr);
    if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
    for (int t = 0; t < P.tpost; ++t) {
      team_phase<T, S, GOP_SWEEP>(L.tlA, L.n, L.arp, L.acol, L.aval, L.W, xa, L.b, xb, nullptr);
      T *tmp = xa;
      xa = xb;
      xb = tmp;
      if (q == 0 && t + 1 == P.tpost) break;   // the launch ends here
      if (!grid_sync(P.bar, ++nb, P.err, deadline)) return;
    }
    cur[q] = xa;
  }
}

template <typename T, int S>
cudaError_t launch_s(const GridPlan<T> *plan_dev, int ctas, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(kGridThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, grid_tail_kernel<T, S>, plan_dev);
  note_launch();
  return e;
}

template <typename T, int S>
int ctas_s(int cap) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grid_tail_kernel<T, S>, kGridThreads, 0) !=
      cudaSuccess)
    return 0;
  if (per > cap) per = cap;
  return per * sms;
}

}  // namespace

int grid_team(int s, double avg) {
  int tl = 4;
  while (tl < 32 && tl * 2.5 < avg) tl *= 2;
  while (tl < s) tl *= 2;
  return tl;
}

#define GASA_GRID_S(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

template <typename T>
int grid_tail_ctas(int s, int cap) {
  switch (s) {
#define GASA_CASE(SV) \
  case SV: return ctas_s<T, SV>(cap);
    GASA_GRID_S(GASA_CASE)
#undef GASA_CASE
    default: return 0;
  }
}

template <typename T>
cudaError_t launch_grid_tail(const GridPlan<T> *plan_dev, int s, int ctas, unsigned int *bar,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  switch (s) {
#define GASA_CASE(SV) \
  case SV: return launch_s<T, SV>(plan_dev, ctas, st);
    GASA_GRID_S(GASA_CASE)
#undef GASA_CASE
    default: return cudaErrorNotSupported;
  }
}

template int grid_tail_ctas<float>(int, int);
template int grid_tail_ctas<double>(int, int);
template cudaError_t launch_grid_tail<float>(const GridPlan<float> *, int, int, unsigned int *,
                                             cudaStream_t);
template cudaError_t launch_grid_tail<double>(const GridPlan<double> *, int, int, unsigned int *,
                                              cudaStream_t);

}  // namespace gasa
