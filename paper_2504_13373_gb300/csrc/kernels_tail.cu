// The bottom of the V-cycle (Alg. 2) in one thread-block-cluster launch.
//
// Coarse levels hold a few hundred to a few thousand units whose block rows
// carry tens to hundreds of blocks (each Galerkin product widens the
// stencil).  Run as one launch per smoothing step, residual and transfer,
// they are bound by launch and drain latency, not by bytes: the work of a
// step is microseconds of L2 traffic spread over the whole GPU.  Here one
// cluster of 512-thread CTAs runs every step of levels k0 .. N-1, the
// coarsest dense solve and the way back up, with a hardware cluster barrier
// between dependent steps.
//
// Warp w of the cluster owns block rows w, w + NW, ... of every operator, so
// a warp reads the same matrix rows in every pass and, after the first pass,
// finds them in its SM's L1.  Vectors written inside the launch are read
// through L2 (ld.global.cg); the release/acquire cluster barrier makes each
// step's writes visible to the next step.  Arithmetic per output row: the
// sum over the row's blocks in a fixed order, so results do not depend on
// timing.
#include "common.cuh"
#include "internal.h"
#include "tail.h"

namespace gasa {

namespace {

constexpr int kTailThreads = 512;
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kTailMaxS = 64;

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster arrives; global-memory writes made
// before the barrier are visible to all threads of the cluster after it.
__device__ __forceinline__ void cl_sync() {
  __syncwarp();   // the .aligned barrier wants every warp converged
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int pow2_at_least(int v) {   // 1 <= v <= 32
  return v <= 1 ? 1 : 1 << (32 - __clz(v - 1));
}

template <typename T, int VW>
struct TailVec;
template <> struct TailVec<float, 4> { using V = float4; };
template <> struct TailVec<double, 2> { using V = double2; };
template <> struct TailVec<float, 1> { using V = float; };
template <> struct TailVec<double, 1> { using V = double; };

template <typename T>
__device__ __forceinline__ T vdot(float4 a, float4 x, T acc) {
  acc = fma(a.x, x.x, acc);
  acc = fma(a.y, x.y, acc);
  acc = fma(a.z, x.z, acc);
  return fma(a.w, x.w, acc);
}
template <typename T>
__device__ __forceinline__ T vdot(double2 a, double2 x, T acc) {
  acc = fma(a.x, x.x, acc);
  return fma(a.y, x.y, acc);
}
template <typename T>
__device__ __forceinline__ T vdot(T a, T x, T acc) { return fma(a, x, acc); }

// Rows r0 .. r0 + gs - 1 of one block row (gs a power of two <= 32): lane
// (g, q) takes row r0 + q of blocks beg + g, beg + g + G, ... (G = 32 / gs),
// four blocks at a time so that four gathers of x are in flight; an
// xor-shuffle over the group bits then leaves the sum of row r0 + (lane % gs)
// in every lane.  Matrix values are read through L1 (they never change in a
// launch), x through L2.
template <typename T, int VW>
__device__ __forceinline__ T tail_rows(int beg, int end, int br, int bc, int r0, int gs,
                                       const int *__restrict__ col, const T *__restrict__ val,
                                       const T *x, int lane) {
  using V = typename TailVec<T, VW>::V;
  const int q = lane & (gs - 1), g = lane / gs, G = 32 / gs;
  const int r = r0 + q;
  T acc = T(0);
  if (r < br) {
    int k = beg + g;
    for (; k + 3 * G < end; k += 4 * G) {
      const V *a[4];
      const V *xx[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k + u * G;
        a[u] = reinterpret_cast<const V *>(val + ((size_t)kk * br + r) * bc);
        xx[u] = reinterpret_cast<const V *>(x + (size_t)__ldg(col + kk) * bc);
      }
      T s[4] = {T(0), T(0), T(0), T(0)};
      for (int c = 0; c < bc / VW; ++c) {
        V av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = __ldg(a[u] + c);
          xv[u] = __ldcg(xx[u] + c);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = vdot<T>(av[u], xv[u], s[u]);
      }
      acc += (s[0] + s[1]) + (s[2] + s[3]);
    }
    for (; k < end; k += G) {
      const V *a = reinterpret_cast<const V *>(val + ((size_t)k * br + r) * bc);
      const V *xx = reinterpret_cast<const V *>(x + (size_t)__ldg(col + k) * bc);
      T s = T(0);
      for (int c = 0; c < bc / VW; ++c) s = vdot<T>(__ldg(a + c), __ldcg(xx + c), s);
      acc += s;
    }
  }
  for (int o = gs; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename T>
__device__ __forceinline__ T tail_rows_any(int beg, int end, int br, int bc, int r0, int gs,
                                           const int *__restrict__ col,
                                           const T *__restrict__ val, const T *x, bool vec,
                                           int lane) {
  constexpr int VW = 16 / (int)sizeof(T);
  if (vec && bc % VW == 0) return tail_rows<T, VW>(beg, end, br, bc, r0, gs, col, val, x, lane);
  return tail_rows<T, 1>(beg, end, br, bc, r0, gs, col, val, x, lane);
}

enum { OP_SWEEP = 0, OP_FIRST = 1, OP_RESID = 2, OP_ASSIGN = 3, OP_ADD = 4 };

// y = M x (ASSIGN), y = b - M x (RESID) or y += M x (ADD) for n block rows of
// br x bc blocks, a warp per block row
template <typename T>
__device__ void tail_mv(int op, int n, int br, int bc, const int *__restrict__ rp,
                        const int *__restrict__ col, const T *__restrict__ val, const T *x,
                        const T *b, T *y, bool vec, int gw, int NW, int lane) {
  for (int u = gw; u < n; u += NW) {
    const int beg = __ldg(rp + u), end = __ldg(rp + u + 1);
    for (int r0 = 0; r0 < br; r0 += 32) {
      const int rem = br - r0;
      const int gs = rem >= 32 ? 32 : pow2_at_least(rem);
      const T v = tail_rows_any<T>(beg, end, br, bc, r0, gs, col, val, x, vec, lane);
      const int r = r0 + lane;
      if (lane < gs && r < br) {
        const size_t t = (size_t)u * br + r;
        if (op == OP_ASSIGN) y[t] = v;
        else if (op == OP_RESID) y[t] = __ldcg(b + t) - v;
        else y[t] = __ldcg(y + t) + v;
      }
    }
  }
}

// Smoothing step of Alg. 1 with A~^{-1} = w D^{-1}: xo = x + W (b - A x)
// (SWEEP) or xo = W b (FIRST, from x = 0).  The block row's residual meets
// in the warp's shared-memory row `res`, then lane r applies row r of W_u.
template <typename T>
__device__ void tail_jacobi(int op, const TailLevel<T> &L, const T *x, T *xo, bool vec, int gw,
                            int NW, int lane, T *res) {
  const int s = L.s;
  for (int u = gw; u < L.n; u += NW) {
    int beg = 0, end = 0;
    if (op == OP_SWEEP) {
      beg = __ldg(L.rp + u);
      end = __ldg(L.rp + u + 1);
    }
    for (int r0 = 0; r0 < s; r0 += 32) {
      const int rem = s - r0;
      const int gs = rem >= 32 ? 32 : pow2_at_least(rem);
      T v = T(0);
      if (op == OP_SWEEP) v = tail_rows_any<T>(beg, end, s, s, r0, gs, L.col, L.A, x, vec, lane);
      const int r = r0 + lane;
      if (lane < gs && r < s) res[r] = __ldcg(L.b + (size_t)u * s + r) - v;
    }
    __syncwarp();
    for (int r = lane; r < s; r += 32) {
      const size_t t = (size_t)u * s + r;
      const T *w = L.W + t * s;
      T out = T(0);
      for (int c = 0; c < s; ++c) out = fma(__ldg(w + c), res[c], out);
      if (op == OP_SWEEP) out += __ldcg(x + t);
      xo[t] = out;
    }
    __syncwarp();
  }
}

// x_N = A_N^{-1} b_N in FP64 arithmetic, a warp per row (the same order as
// dense_mv_kernel)
template <typename T>
__device__ void tail_dense(int nc, const double *__restrict__ C, const T *b, T *x, int gw, int NW,
                           int lane) {
  for (int i = gw; i < nc; i += NW) {
    const double *a = C + (size_t)i * nc;
    double acc = 0.0;
    for (int j = lane; j < nc; j += 32) acc = fma(__ldg(a + j), (double)__ldcg(b + j), acc);
    acc = warp_sum(acc);
    if (lane == 0) x[i] = (T)acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
vcycle_tail_kernel(const TailPlan<T> *__restrict__ pl, int part) {
  pdl_entry();
  __shared__ T res_all[kTailWarps][kTailMaxS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int ncta = (int)cl_size();
  const int NW = ncta * kTailWarps;
  const int gw = (int)cl_rank() * kTailWarps + wib;
  T *res = res_all[wib];
  const int nl = pl->nlev, tpre = pl->tpre, tpost = pl->tpost;
  const bool vec = pl->vec != 0;
  const int pre = tail_pre_buffer(tpre), fin = tail_final_buffer(tpre, tpost);
  if (part != TAIL_UP) {
    for (int q = 0; q < nl; ++q) {
      const TailLevel<T> &L = pl->lv[q];
      T *cur = L.x, *oth = L.x2;
      if (tpre == 0) {
        const size_t nd = (size_t)L.n * L.s;
        for (size_t i = (size_t)cl_rank() * kTailThreads + threadIdx.x; i < nd;
             i += (size_t)ncta * kTailThreads)
          cur[i] = T(0);
      } else {
        tail_jacobi<T>(OP_FIRST, L, nullptr, cur, vec, gw, NW, lane, res);
      }
      cl_sync();
      for (int t = 1; t < tpre; ++t) {
        tail_jacobi<T>(OP_SWEEP, L, cur, oth, vec, gw, NW, lane, res);
        cl_sync();
        T *tmp = cur;
        cur = oth;
        oth = tmp;
      }
      tail_mv<T>(OP_RESID, L.n, L.s, L.s, L.rp, L.col, L.A, cur, L.b, L.r, vec, gw, NW, lane);
      cl_sync();
      T *bn = (q + 1 < nl) ? pl->lv[q + 1].b : pl->bN;
      tail_mv<T>(OP_ASSIGN, L.n_next, L.s_next, L.s, L.Rrp, L.Rcol, L.R, L.r, nullptr, bn, vec,
                 gw, NW, lane);
      cl_sync();
    }
  }
  if (part == TAIL_ALL) {
    tail_dense<T>(pl->nc, pl->Cinv, pl->bN, pl->xN, gw, NW, lane);
    cl_sync();
  }
  if (part != TAIL_DOWN) {
    for (int q = nl - 1; q >= 0; --q) {
      const TailLevel<T> &L = pl->lv[q];
      T *cur = pre ? L.x2 : L.x, *oth = pre ? L.x : L.x2;
      const T *xc = pl->xN;
      if (q + 1 < nl) xc = fin ? pl->lv[q + 1].x2 : pl->lv[q + 1].x;
      tail_mv<T>(OP_ADD, L.n, L.s, L.s_next, L.Prp, L.Pcol, L.P, xc, nullptr, cur, vec, gw, NW,
                 lane);
      cl_sync();
      for (int t = 0; t < tpost; ++t) {
        tail_jacobi<T>(OP_SWEEP, L, cur, oth, vec, gw, NW, lane, res);
        cl_sync();
        T *tmp = cur;
        cur = oth;
        oth = tmp;
      }
    }
  }
}

template <typename T>
cudaLaunchConfig_t tail_config(int cluster, cudaLaunchAttribute *attr, int nattr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  if (nattr > 1) {
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  }
  cfg.attrs = attr;
  cfg.numAttrs = nattr;
  return cfg;
}

}  // namespace

template <typename T>
int tail_cluster_size() {
  if (cudaFuncSetAttribute(vcycle_tail_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess) {
    (void)cudaGetLastError();
  }
  for (int cs : {16, 8}) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config<T>(cs, attr, 1, nullptr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, vcycle_tail_kernel<T>, &cfg) == cudaSuccess &&
        nclusters > 0)
      return cs;
    (void)cudaGetLastError();
  }
  return 0;
}
template int tail_cluster_size<double>();
template int tail_cluster_size<float>();

template <typename T>
cudaError_t launch_vcycle_tail(const TailPlan<T> *plan_dev, int part, int cluster,
                               cudaStream_t s) {
  if (cluster <= 0 || !plan_dev || part < TAIL_ALL || part > TAIL_UP) return cudaErrorInvalidValue;
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = tail_config<T>(cluster, attr, 2, s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, vcycle_tail_kernel<T>, plan_dev, part);
  note_launch();
  return e;
}
template cudaError_t launch_vcycle_tail<double>(const TailPlan<double> *, int, int, cudaStream_t);
template cudaError_t launch_vcycle_tail<float>(const TailPlan<float> *, int, int, cudaStream_t);

}  // namespace gasa
