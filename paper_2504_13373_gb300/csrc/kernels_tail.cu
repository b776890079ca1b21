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
// Everything the launch touches after its start sits in shared memory (the
// layout is in tail.h): CTA c owns units c, c + C, ... of every level, copies
// the matrix rows it computes with from a packed global buffer at the start,
// and keeps its units' entries of x, x2, b and r.  A step reads the owned
// unit's own entries locally, gathers neighbour units' entries from the
// owning CTAs with ld.shared::cluster, and writes only owned entries, so the
// release/acquire cluster barrier between steps is the only synchronisation.
// (The barrier's acquire drops the SM's L1, so matrix rows left in global
// memory would come back from L2 in every step; measured on GB300 a barrier
// costs 0.25 us, an L2 round trip after it 0.45 us.)  Arithmetic per output
// row: the sum over the row's blocks in a fixed order, so results do not
// depend on timing.
#include "common.cuh"
#include "internal.h"
#include "tail.h"

namespace gasa {

namespace {

constexpr int kTailMaxS = 64;

extern __shared__ __align__(16) unsigned char tail_smem[];

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
// Every thread of every CTA of the cluster arrives; shared-memory writes made
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

// distributed vector layout (see tail.h): unit j of a level lives in CTA
// j mod C at slot j / C
struct Dist {
  uint32_t sbase;   // shared-window address of tail_smem in this CTA
  int cl;           // CTAs in the cluster
};
template <typename T>
__device__ __forceinline__ T *d_local(int off, int slot, int s) {
  return reinterpret_cast<T *>(tail_smem + off) + (size_t)slot * s;
}
// shared::cluster address of entry 0 of unit j (s entries of esize bytes)
__device__ __forceinline__ uint32_t d_remote(const Dist &d, int off, int j, int s, int esize) {
  const uint32_t la = d.sbase + (uint32_t)off + (uint32_t)((j / d.cl) * s * esize);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(j % d.cl));
  return ra;
}

template <typename V>
__device__ __forceinline__ V ld_cl(uint32_t a);
template <>
__device__ __forceinline__ float ld_cl<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
template <>
__device__ __forceinline__ double ld_cl<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
template <>
__device__ __forceinline__ float4 ld_cl<float4>(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
  return v;
}
template <>
__device__ __forceinline__ double2 ld_cl<double2>(uint32_t a) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
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
// four blocks at a time so that four gathers are in flight; an xor-shuffle
// over the group bits then leaves the sum of row r0 + (lane % gs) in every
// lane.  col and val are the CTA's packed rows in shared memory; x is the
// distributed vector at byte offset xoff (bc entries per unit).
template <typename T, int VW>
__device__ __forceinline__ T tail_rows(int beg, int end, int br, int bc, int r0, int gs,
                                       const int *col, const T *val, const Dist &d, int xoff,
                                       int lane) {
  using V = typename TailVec<T, VW>::V;
  const int q = lane & (gs - 1), g = lane / gs, G = 32 / gs;
  const int r = r0 + q;
  T acc = T(0);
  if (r < br) {
    int k = beg + g;
    for (; k + 3 * G < end; k += 4 * G) {
      const V *a[4];
      uint32_t xa[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k + u * G;
        a[u] = reinterpret_cast<const V *>(val + ((size_t)kk * br + r) * bc);
        xa[u] = d_remote(d, xoff, col[kk], bc, (int)sizeof(T));
      }
      T s[4] = {T(0), T(0), T(0), T(0)};
      for (int c = 0; c < bc / VW; ++c) {
        V av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = a[u][c];
          xv[u] = ld_cl<V>(xa[u] + c * (uint32_t)sizeof(V));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = vdot<T>(av[u], xv[u], s[u]);
      }
      acc += (s[0] + s[1]) + (s[2] + s[3]);
    }
    for (; k < end; k += G) {
      const V *a = reinterpret_cast<const V *>(val + ((size_t)k * br + r) * bc);
      const uint32_t xa = d_remote(d, xoff, col[k], bc, (int)sizeof(T));
      T s = T(0);
      for (int c = 0; c < bc / VW; ++c) s = vdot<T>(a[c], ld_cl<V>(xa + c * (uint32_t)sizeof(V)), s);
      acc += s;
    }
  }
  for (int o = gs; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename T>
__device__ __forceinline__ T tail_rows_any(int beg, int end, int br, int bc, int r0, int gs,
                                           const int *col, const T *val, const Dist &d, int xoff,
                                           bool vec, int lane) {
  constexpr int VW = 16 / (int)sizeof(T);
  if (vec && bc % VW == 0) return tail_rows<T, VW>(beg, end, br, bc, r0, gs, col, val, d, xoff, lane);
  return tail_rows<T, 1>(beg, end, br, bc, r0, gs, col, val, d, xoff, lane);
}

enum { OP_SWEEP = 0, OP_FIRST = 1, OP_RESID = 2, OP_ASSIGN = 3, OP_ADD = 4 };

// y = M x (ASSIGN), y = b - M x (RESID) or y += M x (ADD) for the m block
// rows of br x bc blocks this CTA owns (packed rp / col / val), a warp per
// row; x is the distributed vector at xoff (bc per unit), b and y at boff /
// yoff (br per unit, own slots)
template <typename T>
__device__ void tail_mv(int op, int m, int br, int bc, const int *rp, const int *col, const T *val,
                        const Dist &d, int xoff, int boff, int yoff, bool vec, int wib, int lane) {
  for (int sl = wib; sl < m; sl += kTailWarps) {
    const int beg = rp[sl], end = rp[sl + 1];
    T *y = d_local<T>(yoff, sl, br);
    for (int r0 = 0; r0 < br; r0 += 32) {
      const int rem = br - r0;
      const int gs = rem >= 32 ? 32 : pow2_at_least(rem);
      const T v = tail_rows_any<T>(beg, end, br, bc, r0, gs, col, val, d, xoff, vec, lane);
      const int r = r0 + lane;
      if (lane < gs && r < br) {
        if (op == OP_ASSIGN) y[r] = v;
        else if (op == OP_RESID) y[r] = d_local<T>(boff, sl, br)[r] - v;
        else y[r] += v;
      }
    }
    __syncwarp();
  }
}

// Smoothing step of Alg. 1 with A~^{-1} = w D^{-1}: xo = x + W (b - A x)
// (SWEEP) or xo = W b (FIRST, from x = 0), over the CTA's m units.  The
// block row's residual meets in the warp's shared-memory row `res`, then
// lane r applies row r of W_u.
template <typename T>
__device__ void tail_jacobi(int op, const TailLevel<T> &L, int m, const int *rp, const int *col,
                            const T *val, const T *W, int xoff, int ooff, const Dist &d, bool vec,
                            int wib, int lane, T *res) {
  const int s = L.s;
  for (int sl = wib; sl < m; sl += kTailWarps) {
    int beg = 0, end = 0;
    if (op == OP_SWEEP) {
      beg = rp[sl];
      end = rp[sl + 1];
    }
    const T *bu = d_local<T>(L.off_b, sl, s);
    for (int r0 = 0; r0 < s; r0 += 32) {
      const int rem = s - r0;
      const int gs = rem >= 32 ? 32 : pow2_at_least(rem);
      T v = T(0);
      if (op == OP_SWEEP) v = tail_rows_any<T>(beg, end, s, s, r0, gs, col, val, d, xoff, vec, lane);
      const int r = r0 + lane;
      if (lane < gs && r < s) res[r] = bu[r] - v;
    }
    __syncwarp();
    const T *xu = d_local<T>(xoff, sl, s);
    T *ou = d_local<T>(ooff, sl, s);
    for (int r = lane; r < s; r += 32) {
      const T *w = W + ((size_t)sl * s + r) * s;
      T out = T(0);
      for (int c = 0; c < s; ++c) out = fma(w[c], res[c], out);
      if (op == OP_SWEEP) out += xu[r];
      ou[r] = out;
    }
    __syncwarp();
  }
}

// x_N = A_N^{-1} b_N in FP64 arithmetic, a warp per owned coarse unit and,
// for each of its rows, lanes over the columns
template <typename T>
__device__ void tail_dense(const TailPlan<T> &pl, const double *Crows, const Dist &d, int c,
                           int wib, int lane) {
  const int nc = pl.nc, sN = pl.sN;
  const int m = tail_owned(pl.nN, c, d.cl);
  for (int sl = wib; sl < m; sl += kTailWarps) {
    T *xu = d_local<T>(pl.off_xN, sl, sN);
    for (int rr = 0; rr < sN; ++rr) {
      const double *a = Crows + (size_t)(sl * sN + rr) * nc;
      double acc = 0.0;
      for (int j = lane; j < nc; j += 32) {
        const uint32_t bj = d_remote(d, pl.off_bN, j / sN, sN, (int)sizeof(T)) +
                            (uint32_t)((j % sN) * (int)sizeof(T));
        acc = fma(a[j], (double)ld_cl<T>(bj), acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) xu[rr] = (T)acc;
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
vcycle_tail_kernel(const TailPlan<T> *__restrict__ plp) {
  __shared__ T res_all[kTailWarps][kTailMaxS];
  const TailPlan<T> &pl = *plp;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Dist d;
  d.sbase = (uint32_t)__cvta_generic_to_shared(tail_smem);
  d.cl = (int)cl_size();
  const int c = (int)cl_rank();
  T *res = res_all[wib];
  const int nl = pl.nlev, tpre = pl.tpre, tpost = pl.tpost;
  const bool vec = pl.vec != 0;
  if (d.cl != pl.cl) return;   // uniform over the cluster: the layout needs this size
  // the CTA's packed matrix rows into shared memory, b_{k0} of its units
  unsigned char *mat = tail_smem + pl.mat_base;
  {
    const int4 *src = reinterpret_cast<const int4 *>(pl.pack + pl.pack_off[c]);
    int4 *dst = reinterpret_cast<int4 *>(mat);
    const int n16 = pl.pack_bytes[c] / 16;
    for (int i = threadIdx.x; i < n16; i += kTailThreads) dst[i] = __ldg(src + i);
    const TailLevel<T> &L = pl.lv[0];
    const int m = tail_owned(L.n, c, d.cl);
    for (int i = threadIdx.x; i < m * L.s; i += kTailThreads) {
      const int sl = i / L.s, r = i - sl * L.s;
      d_local<T>(L.off_b, sl, L.s)[r] = pl.b_in[(size_t)(sl * d.cl + c) * L.s + r];
    }
    __syncthreads();
  }
  auto fld = [&](int q, int f) { return mat + pl.moff[c][q][f]; };
  // down: pre-smoothing, residual, restriction
  for (int q = 0; q < nl; ++q) {
    const TailLevel<T> &L = pl.lv[q];
    const int m = tail_owned(L.n, c, d.cl), mn = tail_owned(L.n_next, c, d.cl);
    const int *Arp = reinterpret_cast<const int *>(fld(q, TM_ARP));
    const int *Acol = reinterpret_cast<const int *>(fld(q, TM_ACOL));
    const T *Aval = reinterpret_cast<const T *>(fld(q, TM_AVAL));
    const T *W = reinterpret_cast<const T *>(fld(q, TM_W));
    int cur = L.off_x, oth = L.off_x2;
    if (tpre == 0) {
      for (int i = threadIdx.x; i < m * L.s; i += kTailThreads) d_local<T>(cur, 0, 0)[i] = T(0);
    } else {
      tail_jacobi<T>(OP_FIRST, L, m, Arp, Acol, Aval, W, cur, cur, d, vec, wib, lane, res);
    }
    cl_sync();
    for (int t = 1; t < tpre; ++t) {
      tail_jacobi<T>(OP_SWEEP, L, m, Arp, Acol, Aval, W, cur, oth, d, vec, wib, lane, res);
      cl_sync();
      const int tmp = cur;
      cur = oth;
      oth = tmp;
    }
    tail_mv<T>(OP_RESID, m, L.s, L.s, Arp, Acol, Aval, d, cur, L.off_b, L.off_r, vec, wib, lane);
    cl_sync();
    const int bnext = (q + 1 < nl) ? pl.lv[q + 1].off_b : pl.off_bN;
    tail_mv<T>(OP_ASSIGN, mn, L.s_next, L.s, reinterpret_cast<const int *>(fld(q, TM_RRP)),
               reinterpret_cast<const int *>(fld(q, TM_RCOL)),
               reinterpret_cast<const T *>(fld(q, TM_RVAL)), d, L.off_r, 0, bnext, vec, wib, lane);
    cl_sync();
  }
  // coarsest level
  tail_dense<T>(pl, reinterpret_cast<const double *>(mat + pl.coff[c]), d, c, wib, lane);
  cl_sync();
  // up: prolongation and post-smoothing
  const int pre = tail_pre_buffer(tpre), fin = tail_final_buffer(tpre, tpost);
  for (int q = nl - 1; q >= 0; --q) {
    const TailLevel<T> &L = pl.lv[q];
    const int m = tail_owned(L.n, c, d.cl);
    const int *Arp = reinterpret_cast<const int *>(fld(q, TM_ARP));
    const int *Acol = reinterpret_cast<const int *>(fld(q, TM_ACOL));
    const T *Aval = reinterpret_cast<const T *>(fld(q, TM_AVAL));
    const T *W = reinterpret_cast<const T *>(fld(q, TM_W));
    int cur = pre ? L.off_x2 : L.off_x, oth = pre ? L.off_x : L.off_x2;
    int xc = pl.off_xN;
    if (q + 1 < nl) xc = fin ? pl.lv[q + 1].off_x2 : pl.lv[q + 1].off_x;
    tail_mv<T>(OP_ADD, m, L.s, L.s_next, reinterpret_cast<const int *>(fld(q, TM_PRP)),
               reinterpret_cast<const int *>(fld(q, TM_PCOL)),
               reinterpret_cast<const T *>(fld(q, TM_PVAL)), d, xc, 0, cur, vec, wib, lane);
    cl_sync();
    for (int t = 0; t < tpost; ++t) {
      tail_jacobi<T>(OP_SWEEP, L, m, Arp, Acol, Aval, W, cur, oth, d, vec, wib, lane, res);
      cl_sync();
      const int tmp = cur;
      cur = oth;
      oth = tmp;
    }
  }
  // the corrected x_{k0} (own units) back to global memory
  const TailLevel<T> &L = pl.lv[0];
  const int m = tail_owned(L.n, c, d.cl);
  const int xf = fin ? L.off_x2 : L.off_x;
  for (int i = threadIdx.x; i < m * L.s; i += kTailThreads) {
    const int sl = i / L.s, r = i - sl * L.s;
    pl.x_out[(size_t)(sl * d.cl + c) * L.s + r] = d_local<T>(xf, sl, L.s)[r];
  }
}

template <typename T>
cudaLaunchConfig_t tail_config(int cluster, int smem, cudaLaunchAttribute *attr, int nattr,
                               cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = nattr;
  return cfg;
}

// dynamic shared memory the tail kernel may use (227 KB per CTA on sm_103a,
// minus the static per-warp rows)
constexpr int kTailSmemMax = 200 * 1024;

}  // namespace

template <typename T>
int tail_cluster_size() {
  if (cudaFuncSetAttribute(vcycle_tail_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess)
    (void)cudaGetLastError();
  if (cudaFuncSetAttribute(vcycle_tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kTailSmemMax) != cudaSuccess)
    (void)cudaGetLastError();
  for (int cs : {16, 8}) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config<T>(cs, kTailSmemMax, attr, 1, nullptr);
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

int tail_smem_limit() { return kTailSmemMax; }

template <typename T>
cudaError_t launch_vcycle_tail(const TailPlan<T> *plan_dev, int cluster, int smem_bytes,
                               cudaStream_t s) {
  if (cluster <= 0 || !plan_dev || smem_bytes < 0 || smem_bytes > kTailSmemMax)
    return cudaErrorInvalidValue;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tail_config<T>(cluster, smem_bytes, attr, 1, s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, vcycle_tail_kernel<T>, plan_dev);
  note_launch();
  return e;
}
template cudaError_t launch_vcycle_tail<double>(const TailPlan<double> *, int, int, cudaStream_t);
template cudaError_t launch_vcycle_tail<float>(const TailPlan<float> *, int, int, cudaStream_t);

}  // namespace gasa
