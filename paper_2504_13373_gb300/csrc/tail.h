// The bottom levels of the V-cycle (Alg. 2) in one thread-block-cluster
// launch: descriptors shared by the host driver and kernels_tail.cu.
#pragma once
#include <cuda_runtime.h>

#include "gasa.h"

namespace gasa {

// One smoothed level k of the fused tail.  Every level of the tail keeps
// its operator A_k (no matrix-free level) and has one block size s.
template <typename T>
struct TailLevel {
  int n = 0, s = 0;                   // units, dofs per unit
  int s_next = 0, n_next = 0;         // block size and units of level k+1
  const int *rp = nullptr, *col = nullptr;
  const T *A = nullptr;               // A_k, s x s blocks
  const T *W = nullptr;               // w_k D_k^{-1}, n blocks of s x s
  const int *Prp = nullptr, *Pcol = nullptr;
  const T *P = nullptr;               // P_k: n block rows of s x s_next blocks
  const int *Rrp = nullptr, *Rcol = nullptr;
  const T *R = nullptr;               // R_k = P_k^T: n_next block rows of s_next x s blocks
  // vectors x, x2, b, r of the level live in distributed shared memory: unit
  // u belongs to warp u mod NW of the cluster (NW = CTAs x warps per CTA) and
  // sits in that warp's CTA at slot (u / NW) * warps + u mod warps; off_* are
  // the byte offsets of the level's vectors in every CTA's dynamic shared
  // memory (the same layout in every CTA)
  int off_x = 0, off_x2 = 0, off_b = 0, off_r = 0;
};

// Levels k0 .. k0 + nlev - 1 smoothed in the tail and the coarsest solve
// x_N = A_N^{-1} b_N (n_N units of s_N dofs, nc = n_N s_N).  The launch reads
// b_{k0} from global memory (b_in) and leaves the corrected x_{k0} there
// (x_out); everything in between stays in the cluster's shared memory.
template <typename T>
struct TailPlan {
  int k0 = 0, nlev = 0;
  int tpre = 0, tpost = 0;
  int vec = 0;                        // 1: matrix arrays 16-byte aligned
  int nc = 0, nN = 0, sN = 0;
  const double *Cinv = nullptr;       // row-major A_N^{-1}
  int off_bN = 0, off_xN = 0;         // coarsest-level vectors, distributed like the levels'
  int smem_bytes = 0;                 // dynamic shared memory per CTA
  int nw = 0;                         // warps of the cluster the layout was made for
  const T *b_in = nullptr;
  T *x_out = nullptr;
  TailLevel<T> lv[GASA_MAX_LEVELS];
};

// buffer (0: x, 1: x2) holding a tail level's iterate after pre-smoothing
// and after post-smoothing: the first step writes x, each further step swaps
__host__ __device__ inline int tail_pre_buffer(int tpre) { return tpre >= 1 ? (tpre - 1) & 1 : 0; }
__host__ __device__ inline int tail_final_buffer(int tpre, int tpost) {
  return ((tpre >= 1 ? tpre - 1 : 0) + tpost) & 1;
}

constexpr int kTailThreads = 512;             // threads per CTA of the tail kernel
constexpr int kTailWarps = kTailThreads / 32;
// slots one CTA holds of a level of n units when the cluster has nw warps
inline int tail_slots(int n, int nw) { return ((n + nw - 1) / nw) * kTailWarps; }

// cluster size the tail kernel of precision T launches with (16 where the
// device can co-schedule a 16-CTA cluster of 512-thread CTAs, else 8); 0 if
// the device cannot run it
template <typename T>
int tail_cluster_size();
// dynamic shared memory per CTA the tail kernel may use
int tail_smem_limit();

template <typename T>
cudaError_t launch_vcycle_tail(const TailPlan<T> *plan_dev, int cluster, int smem_bytes,
                               cudaStream_t s);

}  // namespace gasa
