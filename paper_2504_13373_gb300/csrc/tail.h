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
  T *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
};

// Levels k0 .. k0 + nlev - 1 smoothed in the tail; the coarsest solve
// x_N = A_N^{-1} b_N runs inside the launch when Cinv is set (part TAIL_ALL),
// else between a "down" launch and an "up" launch.
template <typename T>
struct TailPlan {
  int k0 = 0, nlev = 0;
  int tpre = 0, tpost = 0;
  int vec = 0;                        // 1: every base pointer is 16-byte aligned
  int nc = 0;
  const double *Cinv = nullptr;       // row-major A_N^{-1}
  T *bN = nullptr, *xN = nullptr;
  TailLevel<T> lv[GASA_MAX_LEVELS];
};

// buffer (0: x, 1: x2) holding a tail level's iterate after pre-smoothing
// and after post-smoothing: the first step writes x, each further step swaps
__host__ __device__ inline int tail_pre_buffer(int tpre) { return tpre >= 1 ? (tpre - 1) & 1 : 0; }
__host__ __device__ inline int tail_final_buffer(int tpre, int tpost) {
  return ((tpre >= 1 ? tpre - 1 : 0) + tpost) & 1;
}

enum { TAIL_ALL = 0, TAIL_DOWN = 1, TAIL_UP = 2 };

// cluster size the tail kernel of precision T launches with (16 where the
// device can co-schedule a 16-CTA cluster of 512-thread CTAs, else 8); 0 if
// the device cannot run it
template <typename T>
int tail_cluster_size();

template <typename T>
cudaError_t launch_vcycle_tail(const TailPlan<T> *plan_dev, int part, int cluster,
                               cudaStream_t s);

}  // namespace gasa
