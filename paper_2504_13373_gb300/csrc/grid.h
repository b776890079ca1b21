// The coarse levels of the V-cycle (Alg. 2) as one persistent launch over
// the whole GPU: descriptors shared by the host driver and kernels_grid.cu.
#pragma once
#include <cuda_runtime.h>

#include "gasa.h"

namespace gasa {

constexpr int kGridThreads = 256;       // threads per CTA of the persistent kernel

// One smoothed level k of the fused range: A_k, w D_k^{-1}, the transfers
// P_k (n fine rows, columns on level k+1) and R_k = P_k^T (n_next rows),
// the level's vectors, and the lane-team width used for each operator.
template <typename T>
struct GridLevel {
  int n = 0, n_next = 0;
  const int *arp = nullptr, *acol = nullptr;
  const T *aval = nullptr, *W = nullptr;
  const int *prp = nullptr, *pcol = nullptr;
  const T *pval = nullptr;
  const int *rrp = nullptr, *rcol = nullptr;
  const T *rval = nullptr;
  T *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
  int tlA = 0, tlP = 0, tlR = 0;
};

// Levels k0 .. k0 + nlev - 1 are smoothed inside the launch, level
// k0 + nlev = N is the coarsest (solved with the explicit FP64 inverse).
// Every level in the range has s dofs per unit.  The launch reads b_{k0}
// from lv[0].b and leaves the corrected x_{k0} in lv[0].x.
template <typename T>
struct GridPlan {
  int k0 = 0, nlev = 0, tpre = 0, tpost = 0, s = 0;
  int nc = 0;                       // coarsest dofs
  const double *cinv = nullptr;     // A_N^{-1}, nc x nc row-major
  T *bN = nullptr, *xN = nullptr;
  unsigned int *bar = nullptr;      // grid barrier counter, zeroed before every launch
  int *err = nullptr;               // set to 1 when a bounded wait runs out
  unsigned long long budget_ns = 0; // wait budget of one launch
  GridLevel<T> lv[GASA_MAX_LEVELS];
};

// CTAs of the persistent kernel for block size s: resident CTAs per SM (at
// most `cap`) times the device's SMs; 0 when the kernel cannot run
template <typename T>
int grid_tail_ctas(int s, int cap);
// lane-team width for a block row of about `avg` s x s blocks: a power of two
// in [4, 32], at least s, about 2.5 blocks per lane
int grid_team(int s, double avg);

template <typename T>
cudaError_t launch_grid_tail(const GridPlan<T> *plan_dev, int s, int ctas, unsigned int *bar,
                             cudaStream_t st);

}  // namespace gasa
