// Device-resident state of a set-up hierarchy, shared by the solver entry
// points and the request server.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "gasa.h"

namespace gasa {

struct DevBSR {
  int nrows = 0, ncols = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  int *rp = nullptr, *col = nullptr;
  double *val = nullptr;
  float *val32 = nullptr;
  float *lo32 = nullptr;       // level 0: FP32 rounding of val - val32 (double-single A x)
  __half *val16 = nullptr;     // FP16 blocks (level 0, MIXED16)
  float *scale16 = nullptr;    // one scale per block
};

struct Level {
  int n = 0;          // units on this level
  int s = 0;          // dofs per unit (stored block size; padded levels pad to it)
  int64_t ndof = 0;   // n * s
  // padded level (kept counts of Eq. sik differ between aggregates): unit u
  // holds usize[u] real dofs followed by zeros
  bool padded = false;
  std::vector<int> usize;
  int *d_usize = nullptr;
  int64_t *d_uoff = nullptr;     // exclusive prefix sums of usize
  int64_t real_dofs = 0;
  DevBSR A;
  double *W = nullptr;        // w D^{-1}
  float *W32 = nullptr;
  __half *W16 = nullptr;       // FP16 blocks of w D^{-1} (level 0, MIXED16)
  float *W16s = nullptr;
  // transfer to the next level
  int *agg = nullptr;
  int n_next = 0, s_next = 0, max_children = 0;
  int *child_ptr = nullptr, *child_idx = nullptr;
  double *T = nullptr;
  DevBSR P, R;
  DevBSR RA;                  // R_k A_k (fused residual + restriction), rows of level k+1
  // folded smoother (option folded_smoother, level 0): W A in A's block
  // pattern, and c = W b of the current V-cycle
  double *WA = nullptr;
  float *WA32 = nullptr;
  double *c = nullptr;
  float *cf = nullptr;
  double *cand = nullptr, *cand_in = nullptr;
  std::vector<int> sweeps;
  double omega = 0.0, rho = 0.0;
  // bulk-copy staged FP32 smoothing step (level 0): plan from tma_plan
  bool tma = false;
  int tma_TR = 0, tma_stageA = 0, tma_stageW = 0, tma_smem = 0, tma_grid = 0;
  // V-cycle vectors
  double *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
  float *xf = nullptr, *x2f = nullptr, *bf = nullptr, *rf = nullptr;
  // matrix-free level (Section 4.4): A is applied as R_{k-1} A_{k-1} P_{k-1};
  // mt / mu are this level's scratch for the product of the level above
  bool mf = false;
  double *mt = nullptr, *mu = nullptr;
  float *mtf = nullptr, *muf = nullptr;
};

struct ProfClass {
  std::vector<cudaEvent_t> ev;    // pairs
  size_t used = 0;
  double bytes = 0.0;
  int64_t launches = 0;
};

}  // namespace gasa

struct gasa_ctx {
  using DevBSR = gasa::DevBSR;
  using Level = gasa::Level;
  using ProfClass = gasa::ProfClass;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool ready = false;
  gasa_options opt{};
  int N = 0;
  int r = 0;
  std::vector<Level> L;
  double *coarse_inv = nullptr;
  int nc = 0;
  std::vector<void *> allocs;     // hierarchy allocations
  // Krylov workspace
  double *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr,
         *kzold = nullptr, *kb = nullptr, *kt = nullptr;
  double *part = nullptr;         // 4 x kRedBlocks partials
  double *scal = nullptr;         // device scalars
  double *hscal = nullptr;        // pinned host mirror
  float *kf_in = nullptr, *kf_out = nullptr;
  float *kzold_f = nullptr;   // previous z of the graph-resident mixed CG step (FP32)
  float *kp_hi = nullptr, *kp_lo = nullptr;   // two-term FP32 split of p (mixed precision)
  double *pq_ds = nullptr;   // p . Ap partials of the double-single product (one per CTA)
  int n_pq_ds = 0;
  double *rz_ds = nullptr, *rzo_ds = nullptr;   // r . z, r . zold partials of the CG step
  int n_rz_cap = 0;                             // their capacity
  double *V = nullptr, *Z = nullptr, *H = nullptr, *gm = nullptr, *mpart = nullptr;
  int gm_restart = 0;
  bool gm_flex = false;
  // graph-resident CG: one instantiated graph per precision, the whole CG
  // iteration (V-cycle included) inside a conditional while node
  // slots 0-2: CG per precision; 3-5: stationary iteration per precision
  cudaGraph_t cg_graph[6] = {};
  cudaGraphExec_t cg_exec[6] = {};
  long long cg_kernels[6] = {};
  int cg_max_iter[6] = {};
  int *d_iters = nullptr;
  int *d_err = nullptr;          // set by kernels whose bounded waits time out
  // fused bottom of the V-cycle per precision (0: FP64, 1: FP32): levels
  // tail_k0[p] .. N-1 and the coarsest solve run in one cluster launch
  // (kernels_tail.cu); no plan: every step is its own launch
  void *tail_plan[2] = {};
  int tail_k0[2] = {0, 0};
  int tail_coarse[2] = {0, 0};   // 1: the coarsest solve runs inside the launch
  int tail_cluster[2] = {0, 0};  // CTAs per cluster
  int tail_smem[2] = {0, 0};     // dynamic shared memory per CTA
  // persistent coarse levels per precision (kernels_grid.cu): levels
  // grid_k0[p] .. N in one cooperative launch of grid_ctas[p] CTAs
  void *grid_plan[2] = {};
  int grid_k0[2] = {0, 0};
  int grid_ctas[2] = {0, 0};
  int grid_s[2] = {0, 0};
  unsigned int *grid_bar = nullptr;
  // dense bottom of the V-cycle (option dense_tail_dofs): levels dtail_k ..
  // N as the FP64 dtail_n x dtail_n operator dtail_M (row-major); none when
  // dtail_M is null (dtail_k = N)
  double *dtail_M = nullptr;
  int dtail_k = 0;
  int dtail_n = 0;
  int dtail_ld = 0;   // row pitch of dtail_M in doubles (n padded against power-of-two strides)
  float *dtail_Mh = nullptr, *dtail_Ml = nullptr;   // its exact two-term FP32 split (FP32 cycle)
  // profiling
  bool prof = false;
  ProfClass pc[5];
  double setup_seconds = 0.0;
  int64_t device_bytes = 0;
};

