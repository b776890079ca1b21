// The bottom levels of the V-cycle (Alg. 2) in one thread-block-cluster
// launch: descriptors shared by the host driver and kernels_tail.cu.
#pragma once
#include <cuda_runtime.h>

#include "gasa.h"

namespace gasa {

constexpr int kTailThreads = 512;             // threads per CTA of the tail kernel
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kTailMaxCluster = 16;

// Ownership: unit u of a level belongs to CTA u mod C of the C-CTA cluster
// and sits at slot u / C there; the CTA's warps take its slots round robin.
// Each CTA keeps in shared memory
//  * the vectors of every tail level (x, x2, b, r) and of the coarsest level
//    (b_N, x_N) for its own units, at offsets that are the same in every CTA
//    (slots for ceil(n / C) units), so that any CTA can read any unit's
//    entries through distributed shared memory;
//  * the matrix rows it computes with: A_k, w D_k^{-1}, P_k rows of its level-k
//    units, R_k rows of its level-(k+1) units, A_N^{-1} rows of its coarsest
//    units, packed per CTA in one global buffer and copied in at the start of
//    the launch.  Row pointers are local to the packed rows; column indices
//    stay global unit ids.
enum { TM_ARP = 0, TM_ACOL, TM_AVAL, TM_W, TM_PRP, TM_PCOL, TM_PVAL, TM_RRP, TM_RCOL, TM_RVAL,
       TM_FIELDS };

template <typename T>
struct TailLevel {
  int n = 0, s = 0;                   // units, dofs per unit
  int s_next = 0, n_next = 0;         // block size and units of level k+1
  int off_x = 0, off_x2 = 0, off_b = 0, off_r = 0;   // vector offsets (bytes, every CTA)
};

template <typename T>
struct TailPlan {
  int k0 = 0, nlev = 0;
  int tpre = 0, tpost = 0;
  int cl = 0;                          // CTAs per cluster the layout was made for
  int vec = 0;                         // 1: 16-byte vector paths allowed
  int nc = 0, nN = 0, sN = 0;
  int off_bN = 0, off_xN = 0;          // coarsest-level vectors (every CTA)
  int mat_base = 0;                    // start of the packed matrix rows in shared memory
  int smem_bytes = 0;                  // dynamic shared memory per CTA
  const unsigned char *pack = nullptr; // packed matrix rows of all CTAs
  int64_t pack_off[kTailMaxCluster] = {};   // byte offset of CTA c's rows in pack
  int pack_bytes[kTailMaxCluster] = {};     // and their size (multiple of 16)
  // byte offsets of each CTA's fields within its packed rows
  int moff[kTailMaxCluster][GASA_MAX_LEVELS][TM_FIELDS] = {};
  int coff[kTailMaxCluster] = {};           // A_N^{-1} rows of the CTA's coarsest units
  const T *b_in = nullptr;             // b_{k0} (global)
  T *x_out = nullptr;                  // x_{k0} after post-smoothing (global)
  TailLevel<T> lv[GASA_MAX_LEVELS];
};

// buffer (0: x, 1: x2) holding a tail level's iterate after pre-smoothing
// and after post-smoothing: the first step writes x, each further step swaps
__host__ __device__ inline int tail_pre_buffer(int tpre) { return tpre >= 1 ? (tpre - 1) & 1 : 0; }
__host__ __device__ inline int tail_final_buffer(int tpre, int tpost) {
  return ((tpre >= 1 ? tpre - 1 : 0) + tpost) & 1;
}
// units of an n-unit level owned by CTA c of a C-CTA cluster
__host__ __device__ inline int tail_owned(int n, int c, int C) { return n > c ? (n - c + C - 1) / C : 0; }

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
