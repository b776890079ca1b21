// Level-0 block-Jacobi step (Alg. 1) with the matrix and block-inverse
// streams staged in shared memory by bulk asynchronous copies (sm_90+ TMA
// engine, cp.async.bulk with an mbarrier transaction count).
//
// A tile is TR consecutive block rows.  Its blocks of A are one contiguous
// range [row_ptr[i0], row_ptr[i1]) and its blocks of W = w D^{-1} another,
// so each tile is two bulk copies.  A persistent grid walks the tiles with
// two shared-memory stages: while a CTA computes tile j from one stage, the
// copy engine fills the other with tile j + grid.  Only the gathered x
// entries (L2-resident) and the row-local vectors go through registers.
//
// The arithmetic and its order are those of jacobi_kernel, so both give the
// same bits.  Every wait on an mbarrier is bounded: on time-out the kernel
// records an error code and leaves (the host turns it into GASA_ERR_TIMEOUT).
#include "common.cuh"
#include "internal.h"

namespace gasa {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait: gives up after one second of wall time (or 2^24 rounds)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}

constexpr int kTmaMaxBlocks = 4;   // blocks per block row whose x loads are issued together

template <typename T, int BS>
__global__ void __launch_bounds__(256)
jacobi_tma_kernel(int n_units, int TR, int n_tiles, int stageA, int stageW,
                  const int *__restrict__ rp, const int *__restrict__ col,
                  const T *__restrict__ val, const T *__restrict__ Wm, const T *__restrict__ x,
                  const T *__restrict__ b, T *__restrict__ xo, int *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar[2];
  __shared__ int ok_s;
  constexpr int BSZ = BS * BS;
  constexpr int W = RowVec<T, BS>::value;
  // stage st: A at smem + st * stageA, W at smem + 2 stageA + st * stageW
  auto sA = [&](int st) { return reinterpret_cast<T *>(smem + st * stageA); };
  auto sW = [&](int st) { return reinterpret_cast<T *>(smem + 2 * stageA + st * stageW); };
  T *res = reinterpret_cast<T *>(smem + 2 * stageA + 2 * stageW);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_async_shared();
  }
  __syncthreads();
  auto issue = [&](int tile, int st) {
    const int i0 = tile * TR;
    const int i1 = min(i0 + TR, n_units);
    const int k0 = __ldg(rp + i0), k1 = __ldg(rp + i1);
    const unsigned ab = (unsigned)((k1 - k0) * BSZ * sizeof(T));
    const unsigned wb = (unsigned)((i1 - i0) * BSZ * sizeof(T));
    mbar_arrive_expect_tx(&bar[st], ab + wb);
    if (ab) bulk_g2s(sA(st), val + (size_t)k0 * BSZ, ab, &bar[st]);
    bulk_g2s(sW(st), Wm + (size_t)i0 * BSZ, wb, &bar[st]);
  };
  if (tid == 0 && blockIdx.x < n_tiles) issue(blockIdx.x, 0);
  const int li = tid / BS;
  const int r = tid - li * BS;
  int j = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++j) {
    const int st = j & 1;
    const int next = tile + gridDim.x;
    if (tid == 0 && next < n_tiles) {
      fence_async_shared();
      issue(next, st ^ 1);
    }
    // thread 0 waits (bounded) and tells the CTA; the decision is uniform,
    // so no thread can be left behind at a barrier
    if (tid == 0) ok_s = mbar_wait_bounded(&bar[st], (unsigned)((j >> 1) & 1)) ? 1 : 0;
    __syncthreads();
    if (!ok_s) {
      if (tid == 0) {
        atomicExch(err, 1);
        // let copies still in flight land before the CTA's memory is released
        mbar_wait_bounded(&bar[st], (unsigned)((j >> 1) & 1));
        if (next < n_tiles) mbar_wait_bounded(&bar[st ^ 1], (unsigned)(((j + 1) >> 1) & 1));
      }
      return;
    }
    // the phase is complete: every thread's own try_wait succeeds at once and
    // gives it acquire ordering on the copied bytes
    for (int it = 0; it < 4096 && !mbar_try_wait(&bar[st], (unsigned)((j >> 1) & 1)); ++it) {
    }
    const int i0 = tile * TR;
    const int i = i0 + li;
    const bool active = (li < TR) && (i < n_units);
    const size_t row = (size_t)i * BS + r;
    T v = T(0);
    if (active) {
      const int k0t = __ldg(rp + i0);
      const int beg = __ldg(rp + i), end = __ldg(rp + i + 1);
      T acc = T(0);
      for (int kb = beg; kb < end; kb += kTmaMaxBlocks) {
        const int nb = min(kTmaMaxBlocks, end - kb);
        int jj[kTmaMaxBlocks];
#pragma unroll
        for (int q = 0; q < kTmaMaxBlocks; ++q) jj[q] = q < nb ? __ldg(col + kb + q) : 0;
        T xv[kTmaMaxBlocks][BS];
#pragma unroll
        for (int q = 0; q < kTmaMaxBlocks; ++q) {
          if (q < nb) {
#pragma unroll
            for (int c = 0; c < BS; c += W) load_vec<T, W>(x + (size_t)jj[q] * BS + c, &xv[q][c]);
          }
        }
#pragma unroll
        for (int q = 0; q < kTmaMaxBlocks; ++q) {
          if (q < nb) {
            const T *a = sA(st) + (size_t)(kb + q - k0t) * BSZ + r * BS;
#pragma unroll
            for (int c = 0; c < BS; ++c) acc = fma(a[c], xv[q][c], acc);
          }
        }
      }
      v = b[row] - acc;
    }
    res[tid] = v;
    __syncthreads();
    if (active) {
      const T *w = sW(st) + (size_t)li * BSZ + r * BS;
      T out = T(0);
#pragma unroll
      for (int c = 0; c < BS; ++c) out = fma(w[c], res[li * BS + c], out);
      out += x[row];
      xo[row] = out;
    }
    __syncthreads();   // stage st is refilled at iteration j + 1
  }
}

// Shared-memory plan for a level: tile height, stage sizes, grid.
bool tma_plan(int n_units, int bs, int wbytes, int max_tile_blocks_per_row, int *TR, int *stageA,
              int *stageW, int *smem, int *grid) {
  if (bs != 10 && bs != 4 && bs != 8 && bs != 6) return false;
  const int bsz = bs * bs * wbytes;
  if (bsz % 16 != 0) return false;
  int tr = 256 / bs;
  // two stages of A (max blocks per row of any row) and W per CTA, two CTAs per SM
  const int budget = 100 * 1024;
  while (tr > 1 && 2 * (tr * max_tile_blocks_per_row * bsz + tr * bsz) + 256 * wbytes > budget) --tr;
  if (tr < 4) return false;
  *TR = tr;
  *stageA = ((tr * max_tile_blocks_per_row * bsz) + 127) / 128 * 128;
  *stageW = ((tr * bsz) + 127) / 128 * 128;
  *smem = 2 * *stageA + 2 * *stageW + 256 * wbytes;
  const int tiles = (n_units + tr - 1) / tr;
  *grid = std::min(tiles, 2 * kNumSM);
  return true;
}

template <typename T>
cudaError_t launch_jacobi_tma(int n_units, int bs, int TR, int stageA, int stageW, int smem,
                              int grid, const int *rp, const int *col, const T *val, const T *W,
                              const T *x, const T *b, T *xo, int *err, cudaStream_t s) {
  const int tiles = (n_units + TR - 1) / TR;
#define GASA_TMA_CASE(BS)                                                                      \
  case BS: {                                                                                   \
    cudaError_t e = cudaFuncSetAttribute(jacobi_tma_kernel<T, BS>,                             \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);   \
    if (e != cudaSuccess) return e;                                                            \
    jacobi_tma_kernel<T, BS><<<grid, 256, smem, s>>>(n_units, TR, tiles, stageA, stageW, rp,   \
                                                    col, val, W, x, b, xo, err);               \
    note_launch();                                                                             \
    return cudaGetLastError();                                                                 \
  }
  switch (bs) {
    GASA_TMA_CASE(4) GASA_TMA_CASE(6) GASA_TMA_CASE(8) GASA_TMA_CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef GASA_TMA_CASE
}

template cudaError_t launch_jacobi_tma<float>(int, int, int, int, int, int, int, const int *,
                                              const int *, const float *, const float *,
                                              const float *, const float *, float *, int *,
                                              cudaStream_t);
template cudaError_t launch_jacobi_tma<double>(int, int, int, int, int, int, int, const int *,
                                               const int *, const double *, const double *,
                                               const double *, const double *, double *, int *,
                                               cudaStream_t);

}  // namespace gasa
