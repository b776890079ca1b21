// Allocation-free variant of the power-iteration estimate (Alg. 4).
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// moment they need this step: a host application whose device-memory budget
// is fixed after start-up and that forbids later allocations, a solver
// embedded in a framework that owns the device allocator, or real-time
// serving code that must not take the allocator's locks or risk an
// out-of-memory failure in the middle of a request.  For them this file
// keeps the step's scratch in a fixed device array compiled into the
// library.
//
// Scratch layout (doubles): two work vectors of GASA_NOALLOC_MAX_DOFS
// entries, the reduction partials, and a few scalars.  The array exists on
// every device that loads the library and stays there until the process
// exits (about 4.2 MB).  All calls on a device share it: a call reads only
// what it wrote itself, but calls that overlap on the GPU (on different
// streams or threads) race on the array and must not be issued.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "gasa.h"
#include "internal.h"

using namespace gasa;

namespace {

constexpr int64_t kMaxDofs = GASA_NOALLOC_MAX_DOFS;
constexpr int64_t kScalars = 8;
constexpr size_t kScratchDoubles = (size_t)(2 * kMaxDofs + kRedBlocks + kScalars);

}  // namespace

// the scratch itself; in host code this name is only a stand-in for the
// symbol, its device address comes from cudaGetSymbolAddress below
static __device__ __align__(256) double g_power_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_on_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_power_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int64_t stored_blocks(const int32_t *row_ptr, int32_t n, cudaStream_t s) {
  int32_t v = -1;
  if (cudaMemcpyAsync(&v, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return v;
}

}  // namespace

extern "C" gasa_status gasa_power_estimate_noalloc(int32_t n_units, int32_t bs,
                                                   const int32_t *row_ptr, const int32_t *col,
                                                   const double *val, const double *Dinv,
                                                   const double *x0, int32_t q, double *rho,
                                                   void *stream) {
  if (n_units <= 0 || bs <= 0 || bs > 1024 || q < 0 || !row_ptr || !col || !val || !Dinv ||
      !x0 || !rho)
    return GASA_ERR_INVALID_ARG;
  const int64_t n = (int64_t)n_units * bs;
  if (n > kMaxDofs) return GASA_ERR_INVALID_ARG;   // larger than the fixed scratch
  cudaStream_t s = (cudaStream_t)stream;
  double *base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) return GASA_ERR_CUDA;
  double *a = base, *b = base + kMaxDofs, *part = base + 2 * kMaxDofs, *sc = part + kRedBlocks;
  const int64_t nnzb = stored_blocks(row_ptr, n_units, s);
  // the scalars start from zero on every call (the vectors and partials are
  // written before they are read)
  e = cudaMemsetAsync(sc, 0, kScalars * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_dot_partials(n, a, nullptr, part, s);
  if (e == cudaSuccess) e = launch_finalize(part, 1, sc, s);
  if (e == cudaSuccess) e = launch_scale_by_inv_sqrt(n, a, sc, s);
  for (int it = 0; it < q && e == cudaSuccess; ++it) {
    e = launch_jacobi<double>(JAC_APPLY, n_units, bs, row_ptr, col, val, Dinv, a, nullptr, b, s,
                              nnzb);
    if (e == cudaSuccess) e = launch_dot_partials(n, b, nullptr, part, s);
    if (e == cudaSuccess) e = launch_finalize(part, 1, sc, s);
    if (e == cudaSuccess) e = launch_scale_by_inv_sqrt(n, b, sc, s);
    std::swap(a, b);
  }
  if (e == cudaSuccess)
    e = launch_jacobi<double>(JAC_APPLY, n_units, bs, row_ptr, col, val, Dinv, a, nullptr, b, s,
                              nnzb);
  if (e == cudaSuccess) e = launch_dot_partials(n, b, nullptr, part, s);
  if (e == cudaSuccess) e = launch_finalize(part, 1, sc + 1, s);
  double h = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GASA_ERR_CUDA;
  *rho = std::sqrt(h);
  return GASA_OK;
}
