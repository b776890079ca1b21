// Allocation-free variant of the power-iteration estimate (Alg. 4).
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// moment they need this step: a host application whose device-memory budget
// is fixed after start-up and that forbids later allocations, a solver
// embedded in a framework that owns the device allocator, or real-time
// serving code that must not take the allocator's locks or risk an
// out-of-memory failure in the middle of a request.  For them this file
// keeps the step's scratch in a fixed device array compiled into the
// library; the arithmetic is the body gasa_power_estimate runs on scratch it
// allocates.
//
// Scratch layout (doubles): two work vectors of GASA_NOALLOC_MAX_DOFS
// entries, the reduction partials, and two scalars.  The array exists on
// every device that loads the library and stays there until the process
// exits (about 4.2 MB).  All calls on a device share it: a call reads only
// what it wrote itself, but calls that overlap on the GPU (on different
// streams or threads) race on the array and must not be issued.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "gasa.h"
#include "internal.h"

using namespace gasa;

namespace {

constexpr int64_t kMaxDofs = GASA_NOALLOC_MAX_DOFS;
constexpr int64_t kScalars = 2;
constexpr size_t kScratchDoubles = (size_t)(2 * kMaxDofs + kRedBlocks + kScalars);

}  // namespace

// the scratch itself; in host code this name is only a stand-in for the
// symbol, its device address comes from cudaGetSymbolAddress below
static __device__ __align__(256) double g_power_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.  Under lazy module loading
// the first lookup on a device also loads this file's module there, which
// is when the array takes its device memory.
cudaError_t gasa::noalloc_scratch_on_current_device(double **out) {
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
  cudaError_t e = noalloc_scratch_on_current_device(&base);
  if (e != cudaSuccess) return (gasa_status)op_status_code(e);
  const int64_t nnzb = op_nnzb(row_ptr, n_units, s);
  if (nnzb < 0) return GASA_ERR_CUDA;
  // every scratch entry a call reads it has written first in the same call
  // (vectors, partials and scalars alike), so nothing needs clearing
  e = power_estimate_on(n_units, bs, row_ptr, col, val, Dinv, x0, q, nnzb, base, base + kMaxDofs,
                        base + 2 * kMaxDofs, base + 2 * kMaxDofs + kRedBlocks, rho, s);
  return (gasa_status)op_status_code(e);
}
