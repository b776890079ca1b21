// Stand-alone timing of the two heaviest FP32-cycle kernels of the P3 SIPG
// benchmark workload, through the library's own launchers (not part of
// libgasa.so; built against it):
//   * the folded level-0 smoothing step xo = x + c - (W A) x (Alg. 1 with
//     A~^{-1} = w D^{-1} folded into the operator), launch_folded_sweep<float>;
//   * the outer Krylov product q = A p with the p.q partial sums, in
//     double-single arithmetic, launch_bsr_mv_ds.
// The block pattern is the face graph of the n x n jittered grid split into
// two P3 triangles per square, in the mesh's element order: triangle 2q
// (lower right of square q = j n + i) meets 2q+1 across the diagonal, the
// square below (2(q-n)+1) and the square to the right (2(q+1)+1); triangle
// 2q+1 meets 2q, the square to the left (2(q-1)) and the square above
// (2(q+n)); tests/test_synth.py pins this rule against the mesh.  With the
// diagonal and 10 x 10 blocks it is exactly the benchmark's level-0 pattern
// (n = 256: 131,072 block rows, 523,264 blocks); the values are seeded
// uniform numbers, which do not change the memory traffic.
// Each kernel is checked on sampled rows against an FP64 host product and
// timed by CUDA events on its stream (median over the rounds).
//
// Build and run (after the library is built):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//     -Iinclude -Ipaper_2504_13373_gb300/csrc paper_2504_13373_gb300/csrc/bench_level0.cu \
//     -o bench_level0 -Lpaper_2504_13373_gb300 -lgasa
//   LD_LIBRARY_PATH=paper_2504_13373_gb300 ./bench_level0 [n=256] [rounds=25]
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "internal.h"

using namespace gasa;

#define CK(x)                                                                                \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) {                                                                 \
      fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);      \
      exit(2);                                                                               \
    }                                                                                        \
  } while (0)

namespace {

constexpr int kB = 10;   // P3 triangle: 10 dofs

// splitmix64 (Steele, Lea & Flood 2014), mapped to uniform(-1, 1)
double uniform(uint64_t stream, uint64_t i) {
  uint64_t z = stream * 0x100000001b3ull + i + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

void pattern(int n, std::vector<int> &rp, std::vector<int> &col) {
  const int nb = 2 * n * n;
  rp.assign(nb + 1, 0);
  col.clear();
  for (int q = 0; q < n * n; ++q) {
    const int i = q % n, j = q / n;
    for (int h = 0; h < 2; ++h) {
      int c[4], m = 0;
      c[m++] = 2 * q;
      c[m++] = 2 * q + 1;
      if (h == 0) {
        if (j > 0) c[m++] = 2 * (q - n) + 1;
        if (i + 1 < n) c[m++] = 2 * (q + 1) + 1;
      } else {
        if (i > 0) c[m++] = 2 * (q - 1);
        if (j + 1 < n) c[m++] = 2 * (q + n);
      }
      std::sort(c, c + m);
      for (int k = 0; k < m; ++k) col.push_back(c[k]);
      rp[2 * q + h + 1] = (int)col.size();
    }
  }
}

template <typename T>
T *upload(const std::vector<T> &h) {
  T *d = nullptr;
  CK(cudaMalloc(&d, h.size() * sizeof(T)));
  CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

template <typename T>
std::vector<T> download(const T *d, size_t n) {
  std::vector<T> h(n);
  CK(cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost));
  return h;
}

template <typename F>
double median_us(F launch, int rounds, cudaStream_t s) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  std::vector<float> t;
  for (int r = 0; r < rounds + 3; ++r) {
    CK(cudaEventRecord(a, s));
    CK(launch());
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (r >= 3) t.push_back(ms);
  }
  CK(cudaEventDestroy(a));
  CK(cudaEventDestroy(b));
  std::sort(t.begin(), t.end());
  return 1e3 * t[t.size() / 2];
}

}  // namespace

int main(int argc, char **argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 256;
  const int rounds = argc > 2 ? atoi(argv[2]) : 25;
  if (n < 1 || n > 1024 || rounds < 1) {
    fprintf(stderr, "usage: bench_level0 [n in 1..1024] [rounds >= 1]\n");
    return 1;
  }
  std::vector<int> rp, col;
  pattern(n, rp, col);
  const int nb = 2 * n * n;
  const size_t nnzb = col.size(), rows = (size_t)nb * kB, nval = nnzb * kB * kB;
  for (int c : col)
    if (c < 0 || c >= nb) return 3;

  // operands: WA and A as exact FP32 splits (hi, lo) of FP64 values; x, c, p
  std::vector<float> wa(nval), ahi(nval), alo(nval), x(rows), c(rows), phi(rows), plo(rows);
  std::vector<double> pd(rows);
  for (size_t i = 0; i < nval; ++i) {
    wa[i] = (float)(0.25 * uniform(1, i));
    const double a = uniform(2, i);
    ahi[i] = (float)a;
    alo[i] = (float)(a - (double)ahi[i]);
  }
  for (size_t i = 0; i < rows; ++i) {
    x[i] = (float)uniform(3, i);
    c[i] = (float)uniform(4, i);
    pd[i] = uniform(5, i);
    phi[i] = (float)pd[i];
    plo[i] = (float)(pd[i] - (double)phi[i]);
  }
  int *d_rp = upload(rp), *d_col = upload(col);
  float *d_wa = upload(wa), *d_ahi = upload(ahi), *d_alo = upload(alo), *d_x = upload(x),
        *d_c = upload(c), *d_phi = upload(phi), *d_plo = upload(plo), *d_xo = nullptr;
  double *d_pd = upload(pd), *d_q = nullptr, *d_part = nullptr;
  const int parts = bsr_mv_ds_grid(nb, kB);
  CK(cudaMalloc(&d_xo, rows * sizeof(float)));
  CK(cudaMalloc(&d_q, rows * sizeof(double)));
  CK(cudaMalloc(&d_part, (size_t)parts * sizeof(double)));
  cudaStream_t s;
  CK(cudaStreamCreate(&s));

  auto folded = [&] { return launch_folded_sweep<float>(nb, kB, d_rp, d_col, d_wa, d_x, d_c, d_xo, s); };
  auto outer = [&] {
    return launch_bsr_mv_ds(nb, kB, kB, d_rp, d_col, d_ahi, d_alo, d_phi, d_plo, d_q, s, d_pd,
                            d_part);
  };
  CK(folded());
  CK(outer());
  CK(cudaStreamSynchronize(s));
  const std::vector<float> xo = download(d_xo, rows);
  const std::vector<double> q = download(d_q, rows);
  const std::vector<double> part = download(d_part, (size_t)parts);

  // sampled rows against FP64 host products
  double worst_f = 0.0, worst_q = 0.0;
  for (size_t t = 0; t < rows; t += 317) {
    const int i = (int)(t / kB), r = (int)(t % kB);
    double acc_f = 0.0, abs_f = 0.0, acc_q = 0.0, abs_q = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      for (int e = 0; e < kB; ++e) {
        const size_t v = ((size_t)k * kB + r) * kB + e, xi = (size_t)col[k] * kB + e;
        acc_f += (double)wa[v] * x[xi];
        abs_f += fabs((double)wa[v] * x[xi]);
        const double a = (double)ahi[v] + (double)alo[v], p = (double)phi[xi] + (double)plo[xi];
        acc_q += a * p;
        abs_q += fabs(a * p);
      }
    const double want_f = (double)x[t] + ((double)c[t] - acc_f);
    worst_f = std::max(worst_f, fabs(xo[t] - want_f) / (fabs(x[t]) + fabs(c[t]) + abs_f));
    worst_q = std::max(worst_q, fabs(q[t] - acc_q) / abs_q);
  }
  double dot = 0.0, dot_ref = 0.0, dot_abs = 0.0;
  for (int b = 0; b < parts; ++b) dot += part[b];
  for (size_t t = 0; t < rows; ++t) {
    dot_ref += pd[t] * q[t];
    dot_abs += fabs(pd[t] * q[t]);
  }
  const bool ok_f = worst_f <= 40 * ldexp(1.0, -24);
  const bool ok_q = worst_q <= ldexp(1.0, -40);
  const bool ok_d = fabs(dot - dot_ref) <= 1e-12 * dot_abs;   // summation order only

  const double us_f = median_us(folded, rounds, s), us_q = median_us(outer, rounds, s);
  // algorithmic bytes: every matrix value, column index and row pointer once,
  // x (gathered, counted once), c and the result; the outer product reads
  // both FP32 words of A and of p, p in FP64 for p.q, and writes q in FP64
  const double idx = nnzb * 4.0 + (nb + 1) * 4.0;
  const double bytes_f = nval * 4.0 + idx + rows * 4.0 * 3;
  const double bytes_q = nval * 8.0 + idx + rows * 8.0 + rows * 8.0 + rows * 8.0 + parts * 8.0;
  printf("pattern: %d x %d grid, %d block rows, %zu blocks of %d x %d\n", n, n, nb, nnzb, kB, kB);
  printf("folded step  : %8.2f us, %7.1f MB algorithmic, %7.1f GB/s; sampled rows within %.2e "
         "of sum|WA x| %s\n",
         us_f, bytes_f / 1e6, bytes_f / us_f / 1e3, worst_f, ok_f ? "ok" : "FAIL");
  printf("outer product: %8.2f us, %7.1f MB algorithmic, %7.1f GB/s; sampled rows within %.2e "
         "of sum|a p| %s; p.q %s\n",
         us_q, bytes_q / 1e6, bytes_q / us_q / 1e3, worst_q, ok_q ? "ok" : "FAIL",
         ok_d ? "ok" : "FAIL");
  CK(cudaStreamDestroy(s));
  for (void *p : {(void *)d_rp, (void *)d_col, (void *)d_wa, (void *)d_ahi, (void *)d_alo,
                  (void *)d_x, (void *)d_c, (void *)d_phi, (void *)d_plo, (void *)d_xo,
                  (void *)d_pd, (void *)d_q, (void *)d_part})
    CK(cudaFree(p));
  return ok_f && ok_q && ok_d ? 0 : 1;
}
