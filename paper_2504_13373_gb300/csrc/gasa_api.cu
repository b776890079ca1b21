// C ABI of the library: context, Alg. 5 setup driver, Alg. 2 V-cycle,
// CG / GMRES outer loops, and single-operation entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "gasa.h"
#include "internal.h"
#include "ctx.h"
#include "tail.h"
#include "grid.h"
#include "batch.h"

using namespace gasa;

namespace {

const char *kStatusText[] = {"ok",
                             "invalid argument",
                             "device allocation failed",
                             "CUDA error",
                             "singular diagonal block or coarse matrix",
                             "matrix not SPD (CG breakdown)",
                             "not converged",
                             "breakdown",
                             "timeout",
                             "over budget",
                             "pending",
                             "unsupported input",
                             "call out of order"};

gasa_status fail(gasa_ctx *c, gasa_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

#define CU(...)                                                                        \
  do {                                                                                 \
    cudaError_t e_ = (__VA_ARGS__);                                                    \
    if (e_ != cudaSuccess) {                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GASA_ERR_OOM : GASA_ERR_CUDA, \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));          \
    }                                                                                  \
  } while (0)

#define ST(...)                         \
  do {                                  \
    gasa_status s_ = (__VA_ARGS__);     \
    if (s_ != GASA_OK) return s_;       \
  } while (0)

template <typename T>
gasa_status dalloc(gasa_ctx *ctx, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, GASA_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->allocs.push_back((void *)*p);
  ctx->device_bytes += (int64_t)(count * sizeof(T));
  return GASA_OK;
}

void dfree(gasa_ctx *ctx, void *p) {
  if (!p) return;
  auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
  if (it != ctx->allocs.end()) ctx->allocs.erase(it);
  cudaFree(p);
}

void free_graphs(gasa_ctx *ctx) {
  for (int p = 0; p < 6; ++p) {
    if (ctx->cg_exec[p]) cudaGraphExecDestroy(ctx->cg_exec[p]);
    if (ctx->cg_graph[p]) cudaGraphDestroy(ctx->cg_graph[p]);
    ctx->cg_exec[p] = nullptr;
    ctx->cg_graph[p] = nullptr;
    ctx->cg_kernels[p] = 0;
  }
}

void free_all(gasa_ctx *ctx) {
  cudaStreamSynchronize(ctx->stream);
  free_graphs(ctx);
  for (void *p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  if (ctx->hscal) {
    cudaFreeHost(ctx->hscal);
    ctx->hscal = nullptr;
  }
  ctx->L.clear();
  ctx->ready = false;
  ctx->device_bytes = 0;
  ctx->coarse_inv = nullptr;
  for (int p = 0; p < 2; ++p) {
    ctx->tail_plan[p] = nullptr;
    ctx->tail_k0[p] = 0;
    ctx->grid_plan[p] = nullptr;
    ctx->grid_k0[p] = 0;
    ctx->grid_ctas[p] = 0;
  }
  ctx->grid_bar = nullptr;
  ctx->dtail_M = nullptr;
  ctx->dtail_Mh = ctx->dtail_Ml = nullptr;
  ctx->dtail_k = 0;
  ctx->dtail_n = 0;
  ctx->dtail_ld = 0;
  ctx->V = ctx->Z = ctx->H = ctx->gm = ctx->mpart = nullptr;
  ctx->gm_restart = 0;
}

// ----------------------------------------------------------------------------
// profiling helpers (CUDA events on the context stream)
// ----------------------------------------------------------------------------
void prof_begin(gasa_ctx *ctx, int cls, cudaEvent_t *e0) {
  *e0 = nullptr;
  if (!ctx->prof) return;
  ProfClass &p = ctx->pc[cls];
  if (p.used + 2 > p.ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      p.ev.push_back(ev);
    }
  }
  *e0 = p.ev[p.used];
  cudaEventRecord(*e0, ctx->stream);
}
void prof_end(gasa_ctx *ctx, int cls, double bytes) {
  if (!ctx->prof) return;
  ProfClass &p = ctx->pc[cls];
  cudaEventRecord(p.ev[p.used + 1], ctx->stream);
  p.used += 2;
  p.bytes += bytes;
  p.launches += 1;
}

// ----------------------------------------------------------------------------
// V-cycle (Alg. 2), one pass from a zero initial guess; T = double or float
// ----------------------------------------------------------------------------
template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double *A(const DevBSR &m) { return m.val; }
  static const double *W(const Level &l) { return l.W; }
  static const double *WA(const Level &l) { return l.WA; }
  static double *c(Level &l) { return l.c; }
  static double *x(Level &l) { return l.x; }
  static double *x2(Level &l) { return l.x2; }
  static double *b(Level &l) { return l.b; }
  static double *r(Level &l) { return l.r; }
  static double *mt(Level &l) { return l.mt; }
  static double *mu(Level &l) { return l.mu; }
};
template <> struct Prec<float> {
  static const float *A(const DevBSR &m) { return m.val32; }
  static const float *W(const Level &l) { return l.W32; }
  static const float *WA(const Level &l) { return l.WA32; }
  static float *c(Level &l) { return l.cf; }
  static float *x(Level &l) { return l.xf; }
  static float *x2(Level &l) { return l.x2f; }
  static float *b(Level &l) { return l.bf; }
  static float *r(Level &l) { return l.rf; }
  static float *mt(Level &l) { return l.mtf; }
  static float *mu(Level &l) { return l.muf; }
};

// y = A_k x (mode ASSIGN) or y = b - A_k x (RESIDUAL) on a matrix-free level
// k >= 1: A_k x = R_{k-1} (A_{k-1} (P_{k-1} x)) (Section 4.4, Eq. matfree2
// with the transfers unrolled), recursively while A_{k-1} is matrix-free too
template <typename T>
cudaError_t mf_apply(gasa_ctx *ctx, int k, int mode, const T *x, const T *b, T *y) {
  using P = Prec<T>;
  cudaStream_t s = ctx->stream;
  Level &lp = ctx->L[k - 1];
  T *t = P::mt(lp), *u = P::mu(lp);
  cudaError_t e = launch_bsr_mv<T>(GASA_MV_ASSIGN, lp.P.nrows, lp.P.br, lp.P.bc, lp.P.rp, lp.P.col,
                                   P::A(lp.P), x, nullptr, t, s, lp.P.nnzb);
  if (e != cudaSuccess) return e;
  if (k - 1 > 0 && lp.mf) e = mf_apply<T>(ctx, k - 1, GASA_MV_ASSIGN, t, nullptr, u);
  else e = launch_bsr_mv<T>(GASA_MV_ASSIGN, lp.n, lp.s, lp.s, lp.A.rp, lp.A.col, P::A(lp.A), t,
                            nullptr, u, s, lp.A.nnzb);
  if (e != cudaSuccess) return e;
  return launch_bsr_mv<T>(mode, lp.R.nrows, lp.R.br, lp.R.bc, lp.R.rp, lp.R.col, P::A(lp.R), u, b,
                          y, s, lp.R.nnzb);
}

// algorithmic bytes of one launch: w bytes per vector entry, wa bytes per
// matrix value (FP16 blocks add one 4-byte scale per block)
// folded: the step reads W A instead of A and W (and c instead of b); the
// first step also writes c
double sweep_bytes(const Level &l, int w, bool first, int wa = 0, bool folded = false) {
  if (wa == 0) wa = w;
  const double vec = (double)l.ndof * w;
  const double Wb = (double)l.n * l.s * l.s * wa + (wa == 2 ? 4.0 * l.n : 0.0);
  if (first) return Wb + (folded ? 3.0 : 2.0) * vec;
  const double Ab = (double)l.A.nnzb * l.s * l.s * wa + (wa == 2 ? 4.0 * l.A.nnzb : 0.0) +
                    4.0 * l.A.nnzb + 4.0 * (l.n + 1);
  return Ab + (folded ? 0.0 : Wb) + 3.0 * vec;
}
double spmv_bytes(const Level &l, int w, bool residual, int wa = 0) {
  if (wa == 0) wa = w;
  const double vec = (double)l.ndof * w;
  const double Ab = (double)l.A.nnzb * l.s * l.s * wa + (wa == 2 ? 4.0 * l.A.nnzb : 0.0) +
                    4.0 * l.A.nnzb + 4.0 * (l.n + 1);
  return Ab + (residual ? 3.0 : 2.0) * vec;
}

// Plan of the fused bottom of the V-cycle for precision T (slot pi: 0 FP64,
// 1 FP32): the deepest run of levels k >= 1 whose A_k is stored and takes at
// most opt.tail_kib KiB, with every level below it down to the coarsest,
// while the coarsest inverse is small (2 MB) and each CTA's share of the
// vectors and matrix rows fits in its shared memory (top levels are dropped
// until it does).  The matrix rows are packed per CTA on the host.
template <typename T>
gasa_status tail_build(gasa_ctx *ctx, int pi) {
  using P = Prec<T>;
  const int N = ctx->N;
  ctx->tail_k0[pi] = N;
  ctx->tail_plan[pi] = nullptr;
  const int64_t limit = (int64_t)ctx->opt.tail_kib * 1024;
  if (limit <= 0 || N < 2) return GASA_OK;
  if ((int64_t)ctx->nc * ctx->nc * 8 > (2 << 20)) return GASA_OK;
  Level &lc = ctx->L[N];
  int k0 = N;
  for (int k = N - 1; k >= 1; --k) {
    Level &l = ctx->L[k];
    if (l.mf || l.tma || l.s > 64 || l.R.br > 64) break;
    if (l.P.nrows != l.n || l.P.br != l.s || l.P.bc != l.R.br || l.R.bc != l.s ||
        l.R.nrows != ctx->L[k + 1].n || l.R.br != ctx->L[k + 1].s)
      break;
    if (l.A.nnzb * l.s * l.s * (int64_t)sizeof(T) > limit) break;
    k0 = k;
  }
  if (k0 == N) return GASA_OK;
  const int cl = tail_cluster_size<T>();
  if (cl == 0 || cl > kTailMaxCluster) return GASA_OK;
  cudaStream_t s = ctx->stream;
  CU(cudaStreamSynchronize(s));
  // host copies of the candidate levels' operators
  struct HostBSR {
    std::vector<int> rp, col;
    std::vector<T> val;
  };
  auto fetch = [&](const DevBSR &m, const T *val, HostBSR &h) -> gasa_status {
    h.rp.resize(m.nrows + 1);
    h.col.resize(m.nnzb);
    h.val.resize((size_t)m.nnzb * m.br * m.bc);
    CU(cudaMemcpy(h.rp.data(), m.rp, h.rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(h.col.data(), m.col, h.col.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(h.val.data(), val, h.val.size() * sizeof(T), cudaMemcpyDeviceToHost));
    return GASA_OK;
  };
  const int nlmax = N - k0;
  std::vector<HostBSR> hA(nlmax), hP(nlmax), hR(nlmax);
  std::vector<std::vector<T>> hW(nlmax);
  for (int q = 0; q < nlmax; ++q) {
    Level &l = ctx->L[k0 + q];
    ST(fetch(l.A, P::A(l.A), hA[q]));
    ST(fetch(l.P, P::A(l.P), hP[q]));
    ST(fetch(l.R, P::A(l.R), hR[q]));
    hW[q].resize((size_t)l.n * l.s * l.s);
    CU(cudaMemcpy(hW[q].data(), P::W(l), hW[q].size() * sizeof(T), cudaMemcpyDeviceToHost));
  }
  std::vector<double> hC((size_t)ctx->nc * ctx->nc);
  CU(cudaMemcpy(hC.data(), ctx->coarse_inv, hC.size() * sizeof(double), cudaMemcpyDeviceToHost));
  auto r16 = [](int64_t b) { return (b + 15) / 16 * 16; };
  auto vec_bytes = [&](int n, int sz) { return r16((int64_t)((n + cl - 1) / cl) * sz * (int64_t)sizeof(T)); };
  for (; k0 < N; ++k0) {
    const int q0 = k0 - (N - nlmax), nl = N - k0;
    TailPlan<T> h;
    h.k0 = k0;
    h.nlev = nl;
    h.tpre = ctx->opt.t_pre;
    h.tpost = ctx->opt.t_post;
    h.cl = cl;
    h.vec = 1;
    h.nc = ctx->nc;
    h.nN = lc.n;
    h.sN = lc.s;
    h.b_in = P::b(ctx->L[k0]);
    h.x_out = P::x(ctx->L[k0]);
    // vectors: the same offsets in every CTA
    int64_t off = 0;
    for (int q = 0; q < nl; ++q) {
      Level &l = ctx->L[k0 + q];
      TailLevel<T> &t = h.lv[q];
      t.n = l.n;
      t.s = l.s;
      t.n_next = l.R.nrows;
      t.s_next = l.R.br;
      const int64_t vb = vec_bytes(l.n, l.s);
      t.off_x = (int)off;
      t.off_x2 = (int)(off + vb);
      t.off_b = (int)(off + 2 * vb);
      t.off_r = (int)(off + 3 * vb);
      off += 4 * vb;
    }
    h.off_bN = (int)off;
    h.off_xN = (int)(off + vec_bytes(lc.n, lc.s));
    off += 2 * vec_bytes(lc.n, lc.s);
    h.mat_base = (int)off;
    // packed matrix rows per CTA
    std::vector<unsigned char> pack;
    int64_t maxb = 0;
    for (int c = 0; c < cl; ++c) {
      std::vector<unsigned char> buf;
      auto put = [&](const void *src, size_t bytes) -> int {
        const size_t at = (size_t)r16((int64_t)buf.size());
        buf.resize(at + bytes);
        if (bytes) std::memcpy(buf.data() + at, src, bytes);
        return (int)at;
      };
      // rows u = c, c + cl, ... of a BSR matrix: local row pointers, cols, values
      auto put_rows = [&](const HostBSR &m, int nrows, int bsz, int *fo) {
        std::vector<int> lrp(1, 0), lcol;
        std::vector<T> lval;
        for (int u = c; u < nrows; u += cl) {
          for (int k = m.rp[u]; k < m.rp[u + 1]; ++k) {
            lcol.push_back(m.col[k]);
            lval.insert(lval.end(), m.val.begin() + (size_t)k * bsz, m.val.begin() + (size_t)(k + 1) * bsz);
          }
          lrp.push_back((int)lcol.size());
        }
        fo[0] = put(lrp.data(), lrp.size() * sizeof(int));
        fo[1] = put(lcol.data(), lcol.size() * sizeof(int));
        fo[2] = put(lval.data(), lval.size() * sizeof(T));
      };
      for (int q = 0; q < nl; ++q) {
        const int qq = q0 + q;
        Level &l = ctx->L[k0 + q];
        int *mo = h.moff[c][q];
        int fo[3];
        put_rows(hA[qq], l.n, l.s * l.s, fo);
        mo[TM_ARP] = fo[0];
        mo[TM_ACOL] = fo[1];
        mo[TM_AVAL] = fo[2];
        std::vector<T> w;
        for (int u = c; u < l.n; u += cl)
          w.insert(w.end(), hW[qq].begin() + (size_t)u * l.s * l.s, hW[qq].begin() + (size_t)(u + 1) * l.s * l.s);
        mo[TM_W] = put(w.data(), w.size() * sizeof(T));
        put_rows(hP[qq], l.n, l.s * l.R.br, fo);
        mo[TM_PRP] = fo[0];
        mo[TM_PCOL] = fo[1];
        mo[TM_PVAL] = fo[2];
        put_rows(hR[qq], l.R.nrows, l.R.br * l.s, fo);
        mo[TM_RRP] = fo[0];
        mo[TM_RCOL] = fo[1];
        mo[TM_RVAL] = fo[2];
      }
      std::vector<double> crows;
      for (int u = c; u < lc.n; u += cl)
        crows.insert(crows.end(), hC.begin() + (size_t)u * lc.s * ctx->nc,
                     hC.begin() + (size_t)(u + 1) * lc.s * ctx->nc);
      h.coff[c] = put(crows.data(), crows.size() * sizeof(double));
      buf.resize((size_t)r16((int64_t)buf.size()));
      h.pack_off[c] = (int64_t)pack.size();
      h.pack_bytes[c] = (int)buf.size();
      pack.insert(pack.end(), buf.begin(), buf.end());
      maxb = std::max<int64_t>(maxb, (int64_t)buf.size());
    }
    h.smem_bytes = (int)(off + maxb);
    if (off + maxb > tail_smem_limit()) continue;   // too big: start one level lower
    unsigned char *dpack = nullptr, *dplan = nullptr;
    ST(dalloc(ctx, &dpack, pack.size()));
    CU(cudaMemcpy(dpack, pack.data(), pack.size(), cudaMemcpyHostToDevice));
    h.pack = dpack;
    ST(dalloc(ctx, &dplan, sizeof(TailPlan<T>)));
    CU(cudaMemcpy(dplan, &h, sizeof(h), cudaMemcpyHostToDevice));
    ctx->tail_plan[pi] = dplan;
    ctx->tail_k0[pi] = k0;
    ctx->tail_coarse[pi] = 1;
    ctx->tail_cluster[pi] = cl;
    ctx->tail_smem[pi] = h.smem_bytes;
    return GASA_OK;
  }
  return GASA_OK;
}

// Plan of the persistent coarse levels for precision T (slot pi: 0 FP64,
// 1 FP32), with opt.grid_tail: levels k0 .. N in one cooperative launch,
// k0 the first level k >= 1 from which every level is stored unpadded with
// one block size s <= 8 (A_k, P_k, R_k all s x s blocks).
template <typename T>
gasa_status grid_build(gasa_ctx *ctx, int pi) {
  using P = Prec<T>;
  const int N = ctx->N;
  ctx->grid_plan[pi] = nullptr;
  ctx->grid_k0[pi] = N;
  ctx->grid_ctas[pi] = 0;
  if (!ctx->opt.grid_tail || N < 2 || ctx->opt.t_pre < 1) return GASA_OK;
  Level &lc = ctx->L[N];
  const int S = lc.s;
  if (S < 1 || S > 8 || lc.padded) return GASA_OK;
  int k0 = N;
  for (int k = N - 1; k >= 1; --k) {
    Level &l = ctx->L[k];
    if (l.mf || l.padded || l.s != S) break;
    if (l.P.nrows != l.n || l.P.br != S || l.P.bc != S || l.R.br != S || l.R.bc != S ||
        l.R.nrows != ctx->L[k + 1].n)
      break;
    if (!P::A(l.A) || !P::W(l) || !P::A(l.P) || !P::A(l.R)) break;
    k0 = k;
  }
  if (k0 == N) return GASA_OK;
  const int ctas = grid_tail_ctas<T>(S, 2);
  if (ctas <= 0) return GASA_OK;
  if (!ctx->grid_bar) ST(dalloc(ctx, &ctx->grid_bar, 1));
  GridPlan<T> h;
  h.k0 = k0;
  h.nlev = N - k0;
  h.tpre = ctx->opt.t_pre;
  h.tpost = ctx->opt.t_post;
  h.s = S;
  h.nc = ctx->nc;
  h.cinv = ctx->coarse_inv;
  h.bN = P::b(lc);
  h.xN = P::x(lc);
  h.bar = ctx->grid_bar;
  h.err = ctx->d_err;
  const double budget = ctx->opt.wait_budget_s > 0.0 ? ctx->opt.wait_budget_s : 1.0;
  h.budget_ns = (unsigned long long)(budget * 1e9) + 1ull;
  for (int q = 0; q < h.nlev; ++q) {
    Level &l = ctx->L[k0 + q];
    GridLevel<T> &g = h.lv[q];
    g.n = l.n;
    g.n_next = ctx->L[k0 + q + 1].n;
    g.arp = l.A.rp;
    g.acol = l.A.col;
    g.aval = P::A(l.A);
    g.W = P::W(l);
    g.prp = l.P.rp;
    g.pcol = l.P.col;
    g.pval = P::A(l.P);
    g.rrp = l.R.rp;
    g.rcol = l.R.col;
    g.rval = P::A(l.R);
    g.x = P::x(l);
    g.x2 = P::x2(l);
    g.b = P::b(l);
    g.r = P::r(l);
    g.tlA = grid_team(S, (double)l.A.nnzb / (double)l.n);
    g.tlP = grid_team(S, (double)l.P.nnzb / (double)l.P.nrows);
    g.tlR = grid_team(S, (double)l.R.nnzb / (double)l.R.nrows);
  }
  GridPlan<T> *dplan = nullptr;
  ST(dalloc(ctx, &dplan, 1));
  CU(cudaMemcpy(dplan, &h, sizeof(h), cudaMemcpyHostToDevice));
  ctx->grid_plan[pi] = dplan;
  ctx->grid_k0[pi] = k0;
  ctx->grid_ctas[pi] = ctas;
  ctx->grid_s[pi] = S;
  return GASA_OK;
}

// Dense bottom of the V-cycle (opt.dense_tail_dofs).  From level kt down,
// Alg. 2 started from u_kt = 0 is a fixed linear map of b_kt: each smoothing
// step, residual, restriction, prolongation and the coarsest solve is linear
// in it.  On the coarse levels each of those steps is a launch whose cost is
// latency rather than bytes, so setup runs exactly those steps (FP64, the
// batched kernels of the request server) on the unit vectors, eight at a
// time, and keeps the results as the columns of M_kt; the V-cycle then
// applies u_kt = M_kt b_kt as one dense product.  kt is the first level
// k >= 1 from which every level holds at most dense_tail_dofs stored dofs
// and is stored (not matrix-free).
gasa_status dense_tail_build(gasa_ctx *ctx) {
  const int N = ctx->N;
  ctx->dtail_M = nullptr;
  ctx->dtail_Mh = ctx->dtail_Ml = nullptr;
  ctx->dtail_k = N;
  ctx->dtail_n = 0;
  const gasa_options &o = ctx->opt;
  if (o.dense_tail_dofs <= 0 || o.tail_kib > 0 || o.grid_tail || N < 2) return GASA_OK;
  int kt = N;
  for (int k = N - 1; k >= 1; --k) {
    const Level &l = ctx->L[k];
    if (l.mf || !l.A.val || l.ndof > o.dense_tail_dofs) break;
    kt = k;
  }
  if (kt == N) return GASA_OK;
  constexpr int K = 8;
  cudaStream_t s = ctx->stream;
  const int n = (int)ctx->L[kt].ndof;
  const int tpre = o.t_pre, tpost = o.t_post;
  // scratch per level kt .. N: x, x2, b, r of K interleaved columns
  size_t tot = 0;
  for (int k = kt; k <= N; ++k) tot += 4 * (size_t)ctx->L[k].ndof * K;
  double *scr = nullptr;
  ST(dalloc(ctx, &scr, tot));
  std::vector<double *> X(N + 1), X2(N + 1), B(N + 1), Rv(N + 1);
  {
    double *p = scr;
    for (int k = kt; k <= N; ++k) {
      const size_t m = (size_t)ctx->L[k].ndof * K;
      X[k] = p;
      X2[k] = p + m;
      B[k] = p + 2 * m;
      Rv[k] = p + 3 * m;
      p += 4 * m;
    }
  }
  // rows of M 128-byte aligned and 129 * 128 bytes apart for n = 2048 (a row
  // pitch that is no power of two)
  const int ld = ((n + 15) / 16) * 16 + 16;
  double *M = nullptr;
  gasa_status st = dalloc(ctx, &M, (size_t)n * ld);
  if (st == GASA_OK) CU(cudaMemsetAsync(M, 0, (size_t)n * ld * sizeof(double), s));
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
    return e == cudaSuccess;
  };
  for (int c0 = 0; st == GASA_OK && e == cudaSuccess && c0 < n; c0 += K) {
    std::vector<double *> xk(N + 1);
    if (!ok(launch_bunit_columns(n, K, c0, B[kt], s))) break;
    for (int k = kt; k < N && e == cudaSuccess; ++k) {
      Level &l = ctx->L[k];
      double *x = X[k], *x2 = X2[k];
      if (tpre == 0) {
        ok(cudaMemsetAsync(x, 0, (size_t)l.ndof * K * sizeof(double), s));
      } else {
        ok(launch_bjacobi<double>(JAC_FIRST, l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, nullptr,
                                  B[k], x, K, s, l.A.nnzb));
        for (int t = 1; t < tpre; ++t) {
          ok(launch_bjacobi<double>(JAC_SWEEP, l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, x, B[k],
                                    x2, K, s, l.A.nnzb));
          std::swap(x, x2);
        }
      }
      xk[k] = x;
      ok(launch_bmv<double>(GASA_MV_RESIDUAL, l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val, x, B[k],
                            Rv[k], K, s, l.A.nnzb));
      ok(launch_bmv<double>(GASA_MV_ASSIGN, l.R.nrows, l.R.br, l.R.bc, l.R.rp, l.R.col, l.R.val,
                            Rv[k], nullptr, B[k + 1], K, s, l.R.nnzb));
    }
    ok(launch_bdense<double>(ctx->nc, ctx->coarse_inv, B[N], X[N], K, s));
    xk[N] = X[N];
    for (int k = N - 1; k >= kt && e == cudaSuccess; --k) {
      Level &l = ctx->L[k];
      double *x = xk[k];
      double *x2 = (x == X[k]) ? X2[k] : X[k];
      ok(launch_bmv<double>(GASA_MV_ADD, l.P.nrows, l.P.br, l.P.bc, l.P.rp, l.P.col, l.P.val,
                            xk[k + 1], nullptr, x, K, s, l.P.nnzb));
      for (int t = 0; t < tpost; ++t) {
        ok(launch_bjacobi<double>(JAC_SWEEP, l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, x, B[k], x2,
                                  K, s, l.A.nnzb));
        std::swap(x, x2);
      }
      xk[k] = x;
    }
    // row i of the K interleaved columns is M[i][c0 .. c0 + K)
    const int w = std::min(K, n - c0);
    ok(cudaMemcpy2DAsync(M + c0, (size_t)ld * sizeof(double), xk[kt], K * sizeof(double),
                         w * sizeof(double), n, cudaMemcpyDeviceToDevice, s));
  }
  // the FP32 cycle applies M from its exact two-term FP32 split
  float *Mh = nullptr, *Ml = nullptr;
  if (st == GASA_OK) st = dalloc(ctx, &Mh, (size_t)n * ld);
  if (st == GASA_OK) st = dalloc(ctx, &Ml, (size_t)n * ld);
  if (st == GASA_OK && e == cudaSuccess) e = launch_split((int64_t)n * ld, M, Mh, Ml, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(ctx, scr);
  ctx->device_bytes -= (int64_t)(tot * sizeof(double));
  if (st != GASA_OK) return st;
  CU(e);
  ctx->dtail_Mh = Mh;
  ctx->dtail_Ml = Ml;
  ctx->dtail_M = M;
  ctx->dtail_k = kt;
  ctx->dtail_n = n;
  ctx->dtail_ld = ld;
  return GASA_OK;
}

// Fused residual and restriction of Alg. 2 on level k: b_{k+1} = R_k b_k -
// (R_k A_k) x_k, the vector R_k (b_k - A_k x_k) without the fine residual.
// FP32 levels run it as one product (lane teams for s <= 8 square blocks,
// the wide-block kernel beyond), which with Wn also takes level k+1's first
// smoothing step xn = Wn b_{k+1}; *first_done tells whether it did.  Elsewhere
// (FP64, or shapes neither kernel takes) it is two products, R b into tmp
// and then tmp - (R A) x.
template <typename T>
cudaError_t restrict_fused(gasa_ctx *ctx, int k, const T *bk, const T *xk, T *bnext,
                           const T *Wn, T *xn, T *tmp, bool *first_done) {
  using P = Prec<T>;
  cudaStream_t s = ctx->stream;
  Level &l = ctx->L[k];
  const DevBSR &R = l.R, &RA = l.RA;
  *first_done = false;
  if constexpr (std::is_same<T, float>::value) {
    const int64_t nz = R.nnzb + RA.nnzb;
    if (R.br == R.bc && blk_applies(R.br, R.nrows, nz)) {
      const cudaError_t e = launch_blk_restrict(R.nrows, R.br, nz, R.rp, R.col, R.val32, RA.rp,
                                                RA.col, RA.val32, bk, xk, bnext, Wn, xn, s);
      if (e != cudaErrorNotSupported) {
        *first_done = Wn != nullptr && e == cudaSuccess;
        return e;
      }
    }
    if (blk_restrict_rect_applies(R.br, R.bc, R.nrows, nz)) {
      const cudaError_t e = launch_blk_restrict_rect(R.nrows, R.br, R.bc, nz, R.rp, R.col,
                                                     R.val32, RA.rp, RA.col, RA.val32, bk, xk,
                                                     bnext, Wn, xn, s);
      if (e != cudaErrorNotSupported) {
        *first_done = Wn != nullptr && e == cudaSuccess;
        return e;
      }
    }
    if (wide_applies(R.br, R.bc, R.nrows, nz)) {
      const cudaError_t e = launch_wide_restrict(R.nrows, R.br, R.bc, nz, R.rp, R.col, R.val32,
                                                 RA.rp, RA.col, RA.val32, bk, xk, bnext, Wn, xn, s);
      if (e != cudaErrorNotSupported) {
        *first_done = Wn != nullptr && e == cudaSuccess;
        return e;
      }
    }
  }
  cudaError_t e = launch_bsr_mv<T>(GASA_MV_ASSIGN, R.nrows, R.br, R.bc, R.rp, R.col, P::A(R), bk,
                                   nullptr, tmp, s, R.nnzb);
  if (e != cudaSuccess) return e;
  return launch_bsr_mv<T>(GASA_MV_RESIDUAL, RA.nrows, RA.br, RA.bc, RA.rp, RA.col, P::A(RA), xk,
                          tmp, bnext, s, RA.nnzb);
}

// bytes of the fused restriction of level l (R, R A, b, x, b_{k+1}; with the
// next level's first step also its W and x)
double restrict_fused_bytes(const Level &l, int w, bool first) {
  auto mat = [&](const DevBSR &m) {
    return (double)m.nnzb * m.br * m.bc * w + 4.0 * m.nnzb + 4.0 * (m.nrows + 1);
  };
  const double vfine = (double)l.ndof * w, vc = (double)l.R.nrows * l.R.br * w;
  double b = mat(l.R) + mat(l.RA) + 2.0 * vfine + vc;
  if (first) b += (double)l.R.nrows * l.R.br * l.R.br * w + vc;
  return b;
}

// The FP32 V-cycle's first level-0 step reads the FP64 right-hand side r
// itself and leaves its FP32 rounding in b32 (the conversion then needs no
// launch of its own; same bits).  Folding the conversion of z and the dot
// products r . z, r . zold into the last step as well was measured slower
// (0.777 vs 0.767 ms per CG iteration on the P3 256x256 workload): the two
// block reductions and FP64 reads slow the HBM-bound sweep by more than the
// launches they save.
struct FusedEnds {
  const double *r;
  float *b32;
};

template <typename T>
gasa_status vcycle_impl(gasa_ctx *ctx, const T *rhs, T *out, bool h16 = false,
                        const FusedEnds *fe = nullptr) {
  using P = Prec<T>;
  cudaStream_t s = ctx->stream;
  const int N = ctx->N;
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  const bool grid = ctx->grid_plan[pi] != nullptr;
  const bool cluster = !grid && ctx->tail_plan[pi] != nullptr;
  const bool dense = !grid && !cluster && ctx->dtail_M != nullptr;
  // first level of the fused bottom (persistent grid launch, cluster launch
  // or dense operator)
  const int kt = grid ? ctx->grid_k0[pi]
                      : (cluster ? ctx->tail_k0[pi] : (dense ? ctx->dtail_k : N));
  const int tpre = ctx->opt.t_pre, tpost = ctx->opt.t_post;
  const int w = (int)sizeof(T);
  // level 0 smooths in the folded form u + c - (W A) u (not with FP16 blocks
  // or the bulk-copy staged step)
  const bool fold0 = std::is_same<T, float>::value && P::WA(ctx->L[0]) && !h16 && !ctx->L[0].tma;
  // level-0 smoothing step and residual; with h16 (FP32 V-cycle only) the
  // level-0 operator and block inverses are read from their FP16 blocks
  auto sweep = [&](int k, int mode, const T *xin, const T *bb, T *xo) -> cudaError_t {
    Level &l = ctx->L[k];
    if (k == 0 && fold0) {
      if (mode == JAC_SWEEP)
        return launch_folded_sweep<T>(l.n, l.s, l.A.rp, l.A.col, P::WA(l), xin, P::c(l), xo, s);
      // first step u = W b, kept as c for the later steps
      cudaError_t e = launch_jacobi<T>(JAC_FIRST, l.n, l.s, l.A.rp, l.A.col, P::A(l.A), P::W(l),
                                       nullptr, bb, xo, s, l.A.nnzb);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(P::c(l), xo, l.ndof * sizeof(T), cudaMemcpyDeviceToDevice, s);
      return e;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (h16 && k == 0)
        return launch_jacobi_h16(mode, l.n, l.s, l.A.rp, l.A.col, l.A.val16, l.A.scale16, l.W16,
                                 l.W16s, xin, bb, xo, s);
      if (l.tma && mode == JAC_SWEEP)
        return launch_jacobi_tma<float>(l.n, l.s, l.tma_TR, l.tma_stageA, l.tma_stageW,
                                        l.tma_smem, l.tma_grid, l.A.rp, l.A.col, l.A.val32,
                                        l.W32, xin, bb, xo, ctx->d_err, s);
    }
    if (l.mf && mode == JAC_SWEEP) {
      // x_out = x + W (b - A_k x) with A_k applied through the transfers
      cudaError_t e = mf_apply<T>(ctx, k, GASA_MV_RESIDUAL, xin, bb, P::r(l));
      if (e == cudaSuccess)
        e = launch_jacobi<T>(JAC_FIRST, l.n, l.s, nullptr, nullptr, nullptr, P::W(l), nullptr,
                             P::r(l), xo, s);
      if (e == cudaSuccess) e = launch_add<T>(l.ndof, xin, xo, s);
      return e;
    }
    return launch_jacobi<T>(mode, l.n, l.s, l.A.rp, l.A.col, P::A(l.A), P::W(l), xin, bb, xo, s,
                            l.A.nnzb);
  };
  auto resid = [&](int k, const T *xin, const T *bb, T *rr) -> cudaError_t {
    Level &l = ctx->L[k];
    if constexpr (std::is_same<T, float>::value) {
      if (h16 && k == 0)
        return launch_bsr_mv_h16(GASA_MV_RESIDUAL, l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val16,
                                 l.A.scale16, xin, bb, rr, s);
    }
    if (l.mf) return mf_apply<T>(ctx, k, GASA_MV_RESIDUAL, xin, bb, rr);
    return launch_bsr_mv<T>(GASA_MV_RESIDUAL, l.n, l.s, l.s, l.A.rp, l.A.col, P::A(l.A), xin, bb,
                            rr, s, l.A.nnzb);
  };
  const int wa = (h16 ? 2 : w);     // level-0 matrix bytes per value
  std::vector<const T *> bk(N + 1);
  std::vector<T *> xk(N + 1);
  bk[0] = rhs;
  for (int k = 1; k <= N; ++k) bk[k] = P::b(ctx->L[k]);
  // levels whose first smoothing step the restriction of the level above took
  std::vector<char> first_done(N + 1, 0);
  for (int k = 0; k < kt; ++k) {
    Level &l = ctx->L[k];
    T *x = P::x(l), *x2 = P::x2(l);
    // pre-smoothing from zero
    if (tpre == 0) {
      CU(cudaMemsetAsync(x, 0, l.ndof * sizeof(T), s));
      // the folded post-smoothing steps read c = W b
      if (k == 0 && fold0)
        CU(launch_jacobi<T>(JAC_FIRST, l.n, l.s, l.A.rp, l.A.col, P::A(l.A), P::W(l), nullptr,
                            bk[0], P::c(l), s, l.A.nnzb));
    } else {
      cudaEvent_t e0;
      if (k == 0) prof_begin(ctx, 3, &e0);
      if constexpr (std::is_same<T, float>::value) {
        if (k == 0 && fe)
          CU(launch_jacobi_first_conv(l.n, l.s, fe->r, fe->b32, P::W(l), x, s,
                                      fold0 ? P::c(l) : nullptr));
        else if (!first_done[k]) CU(sweep(k, JAC_FIRST, nullptr, bk[k], x));
      } else {
        if (!first_done[k]) CU(sweep(k, JAC_FIRST, nullptr, bk[k], x));
      }
      if (k == 0) prof_end(ctx, 3, sweep_bytes(l, w, true, wa, fold0));
      for (int t = 1; t < tpre; ++t) {
        if (k == 0) prof_begin(ctx, 0, &e0);
        CU(sweep(k, JAC_SWEEP, x, bk[k], x2));
        if (k == 0) prof_end(ctx, 0, sweep_bytes(l, w, false, wa, k == 0 && fold0));
        std::swap(x, x2);
      }
    }
    xk[k] = x;
    // residual and restriction: fused as R b - (R A) x where R A is stored
    // (the FP16-block level 0 keeps its own residual)
    if (l.RA.rp && P::A(l.RA) && !(h16 && k == 0)) {
      Level &ln = ctx->L[k + 1];
      const bool take_first = tpre >= 1 && k + 1 < kt && k + 1 < N;
      bool fd = false;
      cudaEvent_t e0;
      if (k == 0) prof_begin(ctx, 1, &e0);
      CU(restrict_fused<T>(ctx, k, bk[k], x, P::b(ln), take_first ? P::W(ln) : nullptr,
                           take_first ? P::x(ln) : nullptr, P::r(ln), &fd));
      if (k == 0) prof_end(ctx, 1, restrict_fused_bytes(l, w, fd));
      first_done[k + 1] = fd ? 1 : 0;
    } else {
      {
        cudaEvent_t e0;
        if (k == 0) prof_begin(ctx, 1, &e0);
        CU(resid(k, x, bk[k], P::r(l)));
        if (k == 0) prof_end(ctx, 1, spmv_bytes(l, w, true, wa));
      }
      CU(launch_bsr_mv<T>(GASA_MV_ASSIGN, l.R.nrows, l.R.br, l.R.bc, l.R.rp, l.R.col, P::A(l.R),
                          P::r(l), nullptr, P::b(ctx->L[k + 1]), s, l.R.nnzb));
    }
  }
  Level &lc = ctx->L[N];
  if (kt < N && grid) {
    // levels kt .. N-1 and the coarsest solve (FP64 arithmetic) in one
    // persistent launch; it leaves the corrected x_kt in L[kt]'s x
    CU(launch_grid_tail<T>(static_cast<const GridPlan<T> *>(ctx->grid_plan[pi]), ctx->grid_s[pi],
                           ctx->grid_ctas[pi], ctx->grid_bar, s));
    xk[kt] = P::x(ctx->L[kt]);
  } else if (kt < N && cluster) {
    // levels kt .. N-1 and the coarsest solve (FP64 arithmetic) in one
    // cluster launch; it leaves the corrected x_kt in L[kt]'s x
    const TailPlan<T> *pl = static_cast<const TailPlan<T> *>(ctx->tail_plan[pi]);
    CU(launch_vcycle_tail<T>(pl, ctx->tail_cluster[pi], ctx->tail_smem[pi], s));
    xk[kt] = P::x(ctx->L[kt]);
  } else if (kt < N) {
    // levels kt .. N-1 and the coarsest solve as their dense operator: FP64
    // arithmetic in the FP64 cycle, double-single arithmetic on FP32 units
    // (the same to about 2^-47 of sum |m x| per row) in the FP32 cycle
    Level &ld = ctx->L[kt];
    if constexpr (std::is_same<T, float>::value)
      CU(launch_dense_mv_ds(ctx->dtail_n, ctx->dtail_ld, ctx->dtail_Mh, ctx->dtail_Ml, P::b(ld),
                            P::x(ld), s));
    else
      CU(launch_dense_mv<T>(ctx->dtail_n, ctx->dtail_M, P::b(ld), P::x(ld), s, ctx->dtail_ld));
    xk[kt] = P::x(ld);
  } else {
    // coarsest solve in FP64
    CU(launch_dense_mv<T>(ctx->nc, ctx->coarse_inv, P::b(lc), P::x(lc), s));
    xk[N] = P::x(lc);
  }
  for (int k = kt - 1; k >= 0; --k) {
    Level &l = ctx->L[k];
    T *x = xk[k];
    T *x2 = (x == P::x(l)) ? P::x2(l) : P::x(l);
    {
      cudaEvent_t e0;
      if (k == 0) prof_begin(ctx, 4, &e0);
      CU(launch_bsr_mv<T>(GASA_MV_ADD, l.P.nrows, l.P.br, l.P.bc, l.P.rp, l.P.col, P::A(l.P),
                          xk[k + 1], nullptr, x, s, l.P.nnzb));
      if (k == 0)
        prof_end(ctx, 4, (double)l.P.nnzb * l.P.br * l.P.bc * w + 4.0 * l.P.nnzb +
                             4.0 * (l.P.nrows + 1) + 2.0 * l.ndof * w +
                             (double)ctx->L[1].ndof * w);
    }
    if (tpost == 0 && k == 0) {
      CU(cudaMemcpyAsync(out, x, l.ndof * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    for (int t = 0; t < tpost; ++t) {
      T *dst = (k == 0 && t == tpost - 1) ? out : x2;
      cudaEvent_t e0;
      if (k == 0) prof_begin(ctx, 0, &e0);
      CU(sweep(k, JAC_SWEEP, x, bk[k], dst));
      if (k == 0) prof_end(ctx, 0, sweep_bytes(l, w, false, wa, fold0));
      if (dst == x2) std::swap(x, x2);
      else x = dst;
    }
    xk[k] = x;
  }
  return GASA_OK;
}

// FP32 V-cycle of the mixed precisions on the FP64 residual rr; z in FP32
// is left in ctx->kf_out
gasa_status vcycle_f32_out(gasa_ctx *ctx, const double *rr, int precision) {
  Level &l0 = ctx->L[0];
  const int64_t n = l0.ndof;
  if (precision == GASA_PREC_MIXED32 && !l0.mf && l0.s <= 16 && ctx->opt.t_pre >= 1) {
    FusedEnds fe{rr, ctx->kf_in};
    return vcycle_impl<float>(ctx, ctx->kf_in, ctx->kf_out, false, &fe);
  }
  CU(launch_convert<double, float>(n, rr, ctx->kf_in, ctx->stream));
  return vcycle_impl<float>(ctx, ctx->kf_in, ctx->kf_out, precision == GASA_PREC_MIXED16);
}

gasa_status apply_M(gasa_ctx *ctx, const double *rr, double *z, int precision) {
  if (precision == GASA_PREC_FP64) return vcycle_impl<double>(ctx, rr, z);
  ST(vcycle_f32_out(ctx, rr, precision));
  CU(launch_convert<float, double>(ctx->L[0].ndof, ctx->kf_out, z, ctx->stream));
  return GASA_OK;
}

// z = M r for the CG step and the partial sums of r . z (and of r . zold
// when zold is given); *n_part receives the number of partials per product
gasa_status apply_M_cg(gasa_ctx *ctx, const double *rr, double *z, const double *zold,
                       int precision, double *part_rz, double *part_rzo, int *n_part) {
  const int64_t n = ctx->L[0].ndof;
  ST(apply_M(ctx, rr, z, precision));
  CU(launch_dot_partials(n, rr, z, part_rz, ctx->stream));
  if (zold) CU(launch_dot_partials(n, rr, zold, part_rzo, ctx->stream));
  *n_part = kRedBlocks;
  return GASA_OK;
}

// scalar slots in ctx->scal
enum { S_RR = 0, S_ALPHA = 1, S_PQ = 2, S_RZ0 = 3, S_RZ1 = 4, S_BB = 5, S_TMP = 6, S_G = 7,
       S_BETA = 8, S_BN = 9, S_TOL = 10, S_COUNT = 16 };

// GASA_ERR_TIMEOUT (flag cleared) when a bounded device-side wait of the
// last launches ran out, else GASA_OK; synchronises the context stream
gasa_status check_wait_flag(gasa_ctx *ctx) {
  int kerr = 0;
  CU(cudaMemcpyAsync(&kerr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (!kerr) return GASA_OK;
  CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return fail(ctx, GASA_ERR_TIMEOUT, "a bounded device-side wait ran out");
}

gasa_status read_scalars(gasa_ctx *ctx, int first, int count) {
  CU(cudaMemcpyAsync(ctx->hscal + first, ctx->scal + first, count * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return GASA_OK;
}

gasa_status norm2(gasa_ctx *ctx, int64_t n, const double *x, int slot, double *out) {
  CU(launch_dot_partials(n, x, nullptr, ctx->part, ctx->stream));
  CU(launch_finalize(ctx->part, 1, ctx->scal + slot, ctx->stream));
  ST(read_scalars(ctx, slot, 1));
  *out = ctx->hscal[slot];
  return GASA_OK;
}

gasa_status spmv_outer(gasa_ctx *ctx, int mode, const double *x, const double *b, double *y) {
  Level &l = ctx->L[0];
  cudaEvent_t e0;
  prof_begin(ctx, 2, &e0);
  CU(launch_bsr_mv<double>(mode, l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val, x, b, y, ctx->stream));
  prof_end(ctx, 2, spmv_bytes(l, 8, mode == GASA_MV_RESIDUAL));
  return GASA_OK;
}

int pq_ds_count(gasa_ctx *ctx) { return ctx->n_pq_ds; }

// q = A p of the mixed-precision Krylov step: double-single arithmetic on
// the FP32 splits of A (val32 + lo32) and of p (kp_hi + kp_lo, written by the
// CG update or, with split_p, here); the same launch leaves the partial sums
// of p . q in ctx->pq_ds
gasa_status spmv_outer_ds(gasa_ctx *ctx, const double *p, double *q) {
  Level &l = ctx->L[0];
  cudaEvent_t e0;
  prof_begin(ctx, 2, &e0);
  CU(launch_bsr_mv_ds(l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val32, l.A.lo32, ctx->kp_hi,
                      ctx->kp_lo, q, ctx->stream, p, ctx->pq_ds));
  prof_end(ctx, 2, spmv_bytes(l, 8, false));   // 4 + 4 bytes per value and per x entry
  return GASA_OK;
}

gasa_status pcg(gasa_ctx *ctx, const double *b, double tol, int precision, int *iters,
                double *relres, bool *conv) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->L[0].ndof;
  const bool flex = precision != GASA_PREC_FP64;
  double *x = ctx->kx, *r = ctx->kr, *z = ctx->kz, *p = ctx->kp, *q = ctx->kq;
  double *pq_part = ctx->part, *rr_part = ctx->part + kRedBlocks;
  *conv = false;
  *iters = 0;
  double bb;
  ST(norm2(ctx, n, b, S_BB, &bb));
  const double bn = std::sqrt(bb);
  CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bn == 0.0) {
    *relres = 0.0;
    *conv = true;
    return GASA_OK;
  }
  CU(launch_copy(n, b, r, s));
  const int max_iter = ctx->opt.max_iter;
  if (flex) {
    // the kernels of the graph-resident step, in its order, one by one:
    // z = M r (FP32), r . z and r . zold, p = z + beta p with its split,
    // q = A p with p . q, x and r; started from p = 0, zold = 0, rz = 1
    CU(cudaMemsetAsync(p, 0, n * sizeof(double), s));
    CU(cudaMemsetAsync(ctx->kzold_f, 0, n * sizeof(float), s));
    ctx->hscal[S_RZ0] = 1.0;
    CU(cudaMemcpyAsync(ctx->scal + S_RZ0, ctx->hscal + S_RZ0, sizeof(double),
                       cudaMemcpyHostToDevice, s));
    int cur = S_RZ0, nxt = S_RZ1;
    for (int it = 1; it <= max_iter; ++it) {
      ST(vcycle_f32_out(ctx, r, precision));
      CU(launch_cg_dots_f32(n, r, ctx->kf_out, ctx->kzold_f, ctx->rz_ds, ctx->rzo_ds, s));
      CU(launch_cg_update_p_f32(n, p, ctx->kf_out, ctx->scal + cur, ctx->rz_ds, ctx->rzo_ds,
                                ctx->scal + nxt, ctx->kzold_f, ctx->kp_hi, ctx->kp_lo, kRedBlocks,
                                s));
      ST(spmv_outer_ds(ctx, p, q));
      CU(launch_cg_update_xr(n, x, r, p, q, ctx->scal + nxt, ctx->pq_ds, rr_part,
                             ctx->scal + S_ALPHA, s, pq_ds_count(ctx)));
      CU(launch_finalize(rr_part, 1, ctx->scal + S_RR, s));
      ST(read_scalars(ctx, 0, 3));
      const double pq = ctx->hscal[S_PQ];
      if (!std::isfinite(pq)) return fail(ctx, GASA_ERR_BREAKDOWN, "CG: non-finite p^T A p");
      const double rel = std::sqrt(ctx->hscal[S_RR]) / bn;
      *iters = it;
      if (!std::isfinite(rel)) return fail(ctx, GASA_ERR_BREAKDOWN, "CG: non-finite residual");
      if (rel <= tol) {
        ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, ctx->kt));
        double tt;
        ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
        const double relt = std::sqrt(tt) / bn;
        if (relt <= tol) {
          *relres = relt;
          *conv = true;
          return GASA_OK;
        }
        CU(launch_copy(n, ctx->kt, r, s));
      }
      std::swap(cur, nxt);
    }
    ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, ctx->kt));
    double tt;
    ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
    *relres = std::sqrt(tt) / bn;
    return GASA_OK;
  }
  int np = 0;
  ST(apply_M_cg(ctx, r, z, nullptr, precision, ctx->rz_ds, ctx->rzo_ds, &np));
  CU(launch_finalize_n(ctx->rz_ds, np, ctx->scal + S_RZ0, s));
  CU(launch_copy(n, z, p, s));
  int cur = S_RZ0, nxt = S_RZ1;
  for (int it = 1; it <= max_iter; ++it) {
    ST(spmv_outer(ctx, GASA_MV_ASSIGN, p, nullptr, q));
    CU(launch_dot_partials(n, p, q, pq_part, s));
    CU(launch_cg_update_xr(n, x, r, p, q, ctx->scal + cur, pq_part, rr_part,
                           ctx->scal + S_ALPHA, s, kRedBlocks));
    CU(launch_finalize(rr_part, 1, ctx->scal + S_RR, s));
    ST(read_scalars(ctx, 0, 3));
    const double pq = ctx->hscal[S_PQ];
    if (!(pq > 0.0)) {
      *iters = it;
      *relres = std::sqrt(ctx->hscal[S_RR]) / bn;
      return fail(ctx, GASA_ERR_NOT_SPD, "CG: p^T A p <= 0");
    }
    if (!std::isfinite(pq)) return fail(ctx, GASA_ERR_BREAKDOWN, "CG: non-finite p^T A p");
    const double rel = std::sqrt(ctx->hscal[S_RR]) / bn;
    *iters = it;
    if (rel <= tol) {
      ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, ctx->kt));
      double tt;
      ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
      const double relt = std::sqrt(tt) / bn;
      if (relt <= tol) {
        *relres = relt;
        *conv = true;
        return GASA_OK;
      }
      CU(launch_copy(n, ctx->kt, r, s));
    }
    ST(apply_M_cg(ctx, r, z, nullptr, precision, ctx->rz_ds, ctx->rzo_ds, &np));
    CU(launch_cg_update_p(n, p, z, ctx->scal + cur, ctx->rz_ds, ctx->rzo_ds, ctx->scal + nxt, 0, s,
                          nullptr, nullptr, nullptr, np));
    std::swap(cur, nxt);
  }
  ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, ctx->kt));
  double tt;
  ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
  *relres = std::sqrt(tt) / bn;
  return GASA_OK;
}

// Build the CG graph of one precision: a conditional while node whose body
// is one CG step in the order z = M r; p = z + beta p; q = A p; x, r update;
// check.  Started with p = 0 and rz = 1, the first step gives p = z, so the
// sequence of iterates is the same as the host-driven loop above.
gasa_status build_cg_graph(gasa_ctx *ctx, int precision) {
  const int pi = precision;   // graph slot: FP64, MIXED32, MIXED16
  const int max_iter = ctx->opt.max_iter;
  if (ctx->cg_exec[pi] && ctx->cg_max_iter[pi] == max_iter) return GASA_OK;
  if (ctx->cg_exec[pi]) cudaGraphExecDestroy(ctx->cg_exec[pi]);
  if (ctx->cg_graph[pi]) cudaGraphDestroy(ctx->cg_graph[pi]);
  ctx->cg_exec[pi] = nullptr;
  ctx->cg_graph[pi] = nullptr;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->L[0].ndof;
  const bool flex = precision != GASA_PREC_FP64;
  cudaGraph_t g = nullptr;
  CU(cudaGraphCreate(&g, 0));
  ctx->cg_graph[pi] = g;
  cudaGraphConditionalHandle h;
  CU(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  double *x = ctx->kx, *r = ctx->kr, *z = ctx->kz, *p = ctx->kp, *q = ctx->kq;
  double *pq_part = ctx->part, *rr_part = ctx->part + kRedBlocks;
  const bool prof = ctx->prof;
  ctx->prof = false;   // no event records inside a graph body
  const long long k0 = launch_count();
  CU(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int np = kRedBlocks;
  gasa_status st = GASA_OK;
  cudaError_t e = cudaSuccess;
  if (flex) {
    // z stays in FP32: one pass for r . z and r . zold, and the p update
    // reads it there and keeps it as the next step's zold
    st = vcycle_f32_out(ctx, r, precision);
    if (st == GASA_OK)
      e = launch_cg_dots_f32(n, r, ctx->kf_out, ctx->kzold_f, ctx->rz_ds, ctx->rzo_ds, s);
  } else {
    st = apply_M_cg(ctx, r, z, nullptr, precision, ctx->rz_ds, ctx->rzo_ds, &np);
  }
  if (st == GASA_OK && e == cudaSuccess) {
    if (flex)
      e = launch_cg_update_p_f32(n, p, ctx->kf_out, ctx->scal + S_RZ0, ctx->rz_ds, ctx->rzo_ds,
                                 ctx->scal + S_RZ1, ctx->kzold_f, ctx->kp_hi, ctx->kp_lo, np, s);
    else
      e = launch_cg_update_p(n, p, z, ctx->scal + S_RZ0, ctx->rz_ds, ctx->rzo_ds,
                             ctx->scal + S_RZ1, 0, s, nullptr, nullptr, nullptr, np);
    Level &l = ctx->L[0];
    if (e == cudaSuccess && flex) {
      // q = A p with the p . q partials in the same launch
      e = launch_bsr_mv_ds(l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val32, l.A.lo32, ctx->kp_hi,
                           ctx->kp_lo, q, s, p, ctx->pq_ds);
    } else if (e == cudaSuccess) {
      e = launch_bsr_mv<double>(GASA_MV_ASSIGN, l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val, p, nullptr,
                                q, s);
      if (e == cudaSuccess) e = launch_dot_partials(n, p, q, pq_part, s);
    }
    if (e == cudaSuccess)
      e = launch_cg_update_xr(n, x, r, p, q, ctx->scal + S_RZ1, flex ? ctx->pq_ds : pq_part,
                              rr_part, ctx->scal + S_ALPHA, s, flex ? pq_ds_count(ctx) : kRedBlocks);
    if (e == cudaSuccess) e = launch_cg_check(rr_part, ctx->scal, ctx->d_iters, max_iter, h, s);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &captured);
  ctx->prof = prof;
  ctx->cg_kernels[pi] = launch_count() - k0;
  if (st != GASA_OK) return st;
  CU(e);
  CU(e2);
  CU(cudaGraphInstantiate(&ctx->cg_exec[pi], g, 0));
  ctx->cg_max_iter[pi] = max_iter;
  return GASA_OK;
}

gasa_status pcg_graph(gasa_ctx *ctx, const double *b, double tol, int precision, int *iters,
                      double *relres, bool *conv) {
  cudaStream_t s = ctx->stream;
  const int pi = precision;   // graph slot: FP64, MIXED32, MIXED16
  const int64_t n = ctx->L[0].ndof;
  *conv = false;
  *iters = 0;
  ST(build_cg_graph(ctx, precision));
  double bb;
  ST(norm2(ctx, n, b, S_BB, &bb));
  const double bn = std::sqrt(bb);
  CU(cudaMemsetAsync(ctx->kx, 0, n * sizeof(double), s));
  if (bn == 0.0) {
    *relres = 0.0;
    *conv = true;
    return GASA_OK;
  }
  CU(launch_copy(n, b, ctx->kr, s));
  CU(cudaMemsetAsync(ctx->kp, 0, n * sizeof(double), s));
  CU(cudaMemsetAsync(ctx->kzold, 0, n * sizeof(double), s));
  CU(cudaMemsetAsync(ctx->kzold_f, 0, n * sizeof(float), s));
  CU(cudaMemsetAsync(ctx->d_iters, 0, sizeof(int), s));
  ctx->hscal[S_RZ0] = 1.0;
  ctx->hscal[S_BN] = bn;
  ctx->hscal[S_TOL] = tol;
  CU(cudaMemcpyAsync(ctx->scal + S_RZ0, ctx->hscal + S_RZ0, sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ctx->scal + S_BN, ctx->hscal + S_BN, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  int done_iters = 0;
  const int max_iter = ctx->opt.max_iter;
  for (;;) {
    CU(cudaGraphLaunch(ctx->cg_exec[pi], s));
    int it = 0, kerr = 0;
    CU(cudaMemcpyAsync(&it, ctx->d_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&kerr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ST(read_scalars(ctx, 0, 3));
    note_launches(ctx->cg_kernels[pi] * (long long)(it - done_iters));
    done_iters = it;
    *iters = it;
    if (kerr) {
      CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
      return fail(ctx, GASA_ERR_TIMEOUT, "a bounded wait on a bulk copy timed out");
    }
    const double pq = ctx->hscal[S_PQ];
    const double rel = std::sqrt(ctx->hscal[S_RR]) / bn;
    if (!std::isfinite(rel) || !std::isfinite(pq))
      return fail(ctx, GASA_ERR_BREAKDOWN, "CG: non-finite residual");
    if (!(pq > 0.0)) {
      *relres = rel;
      return fail(ctx, GASA_ERR_NOT_SPD, "CG: p^T A p <= 0");
    }
    if (rel <= tol) {
      ST(spmv_outer(ctx, GASA_MV_RESIDUAL, ctx->kx, b, ctx->kt));
      double tt;
      ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
      const double relt = std::sqrt(tt) / bn;
      *relres = relt;
      if (relt <= tol) {
        *conv = true;
        return GASA_OK;
      }
      CU(launch_copy(n, ctx->kt, ctx->kr, s));   // continue from the true residual
    }
    if (it >= max_iter) break;
  }
  ST(spmv_outer(ctx, GASA_MV_RESIDUAL, ctx->kx, b, ctx->kt));
  double tt;
  ST(norm2(ctx, n, ctx->kt, S_TMP, &tt));
  *relres = std::sqrt(tt) / bn;
  return GASA_OK;
}

gasa_status ensure_gmres(gasa_ctx *ctx, int m, bool flex) {
  if (ctx->V && ctx->gm_restart == m && (ctx->gm_flex || !flex)) return GASA_OK;
  const int64_t n = ctx->L[0].ndof;
  if (ctx->V) { dfree(ctx, ctx->V); ctx->V = nullptr; }
  if (ctx->Z) { dfree(ctx, ctx->Z); ctx->Z = nullptr; }
  if (ctx->H) { dfree(ctx, ctx->H); ctx->H = nullptr; }
  if (ctx->gm) { dfree(ctx, ctx->gm); ctx->gm = nullptr; }
  if (ctx->mpart) { dfree(ctx, ctx->mpart); ctx->mpart = nullptr; }
  ST(dalloc(ctx, &ctx->V, (size_t)(m + 1) * n));
  if (flex) ST(dalloc(ctx, &ctx->Z, (size_t)m * n));
  ST(dalloc(ctx, &ctx->H, (size_t)(m + 1) * m));
  ST(dalloc(ctx, &ctx->gm, (size_t)6 * (m + 2)));   // cs, sn, g, y, h, h2
  ST(dalloc(ctx, &ctx->mpart, (size_t)(m + 1) * kRedBlocks));
  ctx->gm_restart = m;
  ctx->gm_flex = flex;
  return GASA_OK;
}

gasa_status gmres(gasa_ctx *ctx, const double *b, double tol, int precision, int *iters,
                  double *relres, bool *conv) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->L[0].ndof;
  const bool flex = precision != GASA_PREC_FP64;
  const int m = ctx->opt.restart > 0 ? ctx->opt.restart : 30;
  ST(ensure_gmres(ctx, m, flex));
  double *x = ctx->kx, *w = ctx->kz, *t = ctx->kt;
  const int ldh = m + 1;
  double *cs = ctx->gm, *sn = cs + (m + 2), *g = sn + (m + 2), *y = g + (m + 2), *h = y + (m + 2),
         *h2 = h + (m + 2);
  *conv = false;
  *iters = 0;
  double bb;
  ST(norm2(ctx, n, b, S_BB, &bb));
  const double bn = std::sqrt(bb);
  CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bn == 0.0) {
    *relres = 0.0;
    *conv = true;
    return GASA_OK;
  }
  int total = 0;
  double inner_tol = -1.0;
  const int max_iter = ctx->opt.max_iter;
  while (total < max_iter) {
    ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, t));
    double rr;
    ST(norm2(ctx, n, t, S_TMP, &rr));
    const double rel = std::sqrt(rr) / bn;
    *relres = rel;
    if (rel <= tol) {
      *conv = true;
      *iters = total;
      return GASA_OK;
    }
    if (flex) CU(launch_copy(n, t, w, s));
    else ST(apply_M(ctx, t, w, precision));
    double beta2;
    ST(norm2(ctx, n, w, S_TMP, &beta2));
    const double beta = std::sqrt(beta2);
    if (inner_tol < 0.0) inner_tol = tol * (flex ? bn : beta);
    CU(launch_normalize_into(n, w, ctx->scal + S_TMP, ctx->V, ctx->scal + S_BETA, s));
    CU(cudaMemsetAsync(ctx->H, 0, sizeof(double) * (m + 1) * m, s));
    CU(cudaMemsetAsync(g, 0, sizeof(double) * (m + 2), s));
    CU(cudaMemcpyAsync(g, ctx->scal + S_BETA, sizeof(double), cudaMemcpyDeviceToDevice, s));
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = ctx->V + (size_t)j * n;
      if (flex) {
        double *zj = ctx->Z + (size_t)j * n;
        ST(apply_M(ctx, vj, zj, precision));
        ST(spmv_outer(ctx, GASA_MV_ASSIGN, zj, nullptr, w));
      } else {
        ST(spmv_outer(ctx, GASA_MV_ASSIGN, vj, nullptr, t));
        ST(apply_M(ctx, t, w, precision));
      }
      ++total;
      double *Hj = ctx->H + (size_t)j * ldh;
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; ++pass) {
        CU(launch_multi_dot(n, ctx->V, n, j + 1, w, ctx->mpart, s));
        CU(launch_multi_dot_finalize(ctx->mpart, j + 1, pass == 0 ? h : h2, Hj, s));
        CU(launch_gs_update(n, ctx->V, n, j + 1, pass == 0 ? h : h2, w, s));
      }
      CU(launch_dot_partials(n, w, nullptr, ctx->part, s));
      CU(launch_finalize(ctx->part, 1, ctx->scal + S_TMP, s));
      CU(launch_normalize_into(n, w, ctx->scal + S_TMP, ctx->V + (size_t)(j + 1) * n, Hj + j + 1, s));
      CU(launch_gmres_givens(ctx->H, ldh, j, cs, sn, g, s));
      CU(cudaMemcpyAsync(ctx->scal + S_G, g + j + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
      ST(read_scalars(ctx, S_G, 1));
      jdone = j + 1;
      const double gres = std::fabs(ctx->hscal[S_G]);
      if (!std::isfinite(gres)) return fail(ctx, GASA_ERR_BREAKDOWN, "GMRES: non-finite residual");
      if (gres <= inner_tol || total >= max_iter) break;
    }
    CU(launch_gmres_backsolve(ctx->H, ldh, jdone, g, y, s));
    CU(launch_combine(n, flex ? ctx->Z : ctx->V, n, jdone, y, x, s));
  }
  ST(spmv_outer(ctx, GASA_MV_RESIDUAL, x, b, t));
  double rr;
  ST(norm2(ctx, n, t, S_TMP, &rr));
  *relres = std::sqrt(rr) / bn;
  *iters = total;
  *conv = *relres <= tol;
  return GASA_OK;
}

// ----------------------------------------------------------------------------
// Alg. 2 as a stand-alone solver: x <- x + V(b - A x) until
// ||b - A x|| <= tol ||b||.  t = b - A x of the stopping test is the next
// step's residual.  The loop runs in a conditional while node (or from the
// host when profiling); b is read from ctx->kb.
// ----------------------------------------------------------------------------
gasa_status stationary_step(gasa_ctx *ctx, int precision, int max_iter,
                            cudaGraphConditionalHandle h, bool in_graph) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->L[0].ndof;
  double *rr_part = ctx->part + kRedBlocks;
  ST(apply_M(ctx, ctx->kt, ctx->kz, precision));
  CU(launch_axpy(n, 1.0, ctx->kz, ctx->kx, s));
  ST(spmv_outer(ctx, GASA_MV_RESIDUAL, ctx->kx, ctx->kb, ctx->kt));
  CU(launch_dot_partials(n, ctx->kt, nullptr, rr_part, s));
  if (in_graph) CU(launch_cg_check(rr_part, ctx->scal, ctx->d_iters, max_iter, h, s));
  else CU(launch_finalize(rr_part, 1, ctx->scal + S_RR, s));
  return GASA_OK;
}

gasa_status build_st_graph(gasa_ctx *ctx, int precision) {
  const int pi = 3 + precision;
  const int max_iter = ctx->opt.max_iter;
  if (ctx->cg_exec[pi] && ctx->cg_max_iter[pi] == max_iter) return GASA_OK;
  if (ctx->cg_exec[pi]) cudaGraphExecDestroy(ctx->cg_exec[pi]);
  if (ctx->cg_graph[pi]) cudaGraphDestroy(ctx->cg_graph[pi]);
  ctx->cg_exec[pi] = nullptr;
  ctx->cg_graph[pi] = nullptr;
  cudaStream_t s = ctx->stream;
  cudaGraph_t g = nullptr;
  CU(cudaGraphCreate(&g, 0));
  ctx->cg_graph[pi] = g;
  cudaGraphConditionalHandle h;
  CU(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const bool prof = ctx->prof;
  ctx->prof = false;
  const long long k0 = launch_count();
  CU(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  gasa_status st = stationary_step(ctx, precision, max_iter, h, true);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &captured);
  ctx->prof = prof;
  ctx->cg_kernels[pi] = launch_count() - k0;
  if (st != GASA_OK) return st;
  CU(e2);
  CU(cudaGraphInstantiate(&ctx->cg_exec[pi], g, 0));
  ctx->cg_max_iter[pi] = max_iter;
  return GASA_OK;
}

gasa_status stationary(gasa_ctx *ctx, const double *b, double tol, int precision, int *iters,
                       double *relres, bool *conv) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->L[0].ndof;
  const int max_iter = ctx->opt.max_iter;
  *conv = false;
  *iters = 0;
  if (b != ctx->kb)
    CU(cudaMemcpyAsync(ctx->kb, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double bb;
  ST(norm2(ctx, n, ctx->kb, S_BB, &bb));
  const double bn = std::sqrt(bb);
  CU(cudaMemsetAsync(ctx->kx, 0, n * sizeof(double), s));
  if (bn == 0.0) {
    *relres = 0.0;
    *conv = true;
    return GASA_OK;
  }
  CU(launch_copy(n, ctx->kb, ctx->kt, s));      // t = b - A 0
  ctx->hscal[S_PQ] = 1.0;                        // the shared test also checks p^T A p > 0
  ctx->hscal[S_BN] = bn;
  ctx->hscal[S_TOL] = tol;
  CU(cudaMemcpyAsync(ctx->scal + S_PQ, ctx->hscal + S_PQ, sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ctx->scal + S_BN, ctx->hscal + S_BN, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  if (ctx->prof) {
    for (int it = 1; it <= max_iter; ++it) {
      ST(stationary_step(ctx, precision, max_iter, 0, false));
      ST(read_scalars(ctx, S_RR, 1));
      const double rel = std::sqrt(ctx->hscal[S_RR]) / bn;
      *iters = it;
      *relres = rel;
      if (!std::isfinite(rel)) return fail(ctx, GASA_ERR_BREAKDOWN, "stationary: non-finite residual");
      if (rel <= tol) {
        *conv = true;
        return GASA_OK;
      }
    }
    return GASA_OK;
  }
  ST(build_st_graph(ctx, precision));
  const int pi = 3 + precision;
  CU(cudaMemsetAsync(ctx->d_iters, 0, sizeof(int), s));
  CU(cudaGraphLaunch(ctx->cg_exec[pi], s));
  int it = 0;
  CU(cudaMemcpyAsync(&it, ctx->d_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  ST(read_scalars(ctx, S_RR, 1));
  note_launches(ctx->cg_kernels[pi] * (long long)it);
  *iters = it;
  *relres = std::sqrt(ctx->hscal[S_RR]) / bn;
  if (!std::isfinite(*relres)) return fail(ctx, GASA_ERR_BREAKDOWN, "stationary: non-finite residual");
  *conv = *relres <= tol;
  return GASA_OK;
}

// ----------------------------------------------------------------------------
// setup helpers
// ----------------------------------------------------------------------------
int keep_count(int rows, int r, double n_cut) {
  int s = (int)std::floor((double)rows / n_cut);
  s = std::max(1, s);
  s = std::min(s, r);
  s = std::min(s, rows);
  return s;
}

gasa_status upload_i32(gasa_ctx *ctx, int **d, const int32_t *h, size_t n) {
  ST(dalloc(ctx, d, n));
  CU(cudaMemcpyAsync(*d, h, n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  return GASA_OK;
}

// symbolic + numeric C = A B on BSR patterns (fresh allocations in ctx);
// with max_values > 0, C is left empty (rp == nullptr) when it would hold
// more than max_values scalars
gasa_status spgemm(gasa_ctx *ctx, const DevBSR &A, const DevBSR &B, DevBSR &C,
                   int64_t max_values = 0) {
  cudaStream_t s = ctx->stream;
  const int n = A.nrows;
  int *cand = nullptr, *mx = nullptr, *cnt = nullptr;
  ST(dalloc(ctx, &cand, n + 1));
  ST(dalloc(ctx, &mx, 1));
  ST(dalloc(ctx, &cnt, n + 1));
  CU(launch_cand_count_AB(n, A.rp, A.col, B.rp, cand, s));
  CU(launch_max_int(n, cand, mx, s));
  int maxc = 0;
  CU(cudaMemcpyAsync(&maxc, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (maxc > 4096 && (size_t)((B.ncols + 31) / 32) * 4 > 200 * 1024)
    return fail(ctx, GASA_ERR_UNSUPPORTED, "coarse level too wide for the shared-memory column bitmap");
  C.nrows = n;
  C.ncols = B.ncols;
  C.br = A.br;
  C.bc = B.bc;
  CU(launch_pattern_AB(n, A.rp, A.col, B.rp, B.col, cnt, nullptr, nullptr, maxc, B.ncols, s));
  ST(dalloc(ctx, &C.rp, n + 1));
  CU(launch_exclusive_scan(n, cnt, C.rp, nullptr, s));
  int nnz = 0;
  CU(cudaMemcpyAsync(&nnz, C.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (max_values > 0 && (int64_t)nnz * C.br * C.bc > max_values) {
    dfree(ctx, C.rp);
    dfree(ctx, cand);
    dfree(ctx, mx);
    dfree(ctx, cnt);
    C = DevBSR{};
    return GASA_OK;
  }
  C.nnzb = nnz;
  ST(dalloc(ctx, &C.col, (size_t)nnz));
  ST(dalloc(ctx, &C.val, (size_t)nnz * C.br * C.bc));
  CU(launch_pattern_AB(n, A.rp, A.col, B.rp, B.col, nullptr, C.rp, C.col, maxc, B.ncols, s));
  CU(launch_numeric_AB(n, A.br, A.bc, B.bc, A.rp, A.col, A.val, B.rp, B.col, B.val, C.rp, C.col,
                       C.val, s));
  CU(cudaStreamSynchronize(s));
  dfree(ctx, cand);
  dfree(ctx, mx);
  dfree(ctx, cnt);
  return GASA_OK;
}

gasa_status transpose(gasa_ctx *ctx, const DevBSR &P, DevBSR &R) {
  cudaStream_t s = ctx->stream;
  R.nrows = P.ncols;
  R.ncols = P.nrows;
  R.br = P.bc;
  R.bc = P.br;
  R.nnzb = P.nnzb;
  int *src = nullptr, *cnt = nullptr;
  ST(dalloc(ctx, &R.rp, R.nrows + 1));
  ST(dalloc(ctx, &R.col, (size_t)P.nnzb));
  ST(dalloc(ctx, &R.val, (size_t)P.nnzb * P.br * P.bc));
  ST(dalloc(ctx, &src, (size_t)P.nnzb));
  ST(dalloc(ctx, &cnt, (size_t)R.nrows + 1));
  CU(launch_transpose(P.nrows, P.ncols, P.br, P.bc, P.rp, P.col, P.val, R.rp, R.col, R.val, src,
                      cnt, s));
  CU(cudaStreamSynchronize(s));
  dfree(ctx, src);
  dfree(ctx, cnt);
  return GASA_OK;
}

gasa_status make_f32(gasa_ctx *ctx, DevBSR &m) {
  const int64_t n = m.nnzb * m.br * m.bc;
  ST(dalloc(ctx, &m.val32, (size_t)n));
  CU(launch_convert<double, float>(n, m.val, m.val32, ctx->stream));
  return GASA_OK;
}

gasa_status validate_bsr(gasa_ctx *ctx, int n, int b, int nnzb, const int32_t *rp,
                         const int32_t *col) {
  if (n <= 0 || b <= 0 || b > 64 || nnzb < n)
    return fail(ctx, GASA_ERR_INVALID_ARG, "A: bad sizes (need n_blocks > 0, 0 < block <= 64)");
  if (rp[0] != 0 || rp[n] != nnzb) return fail(ctx, GASA_ERR_INVALID_ARG, "A: row_ptr ends");
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return fail(ctx, GASA_ERR_INVALID_ARG, "A: row_ptr not monotone");
    bool diag = false;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n) return fail(ctx, GASA_ERR_INVALID_ARG, "A: column out of range");
      if (k > rp[i] && col[k] <= col[k - 1])
        return fail(ctx, GASA_ERR_INVALID_ARG, "A: columns not strictly increasing");
      if (col[k] == i) diag = true;
    }
    if (!diag) return fail(ctx, GASA_ERR_INVALID_ARG, "A: missing diagonal block");
  }
  return GASA_OK;
}

gasa_status validate_graph(gasa_ctx *ctx, int n, const int32_t *ap, const int32_t *ai) {
  if (!ap) return GASA_OK;
  if (!ai && ap[n] > 0) return fail(ctx, GASA_ERR_INVALID_ARG, "adjacency: null indices");
  if (ap[0] != 0) return fail(ctx, GASA_ERR_INVALID_ARG, "adjacency: ptr[0] != 0");
  std::vector<std::pair<int, int>> e;
  for (int i = 0; i < n; ++i) {
    if (ap[i + 1] < ap[i]) return fail(ctx, GASA_ERR_INVALID_ARG, "adjacency: ptr not monotone");
    for (int k = ap[i]; k < ap[i + 1]; ++k) {
      const int j = ai[k];
      if (j < 0 || j >= n || j == i) return fail(ctx, GASA_ERR_INVALID_ARG, "adjacency: bad neighbour");
      e.emplace_back(i, j);
    }
  }
  std::vector<std::pair<int, int>> t(e.size());
  for (size_t q = 0; q < e.size(); ++q) t[q] = {e[q].second, e[q].first};
  std::sort(e.begin(), e.end());
  std::sort(t.begin(), t.end());
  if (e != t) return fail(ctx, GASA_ERR_INVALID_ARG, "adjacency: not symmetric");
  return GASA_OK;
}

gasa_status setup_impl(gasa_ctx *ctx, const gasa_bsr *Ain, const int32_t *adj_ptr,
                       const int32_t *adj_idx, const double *centroids,
                       const gasa_hierarchy *hier, const gasa_options *opt,
                       gasa_setup_info *info) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = ctx->stream;
  if (!Ain || !opt) return fail(ctx, GASA_ERR_INVALID_ARG, "null A or options");
  if (!hier) return fail(ctx, GASA_ERR_UNSUPPORTED, "a hierarchy must be given");
  if (hier->n_levels < 2 || hier->n_levels > GASA_MAX_LEVELS || !hier->agg_of)
    return fail(ctx, GASA_ERR_INVALID_ARG, "hierarchy: need 2..GASA_MAX_LEVELS levels");
  if (opt->t_pre < 0 || opt->t_post < 0 || opt->q_power < 0 || opt->max_relax < 0 ||
      opt->gamma < 0.0 || !(opt->omega_factor > 0.0) || opt->dim < 1 || opt->dim > 3 ||
      opt->solver < GASA_SOLVER_CG || opt->solver > GASA_SOLVER_STATIONARY || opt->max_iter < 1 ||
      opt->matrix_free_levels < 0 || opt->delta < 0.0 || (opt->hstar && !(opt->delta < 1.0)) ||
      opt->dense_tail_dofs < 0 || opt->dense_tail_dofs > 8192)
    return fail(ctx, GASA_ERR_INVALID_ARG, "options out of range");
  if (opt->hstar && hier->n_levels + 1 > GASA_MAX_LEVELS)
    return fail(ctx, GASA_ERR_INVALID_ARG, "hierarchy: too many levels with the h* step");
  const int n0 = Ain->n_blocks, b0 = Ain->block, nnzb0 = Ain->nnzb;
  if (n0 <= 0 || b0 <= 0 || nnzb0 <= 0 || !Ain->row_ptr || !Ain->col || !Ain->val)
    return fail(ctx, GASA_ERR_INVALID_ARG, "A: null or empty");
  // host copies of the pattern for validation
  std::vector<int32_t> hrp(n0 + 1), hcol(nnzb0);
  if (Ain->on_device) {
    CU(cudaMemcpy(hrp.data(), Ain->row_ptr, sizeof(int) * (n0 + 1), cudaMemcpyDeviceToHost));
    if (hrp[n0] != nnzb0) return fail(ctx, GASA_ERR_INVALID_ARG, "A: row_ptr[n] != nnzb");
    CU(cudaMemcpy(hcol.data(), Ain->col, sizeof(int) * nnzb0, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(hrp.data(), Ain->row_ptr, sizeof(int) * (n0 + 1));
    if (hrp[n0] != nnzb0) return fail(ctx, GASA_ERR_INVALID_ARG, "A: row_ptr[n] != nnzb");
    std::memcpy(hcol.data(), Ain->col, sizeof(int) * nnzb0);
  }
  ST(validate_bsr(ctx, n0, b0, nnzb0, hrp.data(), hcol.data()));
  ST(validate_graph(ctx, n0, adj_ptr, adj_idx));
  if (centroids) {
    for (int64_t i = 0; i < (int64_t)n0 * opt->dim; ++i)
      if (!std::isfinite(centroids[i])) return fail(ctx, GASA_ERR_INVALID_ARG, "centroids: non-finite");
  }
  // hierarchy validation; with an h*-step the top level is duplicated (every
  // element its own aggregate, Section 4.3) and the given levels follow
  const int hs = opt->hstar ? 1 : 0;
  const int N = hier->n_levels - 1 + hs;
  std::vector<int32_t> ident(hs ? n0 : 0);
  for (int i = 0; i < (int)ident.size(); ++i) ident[i] = i;
  std::vector<const int32_t *> aggs(N);
  for (int k = 0; k < N; ++k) aggs[k] = (hs && k == 0) ? ident.data() : hier->agg_of[k - hs];
  std::vector<int> units(N + 1);
  std::vector<std::vector<int>> children_count(N);
  units[0] = n0;
  for (int k = 1; k <= N; ++k) {
    const int32_t *a = aggs[k - 1];
    if (!a) return fail(ctx, GASA_ERR_INVALID_ARG, "hierarchy: null level");
    int mx = -1;
    for (int i = 0; i < units[k - 1]; ++i) {
      if (a[i] < 0) return fail(ctx, GASA_ERR_INVALID_ARG, "hierarchy: negative aggregate id");
      mx = std::max(mx, (int)a[i]);
    }
    units[k] = mx + 1;
    children_count[k - 1].assign(units[k], 0);
    for (int i = 0; i < units[k - 1]; ++i) children_count[k - 1][a[i]]++;
    for (int J = 0; J < units[k]; ++J)
      if (children_count[k - 1][J] == 0)
        return fail(ctx, GASA_ERR_INVALID_ARG, "hierarchy: empty aggregate");
  }
  // candidate count r (Section 4.2: median level-1 aggregate dofs, lower
  // median; with the h*-step, of the first geometric aggregates)
  int r = opt->n_cand;
  if (r <= 0) {
    std::vector<int> d(children_count[hs]);
    for (auto &v : d) v *= b0;
    std::sort(d.begin(), d.end());
    r = d[(d.size() - 1) / 2];
  }
  if (r > 256) return fail(ctx, GASA_ERR_UNSUPPORTED, "more than 256 candidates");
  const double n_cut = opt->n_cut > 0.0 ? opt->n_cut : (double)((1 << opt->dim) - (opt->dim - 1));
  const double delta = opt->delta > 0.0 ? opt->delta : 1e-3;
  std::vector<int> maxch(N);
  for (int k = 0; k < N; ++k) {
    int mc = 0;
    for (int J = 0; J < units[k + 1]; ++J) mc = std::max(mc, children_count[k][J]);
    maxch[k] = mc;
  }
  int smem_optin = 0;
  CU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  // block sizes whose aggregates keep h-branch counts are known now; a level
  // fed by the h*-step learns its sizes from the singular values in the loop
  {
    std::vector<int> usz(n0, b0);
    for (int k = 0; k < N && !(hs && k == 0); ++k) {
      int smax = 0, sk = 0;
      std::vector<int> nxt(units[k + 1], 0), rows(units[k + 1], 0);
      for (int i = 0; i < units[k]; ++i) rows[aggs[k][i]] += usz[i];
      for (int J = 0; J < units[k + 1]; ++J) {
        nxt[J] = keep_count(rows[J], r, n_cut);
        smax = std::max(smax, nxt[J]);
      }
      for (int i = 0; i < units[k]; ++i) sk = std::max(sk, usz[i]);
      if ((size_t)maxch[k] * sk * r * sizeof(double) > (size_t)smem_optin)
        return fail(ctx, GASA_ERR_UNSUPPORTED, "aggregate x candidates exceed shared memory");
      usz.swap(nxt);
      if (k + 1 == N && (int64_t)units[N] * smax > 16384)
        return fail(ctx, GASA_ERR_UNSUPPORTED, "coarsest level larger than 16384 dofs");
    }
  }

  free_all(ctx);
  ctx->opt = *opt;
  if (ctx->opt.max_iter <= 0) ctx->opt.max_iter = 10000;
  ctx->N = N;
  ctx->r = r;
  ctx->L.assign(N + 1, Level());
  const bool keep = opt->keep_setup_data != 0;
  for (int k = 0; k <= N; ++k) ctx->L[k].n = units[k];
  ctx->L[0].s = b0;
  ctx->L[0].ndof = (int64_t)n0 * b0;
  ctx->L[0].real_dofs = ctx->L[0].ndof;
  // level-0 operator
  {
    Level &l = ctx->L[0];
    DevBSR &A = l.A;
    A.nrows = A.ncols = n0;
    A.br = A.bc = b0;
    A.nnzb = nnzb0;
    ST(upload_i32(ctx, &A.rp, hrp.data(), n0 + 1));
    ST(upload_i32(ctx, &A.col, hcol.data(), nnzb0));
    ST(dalloc(ctx, &A.val, (size_t)nnzb0 * b0 * b0));
    CU(cudaMemcpyAsync(A.val, Ain->val, sizeof(double) * (size_t)nnzb0 * b0 * b0,
                       Ain->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  }
  // candidates B^0
  double *B = nullptr;
  ST(dalloc(ctx, &B, (size_t)ctx->L[0].ndof * r));
  if (opt->init_candidates) {
    CU(cudaMemcpyAsync(B, opt->init_candidates, sizeof(double) * ctx->L[0].ndof * r,
                       cudaMemcpyHostToDevice, s));
  } else {
    CU(launch_normal(ctx->L[0].ndof * r, opt->seed, 3, B, s));
  }
  int *dstat = nullptr;
  ST(dalloc(ctx, &dstat, 4));
  double *pv = nullptr, *pv2 = nullptr;   // power-iteration vectors (level 0 is the largest)
  ST(dalloc(ctx, &pv, (size_t)ctx->L[0].ndof));
  ST(dalloc(ctx, &pv2, (size_t)ctx->L[0].ndof));
  ST(dalloc(ctx, &ctx->part, (size_t)4 * kRedBlocks * std::max(1, r)));
  ST(dalloc(ctx, &ctx->scal, S_COUNT));
  CU(cudaMallocHost((void **)&ctx->hscal, S_COUNT * sizeof(double)));
  double **ptab = nullptr;
  ST(dalloc(ctx, &ptab, (size_t)2 * r));
  double *nrmbuf = nullptr;
  ST(dalloc(ctx, &nrmbuf, (size_t)r));
  double *B2 = nullptr;
  ST(dalloc(ctx, &B2, (size_t)ctx->L[0].ndof * r));

  for (int k = 0; k < N; ++k) {
    Level &l = ctx->L[k];
    Level &ln = ctx->L[k + 1];
    const int64_t nd = l.ndof;
    if (nd > ctx->L[0].ndof)
      return fail(ctx, GASA_ERR_UNSUPPORTED, "a padded level larger than level 0");
    // ---- smoother: block inverses, Alg. 4, Eq. omega ----
    ST(dalloc(ctx, &l.W, (size_t)l.n * l.s * l.s));
    CU(cudaMemsetAsync(dstat, 0, sizeof(int) * 4, s));
    CU(launch_block_inverse(l.n, l.s, l.A.rp, l.A.col, l.A.val, 1.0, l.W, dstat, s));
    int nsing = 0;
    CU(cudaMemcpyAsync(&nsing, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (nsing) return fail(ctx, GASA_ERR_SINGULAR_BLOCK, "singular diagonal block on level " + std::to_string(k));
    if (l.padded)
      CU(launch_uniform_pm1_padded(l.n, l.s, l.d_usize, l.d_uoff, opt->seed, 4 + 16 * (uint64_t)k,
                                   pv, s));
    else
      CU(launch_uniform_pm1(nd, opt->seed, 4 + 16 * (uint64_t)k, pv, s));
    CU(launch_dot_partials(nd, pv, nullptr, ctx->part, s));
    CU(launch_finalize(ctx->part, 1, ctx->scal + S_TMP, s));
    CU(launch_scale_by_inv_sqrt(nd, pv, ctx->scal + S_TMP, s));
    for (int it = 0; it < opt->q_power; ++it) {
      CU(launch_jacobi<double>(JAC_APPLY, l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, pv, nullptr, pv2, s, l.A.nnzb));
      CU(launch_dot_partials(nd, pv2, nullptr, ctx->part, s));
      CU(launch_finalize(ctx->part, 1, ctx->scal + S_TMP, s));
      CU(launch_scale_by_inv_sqrt(nd, pv2, ctx->scal + S_TMP, s));
      std::swap(pv, pv2);
    }
    CU(launch_jacobi<double>(JAC_APPLY, l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, pv, nullptr, pv2, s, l.A.nnzb));
    double rr;
    ST(norm2(ctx, nd, pv2, S_TMP, &rr));
    l.rho = std::sqrt(rr);
    if (!(l.rho > 0.0) || !std::isfinite(l.rho))
      return fail(ctx, GASA_ERR_BREAKDOWN, "power iteration gave a zero or non-finite estimate");
    l.omega = opt->omega_factor / l.rho;
    CU(launch_scale((int64_t)l.n * l.s * l.s, l.omega, l.W, s));
    // ---- Eq. bsmooth: relax every candidate column ----
    if (keep) {
      ST(dalloc(ctx, &l.cand_in, (size_t)nd * r));
      CU(cudaMemcpyAsync(l.cand_in, B, sizeof(double) * nd * r, cudaMemcpyDeviceToDevice, s));
    }
    {
      std::vector<double *> cur(r), nxt(r);
      std::vector<double> nrm(r);
      std::vector<int> active, sweeps(r, 0);
      for (int c = 0; c < r; ++c) {
        cur[c] = B + (size_t)c * nd;
        nxt[c] = B2 + (size_t)c * nd;
        active.push_back(c);
      }
      // initial norms
      {
        std::vector<const double *> tab(r);
        for (int c = 0; c < r; ++c) tab[c] = cur[c];
        CU(cudaMemcpyAsync(ptab, tab.data(), sizeof(double *) * r, cudaMemcpyHostToDevice, s));
        CU(launch_colnorm_partials(nd, (const double *const *)ptab, r, ctx->part, s));
        CU(launch_finalize(ctx->part, r, nrmbuf, s));
        CU(cudaMemcpyAsync(nrm.data(), nrmbuf, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (auto &v : nrm) v = std::sqrt(v);
      }
      std::vector<double *> tab(2 * r);
      std::vector<double> nn(r);
      for (int m = 0; m < opt->max_relax && !active.empty(); ++m) {
        const int na = (int)active.size();
        for (int q = 0; q < na; ++q) {
          tab[q] = cur[active[q]];
          tab[na + q] = nxt[active[q]];
        }
        CU(cudaMemcpyAsync(ptab, tab.data(), sizeof(double *) * 2 * na, cudaMemcpyHostToDevice, s));
        CU(launch_relax_multi(l.n, l.s, l.A.rp, l.A.col, l.A.val, l.W, (const double *const *)ptab,
                              (double *const *)(ptab + na), na, s));
        CU(launch_colnorm_partials(nd, (const double *const *)(ptab + na), na, ctx->part, s));
        CU(launch_finalize(ctx->part, na, nrmbuf, s));
        CU(cudaMemcpyAsync(nn.data(), nrmbuf, sizeof(double) * na, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::vector<int> still;
        for (int q = 0; q < na; ++q) {
          const int c = active[q];
          std::swap(cur[c], nxt[c]);
          sweeps[c] = m + 1;
          const double nnew = std::sqrt(nn[q]);
          if (nrm[c] / nnew < 1.0 + opt->gamma) continue;   // stagnated: keep this sweep, stop
          nrm[c] = nnew;
          still.push_back(c);
        }
        active.swap(still);
      }
      // gather the final columns into B
      for (int c = 0; c < r; ++c)
        if (cur[c] != B + (size_t)c * nd)
          CU(cudaMemcpyAsync(B + (size_t)c * nd, cur[c], sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
      l.sweeps = sweeps;
    }
    if (keep) {
      ST(dalloc(ctx, &l.cand, (size_t)nd * r));
      CU(cudaMemcpyAsync(l.cand, B, sizeof(double) * nd * r, cudaMemcpyDeviceToDevice, s));
    }
    // ---- Eq. splitB_dg + Eq. sik: tentative prolongator ----
    l.max_children = maxch[k];
    if ((size_t)l.max_children * l.s * r * sizeof(double) > (size_t)smem_optin)
      return fail(ctx, GASA_ERR_UNSUPPORTED, "aggregate x candidates exceed shared memory");
    ST(upload_i32(ctx, &l.agg, aggs[k], l.n));
    ST(dalloc(ctx, &l.child_ptr, ln.n + 1));
    ST(dalloc(ctx, &l.child_idx, l.n));
    int *scr = nullptr;
    ST(dalloc(ctx, &scr, ln.n + 1));
    CU(build_children(l.n, ln.n, l.agg, l.child_ptr, l.child_idx, scr, s));
    // kept counts of the next level's units (Eq. sik): h*-branch from the
    // singular values of each element's candidate rows, else the h-branch
    {
      std::vector<int> kp(ln.n, 0);
      if (hs && k == 0) {
        double *sig = nullptr;
        ST(dalloc(ctx, &sig, (size_t)ln.n * r));
        CU(launch_tentative(l.s, ln.n, l.max_children, l.child_ptr, l.child_idx, B, nd, r, 0,
                            nullptr, sig, dstat, s, l.padded ? l.d_usize : nullptr, nullptr));
        std::vector<double> hs_sig((size_t)ln.n * r);
        CU(cudaMemcpyAsync(hs_sig.data(), sig, sizeof(double) * hs_sig.size(), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        dfree(ctx, sig);
        for (int J = 0; J < ln.n; ++J) {
          const double *sj = hs_sig.data() + (size_t)J * r;
          int c = 0;
          for (int q = 0; q < r; ++q) c += sj[q] > delta * sj[0] ? 1 : 0;
          kp[J] = std::max(1, c);
        }
      } else {
        std::vector<int> rows(ln.n, 0);
        for (int i = 0; i < l.n; ++i) rows[aggs[k][i]] += l.padded ? l.usize[i] : l.s;
        for (int J = 0; J < ln.n; ++J) kp[J] = keep_count(rows[J], r, n_cut);
      }
      int smax = 0;
      int64_t real = 0;
      for (int v : kp) {
        smax = std::max(smax, v);
        real += v;
      }
      ln.s = smax;
      ln.ndof = (int64_t)ln.n * smax;
      ln.real_dofs = real;
      ln.padded = real != ln.ndof;
      if (ln.padded) {
        ln.usize = kp;
        std::vector<int64_t> off(ln.n);
        int64_t acc = 0;
        for (int J = 0; J < ln.n; ++J) {
          off[J] = acc;
          acc += kp[J];
        }
        ST(upload_i32(ctx, &ln.d_usize, kp.data(), ln.n));
        ST(dalloc(ctx, &ln.d_uoff, (size_t)ln.n));
        CU(cudaMemcpyAsync(ln.d_uoff, off.data(), sizeof(int64_t) * ln.n, cudaMemcpyHostToDevice, s));
      }
      if (k + 1 == N && ln.ndof > 16384)
        return fail(ctx, GASA_ERR_UNSUPPORTED, "coarsest level larger than 16384 dofs");
    }
    l.n_next = ln.n;
    l.s_next = ln.s;
    ST(dalloc(ctx, &l.T, (size_t)l.n * l.s * l.s_next));
    CU(cudaMemsetAsync(dstat, 0, sizeof(int) * 4, s));
    CU(launch_tentative(l.s, ln.n, l.max_children, l.child_ptr, l.child_idx, B, nd, r, l.s_next, l.T,
                        nullptr, dstat, s, l.padded ? l.d_usize : nullptr,
                        ln.padded ? ln.d_usize : nullptr));
    int tstat = 0;
    CU(cudaMemcpyAsync(&tstat, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    dfree(ctx, scr);
    if (tstat) return fail(ctx, GASA_ERR_BREAKDOWN, "candidate block rank below the kept count on level " + std::to_string(k));
    // ---- Eq. TR0: P = T - w D^{-1} A T (pattern of A times the aggregation) ----
    {
      DevBSR &P = l.P;
      P.nrows = l.n;
      P.ncols = ln.n;
      P.br = l.s;
      P.bc = ln.s;
      int maxrow = 0;
      for (int i = 0; i < l.n && k == 0; ++i) maxrow = std::max(maxrow, hrp[i + 1] - hrp[i]);
      if (k > 0) {
        std::vector<int> rp(l.n + 1);
        CU(cudaMemcpy(rp.data(), l.A.rp, sizeof(int) * (l.n + 1), cudaMemcpyDeviceToHost));
        for (int i = 0; i < l.n; ++i) maxrow = std::max(maxrow, rp[i + 1] - rp[i]);
      }
      int *cnt = nullptr;
      ST(dalloc(ctx, &cnt, l.n + 1));
      CU(launch_pattern_P(l.n, l.A.rp, l.A.col, l.agg, cnt, nullptr, nullptr, maxrow, ln.n, s));
      ST(dalloc(ctx, &P.rp, l.n + 1));
      CU(launch_exclusive_scan(l.n, cnt, P.rp, nullptr, s));
      int nnz = 0;
      CU(cudaMemcpyAsync(&nnz, P.rp + l.n, sizeof(int), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      P.nnzb = nnz;
      ST(dalloc(ctx, &P.col, (size_t)nnz));
      ST(dalloc(ctx, &P.val, (size_t)nnz * P.br * P.bc));
      CU(launch_pattern_P(l.n, l.A.rp, l.A.col, l.agg, nullptr, P.rp, P.col, maxrow, ln.n, s));
      CU(launch_numeric_P(l.n, l.s, ln.s, l.A.rp, l.A.col, l.A.val, l.W, l.T, l.agg, P.rp, P.col,
                          P.val, s));
      CU(cudaStreamSynchronize(s));
      dfree(ctx, cnt);
    }
    // ---- Eq. SA_restrict: R = P^T ----
    ST(transpose(ctx, l.P, l.R));
    // ---- Galerkin: A_{k+1} = R (A P) ----
    {
      DevBSR AP;
      ST(spgemm(ctx, l.A, l.P, AP));
      ST(spgemm(ctx, l.R, AP, ln.A));
      if (ln.padded)
        CU(launch_pad_identity(ln.n, ln.s, ln.d_usize, ln.A.rp, ln.A.col, ln.A.val, s));
      dfree(ctx, AP.rp);
      dfree(ctx, AP.col);
      dfree(ctx, AP.val);
    }
    // ---- next candidates: B^{k+1} = R B^k (Alg. 5) or T^T B^k (Eq. SA_Bk) ----
    {
      const int64_t ndn = ln.ndof;
      double *Bn = nullptr;
      ST(dalloc(ctx, &Bn, (size_t)ndn * r));
      if (opt->cand_init == GASA_CAND_TT) {
        DevBSR Tm, Tt;
        Tm.nrows = l.n;
        Tm.ncols = ln.n;
        Tm.br = l.s;
        Tm.bc = ln.s;
        Tm.nnzb = l.n;
        std::vector<int> seq(l.n + 1);
        for (int i = 0; i <= l.n; ++i) seq[i] = i;
        ST(upload_i32(ctx, &Tm.rp, seq.data(), l.n + 1));
        Tm.col = l.agg;
        Tm.val = l.T;
        ST(transpose(ctx, Tm, Tt));
        CU(launch_bsr_mm(Tt.nrows, Tt.br, Tt.bc, Tt.rp, Tt.col, Tt.val, B, nd, Bn, ndn, r, s));
        CU(cudaStreamSynchronize(s));
        dfree(ctx, Tm.rp);
        dfree(ctx, Tt.rp);
        dfree(ctx, Tt.col);
        dfree(ctx, Tt.val);
      } else {
        CU(launch_bsr_mm(l.R.nrows, l.R.br, l.R.bc, l.R.rp, l.R.col, l.R.val, B, nd, Bn, ndn, r, s));
      }
      CU(cudaStreamSynchronize(s));
      dfree(ctx, B);
      B = Bn;
    }
    if (!keep) {
      dfree(ctx, l.T);
      l.T = nullptr;
    }
    // ---- R_k A_k for the fused restriction b_{k+1} = R b - (R A) u, kept
    // where it holds no more values than A_k (then the fused product also
    // moves fewer bytes than the residual and the restriction) ----
    if (opt->fused_restriction)
      ST(spgemm(ctx, l.R, l.A, l.RA, l.A.nnzb * (int64_t)l.s * l.s));
    // ---- FP32 copies for the mixed-precision V-cycle ----
    ST(make_f32(ctx, l.A));
    ST(make_f32(ctx, l.P));
    ST(make_f32(ctx, l.R));
    if (l.RA.val) ST(make_f32(ctx, l.RA));
    if (k == 0) {
      // low FP32 words of A_0 for the double-single outer product
      ST(dalloc(ctx, &l.A.lo32, (size_t)l.A.nnzb * l.s * l.s));
      CU(launch_split((int64_t)l.A.nnzb * l.s * l.s, l.A.val, l.A.val32, l.A.lo32, s));
      // FP16 blocks with one FP32 scale per block for the MIXED16 V-cycle
      ST(dalloc(ctx, &l.A.val16, (size_t)l.A.nnzb * l.s * l.s));
      ST(dalloc(ctx, &l.A.scale16, (size_t)l.A.nnzb));
      CU(launch_to_h16_blocks(l.A.nnzb, l.s * l.s, l.A.val, l.A.val16, l.A.scale16, s));
      ST(dalloc(ctx, &l.W16, (size_t)l.n * l.s * l.s));
      ST(dalloc(ctx, &l.W16s, (size_t)l.n));
      CU(launch_to_h16_blocks(l.n, l.s * l.s, l.W, l.W16, l.W16s, s));
    }
    ST(dalloc(ctx, &l.W32, (size_t)l.n * l.s * l.s));
    CU(launch_convert<double, float>((int64_t)l.n * l.s * l.s, l.W, l.W32, s));
    // ---- folded smoother on level 0: W A in A's block pattern ----
    if (k == 0 && opt->folded_smoother && l.s <= 16) {
      const size_t nv = (size_t)l.A.nnzb * l.s * l.s;
      ST(dalloc(ctx, &l.WA, nv));
      CU(launch_fold_block_rows(l.n, l.s, l.A.rp, l.W, l.A.val, l.WA, s));
      ST(dalloc(ctx, &l.WA32, nv));
      CU(launch_convert<double, float>((int64_t)nv, l.WA, l.WA32, s));
      if (!keep) {
        // the FP64 cycle keeps the plain step: the FP64 copy is inspection data
        CU(cudaStreamSynchronize(s));
        dfree(ctx, l.WA);
        ctx->device_bytes -= (int64_t)(nv * sizeof(double));
        l.WA = nullptr;
      }
    }
  }
  dfree(ctx, B);
  dfree(ctx, B2);
  dfree(ctx, pv);
  dfree(ctx, pv2);
  dfree(ctx, ptab);
  dfree(ctx, nrmbuf);
  // ---- coarsest level: dense inverse ----
  {
    Level &lc = ctx->L[N];
    ctx->nc = (int)lc.ndof;
    const size_t nc = (size_t)ctx->nc;
    double *D = nullptr, *work = nullptr;
    ST(dalloc(ctx, &D, nc * nc));
    ST(dalloc(ctx, &work, 2 * nc * nc + nc));
    ST(dalloc(ctx, &ctx->coarse_inv, nc * nc));
    CU(launch_bsr_to_dense(lc.n, lc.s, lc.A.rp, lc.A.col, lc.A.val, D, s));
    CU(cudaMemsetAsync(dstat, 0, sizeof(int) * 4, s));
    CU(launch_dense_inverse(ctx->nc, D, ctx->coarse_inv, work, dstat, s));
    int sing = 0;
    CU(cudaMemcpyAsync(&sing, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    dfree(ctx, D);
    dfree(ctx, work);
    if (sing) return fail(ctx, GASA_ERR_SINGULAR_BLOCK, "coarsest matrix is singular");
    ST(make_f32(ctx, lc.A));
  }
  // ---- V-cycle vectors and Krylov workspace ----
  for (int k = 0; k <= N; ++k) {
    Level &l = ctx->L[k];
    ST(dalloc(ctx, &l.x, (size_t)l.ndof));
    ST(dalloc(ctx, &l.x2, (size_t)l.ndof));
    ST(dalloc(ctx, &l.b, (size_t)l.ndof));
    ST(dalloc(ctx, &l.r, (size_t)l.ndof));
    ST(dalloc(ctx, &l.xf, (size_t)l.ndof));
    ST(dalloc(ctx, &l.x2f, (size_t)l.ndof));
    ST(dalloc(ctx, &l.bf, (size_t)l.ndof));
    ST(dalloc(ctx, &l.rf, (size_t)l.ndof));
    if (l.WA32) ST(dalloc(ctx, &l.cf, (size_t)l.ndof));
  }
  const int64_t n = ctx->L[0].ndof;
  for (double **p : {&ctx->kx, &ctx->kr, &ctx->kz, &ctx->kp, &ctx->kq, &ctx->kzold, &ctx->kb, &ctx->kt})
    ST(dalloc(ctx, p, (size_t)n));
  ST(dalloc(ctx, &ctx->kf_in, (size_t)n));
  ST(dalloc(ctx, &ctx->kf_out, (size_t)n));
  ST(dalloc(ctx, &ctx->kzold_f, (size_t)n));
  ST(dalloc(ctx, &ctx->kp_hi, (size_t)n));
  ST(dalloc(ctx, &ctx->kp_lo, (size_t)n));
  ctx->n_pq_ds = bsr_mv_ds_grid(ctx->L[0].n, ctx->L[0].s);
  ST(dalloc(ctx, &ctx->pq_ds, (size_t)ctx->n_pq_ds));
  ctx->n_rz_cap = std::max(kRedBlocks, jacobi_grid(ctx->L[0].n, std::min(ctx->L[0].s, 256)));
  ST(dalloc(ctx, &ctx->rz_ds, (size_t)ctx->n_rz_cap));
  ST(dalloc(ctx, &ctx->rzo_ds, (size_t)ctx->n_rz_cap));
  ST(dalloc(ctx, &ctx->d_iters, 4));
  ST(dalloc(ctx, &ctx->d_err, 4));
  CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
  // ---- matrix-free levels (Section 4.4): drop A_1 .. A_kappa ----
  {
    const int kappa = std::min(opt->matrix_free_levels, N - 1);
    CU(cudaStreamSynchronize(s));
    for (int k = 1; k <= kappa; ++k) {
      Level &l = ctx->L[k], &lp = ctx->L[k - 1];
      const int64_t nb = l.A.nnzb;
      const int64_t freed = nb * l.s * l.s * (int64_t)(sizeof(double) + sizeof(float)) +
                            nb * (int64_t)sizeof(int) + (int64_t)(l.n + 1) * sizeof(int);
      for (void *p : {(void *)l.A.val, (void *)l.A.val32, (void *)l.A.rp, (void *)l.A.col})
        dfree(ctx, p);
      ctx->device_bytes -= freed;
      l.A.val = nullptr;
      l.A.val32 = nullptr;
      l.A.rp = nullptr;
      l.A.col = nullptr;
      l.mf = true;
      // a matrix-free level keeps no product with A_k either
      if (l.RA.val) {
        const int64_t nr = l.RA.nnzb;
        ctx->device_bytes -= nr * l.RA.br * l.RA.bc * (int64_t)(sizeof(double) + sizeof(float)) +
                             nr * (int64_t)sizeof(int) + (int64_t)(l.RA.nrows + 1) * sizeof(int);
        for (void *p : {(void *)l.RA.val, (void *)l.RA.val32, (void *)l.RA.rp, (void *)l.RA.col})
          dfree(ctx, p);
        l.RA = DevBSR{};
      }
      ST(dalloc(ctx, &lp.mt, (size_t)lp.ndof));
      ST(dalloc(ctx, &lp.mu, (size_t)lp.ndof));
      ST(dalloc(ctx, &lp.mtf, (size_t)lp.ndof));
      ST(dalloc(ctx, &lp.muf, (size_t)lp.ndof));
    }
  }
  if (opt->bulk_staging) {
    Level &l = ctx->L[0];
    int maxrow = 0;
    for (int i = 0; i < l.n; ++i) maxrow = std::max(maxrow, hrp[i + 1] - hrp[i]);
    l.tma = tma_plan(l.n, l.s, (int)sizeof(float), maxrow, &l.tma_TR, &l.tma_stageA,
                     &l.tma_stageW, &l.tma_smem, &l.tma_grid);
  }
  ST(dense_tail_build(ctx));
  ST(tail_build<double>(ctx, 0));
  ST(tail_build<float>(ctx, 1));
  ST(grid_build<double>(ctx, 0));
  ST(grid_build<float>(ctx, 1));
  CU(cudaStreamSynchronize(s));
  ctx->ready = true;
  ctx->setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n_levels = N + 1;
    info->n_cand = r;
    for (int k = 0; k <= N; ++k) {
      Level &l = ctx->L[k];
      info->units[k] = l.n;
      info->block[k] = l.s;
      info->dofs[k] = l.padded ? l.real_dofs : l.ndof;
      info->nnzb[k] = l.A.nnzb;
      info->nnz[k] = l.A.nnzb * l.s * l.s;
      info->omega[k] = l.omega;
      info->rho[k] = l.rho;
      int mx = 0;
      for (int v : l.sweeps) mx = std::max(mx, v);
      info->relax_sweeps_max[k] = mx;
    }
    info->seconds = ctx->setup_seconds;
    info->device_bytes = ctx->device_bytes;
  }
  return GASA_OK;
}

}  // namespace

// ============================================================================
// a CUDA error as the single-operation entry points report it
static gasa_status op_status(cudaError_t e) {
  if (e == cudaSuccess) return GASA_OK;
  return e == cudaErrorMemoryAllocation ? GASA_ERR_OOM : GASA_ERR_CUDA;
}

int gasa::op_status_code(cudaError_t e) { return (int)op_status(e); }

// stored blocks of a device BSR matrix (row_ptr[n]); -1 when it cannot be read
int64_t gasa::op_nnzb(const int32_t *row_ptr, int32_t n, cudaStream_t s) {
  if (!row_ptr) return -1;
  int32_t v = -1;
  if (cudaMemcpyAsync(&v, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return v;
}

cudaError_t gasa::power_estimate_on(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                    const int32_t *col, const double *val, const double *Dinv,
                                    const double *x0, int32_t q, int64_t nnzb, double *a,
                                    double *b, double *part, double *sc, double *rho,
                                    cudaStream_t s) {
  const int64_t n = (int64_t)n_units * bs;
  // Alg. 4: x = x0 / ||x0||, then q times x <- D^-1 A x / ||D^-1 A x||,
  // then ||D^-1 A x||
  cudaError_t e = cudaMemcpyAsync(a, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
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
  if (e == cudaSuccess) *rho = std::sqrt(h);
  return e;
}

// extern "C" entry points
// ============================================================================
extern "C" {

void gasa_default_options(gasa_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->dim = 2;
  opt->solver = GASA_SOLVER_CG;
  opt->restart = 30;
  opt->precision = GASA_PREC_FP64;
  opt->t_pre = 3;
  opt->t_post = 3;
  opt->q_power = 3;
  opt->n_cand = 0;
  opt->max_relax = 100;
  opt->max_iter = 10000;
  opt->cand_init = GASA_CAND_R;
  opt->gamma = 0.03;
  opt->omega_factor = 4.0 / 3.0;
  opt->n_cut = 0.0;
  opt->seed = 13373;
  opt->init_candidates = nullptr;
  opt->bulk_staging = 0;
  opt->matrix_free_levels = 0;
  opt->hstar = 0;
  opt->delta = 1e-3;
  opt->tail_kib = 0;
  opt->grid_tail = 0;
  opt->wait_budget_s = 0.0;
  opt->fused_restriction = 1;
  opt->dense_tail_dofs = 2048;
  opt->folded_smoother = 1;
}

gasa_status gasa_create(gasa_ctx **out, int32_t device, void *stream) {
  if (!out) return GASA_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return GASA_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return GASA_ERR_CUDA;
  gasa_ctx *c = new gasa_ctx();
  c->device = device;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return GASA_ERR_CUDA;
    }
    c->own_stream = true;
  }
  gasa_default_options(&c->opt);
  // look up the allocation-free entry point's scratch on this device now, so
  // that its module is loaded here rather than inside an allocation-free call
  double *scratch = nullptr;
  if (noalloc_scratch_on_current_device(&scratch) != cudaSuccess) (void)cudaGetLastError();
  *out = c;
  return GASA_OK;
}

gasa_status gasa_setup(gasa_ctx *ctx, const gasa_bsr *A, const int32_t *adj_ptr,
                       const int32_t *adj_idx, const double *centroids,
                       const gasa_hierarchy *hier, const gasa_options *opt,
                       gasa_setup_info *info) {
  if (!ctx) return GASA_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, GASA_ERR_CUDA, "cudaSetDevice");
  (void)cudaGetLastError();   // an error left by an earlier, unrelated call is not ours
  gasa_status st = setup_impl(ctx, A, adj_ptr, adj_idx, centroids, hier, opt, info);
  if (st != GASA_OK) (void)cudaGetLastError();
  if (st != GASA_OK) {
    cudaStreamSynchronize(ctx->stream);
    ctx->ready = false;
  }
  return st;
}

gasa_status gasa_solve(gasa_ctx *ctx, const double *b, double *x, double tol, int32_t precision,
                       int32_t on_device, gasa_solve_info *info) {
  if (!ctx) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "solve before setup");
  if (!b || !x || !(tol > 0.0)) return fail(ctx, GASA_ERR_INVALID_ARG, "null vector or tol <= 0");
  if (precision < GASA_PREC_FP64 || precision > GASA_PREC_MIXED16)
    return fail(ctx, GASA_ERR_INVALID_ARG, "unknown precision");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, GASA_ERR_CUDA, "cudaSetDevice");
  (void)cudaGetLastError();
  auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->L[0].ndof;
  const double *bd = b;
  if (!on_device) {
    CU(cudaMemcpyAsync(ctx->kb, b, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    bd = ctx->kb;
  }
  int iters = 0;
  double rel = 0.0;
  bool conv = false;
  gasa_status st =
      ctx->opt.solver == GASA_SOLVER_GMRES ? gmres(ctx, bd, tol, precision, &iters, &rel, &conv)
      : ctx->opt.solver == GASA_SOLVER_STATIONARY
          ? stationary(ctx, bd, tol, precision, &iters, &rel, &conv)
          : (ctx->prof ? pcg(ctx, bd, tol, precision, &iters, &rel, &conv)
                       : pcg_graph(ctx, bd, tol, precision, &iters, &rel, &conv));
  if (st != GASA_ERR_TIMEOUT) {
    // a wait that ran out inside a V-cycle leaves its result unusable
    const gasa_status wst = check_wait_flag(ctx);
    if (wst != GASA_OK) st = wst;
  }
  if (st == GASA_OK || st == GASA_ERR_NOT_SPD) {
    if (on_device) {
      CU(cudaMemcpyAsync(x, ctx->kx, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
      CU(cudaMemcpyAsync(x, ctx->kx, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
  }
  if (info) {
    info->iterations = iters;
    info->converged = conv ? 1 : 0;
    info->rel_residual = rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (st != GASA_OK) return st;
  return conv ? GASA_OK : fail(ctx, GASA_ERR_NOT_CONVERGED, "max_iter reached");
}

gasa_status gasa_vcycle(gasa_ctx *ctx, const double *r, double *z, int32_t precision) {
  if (!ctx) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "vcycle before setup");
  if (!r || !z) return fail(ctx, GASA_ERR_INVALID_ARG, "null vector");
  if (precision < GASA_PREC_FP64 || precision > GASA_PREC_MIXED16)
    return fail(ctx, GASA_ERR_INVALID_ARG, "unknown precision");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, GASA_ERR_CUDA, "cudaSetDevice");
  ST(apply_M(ctx, r, z, precision));
  return check_wait_flag(ctx);
}

gasa_status gasa_level_shape(gasa_ctx *ctx, int32_t level, int64_t shape[8]) {
  if (!ctx || !shape) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "no hierarchy");
  if (level < 0 || level > ctx->N) return fail(ctx, GASA_ERR_INVALID_ARG, "level out of range");
  Level &l = ctx->L[level];
  shape[0] = l.n;
  shape[1] = l.s;
  shape[2] = l.A.nnzb;
  shape[3] = level < ctx->N ? l.P.nnzb : 0;
  shape[4] = level < ctx->N ? l.R.nnzb : 0;
  shape[5] = level < ctx->N ? l.s_next : 0;
  shape[6] = ctx->r;
  shape[7] = l.padded ? l.real_dofs : l.ndof;
  return GASA_OK;
}

gasa_status gasa_tail_info(gasa_ctx *ctx, int32_t precision, int32_t out[3]) {
  if (!ctx || !out) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "no hierarchy");
  if (precision < GASA_PREC_FP64 || precision > GASA_PREC_MIXED16)
    return fail(ctx, GASA_ERR_INVALID_ARG, "unknown precision");
  const int pi = precision == GASA_PREC_FP64 ? 0 : 1;
  if (ctx->grid_plan[pi]) {
    out[0] = ctx->grid_k0[pi];
    out[1] = ctx->grid_ctas[pi];
    out[2] = 1;
    return GASA_OK;
  }
  const bool on = ctx->tail_plan[pi] != nullptr;
  out[0] = on ? ctx->tail_k0[pi] : ctx->N;
  out[1] = on ? ctx->tail_cluster[pi] : 0;
  out[2] = on ? ctx->tail_coarse[pi] : 0;
  return GASA_OK;
}

gasa_status gasa_cycle_info(gasa_ctx *ctx, int32_t out[3]) {
  if (!ctx || !out) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "no hierarchy");
  const bool on = ctx->dtail_M != nullptr;
  out[0] = on ? ctx->dtail_k : ctx->N;
  out[1] = on ? ctx->dtail_n : 0;
  out[2] = (ctx->L[0].WA32 && !ctx->L[0].tma) ? 1 : 0;
  return GASA_OK;
}

gasa_status gasa_get_level(gasa_ctx *ctx, int32_t level, int32_t what, void *host_out,
                           int64_t n_bytes) {
  if (!ctx || !host_out) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return fail(ctx, GASA_ERR_STATE, "no hierarchy");
  if (level < 0 || level > ctx->N) return fail(ctx, GASA_ERR_INVALID_ARG, "level out of range");
  Level &l = ctx->L[level];
  const bool fine = level < ctx->N;
  const void *src = nullptr;
  int64_t bytes = 0;
  switch (what) {
    case GASA_LV_A_ROWPTR: src = l.A.rp; bytes = 4 * (l.n + 1); break;
    case GASA_LV_A_COL: src = l.A.col; bytes = 4 * l.A.nnzb; break;
    case GASA_LV_A_VAL: src = l.A.val; bytes = 8 * l.A.nnzb * l.s * l.s; break;
    case GASA_LV_P_ROWPTR: if (fine) { src = l.P.rp; bytes = 4 * (l.n + 1); } break;
    case GASA_LV_P_COL: if (fine) { src = l.P.col; bytes = 4 * l.P.nnzb; } break;
    case GASA_LV_P_VAL: if (fine) { src = l.P.val; bytes = 8 * l.P.nnzb * l.s * l.s_next; } break;
    case GASA_LV_R_ROWPTR: if (fine) { src = l.R.rp; bytes = 4 * (int64_t)(l.n_next + 1); } break;
    case GASA_LV_R_COL: if (fine) { src = l.R.col; bytes = 4 * l.R.nnzb; } break;
    case GASA_LV_R_VAL: if (fine) { src = l.R.val; bytes = 8 * l.R.nnzb * l.s * l.s_next; } break;
    case GASA_LV_T_VAL: if (fine && l.T) { src = l.T; bytes = 8 * (int64_t)l.n * l.s * l.s_next; } break;
    case GASA_LV_W: if (fine) { src = l.W; bytes = 8 * (int64_t)l.n * l.s * l.s; } break;
    case GASA_LV_CAND: if (fine && l.cand) { src = l.cand; bytes = 8 * l.ndof * ctx->r; } break;
    case GASA_LV_CAND_IN: if (fine && l.cand_in) { src = l.cand_in; bytes = 8 * l.ndof * ctx->r; } break;
    case GASA_LV_SWEEPS:
      if (fine) {
        if (n_bytes < 4 * (int64_t)l.sweeps.size())
          return fail(ctx, GASA_ERR_INVALID_ARG, "output buffer too small");
        std::memcpy(host_out, l.sweeps.data(), 4 * l.sweeps.size());
        return GASA_OK;
      }
      break;
    case GASA_LV_COARSE_INV:
      if (!fine) { src = ctx->coarse_inv; bytes = 8 * (int64_t)ctx->nc * ctx->nc; }
      break;
    case GASA_LV_RA_ROWPTR: if (fine && l.RA.rp) { src = l.RA.rp; bytes = 4 * (int64_t)(l.RA.nrows + 1); } break;
    case GASA_LV_RA_COL: if (fine && l.RA.col) { src = l.RA.col; bytes = 4 * l.RA.nnzb; } break;
    case GASA_LV_RA_VAL:
      if (fine && l.RA.val) { src = l.RA.val; bytes = 8 * l.RA.nnzb * l.RA.br * l.RA.bc; }
      break;
    case GASA_LV_DENSE_TAIL:
      if (ctx->dtail_M && level == ctx->dtail_k) {
        // rows are stored with a padded pitch: copy them out unpadded
        const size_t n = (size_t)ctx->dtail_n;
        if (n_bytes < (int64_t)(8 * n * n))
          return fail(ctx, GASA_ERR_INVALID_ARG, "output buffer too small");
        if (cudaSetDevice(ctx->device) != cudaSuccess)
          return fail(ctx, GASA_ERR_CUDA, "cudaSetDevice");
        CU(cudaStreamSynchronize(ctx->stream));
        CU(cudaMemcpy2D(host_out, n * sizeof(double), ctx->dtail_M,
                        (size_t)ctx->dtail_ld * sizeof(double), n * sizeof(double), n,
                        cudaMemcpyDeviceToHost));
        return GASA_OK;
      }
      break;
    case GASA_LV_WA:
      if (l.WA) { src = l.WA; bytes = 8 * l.A.nnzb * l.s * l.s; }
      break;
    case GASA_LV_SIZES: {
      if (n_bytes < 4 * (int64_t)l.n) return fail(ctx, GASA_ERR_INVALID_ARG, "output buffer too small");
      int32_t *o = static_cast<int32_t *>(host_out);
      for (int i = 0; i < l.n; ++i) o[i] = l.padded ? l.usize[i] : l.s;
      return GASA_OK;
    }
    default: return fail(ctx, GASA_ERR_INVALID_ARG, "unknown level item");
  }
  if (!src) return fail(ctx, GASA_ERR_INVALID_ARG, "item not available on this level (setup data is kept only with options.keep_setup_data; a matrix-free level keeps no A)");
  if (n_bytes < bytes) return fail(ctx, GASA_ERR_INVALID_ARG, "output buffer too small");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, GASA_ERR_CUDA, "cudaSetDevice");
  CU(cudaStreamSynchronize(ctx->stream));
  CU(cudaMemcpy(host_out, src, bytes, cudaMemcpyDeviceToHost));
  return GASA_OK;
}

gasa_status gasa_profile_enable(gasa_ctx *ctx, int32_t on) {
  if (!ctx) return GASA_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  ctx->prof = on != 0;
  for (auto &p : ctx->pc) {
    p.used = 0;
    p.bytes = 0.0;
    p.launches = 0;
  }
  return GASA_OK;
}

gasa_status gasa_profile_read(gasa_ctx *ctx, int32_t cls, double *ms, int64_t *launches,
                              double *bytes) {
  if (!ctx || cls < 0 || cls > 4) return GASA_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  ProfClass &p = ctx->pc[cls];
  double tot = 0.0;
  for (size_t i = 0; i + 1 < p.used; i += 2) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, p.ev[i], p.ev[i + 1]));
    tot += t;
  }
  if (ms) *ms = tot;
  if (launches) *launches = p.launches;
  if (bytes) *bytes = p.bytes;
  return GASA_OK;
}

gasa_status gasa_destroy(gasa_ctx *ctx) {
  if (!ctx) return GASA_OK;
  cudaSetDevice(ctx->device);
  free_all(ctx);
  for (auto &p : ctx->pc)
    for (auto e : p.ev) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return GASA_OK;
}

const char *gasa_status_string(gasa_status s) {
  if ((int)s < 0 || (int)s > (int)GASA_ERR_STATE) return "unknown status";
  return kStatusText[(int)s];
}

const char *gasa_last_error(const gasa_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int64_t gasa_kernel_launches(void) { return (int64_t)launch_count(); }

// ---------------------------------------------------------------------------
// single operations
// ---------------------------------------------------------------------------



gasa_status gasa_bsr_mv(int32_t mode, int32_t n_brows, int32_t br, int32_t bc,
                        const int32_t *row_ptr, const int32_t *col, const double *val,
                        const double *x, const double *b, double *y, void *stream) {
  if (n_brows < 0 || br <= 0 || bc <= 0 || mode < 0 || mode > 2) return GASA_ERR_INVALID_ARG;
  if (n_brows == 0) return GASA_OK;
  if (!row_ptr || !col || !val || !x || !y || (mode == GASA_MV_RESIDUAL && !b))
    return GASA_ERR_INVALID_ARG;
  return op_status(launch_bsr_mv<double>(mode, n_brows, br, bc, row_ptr, col, val, x, b, y,
                                         (cudaStream_t)stream,
                                         op_nnzb(row_ptr, n_brows, (cudaStream_t)stream)));
}

gasa_status gasa_bsr_mv_f32(int32_t mode, int32_t n_brows, int32_t br, int32_t bc,
                            const int32_t *row_ptr, const int32_t *col, const float *val,
                            const float *x, const float *b, float *y, void *stream) {
  if (n_brows < 0 || br <= 0 || bc <= 0 || mode < 0 || mode > 2) return GASA_ERR_INVALID_ARG;
  if (n_brows == 0) return GASA_OK;
  if (!row_ptr || !col || !val || !x || !y || (mode == GASA_MV_RESIDUAL && !b))
    return GASA_ERR_INVALID_ARG;
  return op_status(launch_bsr_mv<float>(mode, n_brows, br, bc, row_ptr, col, val, x, b, y,
                                        (cudaStream_t)stream,
                                        op_nnzb(row_ptr, n_brows, (cudaStream_t)stream)));
}

gasa_status gasa_bsr_mv_ds(int32_t n_brows, int32_t br, int32_t bc, const int32_t *row_ptr,
                           const int32_t *col, const float *a_hi, const float *a_lo,
                           const float *x_hi, const float *x_lo, double *y, void *stream) {
  if (n_brows < 0 || br <= 0 || bc <= 0) return GASA_ERR_INVALID_ARG;
  if (n_brows == 0) return GASA_OK;
  if (!row_ptr || !col || !a_hi || !a_lo || !x_hi || !x_lo || !y) return GASA_ERR_INVALID_ARG;
  return op_status(launch_bsr_mv_ds(n_brows, br, bc, row_ptr, col, a_hi, a_lo, x_hi, x_lo, y,
                                    (cudaStream_t)stream));
}

gasa_status gasa_jacobi_sweep(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                              const int32_t *col, const double *val, const double *W,
                              const double *x, const double *b, double *x_out, int32_t first,
                              void *stream) {
  if (n_units < 0 || bs <= 0 || bs > 1024) return GASA_ERR_INVALID_ARG;
  if (n_units == 0) return GASA_OK;
  if (!W || !b || !x_out || (!first && (!row_ptr || !col || !val || !x)) || x == x_out)
    return GASA_ERR_INVALID_ARG;
  return op_status(launch_jacobi<double>(first ? JAC_FIRST : JAC_SWEEP, n_units, bs, row_ptr, col,
                                         val, W, x, b, x_out, (cudaStream_t)stream,
                                         first ? -1 : op_nnzb(row_ptr, n_units, (cudaStream_t)stream)));
}

gasa_status gasa_jacobi_sweep_f32(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                  const int32_t *col, const float *val, const float *W,
                                  const float *x, const float *b, float *x_out, int32_t first,
                                  void *stream) {
  if (n_units < 0 || bs <= 0 || bs > 1024) return GASA_ERR_INVALID_ARG;
  if (n_units == 0) return GASA_OK;
  if (!W || !b || !x_out || (!first && (!row_ptr || !col || !val || !x)) || x == x_out)
    return GASA_ERR_INVALID_ARG;
  return op_status(launch_jacobi<float>(first ? JAC_FIRST : JAC_SWEEP, n_units, bs, row_ptr, col,
                                        val, W, x, b, x_out, (cudaStream_t)stream,
                                        first ? -1 : op_nnzb(row_ptr, n_units, (cudaStream_t)stream)));
}

gasa_status gasa_block_inverse(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                               const int32_t *col, const double *val, double scale,
                               double *W_out, int32_t *n_singular, void *stream) {
  if (n_units < 0 || bs <= 0 || bs > 64 || !n_singular) return GASA_ERR_INVALID_ARG;
  *n_singular = 0;
  if (n_units == 0) return GASA_OK;
  if (!row_ptr || !col || !val || !W_out) return GASA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int *d = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&d, sizeof(int), s);
  if (e != cudaSuccess) return op_status(e);
  e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_block_inverse(n_units, bs, row_ptr, col, val, scale, W_out, d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n_singular, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return op_status(e);
}


gasa_status gasa_power_estimate(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                const int32_t *col, const double *val, const double *Dinv,
                                const double *x0, int32_t q, double *rho, void *stream) {
  if (n_units <= 0 || bs <= 0 || bs > 1024 || q < 0 || !row_ptr || !col || !val || !Dinv ||
      !x0 || !rho)
    return GASA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)n_units * bs;
  const int64_t nnzb = op_nnzb(row_ptr, n_units, s);
  if (nnzb < 0) return GASA_ERR_CUDA;
  double *buf = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(double) * (2 * n + kRedBlocks + 2), s);
  if (e != cudaSuccess) return op_status(e);
  e = power_estimate_on(n_units, bs, row_ptr, col, val, Dinv, x0, q, nnzb, buf, buf + n,
                        buf + 2 * n, buf + 2 * n + kRedBlocks, rho, s);
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return op_status(e);
}

gasa_status gasa_relax_candidates(int32_t n_units, int32_t bs, const int32_t *row_ptr,
                                  const int32_t *col, const double *val, const double *W,
                                  double *B, int32_t r, double gamma, int32_t max_relax,
                                  int32_t *sweeps, void *stream) {
  if (n_units <= 0 || bs <= 0 || bs > 1024 || r <= 0 || r > 1024 || max_relax < 0 || !row_ptr ||
      !col || !val || !W || !B || !sweeps || gamma < 0.0)
    return GASA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)n_units * bs;
  double *B2 = nullptr, *part = nullptr, *nr = nullptr;
  double **tab = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&B2, sizeof(double) * n * r, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&part, sizeof(double) * kRedBlocks * r, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&nr, sizeof(double) * r, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&tab, sizeof(double *) * 2 * r, s);
  std::vector<double *> cur(r), nxt(r), htab(2 * r);
  std::vector<double> nrm(r), nn(r);
  std::vector<int> active;
  for (int c = 0; c < r; ++c) {
    cur[c] = B + (size_t)c * n;
    nxt[c] = B2 + (size_t)c * n;
    active.push_back(c);
    sweeps[c] = 0;
  }
  if (e == cudaSuccess) {
    for (int c = 0; c < r; ++c) htab[c] = cur[c];
    e = cudaMemcpyAsync(tab, htab.data(), sizeof(double *) * r, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_colnorm_partials(n, (const double *const *)tab, r, part, s);
    if (e == cudaSuccess) e = launch_finalize(part, r, nr, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nrm.data(), nr, sizeof(double) * r, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (auto &v : nrm) v = std::sqrt(v);
  }
  for (int m = 0; m < max_relax && !active.empty() && e == cudaSuccess; ++m) {
    const int na = (int)active.size();
    for (int q = 0; q < na; ++q) {
      htab[q] = cur[active[q]];
      htab[na + q] = nxt[active[q]];
    }
    e = cudaMemcpyAsync(tab, htab.data(), sizeof(double *) * 2 * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_relax_multi(n_units, bs, row_ptr, col, val, W, (const double *const *)tab,
                             (double *const *)(tab + na), na, s);
    if (e == cudaSuccess) e = launch_colnorm_partials(n, (const double *const *)(tab + na), na, part, s);
    if (e == cudaSuccess) e = launch_finalize(part, na, nr, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nn.data(), nr, sizeof(double) * na, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    std::vector<int> still;
    for (int q = 0; q < na; ++q) {
      const int c = active[q];
      std::swap(cur[c], nxt[c]);
      sweeps[c] = m + 1;
      const double nnew = std::sqrt(nn[q]);
      if (nrm[c] / nnew < 1.0 + gamma) continue;
      nrm[c] = nnew;
      still.push_back(c);
    }
    active.swap(still);
  }
  for (int c = 0; c < r && e == cudaSuccess; ++c)
    if (cur[c] != B + (size_t)c * n)
      e = cudaMemcpyAsync(B + (size_t)c * n, cur[c], sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (B2) cudaFreeAsync(B2, s);
  if (part) cudaFreeAsync(part, s);
  if (nr) cudaFreeAsync(nr, s);
  if (tab) cudaFreeAsync(tab, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  return op_status(e != cudaSuccess ? e : e2);
}

gasa_status gasa_tentative(int32_t n_units, int32_t bs, int32_t n_agg, const int32_t *agg_of,
                           const double *B, int32_t r, int32_t s_next, double *T_out,
                           double *sigma_out, void *stream) {
  if (n_units <= 0 || bs <= 0 || n_agg <= 0 || n_agg > n_units || r <= 0 || r > 256 ||
      s_next <= 0 || s_next > r || !agg_of || !B || !T_out)
    return GASA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int *cp = nullptr, *ci = nullptr, *scr = nullptr, *st = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&cp, sizeof(int) * (n_agg + 1), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&ci, sizeof(int) * n_units, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&scr, sizeof(int) * (n_agg + 1), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&st, sizeof(int) * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int) * 2, s);
  if (e == cudaSuccess) e = build_children(n_units, n_agg, agg_of, cp, ci, scr, s);
  // largest aggregate (children per aggregate = cp[J+1] - cp[J])
  int maxc = 0;
  if (e == cudaSuccess) {
    std::vector<int> hcp(n_agg + 1);
    e = cudaMemcpyAsync(hcp.data(), cp, sizeof(int) * (n_agg + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int J = 0; J < n_agg && e == cudaSuccess; ++J) {
      const int c = hcp[J + 1] - hcp[J];
      if (c <= 0) e = cudaErrorInvalidValue;   // every aggregate must own a unit
      maxc = std::max(maxc, c);
    }
  }
  int smem = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0);
  if (e == cudaSuccess && (size_t)maxc * bs * r * sizeof(double) > (size_t)smem) e = cudaErrorInvalidValue;
  if (e == cudaSuccess)
    e = launch_tentative(bs, n_agg, maxc, cp, ci, B, (int64_t)n_units * bs, r, s_next, T_out,
                         sigma_out, st, s);
  int hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s);
  for (int *p : {cp, ci, scr, st})
    if (p) cudaFreeAsync(p, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaErrorInvalidValue) return GASA_ERR_INVALID_ARG;
  if (e != cudaSuccess || e2 != cudaSuccess) return op_status(e != cudaSuccess ? e : e2);
  return hst ? GASA_ERR_BREAKDOWN : GASA_OK;
}

gasa_status gasa_dense_inverse(int32_t n, const double *A, double *Ainv, int32_t *singular,
                               void *stream) {
  if (n <= 0 || n > 16384 || !A || !Ainv || !singular) return GASA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double *work = nullptr;
  int *d = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&work, sizeof(double) * (2 * (size_t)n * n + n), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&d, sizeof(int), s);
  if (e == cudaSuccess) e = launch_dense_inverse(n, A, Ainv, work, d, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (work) cudaFreeAsync(work, s);
  if (d) cudaFreeAsync(d, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  *singular = h;
  return op_status(e != cudaSuccess ? e : e2);
}

}  // extern "C"
