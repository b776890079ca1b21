// Request server: continuous batching of solves on resident hierarchies.
//
// For each (mesh, precision) with work, an engine owns K slots.  The slots'
// right-hand sides, iterates and Krylov vectors are stored interleaved
// (entry i of slot c at i * K + c), and the V-cycle of Alg. 2 plus the outer
// A x run on all K columns per launch (kernels_batch.cu).  An engine step is
// a CUDA graph launch: for CG a conditional while loop of whole iterations
// that stops when some column leaves the running state or after a cap; for
// GMRES one restart cycle (start, a while loop over Arnoldi steps, update).
// Between launches the engine's host thread retires finished columns and
// admits queued requests into free slots, so a batch changes while other
// solves are in flight.  Each engine has its own stream and thread; engines
// of different meshes overlap on the device.
//
// Device memory: a mesh's hierarchy counts against the budget when added; an
// engine reserves its vectors when created.  A request whose engine does not
// fit waits; engines with no work are released when others need the room.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <type_traits>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "ctx.h"
#include "gasa.h"
#include "internal.h"

using namespace gasa;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0;
  int mesh = 0;
  int prec = 0;
  double tol = 0.0;
  std::vector<double> b, x;
  gasa_status status = GASA_PENDING;
  gasa_solve_info info{};
  Clock::time_point t0;
};

struct Engine;

struct MeshEntry {
  gasa_ctx *ctx = nullptr;
  int64_t bytes = 0;
};

}  // namespace

struct gasa_server {
  int device = 0;
  int64_t budget = 0;
  int max_batch = 8;
  std::mutex mu;
  std::condition_variable cv_done;
  std::vector<MeshEntry> meshes;
  std::deque<Request *> queue;                      // not yet in a slot, FIFO
  std::unordered_map<uint64_t, Request *> tickets;  // every request not yet polled
  std::vector<Engine *> engines;                    // live
  std::vector<Engine *> retired;                    // threads to join
  uint64_t next_ticket = 1;
  int64_t used = 0, peak = 0;
  int64_t submitted = 0, completed = 0, running = 0, peak_running = 0;
  int64_t created = 0, released = 0;
  int retiring = 0;                                 // engines on their way out
  std::atomic<long long> graph_launches{0};
  bool stopping = false;
  std::string err;
};

namespace {

struct LevelVec {
  double *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
  float *xf = nullptr, *x2f = nullptr, *bf = nullptr, *rf = nullptr;
  // scratch of the product A_{k+1} x when level k + 1 is matrix-free
  double *mt = nullptr, *mu = nullptr;
  float *mtf = nullptr, *muf = nullptr;
};

struct Engine {
  gasa_server *srv = nullptr;
  int mesh = 0, prec = 0, K = 1, m = 0;
  bool gm = false, flex = false;
  gasa_ctx *ctx = nullptr;
  int64_t n = 0;
  cudaStream_t s = nullptr;
  std::vector<void *> allocs;
  int64_t bytes = 0;
  // interleaved n x K vectors
  double *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *Zold = nullptr,
         *Bv = nullptr, *T = nullptr, *W = nullptr, *Vcur = nullptr;
  double *V = nullptr, *Zb = nullptr;     // GMRES bases: (m + 1) and m vectors
  float *fin = nullptr, *fout = nullptr;
  std::vector<LevelVec> lv;
  double *part[4] = {nullptr, nullptr, nullptr, nullptr};   // K x kRedBlocks each
  double *mpart = nullptr;                                  // (m + 1) x K x kRedBlocks
  double *sc = nullptr;                                     // BD_COUNT x K
  int *st = nullptr;                                        // BI_COUNT x K
  int *ctl = nullptr;                                       // loop count, cap, changed, j
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *hbuf = nullptr,
         *beta = nullptr;
  double *stage = nullptr;                                  // n (device)
  double *hstage = nullptr;                                 // n (pinned host)
  double *hsc = nullptr;                                    // pinned mirrors
  int *hst = nullptr, *hctl = nullptr;
  cudaGraph_t graph = nullptr, g_start = nullptr, g_end = nullptr;
  cudaGraphExec_t exec = nullptr, x_start = nullptr, x_end = nullptr;
  std::vector<Request *> slot;
  std::thread th;
  std::condition_variable cv;
  bool retire = false;
  std::string err;
};

// ----------------------------------------------------------------------------
// memory layout (counted first, then allocated with the same walk)
// ----------------------------------------------------------------------------
struct Alloc {
  Engine *e;
  bool real;
  int64_t bytes = 0;
  cudaError_t status = cudaSuccess;
  template <typename T>
  void operator()(T **p, int64_t count) {
    if (count <= 0) count = 1;
    const int64_t b = (count * (int64_t)sizeof(T) + 255) / 256 * 256;
    bytes += b;
    if (!real || status != cudaSuccess) return;
    status = cudaMalloc((void **)p, (size_t)count * sizeof(T));
    if (status == cudaSuccess) e->allocs.push_back((void *)*p);
    else *p = nullptr;
  }
};

void layout(Engine &e, Alloc &a) {
  gasa_ctx *ctx = e.ctx;
  const int64_t nk = e.n * e.K;
  const int K = e.K;
  a(&e.X, nk);
  a(&e.Bv, nk);
  a(&e.T, nk);
  if (!e.gm) {
    a(&e.R, nk);
    a(&e.Z, nk);
    a(&e.P, nk);
    a(&e.Q, nk);
    if (e.flex) a(&e.Zold, nk);
  } else {
    a(&e.W, nk);
    a(&e.Vcur, nk);
    a(&e.V, (int64_t)(e.m + 1) * nk);
    if (e.flex) a(&e.Zb, (int64_t)e.m * nk);
    a(&e.mpart, (int64_t)(e.m + 1) * K * kRedBlocks);
    a(&e.H, (int64_t)(e.m + 1) * e.m * K);
    a(&e.cs, (int64_t)(e.m + 1) * K);
    a(&e.sn, (int64_t)(e.m + 1) * K);
    a(&e.g, (int64_t)(e.m + 2) * K);
    a(&e.y, (int64_t)(e.m + 1) * K);
    a(&e.hbuf, (int64_t)(e.m + 1) * K);
    a(&e.beta, K);
  }
  if (e.prec != GASA_PREC_FP64) {
    a(&e.fin, nk);
    a(&e.fout, nk);
  }
  e.lv.assign(ctx->N + 1, LevelVec{});
  for (int k = 0; k <= ctx->N; ++k) {
    const int64_t d = ctx->L[k].ndof * K;
    LevelVec &v = e.lv[k];
    const bool mf_above = k < ctx->N && ctx->L[k + 1].mf;
    if (e.prec == GASA_PREC_FP64) {
      a(&v.x, d);
      a(&v.x2, d);
      a(&v.b, d);
      a(&v.r, d);
      if (mf_above) {
        a(&v.mt, d);
        a(&v.mu, d);
      }
    } else {
      a(&v.xf, d);
      a(&v.x2f, d);
      a(&v.bf, d);
      a(&v.rf, d);
      if (mf_above) {
        a(&v.mtf, d);
        a(&v.muf, d);
      }
    }
  }
  for (auto &p : e.part) a(&p, (int64_t)K * kRedBlocks);
  a(&e.sc, (int64_t)BD_COUNT * K);
  a(&e.st, (int64_t)BI_COUNT * K);
  a(&e.ctl, 8);
  a(&e.stage, e.n);
}

// ----------------------------------------------------------------------------
// batched V-cycle (Alg. 2) on the engine's K columns
// ----------------------------------------------------------------------------
template <typename T> struct EP;
template <> struct EP<double> {
  static const double *A(const DevBSR &m) { return m.val; }
  static const double *W(const Level &l) { return l.W; }
  static double *x(LevelVec &v) { return v.x; }
  static double *x2(LevelVec &v) { return v.x2; }
  static double *b(LevelVec &v) { return v.b; }
  static double *r(LevelVec &v) { return v.r; }
  static double *mt(LevelVec &v) { return v.mt; }
  static double *mu(LevelVec &v) { return v.mu; }
};
template <> struct EP<float> {
  static const float *A(const DevBSR &m) { return m.val32; }
  static const float *W(const Level &l) { return l.W32; }
  static float *x(LevelVec &v) { return v.xf; }
  static float *x2(LevelVec &v) { return v.x2f; }
  static float *b(LevelVec &v) { return v.bf; }
  static float *r(LevelVec &v) { return v.rf; }
  static float *mt(LevelVec &v) { return v.mtf; }
  static float *mu(LevelVec &v) { return v.muf; }
};

#define ECU(...)                              \
  do {                                        \
    cudaError_t e_ = (__VA_ARGS__);           \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

// A_k X (mode ASSIGN) or B - A_k X (RESIDUAL) on a matrix-free level k >= 1,
// through the transfers: R_{k-1} (A_{k-1} (P_{k-1} X)) (Section 4.4)
template <typename T>
cudaError_t bmf_apply(Engine &e, int k, int mode, const T *x, const T *b, T *y) {
  using P = EP<T>;
  gasa_ctx *ctx = e.ctx;
  Level &lp = ctx->L[k - 1];
  LevelVec &v = e.lv[k - 1];
  T *t = P::mt(v), *u = P::mu(v);
  ECU(launch_bmv<T>(GASA_MV_ASSIGN, lp.P.nrows, lp.P.br, lp.P.bc, lp.P.rp, lp.P.col, P::A(lp.P),
                    x, nullptr, t, e.K, e.s, lp.P.nnzb));
  if (k - 1 > 0 && lp.mf) ECU(bmf_apply<T>(e, k - 1, GASA_MV_ASSIGN, t, nullptr, u));
  else ECU(launch_bmv<T>(GASA_MV_ASSIGN, lp.n, lp.s, lp.s, lp.A.rp, lp.A.col, P::A(lp.A), t,
                         nullptr, u, e.K, e.s, lp.A.nnzb));
  return launch_bmv<T>(mode, lp.R.nrows, lp.R.br, lp.R.bc, lp.R.rp, lp.R.col, P::A(lp.R), u, b, y,
                       e.K, e.s, lp.R.nnzb);
}

// one smoothing step of Alg. 1 on K columns
template <typename T>
cudaError_t bsweep(Engine &e, int k, int mode, const T *x, const T *b, T *xo) {
  using P = EP<T>;
  Level &l = e.ctx->L[k];
  if (l.mf && mode == JAC_SWEEP) {
    T *r = P::r(e.lv[k]);
    ECU(bmf_apply<T>(e, k, GASA_MV_RESIDUAL, x, b, r));
    ECU(launch_bjacobi<T>(JAC_FIRST, l.n, l.s, nullptr, nullptr, nullptr, P::W(l), nullptr, r, xo,
                          e.K, e.s, 0));
    return launch_add<T>(l.ndof * e.K, x, xo, e.s);
  }
  if constexpr (std::is_same<T, float>::value) {
    // FP16-block engines read level 0's A and w D^-1 from their FP16 blocks
    if (k == 0 && e.prec == GASA_PREC_MIXED16 && l.A.val16 && l.W16)
      return launch_bjacobi_h16(mode, l.n, l.s, l.A.rp, l.A.col, l.A.val16, l.A.scale16, l.W16,
                                l.W16s, x, b, xo, e.K, e.s);
  }
  return launch_bjacobi<T>(mode, l.n, l.s, l.A.rp, l.A.col, P::A(l.A), P::W(l), x, b, xo, e.K,
                           e.s, l.A.nnzb);
}

template <typename T>
cudaError_t bresid(Engine &e, int k, const T *x, const T *b, T *r) {
  using P = EP<T>;
  Level &l = e.ctx->L[k];
  if (l.mf) return bmf_apply<T>(e, k, GASA_MV_RESIDUAL, x, b, r);
  if constexpr (std::is_same<T, float>::value) {
    if (k == 0 && e.prec == GASA_PREC_MIXED16 && l.A.val16)
      return launch_bmv_h16(GASA_MV_RESIDUAL, l.n, l.s, l.A.rp, l.A.col, l.A.val16, l.A.scale16, x,
                            b, r, e.K, e.s);
  }
  return launch_bmv<T>(GASA_MV_RESIDUAL, l.n, l.s, l.s, l.A.rp, l.A.col, P::A(l.A), x, b, r, e.K,
                       e.s, l.A.nnzb);
}

template <typename T>
cudaError_t vcycle_b(Engine &e, const T *rhs, T *out) {
  using P = EP<T>;
  gasa_ctx *ctx = e.ctx;
  const int N = ctx->N, K = e.K;
  const int tpre = ctx->opt.t_pre, tpost = ctx->opt.t_post;
  cudaStream_t s = e.s;
  // levels kt .. N as the hierarchy's dense bottom operator, when it has one
  const int kt = ctx->dtail_M ? ctx->dtail_k : N;
  std::vector<const T *> bk(N + 1);
  std::vector<T *> xk(N + 1);
  bk[0] = rhs;
  for (int k = 1; k <= N; ++k) bk[k] = P::b(e.lv[k]);
  for (int k = 0; k < kt; ++k) {
    Level &l = ctx->L[k];
    LevelVec &v = e.lv[k];
    T *x = P::x(v), *x2 = P::x2(v);
    if (tpre == 0) {
      ECU(cudaMemsetAsync(x, 0, (size_t)l.ndof * K * sizeof(T), s));
    } else {
      ECU(bsweep<T>(e, k, JAC_FIRST, nullptr, bk[k], x));
      for (int t = 1; t < tpre; ++t) {
        ECU(bsweep<T>(e, k, JAC_SWEEP, x, bk[k], x2));
        std::swap(x, x2);
      }
    }
    xk[k] = x;
    ECU(bresid<T>(e, k, x, bk[k], P::r(v)));
    ECU(launch_bmv<T>(GASA_MV_ASSIGN, l.R.nrows, l.R.br, l.R.bc, l.R.rp, l.R.col, P::A(l.R),
                      P::r(v), nullptr, P::b(e.lv[k + 1]), K, s, l.R.nnzb));
  }
  if (kt < N)
    ECU(launch_bdense<T>(ctx->dtail_n, ctx->dtail_M, P::b(e.lv[kt]), P::x(e.lv[kt]), K, s,
                         ctx->dtail_ld));
  else
    ECU(launch_bdense<T>(ctx->nc, ctx->coarse_inv, P::b(e.lv[N]), P::x(e.lv[N]), K, s));
  xk[kt] = P::x(e.lv[kt]);
  for (int k = kt - 1; k >= 0; --k) {
    Level &l = ctx->L[k];
    LevelVec &v = e.lv[k];
    T *x = xk[k];
    T *x2 = (x == P::x(v)) ? P::x2(v) : P::x(v);
    ECU(launch_bmv<T>(GASA_MV_ADD, l.P.nrows, l.P.br, l.P.bc, l.P.rp, l.P.col, P::A(l.P),
                      xk[k + 1], nullptr, x, K, s, l.P.nnzb));
    if (tpost == 0 && k == 0)
      ECU(cudaMemcpyAsync(out, x, (size_t)l.ndof * K * sizeof(T), cudaMemcpyDeviceToDevice, s));
    for (int t = 0; t < tpost; ++t) {
      T *dst = (k == 0 && t == tpost - 1) ? out : x2;
      ECU(bsweep<T>(e, k, JAC_SWEEP, x, bk[k], dst));
      if (dst == x2) std::swap(x, x2);
      else x = dst;
    }
    xk[k] = x;
  }
  return cudaSuccess;
}

cudaError_t apply_Mb(Engine &e, const double *r, double *z) {
  if (e.prec == GASA_PREC_FP64) return vcycle_b<double>(e, r, z);
  const int64_t nk = e.n * e.K;
  ECU(launch_convert<double, float>(nk, r, e.fin, e.s));
  ECU(vcycle_b<float>(e, e.fin, e.fout));
  return launch_convert<float, double>(nk, e.fout, z, e.s);
}

cudaError_t outer_mv(Engine &e, int mode, const double *x, const double *b, double *y) {
  Level &l = e.ctx->L[0];
  return launch_bmv<double>(mode, l.n, l.s, l.s, l.A.rp, l.A.col, l.A.val, x, b, y, e.K, e.s,
                            l.A.nnzb);
}

// ----------------------------------------------------------------------------
// graphs
// ----------------------------------------------------------------------------
// one CG iteration per pass of a conditional while node (order as in the
// single-solve CG: z = M r, p update, q = A p, x and r update, test)
cudaError_t build_cg(Engine &e) {
  const int K = e.K;
  const int64_t n = e.n;
  ECU(cudaGraphCreate(&e.graph, 0));
  cudaGraphConditionalHandle h;
  ECU(cudaGraphConditionalHandleCreate(&h, e.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ECU(cudaGraphAddNode(&node, e.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ECU(cudaStreamBeginCaptureToGraph(e.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = [&]() -> cudaError_t {
    ECU(apply_Mb(e, e.R, e.Z));
    ECU(launch_bdot(n, e.R, e.Z, e.part[0], K, e.s));
    if (e.flex) ECU(launch_bdot(n, e.R, e.Zold, e.part[1], K, e.s));
    ECU(launch_bcg_beta(e.part[0], e.part[1], e.sc, e.st, e.flex ? 1 : 0, K, e.s));
    ECU(launch_bcg_update_p(n, e.P, e.Z, e.flex ? e.Zold : nullptr, e.sc, K, e.s));
    ECU(outer_mv(e, GASA_MV_ASSIGN, e.P, nullptr, e.Q));
    ECU(launch_bdot(n, e.P, e.Q, e.part[2], K, e.s));
    ECU(launch_bcg_alpha(e.part[2], e.sc, e.st, K, e.s));
    ECU(launch_bcg_update_xr(n, e.X, e.R, e.P, e.Q, e.sc, e.part[3], K, e.s));
    return launch_bcg_check(e.part[3], e.sc, e.st, e.ctl, e.flex ? 1 : 0, h, K, e.s);
  }();
  cudaGraph_t cap = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(e.s, &cap);
  ECU(err);
  ECU(e2);
  return cudaGraphInstantiate(&e.exec, e.graph, 0);
}

// GMRES restart cycle: start graph, step loop graph, end graph
cudaError_t build_gm(Engine &e) {
  const int K = e.K, m = e.m;
  const int64_t n = e.n, nk = n * K;
  int *dj = e.ctl + 3;
  // start: t = b - A x; w = M t (left) or t (flexible); beta; v0; g
  ECU(cudaStreamBeginCapture(e.s, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = [&]() -> cudaError_t {
    ECU(outer_mv(e, GASA_MV_RESIDUAL, e.X, e.Bv, e.T));
    const double *w = e.T;
    if (!e.flex) {
      ECU(apply_Mb(e, e.T, e.W));
      w = e.W;
    }
    ECU(launch_bdot(n, w, nullptr, e.part[0], K, e.s));
    ECU(launch_bnorm(e.part[0], e.beta, K, e.s));
    ECU(launch_bnormalize(n, w, e.beta, e.V, K, e.s));
    return launch_bgm_start(m, e.beta, e.g, e.sc, e.st, e.flex ? 1 : 0, dj, K, e.s);
  }();
  cudaError_t e2 = cudaStreamEndCapture(e.s, &e.g_start);
  ECU(err);
  ECU(e2);
  ECU(cudaGraphInstantiate(&e.x_start, e.g_start, 0));
  // steps: a while node whose body is one Arnoldi step at j = *dj
  ECU(cudaGraphCreate(&e.graph, 0));
  cudaGraphConditionalHandle h;
  ECU(cudaGraphConditionalHandleCreate(&h, e.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ECU(cudaGraphAddNode(&node, e.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ECU(cudaStreamBeginCaptureToGraph(e.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  err = [&]() -> cudaError_t {
    ECU(launch_bgm_load(nk, e.V, nk, dj, 0, e.Vcur, e.s));
    if (e.flex) {
      ECU(apply_Mb(e, e.Vcur, e.T));                       // z_j = M v_j
      ECU(launch_bgm_store(nk, e.T, e.Zb, nk, dj, 0, e.s));
      ECU(outer_mv(e, GASA_MV_ASSIGN, e.T, nullptr, e.W));  // w = A z_j
    } else {
      ECU(outer_mv(e, GASA_MV_ASSIGN, e.Vcur, nullptr, e.T));
      ECU(apply_Mb(e, e.T, e.W));                          // w = M A v_j
    }
    for (int pass = 0; pass < 2; ++pass) {
      ECU(launch_bmulti_dot(n, e.V, nk, m + 1, dj, e.W, e.mpart, K, e.s));
      ECU(launch_bmulti_finalize(e.mpart, m, dj, e.hbuf, e.H, pass, K, e.s));
      ECU(launch_bgs_update(n, e.V, nk, dj, e.hbuf, e.W, K, e.s));
    }
    ECU(launch_bdot(n, e.W, nullptr, e.part[1], K, e.s));
    ECU(launch_bgm_norm(e.part[1], m, dj, e.H, K, e.s));
    ECU(launch_bgm_normalize(n, e.W, e.H, m, dj, e.V, K, e.s));
    return launch_bgm_givens(m, e.H, e.cs, e.sn, e.g, e.sc, e.st, dj, h, K, e.s);
  }();
  cudaGraph_t cap = nullptr;
  e2 = cudaStreamEndCapture(e.s, &cap);
  ECU(err);
  ECU(e2);
  ECU(cudaGraphInstantiate(&e.exec, e.graph, 0));
  // end: y, x update, true residual, per-column decision
  ECU(cudaStreamBeginCapture(e.s, cudaStreamCaptureModeThreadLocal));
  err = [&]() -> cudaError_t {
    ECU(launch_bgm_backsolve(m, e.H, e.g, e.y, e.st, K, e.s));
    ECU(launch_bgm_combine(n, e.flex ? e.Zb : e.V, nk, e.y, e.st, e.X, K, e.s));
    ECU(outer_mv(e, GASA_MV_RESIDUAL, e.X, e.Bv, e.T));
    ECU(launch_bdot(n, e.T, nullptr, e.part[2], K, e.s));
    return launch_bgm_check(e.part[2], e.sc, e.st, K, e.s);
  }();
  e2 = cudaStreamEndCapture(e.s, &e.g_end);
  ECU(err);
  ECU(e2);
  return cudaGraphInstantiate(&e.x_end, e.g_end, 0);
}

void free_engine(Engine &e) {
  if (e.s) cudaStreamSynchronize(e.s);
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.x_start) cudaGraphExecDestroy(e.x_start);
  if (e.x_end) cudaGraphExecDestroy(e.x_end);
  if (e.graph) cudaGraphDestroy(e.graph);
  if (e.g_start) cudaGraphDestroy(e.g_start);
  if (e.g_end) cudaGraphDestroy(e.g_end);
  e.exec = e.x_start = e.x_end = nullptr;
  e.graph = e.g_start = e.g_end = nullptr;
  for (void *p : e.allocs) cudaFree(p);
  e.allocs.clear();
  if (e.hstage) cudaFreeHost(e.hstage);
  if (e.hsc) cudaFreeHost(e.hsc);
  if (e.hst) cudaFreeHost(e.hst);
  if (e.hctl) cudaFreeHost(e.hctl);
  e.hstage = nullptr;
  e.hsc = nullptr;
  e.hst = nullptr;
  e.hctl = nullptr;
  if (e.s) cudaStreamDestroy(e.s);
  e.s = nullptr;
}

int64_t engine_bytes(gasa_ctx *ctx, int mesh, int prec, int K, int max_iter_unused = 0) {
  (void)max_iter_unused;
  Engine e;
  e.ctx = ctx;
  e.mesh = mesh;
  e.prec = prec;
  e.K = K;
  e.gm = ctx->opt.solver != GASA_SOLVER_CG;
  e.flex = prec != GASA_PREC_FP64;
  e.m = ctx->opt.restart > 0 ? ctx->opt.restart : 30;
  e.n = ctx->L[0].ndof;
  Alloc a{&e, false};
  layout(e, a);
  return a.bytes;
}

cudaError_t create_engine(Engine &e) {
  ECU(cudaSetDevice(e.srv->device));
  // smaller meshes get higher stream priority (shortest work first): their
  // kernels are scheduled ahead of a large mesh's between its launches
  int least = 0, greatest = 0;
  ECU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  const double lg = std::log2((double)std::max<int64_t>(e.n, 1));
  int prio = greatest + std::max(0, (int)((lg - 10.0) / 2.0));
  prio = std::min(prio, least);
  ECU(cudaStreamCreateWithPriority(&e.s, cudaStreamNonBlocking, prio));
  Alloc a{&e, true};
  layout(e, a);
  e.bytes = a.bytes;
  ECU(a.status);
  ECU(cudaMallocHost((void **)&e.hstage, (size_t)e.n * sizeof(double)));
  ECU(cudaMallocHost((void **)&e.hsc, (size_t)BD_COUNT * e.K * sizeof(double)));
  ECU(cudaMallocHost((void **)&e.hst, (size_t)BI_COUNT * e.K * sizeof(int)));
  ECU(cudaMallocHost((void **)&e.hctl, 8 * sizeof(int)));
  const int64_t nk = e.n * e.K;
  // every vector starts at zero so that empty columns stay finite
  for (double *p : {e.X, e.Bv, e.T, e.R, e.Z, e.P, e.Q, e.Zold, e.W, e.Vcur})
    if (p) ECU(cudaMemsetAsync(p, 0, (size_t)nk * sizeof(double), e.s));
  if (e.V) ECU(cudaMemsetAsync(e.V, 0, (size_t)(e.m + 1) * nk * sizeof(double), e.s));
  if (e.Zb) ECU(cudaMemsetAsync(e.Zb, 0, (size_t)e.m * nk * sizeof(double), e.s));
  if (e.H) ECU(cudaMemsetAsync(e.H, 0, (size_t)(e.m + 1) * e.m * e.K * sizeof(double), e.s));
  ECU(cudaMemsetAsync(e.sc, 0, (size_t)BD_COUNT * e.K * sizeof(double), e.s));
  ECU(cudaMemsetAsync(e.st, 0, (size_t)BI_COUNT * e.K * sizeof(int), e.s));
  ECU(cudaMemsetAsync(e.ctl, 0, 8 * sizeof(int), e.s));
  std::memset(e.hst, 0, (size_t)BI_COUNT * e.K * sizeof(int));
  std::memset(e.hsc, 0, (size_t)BD_COUNT * e.K * sizeof(double));
  cudaError_t ge = e.gm ? build_gm(e) : build_cg(e);
  ECU(ge);
  ECU(cudaStreamSynchronize(e.s));
  e.slot.assign(e.K, nullptr);
  return cudaSuccess;
}

// ----------------------------------------------------------------------------
// slot traffic (engine thread only)
// ----------------------------------------------------------------------------
cudaError_t put_state(Engine &e, int c) {
  const int K = e.K;
  for (int f = 0; f < BI_COUNT; ++f)
    ECU(cudaMemcpyAsync(e.st + f * K + c, e.hst + f * K + c, sizeof(int), cudaMemcpyHostToDevice, e.s));
  return cudaSuccess;
}

cudaError_t admit(Engine &e, int c, Request *rq) {
  const int K = e.K;
  const int64_t n = e.n;
  std::memcpy(e.hstage, rq->b.data(), (size_t)n * sizeof(double));
  ECU(cudaMemcpyAsync(e.stage, e.hstage, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, e.s));
  ECU(cudaStreamSynchronize(e.s));     // the pinned stage is reused by the next admission
  ECU(launch_bscatter<double>(n, K, c, e.stage, e.Bv, e.s));
  ECU(launch_bscatter<double>(n, K, c, nullptr, e.X, e.s));
  if (!e.gm) {
    ECU(launch_bscatter<double>(n, K, c, e.stage, e.R, e.s));
    ECU(launch_bscatter<double>(n, K, c, nullptr, e.P, e.s));
    if (e.Zold) ECU(launch_bscatter<double>(n, K, c, nullptr, e.Zold, e.s));
  }
  // ||b_c|| (every column is recomputed from its own data: same bits)
  ECU(launch_bdot(n, e.Bv, nullptr, e.part[0], K, e.s));
  ECU(launch_bnorm(e.part[0], e.sc + BD_BN * K, K, e.s));
  e.hsc[BD_TOL * K + c] = rq->tol;
  ECU(cudaMemcpyAsync(e.sc + BD_TOL * K + c, e.hsc + BD_TOL * K + c, sizeof(double),
                      cudaMemcpyHostToDevice, e.s));
  e.hst[BI_STATE * K + c] = BS_RUNNING;
  e.hst[BI_FRESH * K + c] = 1;
  e.hst[BI_ITERS * K + c] = 0;
  e.hst[BI_MAXIT * K + c] = e.ctx->opt.max_iter;
  e.hst[BI_CYCLE * K + c] = 0;
  e.hst[BI_JDONE * K + c] = 0;
  ECU(put_state(e, c));
  e.slot[c] = rq;
  return cudaSuccess;
}

cudaError_t read_back(Engine &e) {
  const int K = e.K;
  ECU(cudaMemcpyAsync(e.hst, e.st, (size_t)BI_COUNT * K * sizeof(int), cudaMemcpyDeviceToHost, e.s));
  ECU(cudaMemcpyAsync(e.hsc, e.sc, (size_t)BD_COUNT * K * sizeof(double), cudaMemcpyDeviceToHost, e.s));
  return cudaStreamSynchronize(e.s);
}

// true residual norms of all columns into hsc[BD_RR]
cudaError_t true_residual(Engine &e) {
  const int K = e.K;
  ECU(outer_mv(e, GASA_MV_RESIDUAL, e.X, e.Bv, e.T));
  ECU(launch_bdot(e.n, e.T, nullptr, e.part[0], K, e.s));
  ECU(launch_bfinalize(e.part[0], e.sc + BD_RR * K, K, e.s));
  return read_back(e);
}

cudaError_t fetch_x(Engine &e, int c, Request *rq) {
  ECU(launch_bgather<double>(e.n, e.K, c, e.X, e.stage, e.s));
  ECU(cudaMemcpyAsync(e.hstage, e.stage, (size_t)e.n * sizeof(double), cudaMemcpyDeviceToHost, e.s));
  ECU(cudaStreamSynchronize(e.s));
  rq->x.assign(e.hstage, e.hstage + e.n);
  return cudaSuccess;
}

void finish(Engine &e, int c, gasa_status st, double rel) {
  Request *rq = e.slot[c];
  gasa_server *srv = e.srv;
  rq->info.iterations = e.hst[BI_ITERS * e.K + c];
  rq->info.rel_residual = rel;
  rq->info.converged = st == GASA_OK ? 1 : 0;
  rq->info.seconds = std::chrono::duration<double>(Clock::now() - rq->t0).count();
  e.slot[c] = nullptr;
  e.hst[BI_STATE * e.K + c] = BS_EMPTY;
  put_state(e, c);
  std::lock_guard<std::mutex> lk(srv->mu);
  rq->status = st;
  srv->completed += 1;
  srv->running -= 1;
  srv->cv_done.notify_all();
}

void fail_all(Engine &e, const std::string &msg) {
  gasa_server *srv = e.srv;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->err = msg;
  for (int c = 0; c < e.K; ++c) {
    if (!e.slot[c]) continue;
    e.slot[c]->status = GASA_ERR_CUDA;
    e.slot[c] = nullptr;
    srv->completed += 1;
    srv->running -= 1;
  }
  srv->cv_done.notify_all();
}

void schedule_locked(gasa_server *srv);
void engine_loop(Engine *e);

bool has_engine(gasa_server *srv, const Request *rq) {
  for (Engine *o : srv->engines)
    if (o->mesh == rq->mesh && o->prec == rq->prec && !o->retire) return true;
  return false;
}

// Handle columns that left the running state after a launch.
cudaError_t settle(Engine &e) {
  const int K = e.K;
  bool need_true = false;
  for (int c = 0; c < K; ++c)
    if (e.slot[c] && e.hst[BI_STATE * K + c] != BS_RUNNING) need_true = true;
  if (!need_true) return cudaSuccess;
  if (!e.gm) ECU(true_residual(e));     // GMRES: the cycle's end already holds it
  for (int c = 0; c < K; ++c) {
    Request *rq = e.slot[c];
    if (!rq) continue;
    const int s = e.hst[BI_STATE * K + c];
    if (s == BS_RUNNING) continue;
    const double bn = e.hsc[BD_BN * K + c];
    const double tn = std::sqrt(e.hsc[BD_RR * K + c]);
    const double rel = bn > 0.0 ? tn / bn : 0.0;
    if (s == BS_CONVERGED) {
      if (tn <= rq->tol * bn) {     // the device's test, in the same form
        ECU(fetch_x(e, c, rq));
        finish(e, c, GASA_OK, rel);
      } else {
        // the recurrence residual passed but the true one did not: restart
        // from the true residual
        if (!e.gm) ECU(launch_bcolcopy(e.n, K, c, e.T, e.R, e.s));
        e.hst[BI_STATE * K + c] = BS_RUNNING;
        e.hst[BI_FRESH * K + c] = 1;
        ECU(put_state(e, c));
      }
    } else if (s == BS_MAXIT) {
      ECU(fetch_x(e, c, rq));
      finish(e, c, GASA_ERR_NOT_CONVERGED, rel);
    } else {
      finish(e, c, s == BS_NOT_SPD ? GASA_ERR_NOT_SPD : GASA_ERR_BREAKDOWN, rel);
    }
  }
  return cudaSuccess;
}

void engine_loop(Engine *ep) {
  Engine &e = *ep;
  gasa_server *srv = e.srv;
  cudaSetDevice(srv->device);
  const int K = e.K;
  for (;;) {
    // admit queued requests of this engine into free slots
    std::vector<std::pair<int, Request *>> fresh;
    int active = 0;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      for (;;) {
        if (srv->stopping || e.retire) break;
        for (int c = 0; c < K; ++c) {
          if (e.slot[c]) continue;
          bool taken = false;
          for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
            Request *rq = *it;
            if (rq->mesh == e.mesh && rq->prec == e.prec) {
              srv->queue.erase(it);
              e.slot[c] = rq;
              fresh.push_back({c, rq});
              srv->running += 1;
              taken = true;
              break;
            }
            // first come, first served: a request ahead in the queue that
            // waits for memory stops admissions here, so this engine drains
            // and can give its memory back
            if (!has_engine(srv, rq)) break;
          }
          if (!taken) break;
        }
        srv->peak_running = std::max(srv->peak_running, srv->running);
        active = 0;
        for (int c = 0; c < K; ++c) active += e.slot[c] ? 1 : 0;
        if (active) break;
        // idle: release the engine if a queued request needs the memory
        // (one engine at a time, so that no more than needed is released)
        bool blocked = false;
        for (Request *rq : srv->queue)
          if (!has_engine(srv, rq)) blocked = true;
        if (blocked && srv->retiring == 0) {
          e.retire = true;
          srv->retiring += 1;
          break;
        }
        e.cv.wait(lk);
      }
      if (srv->stopping) break;
      if (e.retire && !active) break;
    }
    cudaError_t err = cudaSuccess;
    for (auto &f : fresh) {
      err = admit(e, f.first, f.second);
      if (err != cudaSuccess) break;
    }
    if (err == cudaSuccess) {
      // between launches new requests may join: keep launches short while
      // slots are free and requests could arrive, long when the batch is full
      int free_slots = 0;
      for (int c = 0; c < K; ++c) free_slots += e.slot[c] ? 0 : 1;
      e.hctl[0] = 0;
      e.hctl[1] = free_slots ? 8 : (1 << 30);
      e.hctl[2] = 0;
      err = cudaMemcpyAsync(e.ctl, e.hctl, 3 * sizeof(int), cudaMemcpyHostToDevice, e.s);
    }
    if (err == cudaSuccess) {
      if (e.gm) {
        err = cudaGraphLaunch(e.x_start, e.s);
        if (err == cudaSuccess) err = cudaGraphLaunch(e.exec, e.s);
        if (err == cudaSuccess) err = cudaGraphLaunch(e.x_end, e.s);
        srv->graph_launches += 3;
      } else {
        err = cudaGraphLaunch(e.exec, e.s);
        srv->graph_launches += 1;
      }
    }
    if (err == cudaSuccess) err = read_back(e);
    if (err == cudaSuccess) err = settle(e);
    if (err != cudaSuccess) {
      fail_all(e, std::string("server engine: ") + cudaGetErrorString(err));
      std::lock_guard<std::mutex> lk(srv->mu);
      if (!e.retire) srv->retiring += 1;
      e.retire = true;
      break;
    }
  }
  // leave: free memory, give the room back, let the scheduler use it
  free_engine(e);
  std::lock_guard<std::mutex> lk(srv->mu);
  for (int c = 0; c < K; ++c) {
    if (!e.slot[c]) continue;
    e.slot[c]->status = GASA_ERR_STATE;
    srv->completed += 1;
    srv->running -= 1;
    e.slot[c] = nullptr;
  }
  srv->used -= e.bytes;
  srv->released += 1;
  if (e.retire) srv->retiring -= 1;
  srv->engines.erase(std::find(srv->engines.begin(), srv->engines.end(), ep));
  srv->retired.push_back(ep);
  if (!srv->stopping) schedule_locked(srv);
  srv->cv_done.notify_all();
}

// Create engines for queued requests that have none, in queue order, while
// the budget allows; stop at the first request whose engine does not fit.
void schedule_locked(gasa_server *srv) {
  for (Request *rq : srv->queue) {
    bool has = false;
    for (Engine *o : srv->engines)
      if (o->mesh == rq->mesh && o->prec == rq->prec && !o->retire) {
        has = true;
        o->cv.notify_one();
      }
    if (has) continue;
    if (srv->retiring) break;        // wait until the leaving engine has freed its memory
    gasa_ctx *ctx = srv->meshes[rq->mesh].ctx;
    int K = srv->max_batch;
    int64_t need = 0;
    for (; K >= 1; K /= 2) {
      need = engine_bytes(ctx, rq->mesh, rq->prec, K);
      if (srv->used + need <= srv->budget) break;
    }
    if (K < 1) {
      // first come, first served: nothing behind a waiting request starts.
      // Wake idle engines: they release themselves while requests wait.
      for (Engine *o : srv->engines) o->cv.notify_one();
      break;
    }
    Engine *e = new Engine();
    e->srv = srv;
    e->ctx = ctx;
    e->mesh = rq->mesh;
    e->prec = rq->prec;
    e->K = K;
    e->gm = ctx->opt.solver != GASA_SOLVER_CG;
    e->flex = rq->prec != GASA_PREC_FP64;
    e->m = ctx->opt.restart > 0 ? ctx->opt.restart : 30;
    e->n = ctx->L[0].ndof;
    cudaError_t err = create_engine(*e);
    if (err != cudaSuccess) {
      srv->err = std::string("server engine creation: ") + cudaGetErrorString(err);
      free_engine(*e);
      delete e;
      (void)cudaGetLastError();
      continue;
    }
    srv->used += e->bytes;
    srv->peak = std::max(srv->peak, srv->used);
    srv->created += 1;
    srv->engines.push_back(e);
    e->th = std::thread(engine_loop, e);
  }
}

void join_retired(gasa_server *srv, std::unique_lock<std::mutex> &lk) {
  std::vector<Engine *> r;
  r.swap(srv->retired);
  lk.unlock();
  for (Engine *e : r) {
    if (e->th.joinable()) e->th.join();
    delete e;
  }
  lk.lock();
}

}  // namespace

extern "C" {

gasa_status gasa_server_create(gasa_server **out, int32_t device, int64_t budget, int32_t max_batch) {
  if (!out || budget <= 0 || !(max_batch == 1 || max_batch == 2 || max_batch == 4 || max_batch == 8))
    return GASA_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return GASA_ERR_CUDA;
  }
  gasa_server *srv = new gasa_server();
  srv->device = device;
  srv->budget = budget;
  srv->max_batch = max_batch;
  *out = srv;
  return GASA_OK;
}

gasa_status gasa_server_add_mesh(gasa_server *srv, gasa_ctx *ctx, int32_t *mesh_id) {
  if (!srv || !ctx || !mesh_id) return GASA_ERR_INVALID_ARG;
  if (!ctx->ready) return GASA_ERR_STATE;
  if (ctx->device != srv->device) return GASA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->used + ctx->device_bytes > srv->budget) {
    srv->err = "hierarchy does not fit in the server's budget";
    return GASA_ERR_BUDGET;
  }
  srv->used += ctx->device_bytes;
  srv->peak = std::max(srv->peak, srv->used);
  srv->meshes.push_back({ctx, ctx->device_bytes});
  *mesh_id = (int32_t)srv->meshes.size() - 1;
  return GASA_OK;
}

gasa_status gasa_server_submit(gasa_server *srv, int32_t mesh_id, const double *b, double tol,
                               int32_t precision, uint64_t *ticket) {
  if (!srv || !b || !ticket || !(tol > 0.0)) return GASA_ERR_INVALID_ARG;
  if (precision < GASA_PREC_FP64 || precision > GASA_PREC_MIXED16) return GASA_ERR_INVALID_ARG;
  Request *rq = new Request();
  gasa_ctx *ctx = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (mesh_id < 0 || mesh_id >= (int)srv->meshes.size()) {
      delete rq;
      return GASA_ERR_INVALID_ARG;
    }
    if (srv->stopping) {
      delete rq;
      return GASA_ERR_STATE;
    }
    ctx = srv->meshes[mesh_id].ctx;
    // a request whose single-slot engine cannot fit beside the resident
    // hierarchies would wait forever
    int64_t resident = 0;
    for (const MeshEntry &m : srv->meshes) resident += m.bytes;
    if (resident + engine_bytes(ctx, mesh_id, precision, 1) > srv->budget) {
      delete rq;
      srv->err = "the request's engine does not fit in the server's budget";
      return GASA_ERR_BUDGET;
    }
  }
  const int64_t n = ctx->L[0].ndof;
  rq->b.assign(b, b + n);
  rq->mesh = mesh_id;
  rq->prec = precision;
  rq->tol = tol;
  rq->t0 = Clock::now();
  std::unique_lock<std::mutex> lk(srv->mu);
  rq->ticket = srv->next_ticket++;
  srv->tickets[rq->ticket] = rq;
  srv->submitted += 1;
  // a zero right-hand side is solved by x = 0 at once
  double bb = 0.0;
  for (int64_t i = 0; i < n; ++i) bb += b[i] * b[i];
  if (bb == 0.0) {
    rq->x.assign(n, 0.0);
    rq->status = GASA_OK;
    rq->info.converged = 1;
    srv->completed += 1;
    *ticket = rq->ticket;
    return GASA_OK;
  }
  srv->queue.push_back(rq);
  schedule_locked(srv);
  join_retired(srv, lk);
  *ticket = rq->ticket;
  return GASA_OK;
}

gasa_status gasa_server_poll(gasa_server *srv, uint64_t ticket, double *x_out, gasa_solve_info *info) {
  if (!srv) return GASA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) return GASA_ERR_INVALID_ARG;
  Request *rq = it->second;
  if (rq->status == GASA_PENDING) return GASA_PENDING;
  if (x_out && !rq->x.empty()) std::memcpy(x_out, rq->x.data(), rq->x.size() * sizeof(double));
  if (info) *info = rq->info;
  const gasa_status st = rq->status;
  srv->tickets.erase(it);
  delete rq;
  join_retired(srv, lk);
  return st;
}

gasa_status gasa_server_drain(gasa_server *srv, double timeout_s) {
  if (!srv) return GASA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(timeout_s));
  while (srv->completed < srv->submitted) {
    if (srv->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
        srv->completed < srv->submitted)
      return GASA_ERR_TIMEOUT;
  }
  join_retired(srv, lk);
  return GASA_OK;
}

gasa_status gasa_server_stats_read(gasa_server *srv, gasa_server_stats *out) {
  if (!srv || !out) return GASA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->queued = (int64_t)srv->queue.size();
  out->running = srv->running;
  out->engines = (int64_t)srv->engines.size();
  out->engines_created = srv->created;
  out->engines_released = srv->released;
  out->budget_bytes = srv->budget;
  out->used_bytes = srv->used;
  out->peak_bytes = srv->peak;
  out->peak_running = srv->peak_running;
  out->graph_launches = srv->graph_launches.load();
  return GASA_OK;
}

gasa_status gasa_server_destroy(gasa_server *srv) {
  if (!srv) return GASA_OK;
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->stopping = true;
  for (Engine *e : srv->engines) e->cv.notify_all();
  // engines finish their current launch, then leave
  while (!srv->engines.empty()) {
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
    lk.lock();
    for (Engine *e : srv->engines) e->cv.notify_all();
  }
  join_retired(srv, lk);
  for (Request *rq : srv->queue) rq->status = GASA_ERR_STATE;
  srv->queue.clear();
  for (auto &kv : srv->tickets) delete kv.second;
  srv->tickets.clear();
  lk.unlock();
  delete srv;
  return GASA_OK;
}

const char *gasa_server_last_error(const gasa_server *srv) {
  return srv ? srv->err.c_str() : "null server";
}

}  // extern "C"
