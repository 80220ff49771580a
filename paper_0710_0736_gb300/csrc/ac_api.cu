// ac_api.cu -- the C ABI of libac (include/ac.h) and the host-side driver of
// the time step (Sec. 3.2 of Kay & Tomasi): colour means and right-hand side,
// then truncated monotone multigrid V-cycles until the natural residual
// reaches tol.  The cycle is described at solve_mg; the mixed-precision form
// wraps an FP32 solve in a defect correction on the FP64 state (solve_mixed).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/ac.h"
#include "ac_device.cuh"
#include "ac_ops.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define AC_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(AC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

const ac::Ops *ops_for(int N) {
  switch (N) {
    case 2: return ac::ops_n2();
    case 3: return ac::ops_n3();
    case 4: return ac::ops_n4();
    case 5: return ac::ops_n5();
    case 6: return ac::ops_n6();
    case 7: return ac::ops_n7();
    case 8: return ac::ops_n8();
    default: return nullptr;
  }
}

bool pixel_exists(int W, int H, int px, int py) { return px >= 0 && px < W && py >= 0 && py < H; }

// Geometry of a W x H level: lumped mass and diagonal of S per node class
// (see ac_device.cuh for the class numbering).
ac::Geo make_geo(int W, int H, double te) {
  ac::Geo g{};
  g.W = W;
  g.H = H;
  g.Wn = W + 1;
  g.te = te;
  const int xs[3] = {0, 1, W}, ys[3] = {0, 1, H};
  for (int cy = 0; cy < 3; ++cy)
    for (int cx = 0; cx < 3; ++cx) {
      const int x = xs[cx], y = ys[cy];
      const int cnt = 2 * pixel_exists(W, H, x, y) + pixel_exists(W, H, x - 1, y) + pixel_exists(W, H, x, y - 1) +
                      2 * pixel_exists(W, H, x - 1, y - 1);
      const double m0 = cnt / 6.0;
      const double vy = 0.5 * ((y < H) + (y > 0)), vx = 0.5 * ((x < W) + (x > 0));
      const double wsum = (x < W ? vy : 0) + (x > 0 ? vy : 0) + (y < H ? vx : 0) + (y > 0 ? vx : 0);
      const int k = cy * 3 + cx;
      g.m0[k] = m0;
      g.D[k] = m0 + te * wsum;
      g.invD[k] = g.D[k] > 0 ? 1.0 / g.D[k] : 0.0;
    }
  g.half = ((int64_t)(W + 1) * (H + 1) + 1) / 2;
  g.tef = (float)g.te;
  g.teh = (float)g.te;
  g.tel = (float)(g.te - (double)g.teh);
  for (int k = 0; k < 9; ++k) {
    g.Df[k] = (float)g.D[k];
    g.invDf[k] = (float)g.invD[k];
    g.m0h[k] = (float)g.m0[k];
    g.m0l[k] = (float)(g.m0[k] - (double)g.m0h[k]);
  }
  return g;
}

// Node slots of a fine-level array (FP32 arrays are split by colour, see
// ac::fslot: two halves of (n + 1) / 2 slots).
int64_t fine_slots(int64_t n) { return 2 * ((n + 1) / 2); }

struct Level {
  ac::Geo g;
  int64_t n = 0;
  void *op = nullptr, *r = nullptr, *v = nullptr, *t = nullptr;  // coarse levels only
  ac::LevelLists lists{};  // live-tile flags and work lists (coarse levels; used while the level is tiled)
};

// Bytes of a level's live flags: one per (kJ2X x kJ2Y tile, phase).
size_t tile_flag_bytes(const ac::Geo &g, int N) { return (size_t)ac::tiles_x(g) * ac::tiles_y(g) * N; }


// Untruncated entries of P'SP on the first coarse level, one representative
// coarse node per boundary class.
ac::Galerkin0Table galerkin0_table(const ac::Geo &gf, const ac::Geo &gc) {
  ac::Galerkin0Table t{};
  const int lx[4] = {0, 1, 0, 1}, ly[4] = {0, 0, 1, 1};
  bool seen[25] = {};
  for (int Y = 0; Y <= gc.H; ++Y) {
    if (Y > 2 && Y < gc.H - 2) continue;  // rows of class 2 are all alike
    for (int X = 0; X <= gc.W; ++X) {
      if (X > 2 && X < gc.W - 2) continue;
      const int c = ac::g0_class(Y, gc.H) * 5 + ac::g0_class(X, gc.W);
      if (seen[c]) continue;
      seen[c] = true;
      for (int l = 0; l < 4; ++l) {
        t.v[c][l] = ac::galerkin0_entry(gf, gc, X, Y, lx[l], ly[l], [](int, int) { return true; });
        t.vf[c][l] = (float)t.v[c][l];
      }
    }
  }
  return t;
}

// A captured CUDA graph of a fixed launch sequence, with the launches and
// (when captured while profiling) the event pairs it records per class.
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  int64_t launches[AC_PROF_COUNT] = {};
  double bytes[AC_PROF_COUNT] = {};  // algorithmic HBM bytes of the launches per class
  int64_t total = 0;
  struct Ev {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Ev> evs;
};

// Device-side control of a time step's V-cycle loop (capture_step): the
// loop's state lives here, in device memory, and small one-thread kernels
// update it after each residual and set the conditions of the graph's WHILE
// nodes, so that a whole time step runs as one graph launch with no host
// round trip per cycle.  The same decisions as solve_mg / solve_mixed.
struct LoopCtl {
  // the multigrid solve in progress (the inner FP32 solve in AC_MIXED)
  double tol;        // its tolerance
  double rho_inner;  // its last natural residual
  int cyc, cap;      // its cycles so far and its cycle limit
  int inner_status;  // 0 converged, 1 not converged, 2 non-finite residual
  // the time step in progress
  double rho;        // the step's last natural residual (the outer one in AC_MIXED)
  int cycles, outer, status;
  int zero_x;        // AC_MIXED: the next correction starts from zero
  int warm;          // AC_MIXED: sv.x holds the last step's converged correction
  long long sweeps;
  // summed over the steps since the last k_ctl_reset
  long long total_cycles, total_sweeps, total_outer;
  double last_rho;
  int last_cycles, steps, nonconv, numeric;
};

// A captured time step with the device-side loop: its kernel launches per
// replay are fixed + passes x per_pass + (cycles - solves) x per_cycle.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t fixed = 0, per_pass = 0, per_cycle = 0;
};

// One multigrid solve: min_x sum_i 1/2 x_i'S x_i - rhs_i'x_i over the
// constraint set of the instantiation (see ac_kernels.cuh).
struct Solve {
  const ac::SolverOps *o = nullptr;
  int *list_counts = nullptr;  // the tiled levels' list counts, two per level (cleared by one memset per cycle)
  void *x = nullptr, *rhs = nullptr, *ob = nullptr, *rt = nullptr, *d = nullptr;
  uint8_t *mask = nullptr;
  std::vector<Level> lv;  // lv[0]: fine level geometry
  int depth = 0;          // levels in use (<= lv.size()); a schedule can cut the hierarchy short
  ac::Galerkin0Table tab0{};
  // graphs [profiling][variant]: smoothing + residual of the first / a later
  // cycle, and the coarse correction with its line search [profiling][form:
  // dense levels / tiled levels with live flags and work lists]
  GraphSlot smooth_resid[2][2], correction[2][2];
  // the form of the next coarse correction: tiled while few fine nodes are
  // free (its kernels then skip the dead tiles), dense otherwise (when most
  // tiles are live the work lists cost more than they skip); was_tiled: the
  // last correction ran tiled, so the flags describe its tiles
  bool tiled = false, was_tiled = false;
  int tiling = AC_TILES_AUTO;  // ac_set_coarse_tiling
  bool coarse_gs = true;       // ac_set_coarse_smoother: 3-colour Gauss-Seidel (else l1-Jacobi)
};

// A coarse correction runs tiled when fewer than this fraction of the fine
// nodes have a free phase (about 45% of the first level's tiles are then
// live at 4096^2, N = 8, where both forms take the same time).
constexpr double kTiledFreeFraction = 0.25;

// Pre/post l1-Jacobi sweeps on coarse levels (even); a build option
// (-DAC_COARSE_SWEEPS=k) for tuning.
#ifndef AC_COARSE_SWEEPS
#define AC_COARSE_SWEEPS 2
#endif
constexpr int kCoarseSweeps = AC_COARSE_SWEEPS;
static_assert(kCoarseSweeps >= 2 && kCoarseSweeps % 2 == 0, "coarse sweeps: an even count >= 2");
constexpr int kCoarsestSweeps = 20;  // sweeps of the one-block coarsest solve
constexpr int64_t kCoarsestBlockNodes = 1 << 14;
// AC_MIXED: inner FP32 solve to max(0.9 tol, 1e-5 rho_outer) ...  The inner
// natural residual and the outer one agree to about 0.1% at tol 1e-6 (float
// rounding of S delta against rho), so 0.9 tol still passes the outer check
// in one pass; tol/2 cost 0.4 V-cycles per step more at 4096^2, N=8.
constexpr double kInnerTolFrac = 0.9;
constexpr double kInnerReduction = 1e-5;
constexpr int kInnerMaxCycles = 40;       // ... or at most this many V-cycles per defect-correction pass
// AC_MIXED checks convergence with the natural residual computed in float on
// r = b - S u taken in FP64 and shifted per node by max_i r_i before rounding.
// The shifted z = r/S_nn is <= 0 with maximum 0; near the solution the free
// components' z and the projection's theta are O(rho) and a component on its
// bound has u_i <= rho, so the float projection is exact to a few float ulps
// of rho (about (N + 4) 2^-24 rho <= 7e-7 rho): accepting rho32 <= tol (1 -
// kRho32Rel) keeps a 14x margin at any tol.
constexpr double kRho32Rel = 1e-5;

}  // namespace

// Adjoint bookkeeping (ac_adjoint_forward / ac_adjoint_backward).
struct AdjState {
  bool ready = false;
  int T = 0, every = 0, ncp = 0;
  double *cp_u = nullptr;   // checkpoints: u at steps 0, every, 2 every, ... (ncp x n x N)
  double *cp_c = nullptr;   // the means entering those steps (ncp x N x 3)
  double *uT = nullptr;     // u after the last step (n x N)
  double *seg_u = nullptr;  // recomputed states of one segment ((every + 1) x n x N)
  double *seg_c = nullptr;  // c^t of the segment's steps (every x N x 3)
  double *seg_M = nullptr;  // masses M^t of the segment's steps (every x N)
  double *g = nullptr, *g2 = nullptr;  // dL/du (n x N)
  double *gm = nullptr;     // dL/dm1 (RGB), dL/dm2 per node (n x 4)
  double *part = nullptr, *tot = nullptr, *scal = nullptr;
  double *kw = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr, *kq_prev = nullptr;  // flexible CG vectors
  double *kpart = nullptr, *ktot = nullptr;  // its dot products
  double *gimg = nullptr;   // dL/dI on the refined grid (refine > 0)
  unsigned long long *ndiff = nullptr;  // components where a recomputed segment end differed from the forward
  int64_t recompute_diff = 0;           // its value after the last backward pass
  Solve sv;                 // FP64 tangent-form solve
  Solve sv32;               // its FP32 copy: the preconditioner of the FCG (ac_set_adjoint_preconditioner)
  std::vector<void *> allocs;
};

struct ac_ctx {
  ac_params p{};          // the solve's parameters (on the refined grid when refine > 0)
  int r = 0;              // refinements of the pixel grid
  int W0 = 0, H0 = 0;     // the image size in pixels
  void *img_up = nullptr; // device image copied onto the refined grid (refine > 0)
  size_t img_up_bytes = 0;
  int8_t *lab = nullptr;  // device staging of labels for host copies (nodes of the solve grid)
  int N = 0;
  int64_t n = 0;
  int sms = 1;  // multiprocessors of the device
  const ac::Ops *ops = nullptr;
  cudaStream_t s = nullptr;
  ac::Geo g0{};
  Solve sv;                                    // the multigrid solve of this precision
  bool delta_warm = false;  // AC_MIXED: sv.x holds the last step's converged single correction
  double *u = nullptr, *b = nullptr, *mom = nullptr;
  float *r32 = nullptr, *u32 = nullptr;        // AC_MIXED: FP32 right-hand side and obstacle
  double *part = nullptr, *tot = nullptr, *c = nullptr, *c_tmp = nullptr, *energy = nullptr;
  double *rho = nullptr, *omega = nullptr, *ls_part = nullptr, *ls_tot = nullptr;
  void *img = nullptr;  // device copy of a host image (allocated on demand)
  size_t img_bytes = 0;
  __nv_bfloat16 *img16 = nullptr;  // AC_MIXED: the image stored in bfloat16
  double *img64 = nullptr;         // the image as the moments used it, FP64 (for the adjoint)
  AdjState adj;
  bool adj_pre32 = true;           // the adjoint's FCG preconditioned by the FP32 V-cycle (else FP64)
  double *h_scalars = nullptr;     // pinned: rho, energy
  bool have_image = false, have_rhs = false;
  std::vector<void *> allocs;
  // instrumentation
  int64_t total_launches = 0;
  bool profiling = false;
  unsigned prof_mask = (1u << AC_PROF_COUNT) - 1u;  // classes bracketed by events while profiling
  unsigned prof_graph_mask = (1u << AC_PROF_COUNT) - 1u;  // the mask the profiled graphs were captured with
  struct Pending {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Pending> pending;
  double prof_ms[AC_PROF_COUNT] = {};
  int64_t prof_launches[AC_PROF_COUNT] = {};
  double prof_bytes[AC_PROF_COUNT] = {};
  int64_t prof_corr_launches = 0;  // smoother launches that applied a pending correction
  // CUDA graphs (off on the legacy default stream, which cannot be captured)
  bool use_graphs = false;
  GraphSlot *capturing = nullptr;
  // the device-side cycle loop (ac_set_cycle_loop): its control block (and a
  // pinned copy for the read-back), two streams on which the bodies of the
  // WHILE nodes are captured, and the captured steps [energy of the step]
  int loop_mode = AC_LOOP_AUTO;
  LoopCtl *ctl = nullptr, *h_ctl = nullptr;
  cudaStream_t body_s[2] = {nullptr, nullptr};
  StepGraph step_graph[2];
};

namespace {

// Algorithmic HBM bytes of the solve's kernels, for the profile: every array
// element a launch is defined on, read once and written once (dense: the
// coarse kernels' skipping of rows with a zero diagonal is not credited, so
// their DRAM traffic can be lower).  ns = N values of one node of a level in
// the solve's scalar type (N * elem bytes).
struct ByteModel {
  double ns;   // N * sizeof(scalar)
  double ob;   // 1 when the fine level has an obstacle array (shifted and tangent forms)
  double n;    // fine nodes
  // one launch of the fine smoother (one colour): the colour's rhs (and
  // obstacle) and the other colour's iterate read, the colour's iterate written
  double smooth_launch() const { return 0.5 * n * ns * (3 + ob); }
};

ByteModel byte_model(const ac_ctx *ctx, const Solve &S) {
  ByteModel b;
  b.ns = (double)ctx->N * S.o->elem;
  b.ob = S.ob ? 1.0 : 0.0;
  b.n = (double)S.lv[0].n;
  return b;
}

int dev_alloc(ac_ctx *ctx, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AC_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->allocs.push_back(*p);
  return AC_OK;
}

#define AC_ALLOC(ptr, bytes)                                              \
  do {                                                                    \
    int rc_ = dev_alloc(ctx, reinterpret_cast<void **>(&(ptr)), (bytes)); \
    if (rc_) return rc_;                                                  \
  } while (0)

int validate(const ac_params *p) {
  if (!p) return fail(AC_ERR_ARG, "params is NULL");
  if (p->width < 1 || p->height < 1) return fail(AC_ERR_ARG, "image size must be >= 1x1");
  if (p->refine < 0 || p->refine > 4) return fail(AC_ERR_ARG, "refine must be in [0, 4]");
  const int64_t Wr = (int64_t)p->width << p->refine, Hr = (int64_t)p->height << p->refine;
  if ((Wr + 1) * (Hr + 1) > (int64_t)1 << 31)
    return fail(AC_ERR_ARG, "image too large (more than 2^31 nodes on the solve grid)");
  if (Hr + 1 > 65535) return fail(AC_ERR_ARG, "solve grid height must be below 65535 (one grid row per node row)");
  if (p->n_phases < 2 || p->n_phases > AC_MAX_PHASES)
    return fail(AC_ERR_ARG, "n_phases must be in [2, %d]", AC_MAX_PHASES);
  if (!(p->eps > 0) || !std::isfinite(p->eps)) return fail(AC_ERR_ARG, "eps must be > 0");
  if (!(p->tau > 0) || !std::isfinite(p->tau)) return fail(AC_ERR_ARG, "tau must be > 0");
  if (!(p->lambda >= 0) || !std::isfinite(p->lambda)) return fail(AC_ERR_ARG, "lambda must be >= 0");
  if (!(p->tol > 0)) return fail(AC_ERR_ARG, "tol must be > 0");
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1)
    return fail(AC_ERR_ARG, "need nu1, nu2 >= 0 and nu1 + nu2 >= 1");
  if (p->max_cycles < 1) return fail(AC_ERR_ARG, "max_cycles must be >= 1");
  if (p->coarse_min < 1) return fail(AC_ERR_ARG, "coarse_min must be >= 1");
  if (p->precision != AC_FP64 && p->precision != AC_MIXED)
    return fail(AC_ERR_ARG, "precision must be AC_FP64 or AC_MIXED");
  if (p->projection != AC_PROJ_SIMPLEX && p->projection != AC_PROJ_NODE)
    return fail(AC_ERR_ARG, "projection must be AC_PROJ_SIMPLEX or AC_PROJ_NODE");
  return AC_OK;
}

// ---- instrumentation --------------------------------------------------------

// Sum the finished event pairs into the profile and recycle the events.
int prof_harvest(ac_ctx *ctx) {
  if (ctx->pending.empty()) return AC_OK;
  AC_CUDA(cudaStreamSynchronize(ctx->s));
  for (const auto &p : ctx->pending) {
    float ms = 0.f;
    AC_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    ctx->prof_ms[p.cls] += ms;
  }
  ctx->pending.clear();
  ctx->ev_used = 0;
  return AC_OK;
}

int prof_event(ac_ctx *ctx, cudaEvent_t *e) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t ev;
    AC_CUDA(cudaEventCreate(&ev));
    ctx->ev_pool.push_back(ev);
  }
  *e = ctx->ev_pool[ctx->ev_used++];
  return AC_OK;
}

// Run one launcher call: count its kernels and their algorithmic HBM bytes
// (`bytes`, the caller's count of what the launches must read and write),
// check the launch, and bracket it with events on the context's stream while
// profiling.  While a graph is being captured the launches, bytes and event
// pairs are booked to that graph (and counted each time it is replayed)
// instead.
template <class F>
int timed(ac_ctx *ctx, int cls, double bytes, F &&f) {
  cudaEvent_t a = nullptr, b = nullptr;
  GraphSlot *cap = ctx->capturing;
  const bool ev = ctx->profiling && ((ctx->prof_mask >> cls) & 1u);
  if (ev) {
    if (cap) {
      AC_CUDA(cudaEventCreate(&a));
      cap->evs.push_back({a, nullptr, cls});
      AC_CUDA(cudaEventCreate(&b));
      cap->evs.back().b = b;
      AC_CUDA(cudaEventRecordWithFlags(a, ctx->s, cudaEventRecordExternal));
    } else {
      if (ctx->pending.size() >= (1u << 15)) {
        int rc = prof_harvest(ctx);
        if (rc) return rc;
      }
      int rc = prof_event(ctx, &a);
      if (!rc) rc = prof_event(ctx, &b);
      if (rc) return rc;
      AC_CUDA(cudaEventRecord(a, ctx->s));
    }
  }
  const int k = f();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  if (cap) {
    cap->total += k;
    cap->launches[cls] += k;
    cap->bytes[cls] += bytes;
    if (ev) AC_CUDA(cudaEventRecordWithFlags(b, ctx->s, cudaEventRecordExternal));
    return AC_OK;
  }
  ctx->total_launches += k;
  if (ctx->profiling) {
    ctx->prof_launches[cls] += k;
    ctx->prof_bytes[cls] += bytes;
    if (ev) {
      AC_CUDA(cudaEventRecord(b, ctx->s));
      ctx->pending.push_back({a, b, cls});
    }
  }
  return AC_OK;
}

void slot_release(GraphSlot &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto &e : g.evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g = GraphSlot{};
}

// Run `enqueue` (a fixed launch sequence on ctx->s) through the graph in
// `slot`: captured on first use, replayed afterwards.  Without graphs the
// sequence is launched directly.
template <class F>
int run_graph(ac_ctx *ctx, GraphSlot &slot, F &&enqueue) {
  if (!ctx->use_graphs) return enqueue();
  if (!slot.exec) {
    AC_CUDA(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeRelaxed));
    ctx->capturing = &slot;
    int rc = enqueue();
    ctx->capturing = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      slot_release(slot);
      return rc;
    }
    if (e != cudaSuccess) {
      slot_release(slot);
      return fail(AC_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&slot.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      slot.exec = nullptr;
      slot_release(slot);
      return fail(AC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
  }
  AC_CUDA(cudaGraphLaunch(slot.exec, ctx->s));
  ctx->total_launches += slot.total;
  if (ctx->profiling) {
    for (int k = 0; k < AC_PROF_COUNT; ++k) {
      ctx->prof_launches[k] += slot.launches[k];
      ctx->prof_bytes[k] += slot.bytes[k];
    }
    for (const auto &ev : slot.evs) ctx->pending.push_back({ev.a, ev.b, ev.cls});
  }
  return AC_OK;
}

#define AC_RUN(cls, expr)                                       \
  do {                                                          \
    int rc_ = timed(ctx, (cls), 0.0, [&]() { return (expr); }); \
    if (rc_) return rc_;                                        \
  } while (0)

// The same, booking `bytes` algorithmic HBM bytes to the class.
#define AC_RUNB(cls, bytes, expr)                                       \
  do {                                                                  \
    int rc_ = timed(ctx, (cls), (double)(bytes), [&]() { return (expr); }); \
    if (rc_) return rc_;                                                \
  } while (0)

// Reads rho back (the one device-to-host dependency of a cycle), and the
// count of free nodes that the fine residual stores beside it (*nfree,
// nullable).  While profiling, the finished event pairs are summed here: the
// graphs re-record their events on every replay.
int read_rho(ac_ctx *ctx, double *out, int64_t *nfree = nullptr) {
  AC_CUDA(cudaMemcpyAsync(ctx->h_scalars, ctx->rho, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  AC_CUDA(cudaStreamSynchronize(ctx->s));
  *out = ctx->h_scalars[0];
  if (nfree) {
    unsigned long long c = 0;
    std::memcpy(&c, ctx->h_scalars + 1, sizeof c);
    *nfree = (int64_t)c;
  }
  if (ctx->profiling) return prof_harvest(ctx);
  return AC_OK;
}

// ---- multigrid ---------------------------------------------------------------

// Linear V-cycle for S_k v_k = r_k on coarse levels k >= 1 (operators already
// built), zero initial guess.  Smoothing runs in fused pairs of l1-Jacobi
// sweeps that cannot work in place, so a level's two buffers v and t swap
// roles: *res returns the one that holds v_k.
// First level k0 >= 1 from which the rest of the hierarchy (operators and
// the k0 iterate, right-hand side and residual, kTailArrays values per node)
// fits in one block's shared memory: below it the whole cycle is one launch
// of k_coarse_tail.  S.depth when none does.
int tail_level(const Solve &S, size_t *smem) {
  size_t bytes = 0;
  int k0 = S.depth;
  for (int k = S.depth - 1; k >= 1; --k) {
    const size_t b = bytes + (size_t)ac::kTailArrays * (size_t)S.lv[k].n * (size_t)S.o->elem;
    if (b > ac::kTailSmemBytes || S.depth - k > ac::kTailMaxLevels) break;
    bytes = b;
    k0 = k;
  }
  *smem = bytes;
  return k0;
}

// The coarse levels worked tile by tile with live flags and work lists (see
// kLiveNow): levels above the one-launch tail and above the coarsest that
// have at least kTiledMinItems (tile, phase) items per multiprocessor (on
// smaller levels the lists' bookkeeping costs more than the dead tiles
// they skip).  They form a prefix 1 .. k1 - 1 of the hierarchy; the others
// stay dense.
constexpr int64_t kTiledMinItems = 32;
int tiled_end(const Solve &S) {
  size_t smem = 0;
  const int k0 = tail_level(S, &smem);
  int k1 = k0 < S.depth - 1 ? k0 : S.depth - 1;
  if (S.tiling == AC_TILES_NEVER) return 1;
  if (S.tiling == AC_TILES_ALWAYS) return k1;
  for (int k = 1; k < k1; ++k)
    if (S.lv[k].lists.cap < kTiledMinItems * S.lv[k].lists.sms) {
      k1 = k;
      break;
    }
  return k1;
}

const ac::LevelLists *level_lists(Solve &S, int k) {
  return (S.tiled && k >= 1 && k < tiled_end(S)) ? &S.lv[k].lists : nullptr;
}

int coarse_vcycle(ac_ctx *ctx, Solve &S, int k, void **res) {
  Level &L = S.lv[k];
  const ac::SolverOps *o = S.o;
  const ac::LevelLists *const tf = level_lists(S, k), *const tfc = level_lists(S, k + 1);
  // level arrays: the operator is 4 values (C, E, N, NE) per node and phase,
  // r, v, t one; pair = one fused pair of l1-Jacobi sweeps from v (7 values:
  // operator, r and v read, the result written), from zero 6
  const double ns = (double)ctx->N * o->elem, lk = (double)L.n * ns;
  const double pair = 7 * lk, pair0 = 6 * lk;
  size_t smem = 0;
  if (k == tail_level(S, &smem)) {
    ac::TailArgs a{};
    a.levels = S.depth - k;
    double ops = 0;
    for (int l = 0; l < a.levels; ++l) {
      a.W[l] = S.lv[k + l].g.W;
      a.H[l] = S.lv[k + l].g.H;
      a.op[l] = S.lv[k + l].op;
      ops += 4.0 * (double)S.lv[k + l].n * ns;
    }
    AC_RUNB(AC_PROF_COARSE, ops + 2 * lk, o->coarse_tail(a, L.r, L.v, kCoarseSweeps, kCoarsestSweeps, smem, S.coarse_gs, ctx->s));
    *res = L.v;
    return AC_OK;
  }
  if (k == S.depth - 1) {
    if (L.n <= kCoarsestBlockNodes) {
      AC_CUDA(cudaMemsetAsync(L.v, 0, (size_t)L.n * ctx->N * o->elem, ctx->s));
      AC_RUNB(AC_PROF_COARSE, 6 * lk, o->coarse_solve(L.op, L.r, L.v, L.g, kCoarsestSweeps, ctx->s));
      *res = L.v;
    } else {
      AC_RUNB(AC_PROF_COARSE, pair0 + (kCoarseSweeps - 1) * pair,
              o->coarse_smooth(L.op, L.r, L.v, L.t, L.g, 2 * kCoarseSweeps, true, res, nullptr, S.coarse_gs, ctx->s));
    }
    return AC_OK;
  }
  Level &C = S.lv[k + 1];
  const double lc = (double)C.n * ns;
  // v starts at 0: the first pair of sweeps writes every node without reading v
  void *v = nullptr, *other = nullptr;
  if (kCoarseSweeps == 2) {
    // float: one launch reads the operator and r and writes v and t; double:
    // the pair, then the residual (operator, r, v read, t written)
    AC_RUNB(AC_PROF_COARSE, o->elem == 4 ? 7 * lk : pair0 + 7 * lk,
            o->coarse_pre_resid(L.op, L.r, L.v, L.t, L.g, tf, S.coarse_gs, ctx->s));
    v = L.v;
    other = L.t;
  } else {
    AC_RUNB(AC_PROF_COARSE, pair0 + (kCoarseSweeps / 2 - 1) * pair,
            o->coarse_smooth(L.op, L.r, L.v, L.t, L.g, kCoarseSweeps, true, &v, tf, S.coarse_gs, ctx->s));
    other = v == L.v ? L.t : L.v;
    AC_RUNB(AC_PROF_COARSE, 7 * lk, o->coarse_resid(L.op, L.r, v, L.g, other, tf, ctx->s));
  }
  // restriction: t read, the coarse diagonal read, r written
  AC_RUNB(AC_PROF_TRANSFER, lk + 2 * lc, o->restrict_(other, L.g, C.g, C.op, C.r, tfc, ctx->s));
  void *cv = nullptr;
  int rc = coarse_vcycle(ctx, S, k + 1, &cv);
  if (rc) return rc;
  // prolongation: coarse v and this level's diagonal read, v read and written
  AC_RUNB(AC_PROF_TRANSFER, lc + 3 * lk, o->prolong_add(cv, L.g, C.g, L.op, v, tf, ctx->s));
  AC_RUNB(AC_PROF_COARSE, (kCoarseSweeps / 2) * pair,
          o->coarse_smooth(L.op, L.r, v, other, L.g, kCoarseSweeps, false, res, tf, S.coarse_gs, ctx->s));
  return AC_OK;
}

// The two fixed launch sequences of a cycle, on ctx->s (captured into the
// graphs of solve_mg, or into the bodies of the device-side loop of
// capture_step).
//
// Smoothing and residual: nu1 red-black sweeps in the first cycle (`later`
// false), nu2 + nu1 and the pending coarse correction in a later one; then
// r = rhs - S x, rho and the free-node count (zeroed first), the mask and
// the tangent residual.
int enqueue_smooth_resid(ac_ctx *ctx, Solve &S, bool later) {
  const ac::SolverOps *o = S.o;
  const ac::Geo &g0 = S.lv[0].g;
  const ByteModel bm = byte_model(ctx, S);
  const int nsw = later ? ctx->p.nu1 + ctx->p.nu2 : ctx->p.nu1;
  const void *corr = (later && S.depth > 1) ? S.d : nullptr;
  // after at least one sweep the last pass completes its colour's mask
  // (its tangent residual is 0), and the residual kernel visits the other
  // colour only.  Those rt slots hold zeros: cleared at allocation and
  // written by nothing else unless nu1 = 0 lets a first cycle take the
  // every-node residual, in which case the last pass re-zeroes them.
  const bool fused = nsw >= 1;
  void *rt_zero = (fused && ctx->p.nu1 == 0) ? S.rt : nullptr;
  // 2 nsw colour passes; the first also reads the other colour's pending
  // correction; the last writes its colour's mask (and rt = 0)
  const double sm_bytes = 2.0 * nsw * bm.smooth_launch() + (corr && nsw > 0 ? 0.5 * bm.n * bm.ns : 0.0) +
                          (fused ? 0.5 * bm.n * (1.0 + (rt_zero ? bm.ns : 0.0)) : 0.0);
  // mask changes mark the first coarse level's tiles (whatever its form)
  const ac::MaskDirty dirty = S.lv.size() > 1
                                  ? ac::MaskDirty{S.lv[1].lists.dirty, ac::tiles_x(S.lv[1].g), ac::tiles_y(S.lv[1].g)}
                                  : ac::MaskDirty{nullptr, 0, 0};
  AC_RUNB(AC_PROF_SMOOTH, sm_bytes, o->smooth(S.x, S.rhs, S.ob, corr, ctx->omega, g0, nsw, rt_zero,
                                              fused ? S.mask : nullptr, dirty, ctx->s));
  AC_CUDA(cudaMemsetAsync(ctx->rho, 0, 2 * sizeof(double), ctx->s));  // rho and the free-node count
  // residual at the visited nodes: x (their own and, for one colour, the
  // other colour's as neighbours), rhs, obstacle read, rt and the mask
  // byte written
  const double rs_bytes = fused ? 0.5 * bm.n * (bm.ns * (4 + bm.ob) + 1) : bm.n * (bm.ns * (3 + bm.ob) + 1);
  AC_RUNB(AC_PROF_RESID, rs_bytes,
          o->resid(S.x, S.rhs, S.ob, g0, S.rt, S.mask, ctx->rho, fused ? 0 : -1, dirty, ctx->s));
  return AC_OK;
}

// The coarse correction in the form S.tiled selects: truncated Galerkin
// operators, restriction, the coarse V-cycle, the feasible direction and its
// exact line search (omega; applied by the next smoothing pass).
int enqueue_correction(ac_ctx *ctx, Solve &S) {
  const ac::SolverOps *o = S.o;
  const ac::Geo &g0 = S.lv[0].g;
  const ByteModel bm = byte_model(ctx, S);
  Level &L1 = S.lv[1];
  const double l1 = (double)L1.n * bm.ns;
  // first-level operator from the fine mask; each coarser one from the
  // level above (4 values per node and phase read and written)
  // the tiled levels' work lists are rebuilt by their Galerkin kernels
  if (tiled_end(S) > 1) AC_CUDA(cudaMemsetAsync(S.list_counts, 0, 2 * S.lv.size() * sizeof(int), ctx->s));
  AC_RUNB(AC_PROF_TRANSFER, bm.n + 4 * l1,
          o->galerkin0(S.mask, g0, L1.g, S.tab0, L1.op, level_lists(S, 1), L1.lists.dirty, ctx->s));
  for (int k = 1; k + 1 < S.depth; ++k)
    AC_RUNB(AC_PROF_TRANSFER, 4.0 * (double)(S.lv[k].n + S.lv[k + 1].n) * bm.ns,
            o->galerkin(S.lv[k].op, S.lv[k].g, S.lv[k + 1].g, S.lv[k + 1].op, level_lists(S, k), level_lists(S, k + 1),
                        ctx->s));
  // rt read, the first level's diagonal read and its r written
  AC_RUNB(AC_PROF_TRANSFER, bm.n * bm.ns + 2 * l1,
          o->restrict0(S.rt, g0, L1.g, L1.op, L1.r, level_lists(S, 1), ctx->s));
  void *v1 = nullptr;
  int rc = coarse_vcycle(ctx, S, 1, &v1);
  if (rc) return rc;
  // direction: x, obstacle, rt, mask and the first level's v read, d
  // written; curvature: d and the mask read
  const double ls_bytes = bm.n * (bm.ns * (3 + bm.ob) + 1) + l1 + bm.n * (bm.ns + 1);
  AC_RUNB(AC_PROF_LINESEARCH, ls_bytes,
          o->line_search(S.x, S.ob, S.rt, v1, S.mask, g0, L1.g, S.d, ctx->ls_part, ctx->ls_tot, ctx->omega, ctx->s));
  return AC_OK;
}

// Multigrid solve of one step problem.  Cycle structure:
//   smooth (nu1 red-black projected sweeps; nu2 + nu1 after a correction)
//   -> residual r = rhs - S x, natural residual rho, free-phase mask, tangent
//      projection of r; stop if rho <= tol
//   -> truncated Galerkin operators and restriction, linear V-cycle on the
//      coarse levels
//   -> feasible coarse-correction direction and exact line search.
// Every stage keeps x feasible and does not raise the step energy, so the
// limit is the unique minimiser that plain projected Gauss-Seidel (the
// smoother alone) reaches.
int solve_mg(ac_ctx *ctx, Solve &S, double tol, int max_cycles, int *cycles_out, double *rho_out,
             int64_t *sweeps_out) {
  const bool coarse = S.depth > 1;
  double rho = 0;
  int cyc = 0, status = AC_ERR_NOT_CONVERGED;
  int64_t sweeps = 0;
  const int prof = ctx->profiling ? 1 : 0;
  for (;;) {
    const int later = cyc > 0 ? 1 : 0;  // nu1 + nu2 sweeps, and the pending coarse correction if any
    const int nsw = later ? ctx->p.nu1 + ctx->p.nu2 : ctx->p.nu1;
    int rc = run_graph(ctx, S.smooth_resid[prof][later], [&]() { return enqueue_smooth_resid(ctx, S, later); });
    if (rc) return rc;
    if (ctx->profiling && later && coarse && nsw > 0) ++ctx->prof_corr_launches;
    sweeps += nsw;
    ++cyc;
    int64_t nfree = 0;
    rc = read_rho(ctx, &rho, &nfree);
    if (rc) return rc;
#ifdef AC_TRACE_CYCLES
    {  // build option: one line per cycle (rho, the omega the cycle applied, free nodes, form)
      double om[2] = {0, 0};
      cudaMemcpy(om, ctx->omega, sizeof om, cudaMemcpyDeviceToHost);
      std::fprintf(stderr, "cycle %d rho %.3e omega %.4f free %lld tiled %d elem %d\n", cyc, rho, later ? om[0] : 0.0,
                   (long long)nfree, S.tiled ? 1 : 0, S.o->elem);
    }
#endif
    if (std::isnan(rho) || std::isinf(rho)) {
      status = fail(AC_ERR_NUMERIC, "non-finite residual");
      break;
    }
    if (rho <= tol) {
      status = AC_OK;
      break;
    }
    if (cyc >= max_cycles) break;
    if (!coarse) continue;
    // the coarse correction's form from the free nodes (only one colour is
    // counted after a smoothing sequence: about half of them)
    const double free_frac = (double)nfree * (nsw >= 1 ? 2.0 : 1.0) / (double)S.lv[0].n;
    S.tiled = tiled_end(S) > 1 && (S.tiling == AC_TILES_ALWAYS || free_frac < kTiledFreeFraction);
    if (S.tiled && !S.was_tiled) {
      // the flags are stale: let this correction compute and write every
      // tile (kLiveNow), whatever the mask changes since the last one
      for (int k = 1; k < tiled_end(S); ++k) {
        AC_CUDA(cudaMemsetAsync(S.lv[k].lists.flags, ac::kLiveNow, tile_flag_bytes(S.lv[k].g, ctx->N), ctx->s));
        AC_CUDA(cudaMemsetAsync(S.lv[k].lists.dirty, 1, tile_flag_bytes(S.lv[k].g, 1), ctx->s));
      }
    }
    S.was_tiled = S.tiled;
    rc = run_graph(ctx, S.correction[prof][S.tiled ? 1 : 0], [&]() { return enqueue_correction(ctx, S); });
    if (rc) return rc;
  }
  *cycles_out = cyc;
  *rho_out = rho;
  *sweeps_out = sweeps;
  if (status == AC_ERR_NOT_CONVERGED)
    fail(status, "step did not reach tol %.3g in %d cycles (rho %.3g)", tol, cyc, rho);
  return status;
}

// AC_MIXED: defect correction on the FP64 state around the FP32 multigrid.
// Each pass forms r = b - S u in double-float arithmetic (k_outer_resid_df,
// about 2^-46 of the terms) and the natural residual; if rho > tol the
// correction problem min 1/2 d'Sd - r'd, u + d on the simplices, is solved in
// FP32 to max(0.9 tol, 1e-5 rho) or kInnerMaxCycles V-cycles (FP32 keeps the
// correction's own relative precision, except for components driven onto
// their bound, whose precision is that of u; the next pass removes that) and
// u <- P_G(u + d) in FP64.
int solve_mixed(ac_ctx *ctx, int *cycles_out, double *rho_out, int64_t *sweeps_out, int *outer_out) {
  const ac::Ops *o = ctx->ops;
  double rho = 0;
  int cycles = 0, outer = 0, status = AC_ERR_NOT_CONVERGED;
  int64_t sweeps = 0;
  const bool rho32 = true;
  const double accept = ctx->p.tol * (1.0 - kRho32Rel);
  for (;;) {
    AC_CUDA(cudaMemsetAsync(ctx->rho, 0, sizeof(double), ctx->s));
    // u (binary64) and b (double-float pairs) read, r32 and u32 written
    AC_RUNB(AC_PROF_OUTER, (double)ctx->n * ctx->N * 24,
            o->outer_resid(ctx->u, (const float *)ctx->b, ctx->g0, ctx->r32, ctx->u32, ctx->rho, rho32, ctx->s));
    int rc = read_rho(ctx, &rho);
    if (rc) return rc;
#ifdef AC_TRACE_CYCLES
    std::fprintf(stderr, "outer %d rho %.3e\n", outer, rho);
#endif
    if (std::isnan(rho) || std::isinf(rho)) {
      status = fail(AC_ERR_NUMERIC, "non-finite residual");
      break;
    }
    if (rho <= accept) {
      status = AC_OK;
      break;
    }
    if (cycles >= ctx->p.max_cycles) break;
    // The first correction of a step starts from the previous step's
    // converged correction (u^t - u^(t-1) in float): the step's minimiser is
    // unique, so the start only changes the V-cycle count (7.8 against 8.1
    // per step at 4096^2, N=8).  The first smoothing sweep makes it feasible
    // for the new obstacle, so it needs nu1 >= 1; a later correction of the
    // same step starts from zero.
    const bool warm = outer == 0 && ctx->delta_warm && ctx->p.nu1 >= 1;
    ctx->delta_warm = false;
    if (!warm) AC_CUDA(cudaMemsetAsync(ctx->sv.x, 0, (size_t)fine_slots(ctx->n) * ctx->N * sizeof(float), ctx->s));
    int c = 0;
    int64_t sw = 0;
    double rin = 0;
    const int cap = ctx->p.max_cycles - cycles < kInnerMaxCycles ? ctx->p.max_cycles - cycles : kInnerMaxCycles;
    rc = solve_mg(ctx, ctx->sv, std::fmax(kInnerTolFrac * ctx->p.tol, kInnerReduction * rho), cap, &c, &rin, &sw);
    cycles += c;
    sweeps += sw;
    if (rc && rc != AC_ERR_NOT_CONVERGED) return rc;
    // u read and written, delta read
    AC_RUNB(AC_PROF_OUTER, (double)ctx->n * ctx->N * 20,
            o->outer_update(ctx->u, (const float *)ctx->sv.x, ctx->g0, ctx->s));
    ++outer;
    ctx->delta_warm = rc == AC_OK && outer == 1;
  }
  *cycles_out = cycles;
  *rho_out = rho;
  *sweeps_out = sweeps;
  *outer_out = outer;
  if (status == AC_ERR_NOT_CONVERGED)
    fail(status, "step did not reach tol %.3g in %d cycles (rho %.3g)", ctx->p.tol, cycles, rho);
  return status;
}

// ---- device-side cycle loop ------------------------------------------------
// A time step captured as one graph: the V-cycles of solve_mg and the
// defect-correction passes of solve_mixed run under WHILE nodes whose
// conditions one-thread kernels set from the residual on the device (the
// same tests in the same order as the host loops), so a step needs no host
// round trip per cycle.  The launches are those of the host loops with the
// same arguments, so the results are bit-identical.  Used when the context
// has graphs, profiling is off (event records cannot sit in a conditional
// body) and no coarse level can run tiled (the tiled/dense choice per cycle
// stays on the host).

__global__ void k_ctl_reset(LoopCtl *c, int warm) {
  c->total_cycles = 0;
  c->total_sweeps = 0;
  c->total_outer = 0;
  c->last_rho = 0.0;
  c->last_cycles = 0;
  c->steps = 0;
  c->nonconv = 0;
  c->numeric = 0;
  c->warm = warm;
}

__global__ void k_ctl_step_begin(LoopCtl *c, double tol, int cap) {
  c->cycles = 0;
  c->outer = 0;
  c->sweeps = 0;
  c->status = 1;
  c->rho = 0.0;
  c->tol = tol;
  c->cap = cap;
  c->cyc = 0;
  c->inner_status = 1;
}

// After a cycle's residual (solve_mg): stop on a non-finite rho, on rho <=
// tol, or at the cycle limit; otherwise run another cycle.
__global__ void k_ctl_cycle(LoopCtl *c, const double *rho, int nsw, cudaGraphConditionalHandle h) {
  c->cyc += 1;
  c->cycles += 1;
  c->sweeps += nsw;
  const double r = rho[0];
  c->rho_inner = r;
  unsigned go = 0;
  if (isnan(r) || isinf(r)) {
    c->inner_status = 2;
  } else if (r <= c->tol) {
    c->inner_status = 0;
  } else {
    c->inner_status = 1;
    go = c->cyc < c->cap ? 1u : 0u;
  }
  cudaGraphSetConditional(h, go);
}

// After the outer residual (solve_mixed): stop on a non-finite rho, on rho <=
// accept, or when the step's cycles reached max_cycles; otherwise set up the
// next inner solve (its tolerance, its cycle limit, and whether its
// correction starts from the previous step's).
__global__ void k_ctl_outer(LoopCtl *c, const double *rho, double accept, double tol, double tol_frac,
                            double reduction, int max_cycles, int inner_max, int nu1, cudaGraphConditionalHandle h) {
  const double r = rho[0];
  c->rho = r;
  unsigned go = 0;
  if (isnan(r) || isinf(r)) {
    c->status = 2;
  } else if (r <= accept) {
    c->status = 0;
  } else if (c->cycles >= max_cycles) {
    c->status = 1;
  } else {
    go = 1;
    c->status = 1;
    c->tol = fmax(tol_frac * tol, reduction * r);
    const int left = max_cycles - c->cycles;
    c->cap = left < inner_max ? left : inner_max;
    c->cyc = 0;
    const int warm = c->outer == 0 && c->warm && nu1 >= 1;
    c->warm = 0;
    c->zero_x = !warm;
  }
  cudaGraphSetConditional(h, go);
}

// The correction's start: zero unless k_ctl_outer chose the warm start.
__global__ void k_zero_unless_warm(const LoopCtl *c, float *x, int64_t count) {
  if (!c->zero_x) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    x[k] = 0.0f;
}

__global__ void k_ctl_after_update(LoopCtl *c) {
  c->outer += 1;
  c->warm = c->inner_status == 0 && c->outer == 1;
}

__global__ void k_ctl_step_end(LoopCtl *c, int fp64) {
  if (fp64) {
    c->rho = c->rho_inner;
    c->status = c->inner_status;
  }
  c->total_cycles += c->cycles;
  c->total_sweeps += c->sweeps;
  c->total_outer += c->outer;
  c->last_rho = c->rho;
  c->last_cycles = c->cycles;
  c->steps += 1;
  if (c->status == 1)
    c->nonconv += 1;
  else if (c->status == 2)
    c->numeric += 1;
}

// End a capture begun on s, if any, after a failure.  A body's graph belongs
// to its conditional node and is not destroyed here.
void end_capture_quiet(cudaStream_t s, bool destroy) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (s && cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (destroy && g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

// Append a WHILE node on h to the graph being captured on s, after the work
// captured there so far, and begin capturing its body on `body`.
int begin_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaStream_t body) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  AC_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return fail(AC_ERR_CUDA, "begin_while: the stream is not capturing");
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  AC_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  AC_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  AC_CUDA(cudaStreamBeginCaptureToGraph(body, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed));
  return AC_OK;
}

int end_body(cudaStream_t body) {
  cudaGraph_t g = nullptr;
  AC_CUDA(cudaStreamEndCapture(body, &g));
  return AC_OK;
}

// The control block, its pinned read-back copy and the body streams.
int loop_resources(ac_ctx *ctx) {
  if (!ctx->ctl) {
    void *p = nullptr;
    int rc = dev_alloc(ctx, &p, sizeof(LoopCtl));
    if (rc) return rc;
    ctx->ctl = (LoopCtl *)p;
    AC_CUDA(cudaMemsetAsync(ctx->ctl, 0, sizeof(LoopCtl), ctx->s));
  }
  if (!ctx->h_ctl) AC_CUDA(cudaMallocHost(&ctx->h_ctl, sizeof(LoopCtl)));
  for (auto &bs : ctx->body_s)
    if (!bs) AC_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  return AC_OK;
}

void release_step_graphs(ac_ctx *ctx) {
  for (auto &sg : ctx->step_graph) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    sg = StepGraph{};
  }
}

// Whether ac_step runs the device-side loop (see above).
bool loop_on_device(const ac_ctx *ctx) {
  return ctx->loop_mode == AC_LOOP_AUTO && ctx->use_graphs && !ctx->profiling && tiled_end(ctx->sv) <= 1;
}

// Enqueue one time step with the device-side loop on ctx->s, which is
// capturing into `top`: k_ctl_step_begin, the colour means (and the energy)
// and the right-hand side as in ac_step, then
//   AC_FP64:  smooth+resid, k_ctl_cycle, WHILE { correction, smooth+resid, k_ctl_cycle }
//   AC_MIXED: outer resid, k_ctl_outer, WHILE { start of the correction, the
//             inner solve as above, update, k_ctl_after_update, outer resid, k_ctl_outer }
// and k_ctl_step_end.  sg receives the launches of each part.
int enqueue_step_loop(ac_ctx *ctx, cudaGraph_t top, bool energy, StepGraph &sg) {
  Solve &S = ctx->sv;
  const bool mixed = ctx->p.precision == AC_MIXED, coarse = S.depth > 1;
  const ac::Ops *o = ctx->ops;
  const double a1 = 1.0 + 2.0 * ctx->p.tau / ctx->p.eps, tl = ctx->p.tau * ctx->p.lambda;
  const double mean_bytes = (double)ctx->n * (8.0 * ctx->N + 32), rhs_bytes = mean_bytes + (double)ctx->n * 8.0 * ctx->N;
  cudaGraphConditionalHandle h_cyc = 0, h_out = 0;
  AC_CUDA(cudaGraphConditionalHandleCreate(&h_cyc, top, 0, 0));
  if (mixed) AC_CUDA(cudaGraphConditionalHandleCreate(&h_out, top, 0, 0));
  GraphSlot cnt_fixed, cnt_pass, cnt_cycle;  // launch counters only
  cudaStream_t const top_s = ctx->s;
  GraphSlot *const saved = ctx->capturing;
  // on every exit: back to the top stream and the caller's capture slot;
  // after a failure, end the bodies' captures
  struct Guard {
    ac_ctx *ctx;
    cudaStream_t s;
    GraphSlot *cap;
    bool ok = false;
    ~Guard() {
      if (!ok)
        for (int d = 1; d >= 0; --d) end_capture_quiet(ctx->body_s[d], false);
      ctx->s = s;
      ctx->capturing = cap;
    }
  } guard{ctx, top_s, saved};
  ctx->capturing = &cnt_fixed;
  AC_RUN(AC_PROF_SETUP, (k_ctl_step_begin<<<1, 1, 0, ctx->s>>>(ctx->ctl, ctx->p.tol, ctx->p.max_cycles), 1));
  double *en = energy ? ctx->energy : nullptr;
  if (mixed) {
    AC_RUNB(AC_PROF_SETUP, mean_bytes,
            o->means_df(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c, en, ctx->p.eps, ctx->p.lambda, ctx->s));
    AC_RUNB(AC_PROF_SETUP, rhs_bytes, o->rhs_df(ctx->u, ctx->mom, ctx->c, ctx->g0, a1, tl, (float *)ctx->b, ctx->s));
  } else {
    AC_RUNB(AC_PROF_SETUP, mean_bytes,
            o->means(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c, en, ctx->p.eps, ctx->p.lambda, ctx->s));
    AC_RUNB(AC_PROF_SETUP, rhs_bytes, o->rhs(ctx->u, ctx->mom, ctx->c, ctx->g0, a1, tl, ctx->b, ctx->s));
  }
  // one multigrid solve; its cycles' body is captured on body_s[d]
  auto solve = [&](int d) -> int {
    int rc = enqueue_smooth_resid(ctx, S, false);
    if (rc) return rc;
    AC_RUN(AC_PROF_RESID, (k_ctl_cycle<<<1, 1, 0, ctx->s>>>(ctx->ctl, ctx->rho, ctx->p.nu1, h_cyc), 1));
    rc = begin_while(ctx->s, h_cyc, ctx->body_s[d]);
    if (rc) return rc;
    cudaStream_t const outer_s = ctx->s;
    GraphSlot *const outer_cnt = ctx->capturing;
    ctx->s = ctx->body_s[d];
    ctx->capturing = &cnt_cycle;
    if (coarse) rc = enqueue_correction(ctx, S);
    if (!rc) rc = enqueue_smooth_resid(ctx, S, true);
    if (rc) return rc;
    AC_RUN(AC_PROF_RESID,
           (k_ctl_cycle<<<1, 1, 0, ctx->s>>>(ctx->ctl, ctx->rho, ctx->p.nu1 + ctx->p.nu2, h_cyc), 1));
    rc = end_body(ctx->s);
    if (rc) return rc;
    ctx->s = outer_s;
    ctx->capturing = outer_cnt;
    return AC_OK;
  };
  int rc = AC_OK;
  if (!mixed) {
    rc = solve(0);
    if (rc) return rc;
  } else {
    const double accept = ctx->p.tol * (1.0 - kRho32Rel);
    auto outer_resid = [&]() -> int {
      AC_CUDA(cudaMemsetAsync(ctx->rho, 0, sizeof(double), ctx->s));
      AC_RUNB(AC_PROF_OUTER, (double)ctx->n * ctx->N * 24,
              o->outer_resid(ctx->u, (const float *)ctx->b, ctx->g0, ctx->r32, ctx->u32, ctx->rho, true, ctx->s));
      AC_RUN(AC_PROF_OUTER,
             (k_ctl_outer<<<1, 1, 0, ctx->s>>>(ctx->ctl, ctx->rho, accept, ctx->p.tol, kInnerTolFrac, kInnerReduction,
                                               ctx->p.max_cycles, kInnerMaxCycles, ctx->p.nu1, h_out),
              1));
      return AC_OK;
    };
    rc = outer_resid();
    if (rc) return rc;
    rc = begin_while(ctx->s, h_out, ctx->body_s[0]);
    if (rc) return rc;
    ctx->s = ctx->body_s[0];
    ctx->capturing = &cnt_pass;
    const int64_t xs = fine_slots(ctx->n) * ctx->N;
    AC_RUN(AC_PROF_OUTER, (k_zero_unless_warm<<<(unsigned)std::min<int64_t>((xs + 255) / 256, 8 * ctx->sms), 256, 0,
                                                ctx->s>>>(ctx->ctl, (float *)S.x, xs),
                           1));
    rc = solve(1);
    if (rc) return rc;
    AC_RUNB(AC_PROF_OUTER, (double)ctx->n * ctx->N * 20,
            o->outer_update(ctx->u, (const float *)S.x, ctx->g0, ctx->s));
    AC_RUN(AC_PROF_OUTER, (k_ctl_after_update<<<1, 1, 0, ctx->s>>>(ctx->ctl), 1));
    rc = outer_resid();
    if (rc) return rc;
    rc = end_body(ctx->s);
    if (rc) return rc;
    ctx->s = top_s;
    ctx->capturing = &cnt_fixed;
  }
  AC_RUN(AC_PROF_SETUP, (k_ctl_step_end<<<1, 1, 0, ctx->s>>>(ctx->ctl, mixed ? 0 : 1), 1));
  sg.fixed = cnt_fixed.total;
  sg.per_pass = cnt_pass.total;
  sg.per_cycle = cnt_cycle.total;
  guard.ok = true;
  return AC_OK;
}

// Capture (once) the step graph with or without the energy.
int capture_step(ac_ctx *ctx, bool energy) {
  StepGraph &sg = ctx->step_graph[energy ? 1 : 0];
  if (sg.exec) return AC_OK;
  int rc = loop_resources(ctx);
  if (rc) return rc;
  AC_CUDA(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeRelaxed));
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaGraph_t top = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(ctx->s, &st, nullptr, &top, nullptr, nullptr, nullptr);
  rc = e == cudaSuccess ? enqueue_step_loop(ctx, top, energy, sg)
                        : fail(AC_ERR_CUDA, "cudaStreamGetCaptureInfo: %s", cudaGetErrorString(e));
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->s, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    sg = StepGraph{};
    return rc ? rc : fail(AC_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&sg.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    sg = StepGraph{};
    return fail(AC_ERR_CUDA, "cudaGraphInstantiate (step): %s", cudaGetErrorString(e));
  }
  return AC_OK;
}

// Statistics of the steps since the last k_ctl_reset from the read-back
// control block; books the launches (sg: the counts of the step graph) and
// returns the call's status.
int loop_stats(ac_ctx *ctx, const StepGraph &sg, int n_steps, ac_stats *out) {
  const LoopCtl &c = *ctx->h_ctl;
  const bool mixed = ctx->p.precision == AC_MIXED;
  const int64_t solves = mixed ? c.total_outer : c.steps;
  ctx->total_launches += 1 + (int64_t)n_steps * sg.fixed + c.total_outer * sg.per_pass +
                         (c.total_cycles - solves) * sg.per_cycle;
  ctx->delta_warm = c.warm != 0;
  ctx->have_rhs = true;
  if (out) {
    out->residual = c.last_rho;
    out->cycles = c.last_cycles;
    out->total_cycles = (int)c.total_cycles;
    out->steps = n_steps;
    out->converged = (c.nonconv == 0 && c.numeric == 0) ? 1 : 0;
    out->fine_sweeps = c.total_sweeps;
    out->outer = mixed ? (int)c.total_outer : 0;
  }
  if (c.numeric) return fail(AC_ERR_NUMERIC, "non-finite residual");
  if (c.nonconv)
    return fail(AC_ERR_NOT_CONVERGED, "%d of %d steps did not reach tol %.3g (last rho %.3g)", c.nonconv, n_steps,
                ctx->p.tol, c.last_rho);
  return AC_OK;
}

// ac_step with the device-side loop: one graph launch per time step and one
// synchronisation per call.
int step_device(ac_ctx *ctx, int n_steps, ac_stats *out) {
  AC_CUDA((k_ctl_reset<<<1, 1, 0, ctx->s>>>(ctx->ctl, ctx->delta_warm ? 1 : 0), cudaGetLastError()));
  for (int t = 0; t < n_steps; ++t)
    AC_CUDA(cudaGraphLaunch(ctx->step_graph[(out && t == n_steps - 1) ? 1 : 0].exec, ctx->s));
  AC_CUDA(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, ctx->s));
  if (out) AC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 1, ctx->energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  AC_CUDA(cudaStreamSynchronize(ctx->s));
  ac_stats st{};
  int rc = loop_stats(ctx, ctx->step_graph[0], n_steps, &st);
  if (out) {
    st.energy = std::ldexp(ctx->h_scalars[1], -ctx->r);  // pixel units: E = 2^-r E(eps', lambda')
    *out = st;
  }
  return rc;
}

// Device staging for labels copied to the host: (W+1)(H+1) bytes of the
// solve grid, enough for node and pixel labels.
int label_stage(ac_ctx *ctx, int8_t **out) {
  if (!ctx->lab) {
    cudaError_t e = cudaMalloc(&ctx->lab, (size_t)ctx->n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->lab = nullptr;
      return fail(AC_ERR_NOMEM, "cudaMalloc for the label staging: %s", cudaGetErrorString(e));
    }
  }
  *out = ctx->lab;
  return AC_OK;
}

int copy_out(ac_ctx *ctx, void *dst, const void *src, size_t bytes, int is_device) {
  AC_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->s));
  if (!is_device) AC_CUDA(cudaStreamSynchronize(ctx->s));
  return AC_OK;
}

// Refined image by copy: cell (x, y) of the solve grid takes pixel
// (x >> r, y >> r) of the W0-wide input (3 channels).
template <typename TI>
__global__ void k_refine_copy(const TI *__restrict__ in, int W0, int r, ac::Geo g, TI *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.W) return;
  const TI *p = in + ((int64_t)(y >> r) * W0 + (x >> r)) * 3;
  TI *o = out + ((int64_t)y * g.W + x) * 3;
  o[0] = p[0];
  o[1] = p[1];
  o[2] = p[2];
}

// Adjoint of the copy: pixel (x, y) of the W0-wide image collects the
// gradients of its 2^r x 2^r cells of the refined grid (3 channels).
__global__ void k_refine_sum(const double *__restrict__ fine, int W0, int H0, int r, ac::Geo g,
                             double *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W0 || y >= H0) return;
  double s[3] = {0.0, 0.0, 0.0};
  const int side = 1 << r;
  for (int b = 0; b < side; ++b)
    for (int a = 0; a < side; ++a) {
      const double *p = fine + ((int64_t)((y << r) + b) * g.W + ((x << r) + a)) * 3;
      s[0] += p[0];
      s[1] += p[1];
      s[2] += p[2];
    }
  double *o = out + ((int64_t)y * W0 + x) * 3;
  o[0] = s[0];
  o[1] = s[1];
  o[2] = s[2];
}

template <typename TI>
__global__ void k_img_f64(const TI *__restrict__ in, double *__restrict__ out, int64_t count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) {
    if constexpr (std::is_same<TI, __nv_bfloat16>::value)
      out[k] = (double)__bfloat162float(in[k]);
    else
      out[k] = (double)in[k];
  }
}

__global__ void k_to_bf16(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) out[k] = __float2bfloat16_rn(in[k]);
}

__global__ void k_moments_bf16(const __nv_bfloat16 *__restrict__ img, ac::Geo g, double *__restrict__ mom) {
  // same sums as k_moments, reading the bfloat16 image
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x > g.W || y > g.H) return;
  double s[3] = {0, 0, 0}, s2 = 0;
  const int px[4] = {x, x - 1, x, x - 1};
  const int py[4] = {y, y - 1, y - 1, y};
  const double w[4] = {2.0, 2.0, 1.0, 1.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (px[k] < 0 || px[k] >= g.W || py[k] < 0 || py[k] >= g.H) continue;
    const __nv_bfloat16 *p = img + ((int64_t)py[k] * g.W + px[k]) * 3;
    const double r = (double)__bfloat162float(p[0]), gg = (double)__bfloat162float(p[1]),
                 bb = (double)__bfloat162float(p[2]);
    s[0] += w[k] * r;
    s[1] += w[k] * gg;
    s[2] += w[k] * bb;
    s2 += w[k] * (r * r + gg * gg + bb * bb);
  }
  double *m = mom + ((int64_t)y * g.Wn + x) * 4;
  m[0] = s[0] / 6.0;
  m[1] = s[1] / 6.0;
  m[2] = s[2] / 6.0;
  m[3] = s2 / 6.0;
}

// ---- data projection by node (Sec. 4.2) ------------------------------------
// One image value per node, I_n = pixel (min(x, W-1), min(y, H-1)) (a copy of
// a neighbouring pixel, never an interpolated value), and the standard mass
// matrix M_nm = <eta_n, eta_m>.  On the right-diagonal triangulation a
// triangle of area 1/2 contributes (1 + delta_ab)/24 to M_ab, so M is a
// 7-point stencil: M_nn = (incident triangles)/12 = Mhat_n / 2, and an edge
// to E, W, N, S, NE or SW carries (triangles sharing it)/24.  The axis edges
// are shared by 2 vy (E, W) and 2 vx (N, S) triangles -- twice the stiffness
// edge weights of edge_weights -- and a diagonal by the two triangles of its
// pixel.

__device__ __forceinline__ double img_value(float v) { return (double)v; }
__device__ __forceinline__ double img_value(double v) { return v; }
__device__ __forceinline__ double img_value(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// The seven stencil entries of row (x, y) of M: self, E, W, N, S, NE, SW.
struct MassRow {
  double w[7];
};
__device__ __forceinline__ MassRow mass_row(const ac::Geo &g, int x, int y) {
  const ac::Weights e = ac::edge_weights(g, x, y);
  MassRow r;
  r.w[0] = 0.5 * g.m0[ac::node_class(g, x, y)];
  r.w[1] = (double)e.e / 12.0;
  r.w[2] = (double)e.w / 12.0;
  r.w[3] = (double)e.n / 12.0;
  r.w[4] = (double)e.s / 12.0;
  r.w[5] = (x < g.W && y < g.H) ? 1.0 / 12.0 : 0.0;
  r.w[6] = (x > 0 && y > 0) ? 1.0 / 12.0 : 0.0;
  return r;
}
__constant__ int kMassDx[7] = {0, 1, -1, 0, 0, 1, -1};
__constant__ int kMassDy[7] = {0, 0, 0, 1, -1, 1, -1};

// m1 = M I and m2 = M |I|^2 at every node (m0 = Mhat, the rows' sums, is
// taken from the node class as for projection by simplex).
template <typename TI>
__global__ void k_moments_node(const TI *__restrict__ img, ac::Geo g, double *__restrict__ mom) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W || y > g.H) return;
  const MassRow row = mass_row(g, x, y);
  double s[3] = {0.0, 0.0, 0.0}, s2 = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if (row.w[k] == 0.0) continue;  // no such neighbour (the weight of a missing edge is 0)
    const int mx = x + kMassDx[k], my = y + kMassDy[k];
    const int px = mx < g.W ? mx : g.W - 1, py = my < g.H ? my : g.H - 1;
    const TI *p = img + ((int64_t)py * g.W + px) * 3;
    const double r = img_value(p[0]), gg = img_value(p[1]), bb = img_value(p[2]);
    s[0] += row.w[k] * r;
    s[1] += row.w[k] * gg;
    s[2] += row.w[k] * bb;
    s2 += row.w[k] * (r * r + gg * gg + bb * bb);
  }
  double *m = mom + ((int64_t)y * g.Wn + x) * 4;
  m[0] = s[0];
  m[1] = s[1];
  m[2] = s[2];
  m[3] = s2;
}

// The adjoint of k_moments_node: pixel p collects, over the nodes n that copy
// it, (M dL/dm1)_n + 2 I_p (M dL/dm2)_n (M is symmetric).  A pixel is copied
// by node (px, py), and also by the nodes of column W (row H) when it is in
// the last column (row).
__global__ void k_adj_image_node(const double *__restrict__ gm, const double *__restrict__ img, ac::Geo g,
                                 double *__restrict__ gimg) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= g.W || py >= g.H) return;
  const double *I = img + ((int64_t)py * g.W + px) * 3;
  double out[3] = {0.0, 0.0, 0.0};
  const int nx = px == g.W - 1 ? 2 : 1, ny = py == g.H - 1 ? 2 : 1;
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) {
      const int x = px + a, y = py + b;
      const MassRow row = mass_row(g, x, y);
      double t[4] = {0.0, 0.0, 0.0, 0.0};  // (M gm)_n for the four moment entries
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        if (row.w[k] == 0.0) continue;
        const double *gk = gm + ((int64_t)(y + kMassDy[k]) * g.Wn + (x + kMassDx[k])) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) t[j] += row.w[k] * gk[j];
      }
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) out[ch] += t[ch] + 2.0 * I[ch] * t[3];
    }
  double *o = gimg + ((int64_t)py * g.W + px) * 3;
  o[0] = out[0];
  o[1] = out[1];
  o[2] = out[2];
}

}  // namespace

extern "C" {

int ac_default_params(ac_params *p) {
  if (!p) return fail(AC_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof *p);
  p->tol = 1e-10;
  p->nu1 = 2;
  p->nu2 = 2;
  p->max_cycles = 200;
  p->coarse_min = 4;
  p->precision = AC_FP64;
  p->projection = AC_PROJ_SIMPLEX;
  return AC_OK;
}

int ac_create(ac_ctx **out, const ac_params *p) {
  if (!out) return fail(AC_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  ac_ctx *ctx = new (std::nothrow) ac_ctx;
  if (!ctx) return fail(AC_ERR_NOMEM, "host allocation failed");
  // refinement (Sec. 4.1): the solve runs on cells of side 1 of the refined
  // grid, where the pixel-unit step (mass and fitting integrals scale by
  // 4^-r, the 2-D stiffness is scale-invariant) is 4^-r times the plain step
  // with eps' = 2^r eps, tau' = 2^r tau, lambda' = 2^-r lambda
  ctx->r = p->refine;
  ctx->W0 = p->width;
  ctx->H0 = p->height;
  ctx->p = *p;
  ctx->p.width = p->width << p->refine;
  ctx->p.height = p->height << p->refine;
  ctx->p.eps = std::ldexp(p->eps, p->refine);
  ctx->p.tau = std::ldexp(p->tau, p->refine);
  ctx->p.lambda = std::ldexp(p->lambda, -p->refine);
  p = &ctx->p;
  ctx->N = p->n_phases;
  ctx->ops = ops_for(ctx->N);
  ctx->s = (cudaStream_t)p->stream;
  ctx->use_graphs = ctx->s != nullptr;  // the legacy default stream cannot be captured
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || ctx->sms < 1) {
      cudaGetLastError();
      ctx->sms = 1;
    }
  }
  const bool mixed = p->precision == AC_MIXED;
  const double te = p->tau * p->eps;
  Solve &S = ctx->sv;
  S.o = mixed ? &ctx->ops->mixed : &ctx->ops->fp64;
  int W = p->width, H = p->height;
  ctx->g0 = make_geo(W, H, te);
  S.lv.push_back(Level{ctx->g0, (int64_t)(W + 1) * (H + 1)});
  while (W % 2 == 0 && H % 2 == 0 && (W < H ? W : H) / 2 >= p->coarse_min) {
    W /= 2;
    H /= 2;
    Level L;
    L.g = make_geo(W, H, te);
    L.n = (int64_t)(W + 1) * (H + 1);
    S.lv.push_back(L);
  }
  ctx->n = S.lv[0].n;
  S.depth = (int)S.lv.size();
  if (S.lv.size() > 1) S.tab0 = galerkin0_table(S.lv[0].g, S.lv[1].g);
  const int N = ctx->N;
  const size_t es = (size_t)S.o->elem;
  // FP32 fine arrays are split by colour (fslot): 2 ((n + 1) / 2) node slots
  const size_t fN64 = (size_t)ctx->n * N * sizeof(double), fNs = (size_t)fine_slots(ctx->n) * N * es;
  const int ls_blocks = (int)(((ctx->g0.W + 1 + 255) / 256) * (int64_t)(ctx->g0.H + 1));
  auto body = [&]() -> int {
    AC_ALLOC(ctx->u, fN64);
    AC_ALLOC(ctx->b, fN64);
    AC_ALLOC(ctx->mom, (size_t)ctx->n * 4 * sizeof(double));
    if (mixed) {
      AC_ALLOC(ctx->r32, fNs);
      AC_ALLOC(ctx->u32, fNs);
      AC_ALLOC(S.x, fNs);
      S.rhs = ctx->r32;
      S.ob = ctx->u32;
    } else {
      S.x = ctx->u;
      S.rhs = ctx->b;
      S.ob = nullptr;
    }
    AC_ALLOC(S.rt, fNs);
    AC_ALLOC(S.mask, (size_t)ctx->n);
    if (S.lv.size() > 1) AC_ALLOC(S.d, fNs);
    AC_ALLOC(ctx->part, (size_t)ac::kMaxPartBlocks * 7 * N * sizeof(double));
    AC_ALLOC(ctx->tot, (size_t)7 * N * sizeof(double));
    AC_ALLOC(ctx->c, (size_t)3 * N * sizeof(double));
    AC_ALLOC(ctx->c_tmp, (size_t)3 * N * sizeof(double));
    AC_ALLOC(ctx->energy, sizeof(double));
    AC_ALLOC(ctx->rho, 2 * sizeof(double));  // rho and the free-node count of the fine residual
    AC_ALLOC(ctx->omega, 2 * sizeof(double));  // omega and its float rounding
    AC_ALLOC(ctx->ls_part, (size_t)2 * ls_blocks * sizeof(double));
    AC_ALLOC(ctx->ls_tot, 2 * sizeof(double));
    AC_ALLOC(S.list_counts, 2 * S.lv.size() * sizeof(int));
    for (size_t k = 1; k < S.lv.size(); ++k) {
      Level &L = S.lv[k];
      AC_ALLOC(L.op, (size_t)L.n * 4 * N * es);
      AC_ALLOC(L.r, (size_t)L.n * N * es);
      AC_ALLOC(L.v, (size_t)L.n * N * es);
      AC_ALLOC(L.t, (size_t)L.n * N * es);
      const size_t nt = (size_t)ac::tiles_x(L.g) * ac::tiles_y(L.g);
      AC_ALLOC(L.lists.flags, nt * N);
      AC_ALLOC(L.lists.items, nt * N * sizeof(uint64_t));
      AC_ALLOC(L.lists.tiles, nt * sizeof(uint64_t));
      AC_ALLOC(L.lists.dirty, nt);
      AC_ALLOC(L.lists.changed, nt);
      AC_CUDA(cudaMemsetAsync(L.lists.dirty, 1, nt, ctx->s));
      L.lists.count = S.list_counts + 2 * k;
      L.lists.cap = (int64_t)nt * N;
      L.lists.sms = ctx->sms;
      AC_CUDA(cudaMemsetAsync(L.lists.flags, ac::kLiveNow, nt * N, ctx->s));  // the first cycle writes all tiles
    }
    AC_CUDA(cudaMallocHost(&ctx->h_scalars, 4 * sizeof(double)));
    AC_CUDA(cudaMemsetAsync(ctx->c, 0, (size_t)3 * N * sizeof(double), ctx->s));
    AC_CUDA(cudaMemsetAsync(ctx->omega, 0, 2 * sizeof(double), ctx->s));
    AC_CUDA(cudaMemsetAsync(S.rt, 0, fNs, ctx->s));  // second-colour slots stay 0 (see solve_mg)
    return AC_OK;
  };
  rc = body();
  if (rc) {
    std::string msg = g_last_error;
    ac_destroy(ctx);
    g_last_error = msg;
    return rc;
  }
  *out = ctx;
  return AC_OK;
}

void ac_destroy(ac_ctx *ctx) {
  if (!ctx) return;
  if (ctx->s)
    cudaStreamSynchronize(ctx->s);
  else
    cudaDeviceSynchronize();
  for (Solve *S : {&ctx->sv, &ctx->adj.sv, &ctx->adj.sv32})
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 2; ++b) slot_release(S->smooth_resid[a][b]);
      for (int f = 0; f < 2; ++f) slot_release(S->correction[a][f]);
    }
  release_step_graphs(ctx);
  for (cudaStream_t bs : ctx->body_s)
    if (bs) cudaStreamDestroy(bs);
  if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
  for (void *p : ctx->adj.allocs) cudaFree(p);
  if (ctx->img64) cudaFree(ctx->img64);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (void *p : ctx->allocs) cudaFree(p);
  if (ctx->img) cudaFree(ctx->img);
  if (ctx->img_up) cudaFree(ctx->img_up);
  if (ctx->lab) cudaFree(ctx->lab);
  if (ctx->img16) cudaFree(ctx->img16);
  if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
  delete ctx;
}

static int set_image_impl(ac_ctx *ctx, const void *rgb, int is_device, bool f64) {
  if (!ctx || !rgb) return fail(AC_ERR_ARG, "NULL argument");
  const ac::Geo &g = ctx->g0;
  const int64_t count = (int64_t)g.W * g.H * 3;                // on the solve grid
  const int64_t count0 = (int64_t)ctx->W0 * ctx->H0 * 3;       // the image as given
  const size_t esz = f64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)count0 * esz;
  const bool mixed = ctx->p.precision == AC_MIXED;
  if (mixed && f64) return fail(AC_ERR_ARG, "AC_MIXED takes a float32 image (it is stored in bfloat16)");
  const void *src = rgb;
  if (!is_device) {
    if (ctx->img_bytes < bytes) {
      if (ctx->img) cudaFree(ctx->img);
      ctx->img = nullptr;
      ctx->img_bytes = 0;
      cudaError_t e = cudaMalloc(&ctx->img, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AC_ERR_NOMEM, "cudaMalloc(%zu) for the image: %s", bytes, cudaGetErrorString(e));
      }
      ctx->img_bytes = bytes;
    }
    AC_CUDA(cudaMemcpyAsync(ctx->img, rgb, bytes, cudaMemcpyHostToDevice, ctx->s));
    src = ctx->img;
  }
  if (ctx->r > 0) {
    // data projection by copy (Sec. 4.2): every cell of the refined grid
    // takes its pixel's colour
    const size_t up_bytes = (size_t)count * esz;
    if (ctx->img_up_bytes < up_bytes) {
      if (ctx->img_up) cudaFree(ctx->img_up);
      ctx->img_up = nullptr;
      ctx->img_up_bytes = 0;
      cudaError_t e = cudaMalloc(&ctx->img_up, up_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->img_up = nullptr;
        return fail(AC_ERR_NOMEM, "cudaMalloc(%zu) for the refined image: %s", up_bytes, cudaGetErrorString(e));
      }
      ctx->img_up_bytes = up_bytes;
    }
    const dim3 grid((unsigned)((g.W + 255) / 256), (unsigned)g.H);
    if (f64)
      AC_RUN(AC_PROF_SETUP, (k_refine_copy<double><<<grid, 256, 0, ctx->s>>>((const double *)src, ctx->W0, ctx->r,
                                                                              g, (double *)ctx->img_up), 1));
    else
      AC_RUN(AC_PROF_SETUP, (k_refine_copy<float><<<grid, 256, 0, ctx->s>>>((const float *)src, ctx->W0, ctx->r, g,
                                                                             (float *)ctx->img_up), 1));
    src = ctx->img_up;
  }
  if (mixed) {
    if (!ctx->img16) {
      cudaError_t e = cudaMalloc(&ctx->img16, (size_t)count * sizeof(__nv_bfloat16));
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->img16 = nullptr;
        return fail(AC_ERR_NOMEM, "cudaMalloc for the bfloat16 image: %s", cudaGetErrorString(e));
      }
    }
    AC_RUN(AC_PROF_SETUP, (k_to_bf16<<<(unsigned)((count + 255) / 256), 256, 0, ctx->s>>>(
                               (const float *)src, ctx->img16, count), 1));
  }
  const dim3 mgrid((unsigned)((g.W + 256) / 256), (unsigned)(g.H + 1));
  if (ctx->p.projection == AC_PROJ_NODE) {
    if (mixed)
      AC_RUN(AC_PROF_SETUP, (k_moments_node<__nv_bfloat16><<<mgrid, 256, 0, ctx->s>>>(ctx->img16, g, ctx->mom), 1));
    else if (f64)
      AC_RUN(AC_PROF_SETUP, (k_moments_node<double><<<mgrid, 256, 0, ctx->s>>>((const double *)src, g, ctx->mom), 1));
    else
      AC_RUN(AC_PROF_SETUP, (k_moments_node<float><<<mgrid, 256, 0, ctx->s>>>((const float *)src, g, ctx->mom), 1));
  } else if (mixed) {
    AC_RUN(AC_PROF_SETUP, (k_moments_bf16<<<mgrid, 256, 0, ctx->s>>>(ctx->img16, g, ctx->mom), 1));
  } else if (f64) {
    AC_RUN(AC_PROF_SETUP, ctx->ops->moments_f64((const double *)src, g, ctx->mom, ctx->s));
  } else {
    AC_RUN(AC_PROF_SETUP, ctx->ops->moments_f32((const float *)src, g, ctx->mom, ctx->s));
  }
  if (!ctx->img64) {
    cudaError_t e = cudaMalloc(&ctx->img64, (size_t)count * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->img64 = nullptr;
      return fail(AC_ERR_NOMEM, "cudaMalloc for the FP64 image: %s", cudaGetErrorString(e));
    }
  }
  {
    const unsigned nb = (unsigned)((count + 255) / 256);
    if (mixed)
      AC_RUN(AC_PROF_SETUP, (k_img_f64<__nv_bfloat16><<<nb, 256, 0, ctx->s>>>(ctx->img16, ctx->img64, count), 1));
    else if (f64)
      AC_RUN(AC_PROF_SETUP, (k_img_f64<double><<<nb, 256, 0, ctx->s>>>((const double *)src, ctx->img64, count), 1));
    else
      AC_RUN(AC_PROF_SETUP, (k_img_f64<float><<<nb, 256, 0, ctx->s>>>((const float *)src, ctx->img64, count), 1));
  }
  AC_RUN(AC_PROF_SETUP, ctx->ops->init_random(ctx->u, ctx->n, ctx->p.seed, ctx->s));
  AC_CUDA(cudaMemsetAsync(ctx->c, 0, (size_t)3 * ctx->N * sizeof(double), ctx->s));
  if (!is_device) AC_CUDA(cudaStreamSynchronize(ctx->s));  // the host buffer may be reused after return
  ctx->adj.ready = false;
  ctx->have_image = true;
  ctx->have_rhs = false;
  ctx->delta_warm = false;
  return AC_OK;
}

int ac_set_image(ac_ctx *ctx, const float *rgb, int is_device) { return set_image_impl(ctx, rgb, is_device, false); }
int ac_set_image_f64(ac_ctx *ctx, const double *rgb, int is_device) { return set_image_impl(ctx, rgb, is_device, true); }

int ac_step(ac_ctx *ctx, int n_steps, ac_stats *out) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (n_steps < 0) return fail(AC_ERR_ARG, "n_steps must be >= 0");
  if (!ctx->have_image) return fail(AC_ERR_STATE, "ac_set_image must come first");
  if (n_steps > 0 && loop_on_device(ctx)) {
    // capture the step graphs (once); a device or driver that cannot capture
    // or instantiate them leaves the context on the host loop
    int rc = capture_step(ctx, false);
    if (!rc && out) rc = capture_step(ctx, true);
    if (rc) {
      release_step_graphs(ctx);
      ctx->loop_mode = AC_LOOP_HOST;
    } else {
      return step_device(ctx, n_steps, out);
    }
  }
  ac_stats st{};
  st.converged = 1;
  int status = AC_OK;
  const double a1 = 1.0 + 2.0 * ctx->p.tau / ctx->p.eps, tl = ctx->p.tau * ctx->p.lambda;
  const bool mixed = ctx->p.precision == AC_MIXED;
  // means (and energy): u (binary64) and the moments (4 doubles) read per
  // node; right-hand side: the same read and b (8 bytes per phase) written
  const double mean_bytes = (double)ctx->n * (8.0 * ctx->N + 32), rhs_bytes = mean_bytes + (double)ctx->n * 8.0 * ctx->N;
  for (int t = 0; t < n_steps; ++t) {
    // the energy is only evaluated for the statistics of the last step
    double *energy = (out && t == n_steps - 1) ? ctx->energy : nullptr;
    if (mixed)
      AC_RUNB(AC_PROF_SETUP, mean_bytes, ctx->ops->means_df(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c,
                                                            energy, ctx->p.eps, ctx->p.lambda, ctx->s));
    else
      AC_RUNB(AC_PROF_SETUP, mean_bytes, ctx->ops->means(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c,
                                                         energy, ctx->p.eps, ctx->p.lambda, ctx->s));
    if (mixed)
      AC_RUNB(AC_PROF_SETUP, rhs_bytes,
              ctx->ops->rhs_df(ctx->u, ctx->mom, ctx->c, ctx->g0, a1, tl, (float *)ctx->b, ctx->s));
    else
      AC_RUNB(AC_PROF_SETUP, rhs_bytes, ctx->ops->rhs(ctx->u, ctx->mom, ctx->c, ctx->g0, a1, tl, ctx->b, ctx->s));
    ctx->have_rhs = true;
    int cycles = 0, outer = 0;
    double rho = 0;
    int64_t sweeps = 0;
    int rc = mixed ? solve_mixed(ctx, &cycles, &rho, &sweeps, &outer)
                   : solve_mg(ctx, ctx->sv, ctx->p.tol, ctx->p.max_cycles, &cycles, &rho, &sweeps);
    st.fine_sweeps += sweeps;
    st.outer += outer;
    st.cycles = cycles;
    st.total_cycles += cycles;
    st.residual = rho;
    st.steps = t + 1;
    if (rc == AC_ERR_NOT_CONVERGED) {
      st.converged = 0;
      status = rc;
    } else if (rc) {
      st.converged = 0;
      if (out) *out = st;
      return rc;
    }
  }
  if (out && n_steps > 0) {
    AC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 1, ctx->energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    AC_CUDA(cudaStreamSynchronize(ctx->s));
    st.energy = std::ldexp(ctx->h_scalars[1], -ctx->r);  // pixel units: E = 2^-r E(eps', lambda')
  }
  if (out) *out = st;
  return status;
}

int ac_segment(ac_ctx *ctx, int n_steps, int8_t *pixel_labels, int is_device, ac_stats *out) {
  if (!ctx || !pixel_labels) return fail(AC_ERR_ARG, "NULL argument");
  int rc = ac_step(ctx, n_steps, out);
  if (rc && rc != AC_ERR_NOT_CONVERGED) return rc;
  const ac::Geo &g = ctx->g0;
  const size_t bytes = (size_t)ctx->W0 * ctx->H0;
  int8_t *dst = pixel_labels;
  if (!is_device) {
    int rc2 = label_stage(ctx, &dst);
    if (rc2) return rc2;
  }
  AC_RUN(AC_PROF_SETUP, ctx->ops->labels(ctx->u, g, ctx->r, nullptr, dst, ctx->s));
  if (!is_device) {
    int rc2 = copy_out(ctx, pixel_labels, dst, bytes, 0);
    if (rc2) return rc2;
  }
  return rc;
}

int ac_set_phase(ac_ctx *ctx, const double *u, int is_device) {
  if (!ctx || !u) return fail(AC_ERR_ARG, "NULL argument");
  AC_CUDA(cudaMemcpyAsync(ctx->u, u, (size_t)ctx->n * ctx->N * sizeof(double),
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s));
  AC_CUDA(cudaMemsetAsync(ctx->c, 0, (size_t)3 * ctx->N * sizeof(double), ctx->s));
  ctx->delta_warm = false;  // a new state: the next step's correction starts from zero
  if (!is_device) AC_CUDA(cudaStreamSynchronize(ctx->s));
  return AC_OK;
}

int ac_get_phase(ac_ctx *ctx, double *u, int is_device) {
  if (!ctx || !u) return fail(AC_ERR_ARG, "NULL argument");
  return copy_out(ctx, u, ctx->u, (size_t)ctx->n * ctx->N * sizeof(double), is_device);
}

int ac_get_means(ac_ctx *ctx, double *c) {
  if (!ctx || !c) return fail(AC_ERR_ARG, "NULL argument");
  return copy_out(ctx, c, ctx->c, (size_t)3 * ctx->N * sizeof(double), 0);
}

int ac_get_moments(ac_ctx *ctx, double *m) {
  if (!ctx || !m) return fail(AC_ERR_ARG, "NULL argument");
  if (!ctx->have_image) return fail(AC_ERR_STATE, "no image");
  std::vector<double> mom((size_t)ctx->n * 4);
  int rc = copy_out(ctx, mom.data(), ctx->mom, mom.size() * sizeof(double), 0);
  if (rc) return rc;
  const ac::Geo &g = ctx->g0;
  for (int64_t k = 0; k < ctx->n; ++k) {
    const int x = (int)(k % g.Wn), y = (int)(k / g.Wn);
    const int cx = x == 0 ? 0 : (x == g.W ? 2 : 1), cy = y == 0 ? 0 : (y == g.H ? 2 : 1);
    m[k * 5 + 0] = g.m0[cy * 3 + cx];
    for (int j = 0; j < 4; ++j) m[k * 5 + 1 + j] = mom[k * 4 + j];
  }
  return AC_OK;
}

int ac_get_rhs(ac_ctx *ctx, double *b) {
  if (!ctx || !b) return fail(AC_ERR_ARG, "NULL argument");
  if (!ctx->have_rhs) return fail(AC_ERR_STATE, "no step taken yet");
  int rc = copy_out(ctx, b, ctx->b, (size_t)ctx->n * ctx->N * sizeof(double), 0);
  if (rc || ctx->p.precision != AC_MIXED) return rc;
  // the mixed form holds b as double-floats, N heads then N tails per node
  // (the bytes of the node's N doubles): h + l in place, node by node
  const int N = ctx->N;
  float hl[2 * AC_MAX_PHASES];
  for (int64_t k = 0; k < ctx->n; ++k) {
    std::memcpy(hl, b + k * N, (size_t)2 * N * sizeof(float));
    for (int i = 0; i < N; ++i) b[k * N + i] = (double)hl[i] + (double)hl[N + i];
  }
  return AC_OK;
}

int ac_get_node_labels(ac_ctx *ctx, int8_t *labels, int is_device) {
  if (!ctx || !labels) return fail(AC_ERR_ARG, "NULL argument");
  int8_t *dst = labels;
  if (!is_device) {
    int rc = label_stage(ctx, &dst);
    if (rc) return rc;
  }
  AC_RUN(AC_PROF_SETUP, ctx->ops->labels(ctx->u, ctx->g0, ctx->r, dst, nullptr, ctx->s));
  if (!is_device) return copy_out(ctx, labels, dst, (size_t)ctx->n, 0);
  return AC_OK;
}

int ac_get_composite(ac_ctx *ctx, float *rgb, int rounded, int is_device) {
  if (!ctx || !rgb) return fail(AC_ERR_ARG, "NULL argument");
  if (!ctx->have_image) return fail(AC_ERR_STATE, "no image");
  const size_t bytes = (size_t)ctx->W0 * ctx->H0 * 3 * sizeof(float);
  float *dst = rgb;
  if (!is_device) {
    if (ctx->img_bytes < bytes) {
      if (ctx->img) cudaFree(ctx->img);
      ctx->img = nullptr;
      ctx->img_bytes = 0;
      cudaError_t e = cudaMalloc(&ctx->img, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->img = nullptr;
        return fail(AC_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      }
      ctx->img_bytes = bytes;
    }
    dst = static_cast<float *>(ctx->img);
  }
  // the colour means of the current u (a phase of zero mass keeps its last c)
  AC_CUDA(cudaMemcpyAsync(ctx->c_tmp, ctx->c, (size_t)3 * ctx->N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  AC_RUN(AC_PROF_SETUP, ctx->ops->means(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c_tmp, nullptr,
                                        ctx->p.eps, ctx->p.lambda, ctx->s));
  AC_RUN(AC_PROF_SETUP, ctx->ops->composite(ctx->u, ctx->c_tmp, ctx->g0, ctx->r, rounded ? 1 : 0, dst, ctx->s));
  if (!is_device) return copy_out(ctx, rgb, dst, bytes, 0);
  return AC_OK;
}

int ac_energy(ac_ctx *ctx, double *energy) {
  if (!ctx || !energy) return fail(AC_ERR_ARG, "NULL argument");
  if (!ctx->have_image) return fail(AC_ERR_STATE, "no image");
  AC_CUDA(cudaMemcpyAsync(ctx->c_tmp, ctx->c, (size_t)3 * ctx->N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  AC_RUN(AC_PROF_SETUP, ctx->ops->means(ctx->u, ctx->mom, ctx->g0, ctx->part, ctx->tot, ctx->c_tmp, ctx->energy,
                                        ctx->p.eps, ctx->p.lambda, ctx->s));
  int rc = copy_out(ctx, energy, ctx->energy, sizeof(double), 0);
  *energy = std::ldexp(*energy, -ctx->r);  // pixel units: E = 2^-r E(eps', lambda') on the refined cells
  return rc;
}

int ac_residual(ac_ctx *ctx, double *rho) {
  if (!ctx || !rho) return fail(AC_ERR_ARG, "NULL argument");
  if (!ctx->have_rhs) return fail(AC_ERR_STATE, "no step taken yet");
  AC_CUDA(cudaMemsetAsync(ctx->rho, 0, sizeof(double), ctx->s));
  if (ctx->p.precision == AC_MIXED)
    AC_RUN(AC_PROF_OUTER,
           ctx->ops->outer_resid(ctx->u, (const float *)ctx->b, ctx->g0, ctx->r32, ctx->u32, ctx->rho, false, ctx->s));
  else
    AC_RUN(AC_PROF_RESID,
           ctx->ops->fp64.resid(ctx->u, ctx->b, nullptr, ctx->g0, nullptr, nullptr, ctx->rho, -1,
                                ac::MaskDirty{nullptr, 0, 0}, ctx->s));
  return read_rho(ctx, rho);
}

int ac_project_simplex(const double *y, double *x, int64_t count, int n_phases, void *stream) {
  const ac::Ops *o = ops_for(n_phases);
  if (!o) return fail(AC_ERR_ARG, "n_phases must be in [2, %d]", AC_MAX_PHASES);
  if (count < 0 || (count > 0 && (!y || !x))) return fail(AC_ERR_ARG, "bad buffers");
  o->project(y, x, count, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return AC_OK;
}

int ac_set_profiling_mask(ac_ctx *ctx, unsigned class_mask) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  int rc = prof_harvest(ctx);
  if (rc) return rc;
  for (int k = 0; k < AC_PROF_COUNT; ++k) {
    ctx->prof_ms[k] = 0;
    ctx->prof_launches[k] = 0;
    ctx->prof_bytes[k] = 0;
  }
  ctx->prof_corr_launches = 0;
  class_mask &= (1u << AC_PROF_COUNT) - 1u;
  ctx->profiling = class_mask != 0;
  ctx->prof_mask = class_mask ? class_mask : (1u << AC_PROF_COUNT) - 1u;
  if (ctx->profiling && ctx->prof_mask != ctx->prof_graph_mask) {
    // the profiled graphs carry the events of the old mask: capture them again
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    for (Solve *S : {&ctx->sv, &ctx->adj.sv, &ctx->adj.sv32}) {
      for (int b = 0; b < 2; ++b) slot_release(S->smooth_resid[1][b]);
      for (int f = 0; f < 2; ++f) slot_release(S->correction[1][f]);
    }
    ctx->prof_graph_mask = ctx->prof_mask;
  }
  return AC_OK;
}

int ac_set_coarse_tiling(ac_ctx *ctx, int mode) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (mode != AC_TILES_AUTO && mode != AC_TILES_NEVER && mode != AC_TILES_ALWAYS)
    return fail(AC_ERR_ARG, "mode must be AC_TILES_AUTO, AC_TILES_NEVER or AC_TILES_ALWAYS");
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  release_step_graphs(ctx);
  for (Solve *S : {&ctx->sv, &ctx->adj.sv, &ctx->adj.sv32}) {
    // the tiled correction graphs depend on which levels are tiled
    for (int a = 0; a < 2; ++a) slot_release(S->correction[a][1]);
    S->tiling = mode;
    S->was_tiled = false;  // the next tiled correction writes every tile
  }
  return AC_OK;
}

int ac_set_adjoint_preconditioner(ac_ctx *ctx, int precision) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (precision != AC_ADJ_PRECOND_F32 && precision != AC_ADJ_PRECOND_F64)
    return fail(AC_ERR_ARG, "precision must be AC_ADJ_PRECOND_F32 or AC_ADJ_PRECOND_F64");
  ctx->adj_pre32 = precision == AC_ADJ_PRECOND_F32;
  ctx->adj.ready = false;  // the next ac_adjoint_forward sets up the solves again
  return AC_OK;
}

int ac_set_cycle_loop(ac_ctx *ctx, int mode) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (mode != AC_LOOP_AUTO && mode != AC_LOOP_HOST) return fail(AC_ERR_ARG, "mode must be AC_LOOP_AUTO or AC_LOOP_HOST");
  ctx->loop_mode = mode;
  return AC_OK;
}

int ac_get_cycle_loop(ac_ctx *ctx, int *on_device) {
  if (!ctx || !on_device) return fail(AC_ERR_ARG, "NULL argument");
  *on_device = loop_on_device(ctx) ? 1 : 0;
  return AC_OK;
}

int ac_set_coarse_smoother(ac_ctx *ctx, int mode) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (mode != AC_SMOOTH_GS3 && mode != AC_SMOOTH_JACOBI)
    return fail(AC_ERR_ARG, "mode must be AC_SMOOTH_GS3 or AC_SMOOTH_JACOBI");
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  release_step_graphs(ctx);
  for (Solve *S : {&ctx->sv, &ctx->adj.sv, &ctx->adj.sv32}) {
    // the correction graphs hold the smoother's kernels
    for (int a = 0; a < 2; ++a)
      for (int f = 0; f < 2; ++f) slot_release(S->correction[a][f]);
    S->coarse_gs = mode == AC_SMOOTH_GS3;
  }
  return AC_OK;
}

int ac_set_profiling(ac_ctx *ctx, int enable) {
  return ac_set_profiling_mask(ctx, enable ? (1u << AC_PROF_COUNT) - 1u : 0u);
}

int ac_get_profile(ac_ctx *ctx, ac_profile *out) {
  if (!ctx || !out) return fail(AC_ERR_ARG, "NULL argument");
  int rc = prof_harvest(ctx);
  if (rc) return rc;
  for (int k = 0; k < AC_PROF_COUNT; ++k) {
    out->ms[k] = ctx->prof_ms[k];
    out->launches[k] = ctx->prof_launches[k];
    out->bytes[k] = ctx->prof_bytes[k];
  }
  out->smooth_bytes_per_launch = ctx->p.precision == AC_MIXED ? 2.0 * (double)ctx->n * ctx->N * sizeof(float)
                                                               : 1.5 * (double)ctx->n * ctx->N * sizeof(double);
  out->total_launches = ctx->total_launches;
  out->smooth_corr_launches = ctx->prof_corr_launches;
  out->smooth_corr_extra_bytes = 0.5 * (double)ctx->n * ctx->N * (ctx->p.precision == AC_MIXED ? sizeof(float)
                                                                                                 : sizeof(double));
  return AC_OK;
}

const char *ac_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace ac {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace ac

// ---------------------------------------------------------------------------
// Adjoint (gradients of a loss on u after T steps).
// ---------------------------------------------------------------------------
namespace {

int adj_alloc(ac_ctx *ctx, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AC_ERR_NOMEM, "cudaMalloc(%zu) for the adjoint: %s", bytes, cudaGetErrorString(e));
  }
  ctx->adj.allocs.push_back(*p);
  return AC_OK;
}

#define ADJ_ALLOC(ptr, bytes)                                              \
  do {                                                                     \
    int rc_ = adj_alloc(ctx, reinterpret_cast<void **>(&(ptr)), (bytes));  \
    if (rc_) return rc_;                                                   \
  } while (0)

void adj_release(ac_ctx *ctx) {
  AdjState &A = ctx->adj;
  for (Solve *S : {&A.sv, &A.sv32})
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 2; ++b) slot_release(S->smooth_resid[a][b]);
      for (int f = 0; f < 2; ++f) slot_release(S->correction[a][f]);
    }
  for (void *p : A.allocs) cudaFree(p);
  A = AdjState{};
}

// Buffers of the adjoint for T steps with checkpoints every `every` steps,
// and the FP64 tangent-form solve on the primary solve's level hierarchy.
int adj_setup(ac_ctx *ctx, int T, int every) {
  cudaStreamSynchronize(ctx->s);
  adj_release(ctx);
  AdjState &A = ctx->adj;
  const int N = ctx->N;
  const size_t fN = (size_t)ctx->n * N * sizeof(double);
  A.T = T;
  A.every = every;
  A.ncp = (T + every - 1) / every;
  ADJ_ALLOC(A.cp_u, fN * A.ncp);
  ADJ_ALLOC(A.cp_c, (size_t)A.ncp * N * 3 * sizeof(double));
  ADJ_ALLOC(A.uT, fN);
  ADJ_ALLOC(A.seg_u, fN * (every + 1));
  ADJ_ALLOC(A.seg_c, (size_t)every * N * 3 * sizeof(double));
  ADJ_ALLOC(A.seg_M, (size_t)every * N * sizeof(double));
  ADJ_ALLOC(A.g, fN);
  ADJ_ALLOC(A.g2, fN);
  ADJ_ALLOC(A.gm, (size_t)ctx->n * 4 * sizeof(double));
  const int blocks = (int)(((ctx->g0.W + 1 + 255) / 256) * (int64_t)(ctx->g0.H + 1));
  ADJ_ALLOC(A.part, (size_t)blocks * (2 + 3 * N) * sizeof(double));
  ADJ_ALLOC(A.tot, (size_t)(2 + 3 * N) * sizeof(double));
  ADJ_ALLOC(A.scal, 2 * sizeof(double));
  ADJ_ALLOC(A.kw, fN);
  ADJ_ALLOC(A.kr, fN);
  ADJ_ALLOC(A.kp, fN);
  ADJ_ALLOC(A.kq, fN);
  ADJ_ALLOC(A.kq_prev, fN);
  ADJ_ALLOC(A.kpart, (size_t)ac::kMaxPartBlocks * 2 * sizeof(double));
  if (ctx->r > 0) ADJ_ALLOC(A.gimg, (size_t)ctx->g0.W * ctx->g0.H * 3 * sizeof(double));
  ADJ_ALLOC(A.ktot, 2 * sizeof(double));
  ADJ_ALLOC(A.ndiff, sizeof(unsigned long long));
  // the tangent-form solves on the primary solve's level hierarchy: FP64
  // (elem 8, node-order fine arrays) and its FP32 copy (elem 4, colour-split
  // fine arrays), each with its own arrays, lists and graphs
  auto setup_solve = [&](Solve &S, const ac::SolverOps *ops) -> int {
    const size_t es = (size_t)ops->elem;
    const size_t fS = (size_t)fine_slots(ctx->n) * N * es;
    S.o = ops;
    S.lv = ctx->sv.lv;
    ADJ_ALLOC(S.list_counts, 2 * S.lv.size() * sizeof(int));
    for (size_t k = 1; k < S.lv.size(); ++k) {
      Level &L = S.lv[k];
      ADJ_ALLOC(L.op, (size_t)L.n * 4 * N * es);
      ADJ_ALLOC(L.r, (size_t)L.n * N * es);
      ADJ_ALLOC(L.v, (size_t)L.n * N * es);
      ADJ_ALLOC(L.t, (size_t)L.n * N * es);
      const size_t nt = (size_t)ac::tiles_x(L.g) * ac::tiles_y(L.g);
      ADJ_ALLOC(L.lists.flags, nt * N);
      ADJ_ALLOC(L.lists.items, nt * N * sizeof(uint64_t));
      ADJ_ALLOC(L.lists.tiles, nt * sizeof(uint64_t));
      ADJ_ALLOC(L.lists.dirty, nt);
      ADJ_ALLOC(L.lists.changed, nt);
      AC_CUDA(cudaMemsetAsync(L.lists.dirty, 1, nt, ctx->s));
      L.lists.count = S.list_counts + 2 * k;
      L.lists.cap = (int64_t)nt * N;
      L.lists.sms = ctx->sms;
      AC_CUDA(cudaMemsetAsync(L.lists.flags, ac::kLiveNow, nt * N, ctx->s));
    }
    S.depth = ctx->sv.depth;
    S.tab0 = ctx->sv.tab0;
    S.tiling = ctx->sv.tiling;
    S.coarse_gs = ctx->sv.coarse_gs;
    ADJ_ALLOC(S.x, fS);
    ADJ_ALLOC(S.rhs, fS);
    ADJ_ALLOC(S.ob, fS);
    ADJ_ALLOC(S.rt, fS);
    ADJ_ALLOC(S.d, fS);
    ADJ_ALLOC(S.mask, (size_t)ctx->n);
    AC_CUDA(cudaMemsetAsync(S.rt, 0, fS, ctx->s));  // second-colour slots stay 0 (see solve_mg)
    return AC_OK;
  };
  int rc = setup_solve(A.sv, &ctx->ops->adjoint);
  if (!rc && ctx->adj_pre32) rc = setup_solve(A.sv32, &ctx->ops->adjoint32);
  return rc;
}

// Components where a and b differ (bit patterns compared: a recomputation
// either repeats the forward's arithmetic exactly or it does not).
__global__ void k_count_diff(const double *__restrict__ a, const double *__restrict__ b, int64_t count,
                             unsigned long long *out) {
  unsigned long long k = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    k += __double_as_longlong(a[i]) != __double_as_longlong(b[i]);
  k = ac::warp_sum<unsigned long long>(k);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(out, k);
}

}  // namespace

// Flexible CG (one-vector recurrence) on the adjoint system (Pi S Pi) w = Pi g
// of one step, preconditioned by the truncated V-cycle of the tangent form
// (two cycles of solve_mg from zero: pre-smoothing, coarse correction with
// its line search, post-smoothing).  The line search makes the preconditioner
// nonlinear, hence the flexible direction update
//   p_k = z_k - (z_k . q_{k-1}) / (p_{k-1} . q_{k-1}) p_{k-1},   q = Pi S p,
//   alpha = p_k . r_k / p_k . q_k.
// Stops when max |r| / S_nn <= tol_rho (the plain solve's natural-residual
// rule; min S_nn bounds the scaling).  On return A.kw holds w.
int fcg_adjoint(ac_ctx *ctx, AdjState &A, double tol_rho, int max_iter, int *iters) {
  Solve &S = A.sv;
  const ac::Ops *o = ctx->ops;
  const int64_t nN = ctx->n * ctx->N;
  const size_t fN = (size_t)nN * sizeof(double);
  double dmin = ctx->g0.D[0];
  for (int k = 1; k < 9; ++k) dmin = std::fmin(dmin, ctx->g0.D[k] > 0 ? ctx->g0.D[k] : dmin);
  const double tol_r = tol_rho * dmin;
  AC_CUDA(cudaMemsetAsync(A.kw, 0, fN, ctx->s));
  AC_CUDA(cudaMemcpyAsync(A.kr, S.rhs, fN, cudaMemcpyDeviceToDevice, ctx->s));
  double pq_prev = 0.0;
  int it = 0, status = AC_ERR_NOT_CONVERGED;
  for (; it < max_iter; ++it) {
    AC_CUDA(cudaMemsetAsync(ctx->rho, 0, sizeof(double), ctx->s));
    AC_RUN(AC_PROF_SETUP, o->absmax(A.kr, nN, ctx->rho, ctx->s));
    double rmax = 0;
    int rc = read_rho(ctx, &rmax);
    if (rc) return rc;
    if (std::isnan(rmax)) return fail(AC_ERR_NUMERIC, "non-finite adjoint residual");
    if (rmax <= tol_r) {
      status = AC_OK;
      break;
    }
    // z = B r: the truncated V-cycle from zero on right-hand side r, in
    // FP32 (r rounded, z widened and projected onto the tangent space in
    // FP64; the recurrence, residual and dots stay FP64, and the flexible
    // update absorbs the preconditioner's rounding) or in FP64
    int cyc = 0;
    double rho = 0;
    int64_t sw = 0;
    if (A.sv32.o) {
      Solve &P = A.sv32;
      AC_RUN(AC_PROF_SETUP, o->to_split32(A.kr, ctx->g0, (float *)P.rhs, ctx->s));
      AC_CUDA(cudaMemsetAsync(P.x, 0, (size_t)fine_slots(ctx->n) * ctx->N * sizeof(float), ctx->s));
      rc = solve_mg(ctx, P, 0.0, 2, &cyc, &rho, &sw);
      if (rc && rc != AC_ERR_NOT_CONVERGED) return rc;
      AC_RUN(AC_PROF_SETUP,
             o->from_split32((const float *)P.x, ctx->g0, (const double *)S.ob, (double *)S.x, ctx->s));
    } else {
      AC_CUDA(cudaMemcpyAsync(S.rhs, A.kr, fN, cudaMemcpyDeviceToDevice, ctx->s));
      AC_CUDA(cudaMemsetAsync(S.x, 0, fN, ctx->s));
      rc = solve_mg(ctx, S, 0.0, 2, &cyc, &rho, &sw);
      if (rc && rc != AC_ERR_NOT_CONVERGED) return rc;
    }
    const double *z = (const double *)S.x;
    double beta = 0.0;
    if (it > 0) {
      AC_RUN(AC_PROF_SETUP, o->dot2(z, A.kq_prev, nullptr, nullptr, nN, A.kpart, A.ktot, ctx->s));
      AC_CUDA(cudaMemcpyAsync(ctx->h_scalars, A.ktot, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
      AC_CUDA(cudaStreamSynchronize(ctx->s));
      beta = pq_prev > 0 ? -ctx->h_scalars[0] / pq_prev : 0.0;
    }
    AC_RUN(AC_PROF_SETUP, o->fcg_dir(A.kp, z, beta, nN, ctx->s));
    AC_RUN(AC_PROF_SETUP, o->tangent_apply(A.kp, (const double *)S.ob, ctx->g0, A.kq, ctx->s));
    AC_RUN(AC_PROF_SETUP, o->dot2(A.kp, A.kr, A.kp, A.kq, nN, A.kpart, A.ktot, ctx->s));
    AC_CUDA(cudaMemcpyAsync(ctx->h_scalars, A.ktot, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    AC_CUDA(cudaStreamSynchronize(ctx->s));
    const double pr = ctx->h_scalars[0], pq = ctx->h_scalars[1];
    if (!(pq > 0)) break;  // p = 0 (r already 0 on the tangent space) or a lost direction
    AC_RUN(AC_PROF_SETUP, o->fcg_step(A.kw, A.kr, A.kp, A.kq, pr / pq, nN, ctx->s));
    pq_prev = pq;
    std::swap(A.kq, A.kq_prev);
  }
  *iters = it;
  return status;
}

extern "C" {

int ac_adjoint_forward(ac_ctx *ctx, int n_steps, int checkpoint_every) {
  if (!ctx) return fail(AC_ERR_ARG, "ctx is NULL");
  if (n_steps < 1 || checkpoint_every < 1 || checkpoint_every > n_steps)
    return fail(AC_ERR_ARG, "need n_steps >= 1 and 1 <= checkpoint_every <= n_steps");
  if (!ctx->have_image) return fail(AC_ERR_STATE, "ac_set_image must come first");
  int rc = adj_setup(ctx, n_steps, checkpoint_every);
  if (rc) return rc;
  AdjState &A = ctx->adj;
  const size_t fN = (size_t)ctx->n * ctx->N * sizeof(double), cN = (size_t)ctx->N * 3 * sizeof(double);
  int status = AC_OK;
  for (int t = 0; t < n_steps; ++t) {
    if (t % checkpoint_every == 0) {
      const int j = t / checkpoint_every;
      AC_CUDA(cudaMemcpyAsync(A.cp_u + (size_t)j * ctx->n * ctx->N, ctx->u, fN, cudaMemcpyDeviceToDevice, ctx->s));
      AC_CUDA(cudaMemcpyAsync(A.cp_c + (size_t)j * ctx->N * 3, ctx->c, cN, cudaMemcpyDeviceToDevice, ctx->s));
      // each segment starts its first correction from zero (AC_MIXED), as its
      // recomputation from this checkpoint in ac_adjoint_backward will
      ctx->delta_warm = false;
    }
    rc = ac_step(ctx, 1, nullptr);
    if (rc == AC_ERR_NOT_CONVERGED)
      status = rc;
    else if (rc)
      return rc;
  }
  AC_CUDA(cudaMemcpyAsync(A.uT, ctx->u, fN, cudaMemcpyDeviceToDevice, ctx->s));
  A.ready = true;
  return status;
}

int ac_adjoint_backward(ac_ctx *ctx, const double *grad_u, double *grad_lambda, double *grad_eps, double *grad_image,
                        double *grad_u0) {
  if (!ctx || !grad_u || !grad_lambda || !grad_eps || !grad_image) return fail(AC_ERR_ARG, "NULL argument");
  AdjState &A = ctx->adj;
  if (!A.ready) return fail(AC_ERR_STATE, "ac_adjoint_forward must come first");
  const int N = ctx->N;
  const int64_t nN = ctx->n * N;
  const size_t fN = (size_t)nN * sizeof(double), cN = (size_t)N * 3 * sizeof(double);
  const double tau = ctx->p.tau, eps = ctx->p.eps, lam = ctx->p.lambda, a1 = 1.0 + 2.0 * tau / eps;
  const ac::Ops *o = ctx->ops;
  AC_CUDA(cudaMemcpyAsync(A.g, grad_u, fN, cudaMemcpyDeviceToDevice, ctx->s));
  AC_CUDA(cudaMemsetAsync(A.gm, 0, (size_t)ctx->n * 4 * sizeof(double), ctx->s));
  AC_CUDA(cudaMemsetAsync(A.scal, 0, 2 * sizeof(double), ctx->s));
  AC_CUDA(cudaMemsetAsync(A.ndiff, 0, sizeof(unsigned long long), ctx->s));
  int status = AC_OK;
  for (int j = A.ncp - 1; j >= 0; --j) {
    const int t0 = j * A.every, t1 = std::min(t0 + A.every, A.T), len = t1 - t0;
    // recompute the segment's states from its checkpoint with the forward's
    // arithmetic: like the forward, the segment's first step starts its
    // correction from zero (AC_MIXED), and the later ones from the previous
    // step's, which the recomputation has just produced
    AC_CUDA(cudaMemcpyAsync(ctx->u, A.cp_u + (size_t)j * nN, fN, cudaMemcpyDeviceToDevice, ctx->s));
    AC_CUDA(cudaMemcpyAsync(ctx->c, A.cp_c + (size_t)j * N * 3, cN, cudaMemcpyDeviceToDevice, ctx->s));
    AC_CUDA(cudaMemcpyAsync(A.seg_u, ctx->u, fN, cudaMemcpyDeviceToDevice, ctx->s));
    ctx->delta_warm = false;
    for (int k = 0; k < len; ++k) {
      int rc = ac_step(ctx, 1, nullptr);
      if (rc && rc != AC_ERR_NOT_CONVERGED) return rc;
      AC_CUDA(cudaMemcpyAsync(A.seg_u + (size_t)(k + 1) * nN, ctx->u, fN, cudaMemcpyDeviceToDevice, ctx->s));
      AC_CUDA(cudaMemcpyAsync(A.seg_c + (size_t)k * N * 3, ctx->c, cN, cudaMemcpyDeviceToDevice, ctx->s));
      AC_CUDA(cudaMemcpyAsync(A.seg_M + (size_t)k * N, ctx->tot, N * sizeof(double), cudaMemcpyDeviceToDevice,
                              ctx->s));
    }
    // the segment's end against the forward's own state there
    const double *fwd_end = j + 1 < A.ncp ? A.cp_u + (size_t)(j + 1) * nN : A.uT;
    AC_RUN(AC_PROF_SETUP, (k_count_diff<<<(unsigned)std::min<int64_t>((nN + 255) / 256, 4 * 152), 256, 0, ctx->s>>>(
                               A.seg_u + (size_t)len * nN, fwd_end, nN, A.ndiff), 1));
    for (int k = len - 1; k >= 0; --k) {
      const double *u = A.seg_u + (size_t)k * nN, *up = A.seg_u + (size_t)(k + 1) * nN;
      const double *c = A.seg_c + (size_t)k * N * 3, *M = A.seg_M + (size_t)k * N;
      Solve &S = A.sv;
      AC_RUN(AC_PROF_SETUP, o->adj_prepare(up, A.g, ctx->n, (double *)S.ob, (double *)S.rhs, ctx->s));
      if (A.sv32.o) AC_RUN(AC_PROF_SETUP, o->to_split32((const double *)S.ob, ctx->g0, (float *)A.sv32.ob, ctx->s));
      AC_CUDA(cudaMemsetAsync(S.x, 0, fN, ctx->s));
      AC_CUDA(cudaMemsetAsync(ctx->rho, 0, sizeof(double), ctx->s));
      AC_RUN(AC_PROF_SETUP, o->absmax((const double *)S.rhs, nN, ctx->rho, ctx->s));
      double gmax = 0;
      int rc = read_rho(ctx, &gmax);
      if (rc) return rc;
      const double *w = (const double *)S.x;
      if (gmax > 0) {
#ifdef AC_ADJOINT_PLAIN_VCYCLE
        int cyc = 0;
        double rho = 0;
        int64_t sw = 0;
        rc = solve_mg(ctx, S, 1e-13 * gmax, ctx->p.max_cycles, &cyc, &rho, &sw);
#else
        int iters = 0;
        rc = fcg_adjoint(ctx, A, 1e-13 * gmax, ctx->p.max_cycles, &iters);
        w = A.kw;
#endif
        if (rc == AC_ERR_NOT_CONVERGED)
          status = rc;
        else if (rc)
          return rc;
      }
      AC_RUN(AC_PROF_SETUP, o->adj_accum(w, u, up, ctx->mom, c, ctx->g0, tau, eps, lam, A.gm, A.part, A.tot, A.scal,
                                         ctx->s));
      AC_RUN(AC_PROF_SETUP, o->adj_back(w, u, ctx->mom, c, A.tot, M, ctx->g0, a1, A.g2, A.gm, ctx->s));
      std::swap(A.g, A.g2);
    }
  }
  if (grad_u0) AC_CUDA(cudaMemcpyAsync(grad_u0, A.g, fN, cudaMemcpyDeviceToDevice, ctx->s));
  // dL/dI through the moments of the context's projection (Sec. 4.2)
  const dim3 igrid((unsigned)((ctx->g0.W + 255) / 256), (unsigned)ctx->g0.H);
  auto image_grad = [&](double *out) -> int {
    if (ctx->p.projection == AC_PROJ_NODE)
      AC_RUN(AC_PROF_SETUP, (k_adj_image_node<<<igrid, 256, 0, ctx->s>>>(A.gm, ctx->img64, ctx->g0, out), 1));
    else
      AC_RUN(AC_PROF_SETUP, o->adj_image(A.gm, ctx->img64, ctx->g0, out, ctx->s));
    return AC_OK;
  };
  if (ctx->r > 0) {
    // refined grid: the cells' gradients, then their sums over each pixel
    // (the adjoint of the copy); lambda' = 2^-r lambda, eps' = 2^r eps
    int rc = image_grad(A.gimg);
    if (rc) return rc;
    AC_RUN(AC_PROF_SETUP, (k_refine_sum<<<dim3((unsigned)((ctx->W0 + 255) / 256), (unsigned)ctx->H0), 256, 0, ctx->s>>>(
                               A.gimg, ctx->W0, ctx->H0, ctx->r, ctx->g0, grad_image), 1));
  } else {
    int rc = image_grad(grad_image);
    if (rc) return rc;
  }
  AC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 2, A.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  AC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 1, A.ndiff, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->s));
  AC_CUDA(cudaMemcpyAsync(ctx->u, A.uT, fN, cudaMemcpyDeviceToDevice, ctx->s));  // leave u = u^T
  AC_CUDA(cudaStreamSynchronize(ctx->s));
  *grad_lambda = std::ldexp(ctx->h_scalars[2], -ctx->r);
  *grad_eps = std::ldexp(ctx->h_scalars[3], ctx->r);
  {
    unsigned long long nd = 0;
    std::memcpy(&nd, ctx->h_scalars + 1, sizeof nd);
    A.recompute_diff = (int64_t)nd;
  }
  if (status) fail(status, "an adjoint solve did not reach its tolerance");
  return status;
}

int ac_adjoint_recompute_diff(ac_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return fail(AC_ERR_ARG, "NULL argument");
  *count = ctx->adj.recompute_diff;
  return AC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent images (uneven sizes and phase counts).
//
// Every image has its own context (its own CUDA-graph V-cycles); the images
// are spread over a pool of CUDA streams by longest-processing-time-first on
// the node count times N, and one host worker thread per stream advances its
// images, so the GPU runs many images' kernels at once while each image keeps
// its own convergence control.  Each image's arithmetic is exactly that of a
// single-image context with the same parameters.
// ---------------------------------------------------------------------------

struct ac_batch {
  std::vector<ac_ctx *> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<std::vector<int>> assign;  // image indices per stream
  int launch = AC_BATCH_STREAMS;         // ac_batch_set_launch
  // AC_BATCH_ONE_GRAPH: one graph holding a time step of every image, each
  // with its device-side loop (captured on first use, dropped on a schedule
  // change), and the launches of each image's part of it
  cudaGraphExec_t group = nullptr;
  std::vector<StepGraph> counts;
};

namespace {

// Change a context's schedule: pre/post sweeps, the number of multigrid
// levels in use and the coarse smoother (gs: 3-colour Gauss-Seidel, else
// l1-Jacobi).  The captured graphs depend on them, so they are dropped.
void set_schedule(ac_ctx *ctx, int nu1, int nu2, int depth, bool gs) {
  release_step_graphs(ctx);
  for (int a = 0; a < 2; ++a) {
    for (int b = 0; b < 2; ++b) slot_release(ctx->sv.smooth_resid[a][b]);
    for (int f = 0; f < 2; ++f) slot_release(ctx->sv.correction[a][f]);
  }
  ctx->p.nu1 = nu1;
  ctx->p.nu2 = nu2;
  ctx->sv.coarse_gs = gs;
  const int L = (int)ctx->sv.lv.size();
  ctx->sv.depth = depth < 1 ? 1 : (depth > L ? L : depth);
  ctx->delta_warm = false;  // the next step starts its correction from zero
  ctx->sv.was_tiled = false;
  // the tiled levels may change with the depth: let the next cycle write
  // every tile of every level again (see kLiveNow)
  for (int k = 1; k < L; ++k) {
    cudaMemsetAsync(ctx->sv.lv[k].lists.flags, ac::kLiveNow, tile_flag_bytes(ctx->sv.lv[k].g, ctx->N), ctx->s);
    cudaMemsetAsync(ctx->sv.lv[k].lists.dirty, 1, tile_flag_bytes(ctx->sv.lv[k].g, 1), ctx->s);
  }
}

// AC_BATCH_ONE_GRAPH: capture one time step of every image into a single
// graph.  Each image's step (with its device-side loop, enqueue_step_loop)
// is captured on streams[0] into the same graph with no dependencies, so the
// images form independent chains that the graph runs side by side; the
// images' own buffers keep them apart.
int build_group(ac_batch *b) {
  const int count = (int)b->ctx.size();
  for (int k = 0; k < count; ++k) {
    ac_ctx *c = b->ctx[k];
    if (!c->use_graphs || c->profiling || tiled_end(c->sv) > 1)
      return fail(AC_ERR_STATE, "image %d cannot run its cycle loop on the device (coarse levels that can run "
                                "tiled, or profiling)", k);
    int rc = loop_resources(c);
    if (rc) return rc;
  }
  for (cudaStream_t st : b->streams) AC_CUDA(cudaStreamSynchronize(st));
  cudaGraph_t g = nullptr;
  AC_CUDA(cudaGraphCreate(&g, 0));
  cudaStream_t cs = b->streams[0];
  b->counts.assign(count, StepGraph{});
  int rc = AC_OK;
  for (int k = 0; k < count && !rc; ++k) {
    ac_ctx *c = b->ctx[k];
    cudaStream_t own = c->s;
    c->s = cs;
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      rc = fail(AC_ERR_CUDA, "cudaStreamBeginCaptureToGraph: %s", cudaGetErrorString(e));
    } else {
      rc = enqueue_step_loop(c, g, false, b->counts[k]);
      cudaGraph_t g2 = nullptr;
      e = cudaStreamEndCapture(cs, &g2);
      if (!rc && e != cudaSuccess) rc = fail(AC_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    }
    c->s = own;
  }
  if (!rc) {
    cudaError_t e = cudaGraphInstantiate(&b->group, g, 0);
    if (e != cudaSuccess) {
      b->group = nullptr;
      rc = fail(AC_ERR_CUDA, "cudaGraphInstantiate (batch): %s", cudaGetErrorString(e));
    }
  }
  cudaGraphDestroy(g);
  cudaGetLastError();
  return rc;
}

// ac_batch_step in AC_BATCH_ONE_GRAPH: every image's control block is reset
// on streams[0], the group graph is launched once per time step there, and
// the control blocks are read back after one synchronisation.
int batch_step_one_graph(ac_batch *b, int n_steps, std::vector<ac_stats> &st, std::vector<int> &rcs,
                         std::vector<std::string> &msgs) {
  if (!b->group) {
    int rc = build_group(b);
    if (rc) return rc;
  }
  cudaStream_t s0 = b->streams[0];
  for (cudaStream_t st2 : b->streams) AC_CUDA(cudaStreamSynchronize(st2));
  const int count = (int)b->ctx.size();
  for (int k = 0; k < count; ++k)
    AC_CUDA((k_ctl_reset<<<1, 1, 0, s0>>>(b->ctx[k]->ctl, b->ctx[k]->delta_warm ? 1 : 0), cudaGetLastError()));
  for (int t = 0; t < n_steps; ++t) AC_CUDA(cudaGraphLaunch(b->group, s0));
  for (int k = 0; k < count; ++k)
    AC_CUDA(cudaMemcpyAsync(b->ctx[k]->h_ctl, b->ctx[k]->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s0));
  AC_CUDA(cudaStreamSynchronize(s0));
  for (int k = 0; k < count; ++k) {
    rcs[k] = loop_stats(b->ctx[k], b->counts[k], n_steps, &st[k]);
    if (rcs[k]) msgs[k] = ac_last_error();
  }
  return AC_OK;
}

}  // namespace

extern "C" {

int ac_batch_set_launch(ac_batch *b, int mode) {
  if (!b) return fail(AC_ERR_ARG, "batch is NULL");
  if (mode != AC_BATCH_STREAMS && mode != AC_BATCH_ONE_GRAPH)
    return fail(AC_ERR_ARG, "mode must be AC_BATCH_STREAMS or AC_BATCH_ONE_GRAPH");
  b->launch = mode;
  return AC_OK;
}

int ac_batch_set_cycle_loop(ac_batch *b, int mode) {
  if (!b) return fail(AC_ERR_ARG, "batch is NULL");
  for (ac_ctx *c : b->ctx) {
    int rc = ac_set_cycle_loop(c, mode);
    if (rc) return rc;
  }
  return AC_OK;
}

int ac_batch_create(ac_batch **out, const ac_params *params, int count, int n_streams) {
  if (!out || !params || count < 1 || n_streams < 1) return fail(AC_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  for (int k = 0; k < count; ++k) {
    int rc = validate(&params[k]);
    if (rc) return fail(rc, "image %d: %s", k, g_last_error.c_str());
  }
  ac_batch *b = new (std::nothrow) ac_batch;
  if (!b) return fail(AC_ERR_NOMEM, "host allocation failed");
  if (n_streams > count) n_streams = count;
  auto cleanup = [&](int rc) {
    std::string msg = g_last_error;
    ac_batch_destroy(b);
    g_last_error = msg;
    return rc;
  };
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(AC_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    b->streams.push_back(st);
  }
  // longest-processing-time-first assignment of images to streams
  std::vector<int> order(count);
  for (int k = 0; k < count; ++k) order[k] = k;
  auto cost = [&](int k) { return (double)(params[k].width + 1) * (params[k].height + 1) * params[k].n_phases; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
  std::vector<double> load(n_streams, 0.0);
  b->assign.assign(n_streams, {});
  std::vector<int> stream_of(count);
  for (int k : order) {
    int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[best] += cost(k);
    b->assign[best].push_back(k);
    stream_of[k] = best;
  }
  for (auto &v : b->assign) std::sort(v.begin(), v.end());
  b->ctx.assign(count, nullptr);
  for (int k = 0; k < count; ++k) {
    ac_params p = params[k];
    p.stream = b->streams[stream_of[k]];
    int rc = ac_create(&b->ctx[k], &p);
    if (rc) return cleanup(rc);
    // in the stream pool the host loop measured faster (3.54 against 3.66 s
    // for 30 steps of the 256-image workload): the streams' work already
    // covers each image's round trips, and the WHILE bodies launched on the
    // device overlapped less across the streams
    b->ctx[k]->loop_mode = AC_LOOP_HOST;
  }
  *out = b;
  return AC_OK;
}

void ac_batch_destroy(ac_batch *b) {
  if (!b) return;
  if (b->group) cudaGraphExecDestroy(b->group);
  for (ac_ctx *c : b->ctx) ac_destroy(c);
  for (cudaStream_t st : b->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete b;
}

static int batch_index(ac_batch *b, int k) {
  if (!b) return fail(AC_ERR_ARG, "batch is NULL");
  if (k < 0 || k >= (int)b->ctx.size()) return fail(AC_ERR_ARG, "image index %d out of range", k);
  return AC_OK;
}

int ac_batch_set_image(ac_batch *b, int k, const float *rgb, int is_device) {
  int rc = batch_index(b, k);
  return rc ? rc : ac_set_image(b->ctx[k], rgb, is_device);
}

int ac_batch_set_phase(ac_batch *b, int k, const double *u, int is_device) {
  int rc = batch_index(b, k);
  return rc ? rc : ac_set_phase(b->ctx[k], u, is_device);
}

int ac_batch_get_phase(ac_batch *b, int k, double *u, int is_device) {
  int rc = batch_index(b, k);
  return rc ? rc : ac_get_phase(b->ctx[k], u, is_device);
}

int ac_batch_segment(ac_batch *b, int k, int8_t *labels, int is_device) {
  int rc = batch_index(b, k);
  return rc ? rc : ac_segment(b->ctx[k], 0, labels, is_device, nullptr);
}

int ac_batch_step(ac_batch *b, int n_steps, ac_batch_stats *out) {
  if (!b) return fail(AC_ERR_ARG, "batch is NULL");
  if (n_steps < 0) return fail(AC_ERR_ARG, "n_steps must be >= 0");
  const int count = (int)b->ctx.size();
  std::vector<ac_stats> st(count);
  std::vector<int> rcs(count, AC_OK);
  std::vector<std::string> msgs(count);
  if (b->launch == AC_BATCH_ONE_GRAPH && n_steps > 0) {
    int rc = batch_step_one_graph(b, n_steps, st, rcs, msgs);
    if (rc) return rc;
  } else {
    std::vector<std::thread> workers;
    for (size_t s = 0; s < b->streams.size(); ++s)
      workers.emplace_back([&, s]() {
        for (int k : b->assign[s]) {
          rcs[k] = ac_step(b->ctx[k], n_steps, &st[k]);
          if (rcs[k]) msgs[k] = ac_last_error();
        }
      });
    for (auto &w : workers) w.join();
  }
  ac_batch_stats agg{};
  agg.images = count;
  agg.steps = n_steps;
  int status = AC_OK;
  for (int k = 0; k < count; ++k) {
    agg.total_cycles += st[k].total_cycles;
    agg.fine_sweeps += st[k].fine_sweeps;
    agg.converged_images += st[k].converged;
    agg.nodes += b->ctx[k]->n;
    agg.dof += b->ctx[k]->n * b->ctx[k]->N;
    agg.dof_sweeps += (double)st[k].fine_sweeps * (double)(b->ctx[k]->n * b->ctx[k]->N);
    if (rcs[k] && (status == AC_OK || status == AC_ERR_NOT_CONVERGED)) {
      status = rcs[k];
      g_last_error = "image " + std::to_string(k) + ": " + msgs[k];
    }
  }
  if (out) *out = agg;
  return status;
}

// Empirical schedule search.  Images with the same size, phase count and
// model parameters form a group; on the group's first image every candidate
// coarse smoother (3-colour Gauss-Seidel, l1-Jacobi) x (nu1, nu2) in {(1,1),
// (2,1), (1,2), (2,2)} x depth in {all levels, 5} is run for trial_steps steps
// from the image's current state (restored after each trial) and timed; the
// fastest candidate whose steps all converged is applied to the whole group.
int ac_batch_tune(ac_batch *b, int trial_steps, int *chosen) {
  if (!b || trial_steps < 1) return fail(AC_ERR_ARG, "bad tune arguments");
  if (b->group) {
    // the schedules change: the group graph is captured again on next use
    for (cudaStream_t st : b->streams) cudaStreamSynchronize(st);
    cudaGraphExecDestroy(b->group);
    b->group = nullptr;
  }
  const int count = (int)b->ctx.size();
  std::map<std::tuple<int, int, int, int, double, double, double, double>, std::vector<int>> groups;
  for (int k = 0; k < count; ++k) {
    const ac_params &p = b->ctx[k]->p;
    if (!b->ctx[k]->have_image) return fail(AC_ERR_STATE, "image %d has no image set", k);
    groups[std::make_tuple(p.width, p.height, p.n_phases, p.precision, p.eps, p.lambda, p.tau, p.tol)].push_back(k);
  }
  const int nus[4][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}};
  for (auto &kv : groups) {
    ac_ctx *c = b->ctx[kv.second.front()];
    const int L = (int)c->sv.lv.size();
    // the state a trial starts from and is restored to: u and the colour
    // means of the last step (the empty-phase fallback)
    void *snap = nullptr;
    const size_t bytes = (size_t)c->n * c->N * sizeof(double), cbytes = (size_t)3 * c->N * sizeof(double);
    double c_snap[3 * AC_MAX_PHASES];
    cudaError_t e = cudaMalloc(&snap, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AC_ERR_NOMEM, "cudaMalloc(%zu) for the tuning snapshot: %s", bytes, cudaGetErrorString(e));
    }
    auto restore = [&]() -> int {
      int r = ac_set_phase(c, (const double *)snap, 1);
      if (r) return r;
      cudaError_t e2 = cudaMemcpyAsync(c->c, c_snap, cbytes, cudaMemcpyHostToDevice, c->s);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->s);
      return e2 == cudaSuccess ? AC_OK : fail(AC_ERR_CUDA, "restoring the tuning snapshot: %s", cudaGetErrorString(e2));
    };
    int rc = AC_OK;
    e = cudaMemcpyAsync(snap, c->u, bytes, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c_snap, c->c, cbytes, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) rc = fail(AC_ERR_CUDA, "tuning snapshot: %s", cudaGetErrorString(e));
    double best_t = 1e300;
    int best[4] = {c->p.nu1, c->p.nu2, L, c->sv.coarse_gs ? AC_SMOOTH_GS3 : AC_SMOOTH_JACOBI};
    for (int sm = 0; sm < 2 && !rc; ++sm)
    for (int nu = 0; nu < 4 && !rc; ++nu)
      for (int dd = 0; dd < 2 && !rc; ++dd) {
        const int depth = dd == 0 ? L : (L < 5 ? L : 5);
        if (dd == 1 && depth == L) continue;
        const int smoother = sm == 0 ? AC_SMOOTH_GS3 : AC_SMOOTH_JACOBI;
        set_schedule(c, nus[nu][0], nus[nu][1], depth, smoother == AC_SMOOTH_GS3);
        rc = restore();
        if (rc) break;
        ac_stats st{};
        auto t0 = std::chrono::steady_clock::now();
        int r = ac_step(c, trial_steps, &st);
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (r != AC_OK && r != AC_ERR_NOT_CONVERGED) {
          rc = r;
          break;
        }
        if (st.converged && t < best_t) {
          best_t = t;
          best[0] = nus[nu][0];
          best[1] = nus[nu][1];
          best[2] = depth;
          best[3] = smoother;
        }
      }
    int rc2 = rc ? rc : restore();
    cudaStreamSynchronize(c->s);
    cudaFree(snap);
    if (rc2) return rc2;
    for (int k : kv.second) {
      set_schedule(b->ctx[k], best[0], best[1], best[2], best[3] == AC_SMOOTH_GS3);
      if (chosen)
        for (int q = 0; q < 4; ++q) chosen[4 * k + q] = best[q];
    }
  }
  return AC_OK;
}

}  // extern "C"
