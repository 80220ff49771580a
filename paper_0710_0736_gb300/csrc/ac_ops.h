// ac_ops.h -- host-side launch table of the per-N kernel instantiations.
// Every launcher returns the number of kernels it launched.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ac {

struct Geo;
struct Galerkin0Table;
struct MaskDirty;

// Scratch of the block-partial reductions: at most kMaxPartBlocks rows.
constexpr int kMaxPartBlocks = 1024;

// The bottom levels k0 .. k0 + levels - 1 of a coarse V-cycle, run by one
// block per phase in shared memory (kTailArrays values per node: C, E, N,
// NE, r, v, t); the last level is the coarsest.
constexpr int kTailMaxLevels = 8;
constexpr int kTailArrays = 7;
constexpr size_t kTailSmemBytes = 200 * 1024;  // shared memory cap of one block
struct TailArgs {
  int levels;
  int W[kTailMaxLevels], H[kTailMaxLevels];
  const void *op[kTailMaxLevels];  // phase-major C, E, N, NE planes of each level
};

// The live-tile state of a tiled coarse level (see kLiveNow in
// ac_device.cuh): its flags, the work lists its Galerkin kernel appends --
// (tile, phase) items and, on the first level, tiles with their phase masks --
// with their two counts (cleared before each coarse correction), the lists'
// capacity and the device's multiprocessors.  A launch that strides over a
// list runs as many blocks as can be resident at once (at most the
// capacity), so that no block waits for another to finish its share.  Null
// for a dense level.
struct LevelLists {
  uint8_t *flags;
  uint64_t *items;
  uint64_t *tiles;
  uint8_t *dirty;    // per tile: the fine mask under it changed since its operator was computed (first level)
  uint8_t *changed;  // per tile: its operator was rewritten in this cycle's correction
  int *count;  // [0] items, [1] tiles
  int64_t cap; // tiles x phases
  int sms;
};

// One multigrid solve instantiation (scalar type and constraint form); array
// arguments are typed by that instantiation (double or float).
struct SolverOps {
  int elem;  // sizeof(scalar)
  // sweeps red-black sweeps in place; with corr != null the pending coarse
  // correction x += (*omega) corr is applied inside the first launch; with
  // mask != null the last launch stores its colour's free mask (and rt = 0
  // for that colour if rt != null)
  // (dirty: the first coarse level's tiles to mark where the mask changes)
  int (*smooth)(void *x, const void *rhs, const void *ob, const void *corr, const double *omega, const Geo &g,
                int sweeps, void *rt, uint8_t *mask, const MaskDirty &dirty, cudaStream_t s);
  // color < 0: every node; 0: the first colour only (completes a masked smooth)
  int (*resid)(const void *x, const void *rhs, const void *ob, const Geo &g, void *rt, uint8_t *mask, double *rho,
               int color, const MaskDirty &dirty, cudaStream_t s);
  // transfers skip the rows whose diagonal in the (coarse or fine) level's
  // operator is 0: those rows and their residuals are exactly 0.  LevelLists
  // arguments: the live-tile state of a tiled level, or null for a level
  // kept dense
  int (*restrict0)(const void *rt, const Geo &gf, const Geo &gc, const void *op1, void *r1, const LevelLists *L1,
                   cudaStream_t s);
  // dirty (dense level, nullable): per tile, the fine mask under it changed
  // since its operator was computed; clean tiles are skipped, dirty ones
  // recomputed and cleared
  int (*galerkin0)(const uint8_t *mask, const Geo &gf, const Geo &gc, const Galerkin0Table &tab, void *op,
                   const LevelLists *L1, uint8_t *dirty, cudaStream_t s);
  // Lc != null: a tiled coarse level from a tiled fine level (Lf)
  int (*galerkin)(const void *opf, const Geo &gf, const Geo &gc, void *opc, const LevelLists *Lf,
                  const LevelLists *Lc, cudaStream_t s);
  // `sweeps` (even) smoothing sweeps in fused pairs starting from v, using v
  // and tmp in turn; *out returns the buffer holding the result.  zero_start:
  // v = 0 on entry (it is then neither read nor needs clearing).  gs:
  // 3-colour Gauss-Seidel on shared-memory tiles, else l1-Jacobi
  int (*coarse_smooth)(const void *op, const void *r, void *v, void *tmp, const Geo &g, int sweeps, bool zero_start,
                       void **out, const LevelLists *L, bool gs, cudaStream_t s);
  int (*coarse_solve)(const void *op, const void *r, void *v, const Geo &g, int sweeps, cudaStream_t s);
  int (*coarse_resid)(const void *op, const void *r, const void *v, const Geo &g, void *t, const LevelLists *L,
                      cudaStream_t s);
  // one pair of smoothing sweeps from v = 0, then t = r - S v
  int (*coarse_pre_resid)(const void *op, const void *r, void *v, void *t, const Geo &g, const LevelLists *L,
                          bool gs, cudaStream_t s);
  int (*restrict_)(const void *t, const Geo &gf, const Geo &gc, const void *opc, void *rc, const LevelLists *Lc,
                   cudaStream_t s);
  int (*prolong_add)(const void *vc, const Geo &gf, const Geo &gc, const void *opf, void *vf, const LevelLists *Lf,
                     cudaStream_t s);
  // v of level k0 from r of level k0 by the whole cycle below it (see
  // TailArgs); smem bytes of dynamic shared memory per block
  int (*coarse_tail)(const TailArgs &a, const void *r0, void *v0, int coarse_sweeps, int coarsest_sweeps,
                     size_t smem, bool gs, cudaStream_t s);
  // line search: part needs 2 x (blocks of the fine grid) doubles, tot 2 doubles
  int (*line_search)(const void *x, const void *ob, const void *rt, const void *v1, const uint8_t *mask,
                     const Geo &gf, const Geo &gc, void *d, double *part, double *tot, double *omega, cudaStream_t s);
};

struct Ops {
  int N;
  int (*moments_f32)(const float *img, const Geo &g, double *mom, cudaStream_t s);
  int (*moments_f64)(const double *img, const Geo &g, double *mom, cudaStream_t s);
  int (*init_random)(double *u, int64_t n, uint64_t seed, cudaStream_t s);
  // colour means (+ energy if energy != null): part (kMaxPartBlocks x 7N), tot (7N), c (N x 3 in/out)
  int (*means)(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
               double *energy, double eps, double lam, cudaStream_t s);
  int (*rhs)(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl, double *b,
             cudaStream_t s);
  // the mixed form's colour means (+ energy) and right-hand side in
  // double-float arithmetic; b as N float heads then N float tails per node
  int (*means_df)(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
                  double *energy, double eps, double lam, cudaStream_t s);
  int (*rhs_df)(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl, float *b,
                cudaStream_t s);
  // b from rhs_df.  rho32: the solve's residual, formed in double-float
  // arithmetic, with the natural residual through the float projection
  // (accurate to a few float ulps of rho near the solution); otherwise FP64
  // throughout
  int (*outer_resid)(const double *u, const float *b, const Geo &g, float *r32, float *u32, double *rho, bool rho32,
                     cudaStream_t s);
  int (*outer_update)(double *u, const float *delta, const Geo &g, cudaStream_t s);
  // pixel outputs are on the image's pixels: the solve grid g coarsened r times
  int (*labels)(const double *u, const Geo &g, int r, int8_t *node_lab, int8_t *pix_lab, cudaStream_t s);
  int (*composite)(const double *u, const double *c, const Geo &g, int r, int rounded, float *out, cudaStream_t s);
  int (*project)(const double *y, double *x, int64_t count, cudaStream_t s);
  SolverOps fp64;     // T = double, direct form
  SolverOps mixed;    // T = float, shifted form
  SolverOps adjoint;  // T = double, tangent form (frozen free set)
  SolverOps adjoint32;  // T = float, tangent form: the FP32 preconditioner of the adjoint's FCG
  // node-order binary64 <-> colour-split float node arrays (N values per node);
  // from_split32 projects onto the tangent space of freeset (nullable)
  int (*to_split32)(const double *in, const Geo &g, float *out, cudaStream_t s);
  int (*from_split32)(const float *in, const Geo &g, const double *freeset, double *out, cudaStream_t s);
  // adjoint of a time step
  int (*adj_prepare)(const double *up, const double *g, int64_t n, double *freeset, double *rhs, cudaStream_t s);
  // part: (blocks of the level) x (2 + 3N), tot: 2 + 3N, scal[0..1] += lambda/eps gradients
  int (*adj_accum)(const double *w, const double *u, const double *up, const double *mom, const double *c,
                   const Geo &g, double tau, double eps, double lam, double *gm, double *part, double *tot,
                   double *scal, cudaStream_t s);
  int (*adj_back)(const double *w, const double *u, const double *mom, const double *c, const double *tot,
                  const double *mass, const Geo &g, double a1, double *gout, double *gm, cudaStream_t s);
  int (*adj_image)(const double *gm, const double *img, const Geo &g, double *gimg, cudaStream_t s);
  int (*absmax)(const double *v, int64_t count, double *out, cudaStream_t s);
  // flexible CG on the adjoint's tangent system: q = Pi S p; two dots
  // (part: kMaxPartBlocks x 2, tot: 2); x += alpha p, r -= alpha q; p = z + beta p
  int (*tangent_apply)(const double *p, const double *f, const Geo &g, double *q, cudaStream_t s);
  int (*dot2)(const double *a0, const double *b0, const double *a1, const double *b1, int64_t count, double *part,
              double *tot, cudaStream_t s);
  int (*fcg_step)(double *x, double *r, const double *p, const double *q, double alpha, int64_t count,
                  cudaStream_t s);
  int (*fcg_dir)(double *p, const double *z, double beta, int64_t count, cudaStream_t s);
};

const Ops *ops_n2();
const Ops *ops_n3();
const Ops *ops_n4();
const Ops *ops_n5();
const Ops *ops_n6();
const Ops *ops_n7();
const Ops *ops_n8();

}  // namespace ac
