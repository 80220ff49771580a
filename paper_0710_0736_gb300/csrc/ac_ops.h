// ac_ops.h -- host-side launch table of the per-N kernel instantiations.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ac {

struct Geo;

// Scratch of the block-partial reductions: at most kMaxPartBlocks rows.
constexpr int kMaxPartBlocks = 1024;

// Every launcher returns the number of kernels it launched.
struct Ops {
  int N;
  int (*moments_f32)(const float *img, const Geo &g, double *mom, cudaStream_t s);
  int (*moments_f64)(const double *img, const Geo &g, double *mom, cudaStream_t s);
  int (*init_random)(double *u, int64_t n, uint64_t seed, cudaStream_t s);
  // colour means + energy: part (kMaxPartBlocks x 7N scratch), tot (7N), c (N x 3 in/out), energy (1)
  int (*means)(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
                double *energy, double eps, double lam, cudaStream_t s);
  int (*rhs)(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl, double *b,
              cudaStream_t s);
  int (*smooth_fine)(double *u, const double *b, const Geo &g, int sweeps, cudaStream_t s);
  int (*fine_resid)(const double *u, const double *b, const Geo &g, double *rt, uint8_t *mask, double *rho,
                     cudaStream_t s);
  int (*restrict_)(const double *t, const Geo &gf, const Geo &gc, double *rc, cudaStream_t s);
  int (*galerkin0)(const uint8_t *mask, const Geo &gf, const Geo &gc, double *op, cudaStream_t s);
  int (*galerkin)(const double *opf, const Geo &gf, const Geo &gc, double *opc, cudaStream_t s);
  int (*coarse_smooth)(const double *op, const double *r, double *v, const Geo &g, int sweeps, cudaStream_t s);
  int (*coarse_solve)(const double *op, const double *r, double *v, const Geo &g, int sweeps, cudaStream_t s);
  int (*coarse_resid)(const double *op, const double *r, const double *v, const Geo &g, double *t, cudaStream_t s);
  int (*prolong_add)(const double *vc, const Geo &gf, const Geo &gc, double *vf, cudaStream_t s);
  // line search: part needs 2 x (blocks of the fine grid) doubles, tot 2 doubles
  int (*line_search)(const double *u, const double *rt, const double *v1, const uint8_t *mask, const Geo &gf,
                      const Geo &gc, double *d, double *part, double *tot, double *omega, cudaStream_t s);
  int (*apply)(double *u, const double *d, const double *omega, int64_t n, cudaStream_t s);
  int (*labels)(const double *u, const Geo &g, int8_t *node_lab, int8_t *pix_lab, cudaStream_t s);
  int (*project)(const double *y, double *x, int64_t count, cudaStream_t s);
};

const Ops *ops_n2();
const Ops *ops_n3();
const Ops *ops_n4();
const Ops *ops_n5();
const Ops *ops_n6();
const Ops *ops_n7();
const Ops *ops_n8();

// Number of thread blocks of a row-per-blockIdx.y launch over a level.
int fine_grid_blocks(const Geo &g);

}  // namespace ac
