// ac_launch.cuh -- host launchers wrapping the kernel templates for one N.
#pragma once
#include "ac_kernels.cuh"

namespace ac {

inline dim3 row_grid(int count_per_row, int rows, int block = kBlock) {
  return dim3((unsigned)((count_per_row + block - 1) / block), (unsigned)rows);
}

template <int N>
struct Launch {
  static int moments_f32(const float *img, const Geo &g, double *mom, cudaStream_t s) {
    k_moments<float><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(img, g, mom);
    return 1;
  }
  static int moments_f64(const double *img, const Geo &g, double *mom, cudaStream_t s) {
    k_moments<double><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(img, g, mom);
    return 1;
  }
  static int init_random(double *u, int64_t n, uint64_t seed, cudaStream_t s) {
    k_init_random<N><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(u, n, seed);
    return 1;
  }
  static int part_blocks_(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (int)(b < kMaxPartBlocks ? b : kMaxPartBlocks);
  }
  static int means(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
                    double *energy, double eps, double lam, cudaStream_t s) {
    const int64_t n = (int64_t)g.Wn * (g.H + 1);
    const int blocks = part_blocks_(n);
    k_means_partial<N><<<blocks, kBlock, 0, s>>>(u, mom, g, part);
    k_colsum<<<7 * N, kBlock, 0, s>>>(part, blocks, 7 * N, tot);
    k_means_finish<N><<<1, 32, 0, s>>>(tot, c, energy, eps, lam);
    return 3;
  }
  static int rhs(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl, double *b,
                  cudaStream_t s) {
    const int64_t n = (int64_t)g.Wn * (g.H + 1);
    k_rhs<N><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(u, mom, c, g, a1, tl, b);
    return 1;
  }
  static int smooth_fine(double *u, const double *b, const Geo &g, int sweeps, cudaStream_t s) {
    const dim3 grid = row_grid((g.W + 2) / 2, g.H + 1);
    for (int k = 0; k < sweeps; ++k) {
      k_smooth_fine<double, N><<<grid, kBlock, 0, s>>>(u, b, g, 0);
      k_smooth_fine<double, N><<<grid, kBlock, 0, s>>>(u, b, g, 1);
    }
    return 2 * sweeps;
  }
  static int fine_resid(const double *u, const double *b, const Geo &g, double *rt, uint8_t *mask, double *rho,
                         cudaStream_t s) {
    k_fine_resid<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, b, g, rt, mask, rho);
    return 1;
  }
  static int restrict_(const double *t, const Geo &gf, const Geo &gc, double *rc, cudaStream_t s) {
    k_restrict<N><<<row_grid(gc.W + 1, gc.H + 1), kBlock, 0, s>>>(t, gf, gc, rc);
    return 1;
  }
  static int galerkin0(const uint8_t *mask, const Geo &gf, const Geo &gc, double *op, cudaStream_t s) {
    k_galerkin0<N><<<row_grid(gc.W + 1, gc.H + 1), kBlock, 0, s>>>(mask, gf, gc, op);
    return 1;
  }
  static int galerkin(const double *opf, const Geo &gf, const Geo &gc, double *opc, cudaStream_t s) {
    k_galerkin<N><<<row_grid(gc.W + 1, gc.H + 1), kBlock, 0, s>>>(opf, gf, gc, opc);
    return 1;
  }
  static int coarse_smooth(const double *op, const double *r, double *v, const Geo &g, int sweeps, cudaStream_t s) {
    const dim3 grid = row_grid((g.W + 3) / 3, g.H + 1);
    for (int k = 0; k < sweeps; ++k)
      for (int c = 0; c < 3; ++c) k_coarse_smooth<N><<<grid, kBlock, 0, s>>>(op, r, v, g, c);
    return 3 * sweeps;
  }
  static int coarse_solve(const double *op, const double *r, double *v, const Geo &g, int sweeps, cudaStream_t s) {
    k_coarse_solve_block<N><<<1, 1024, 0, s>>>(op, r, v, g, sweeps);
    return 1;
  }
  static int coarse_resid(const double *op, const double *r, const double *v, const Geo &g, double *t,
                           cudaStream_t s) {
    k_coarse_resid<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(op, r, v, g, t);
    return 1;
  }
  static int prolong_add(const double *vc, const Geo &gf, const Geo &gc, double *vf, cudaStream_t s) {
    k_prolong_add<N><<<row_grid(gf.W + 1, gf.H + 1), kBlock, 0, s>>>(vc, gf, gc, vf);
    return 1;
  }
  static int line_search(const double *u, const double *rt, const double *v1, const uint8_t *mask, const Geo &gf,
                          const Geo &gc, double *d, double *part, double *tot, double *omega, cudaStream_t s) {
    const dim3 grid = row_grid(gf.W + 1, gf.H + 1);
    const int blocks = (int)(grid.x * grid.y);
    k_ls_dir<N><<<grid, kBlock, 0, s>>>(u, rt, v1, mask, gf, gc, d, part);
    k_ls_curv<N><<<grid, kBlock, 0, s>>>(d, gf, part + blocks);
    k_colsum<<<1, kBlock, 0, s>>>(part, blocks, 1, tot);
    k_colsum<<<1, kBlock, 0, s>>>(part + blocks, blocks, 1, tot + 1);
    k_ls_finish<<<1, 32, 0, s>>>(tot, omega);
    return 5;
  }
  static int apply(double *u, const double *d, const double *omega, int64_t n, cudaStream_t s) {
    k_apply<N><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(u, d, omega, n);
    return 1;
  }
  static int labels(const double *u, const Geo &g, int8_t *node_lab, int8_t *pix_lab, cudaStream_t s) {
    k_labels<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, g, node_lab, pix_lab);
    return 1;
  }
  static int project(const double *y, double *x, int64_t count, cudaStream_t s) {
    if (count <= 0) return 0;
    k_project<N><<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, s>>>(y, x, count);
    return 1;
  }
  static const Ops *table() {
    static const Ops t = {N,           moments_f32, moments_f64,   init_random,  means,        rhs,
                          smooth_fine, fine_resid,  restrict_,     galerkin0,    galerkin,     coarse_smooth,
                          coarse_solve, coarse_resid, prolong_add, line_search,  apply,        labels,
                          project};
    return &t;
  }
};

}  // namespace ac
