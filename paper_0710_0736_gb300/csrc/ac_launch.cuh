// ac_launch.cuh -- host launchers wrapping the kernel templates for one N.
#pragma once
#include <algorithm>
#include "ac_kernels.cuh"

namespace ac {

inline dim3 row_grid(int count_per_row, int rows, int block = kBlock) {
  return dim3((unsigned)((count_per_row + block - 1) / block), (unsigned)rows);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// One thread per (node, phase) of a coarse level: rows of count_per_row
// nodes, the phase in blockIdx.z; narrow levels get narrower blocks.
struct PhaseLaunch {
  dim3 grid;
  unsigned block;
};
// Levels at least this large take the node-wide variant of the light
// transfer kernels (one thread per node, all phases).
constexpr int64_t kWideLevelNodes = 1 << 20;

inline PhaseLaunch phase_grid(int count_per_row, int rows, int phases) {
  const unsigned b = count_per_row >= kBlock ? (unsigned)kBlock : (unsigned)(((count_per_row + 31) / 32) * 32);
  return {dim3((unsigned)((count_per_row + (int)b - 1) / (int)b), (unsigned)rows, (unsigned)phases), b};
}

// The TileList view of a level's items (dense: null) and the grid that
// strides over it (dense: the level's tiles x phases).
inline TileList item_list(const LevelLists *L) {
  return L ? TileList{L->items, L->count} : TileList{nullptr, nullptr};
}
// Blocks of kernel k with `threads` threads resident on one SM (at least 1).
template <class K>
inline int resident_blocks(K k, int threads) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, threads, 0) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}
// The grid of a launch of kernel k over a level's lists: every block
// resident at once, no more blocks than list entries can exist.
template <class K>
inline dim3 list_grid(const LevelLists *L, int64_t entries, K k, int threads) {
  static const int per_sm = resident_blocks(k, threads);
  const int64_t b = (int64_t)L->sms * per_sm;
  return dim3((unsigned)(b < entries ? b : (entries > 0 ? entries : 1)));
}
template <class K>
inline dim3 tile_grid(const Geo &g, const LevelLists *L, int N, K k, int threads) {
  return L ? list_grid(L, L->cap, k, threads) : dim3((unsigned)tiles_x(g), (unsigned)tiles_y(g), (unsigned)N);
}

template <typename T, int N, int FORM>
struct SolverLaunch {
  // `sweeps` red-black sweeps in place, one launch per colour; the pending
  // coarse correction (corr != null) is applied inside the first launch.
  // With mask != null the last launch (colour 1) also stores its nodes' free
  // mask (and rt = 0 if rt != null), so that resid(color = 0) completes them.
  static int smooth(void *x, const void *rhs, const void *ob, const void *corr, const double *omega, const Geo &g,
                    int sweeps, void *rt, uint8_t *mask, const MaskDirty &dirty, cudaStream_t s) {
    const dim3 grid = row_grid((g.W + 2) / 2, g.H + 1);
    for (int k = 0; k < sweeps; ++k)
      for (int c = 0; c < 2; ++c) {
        const T *cr = k == 0 && c == 0 ? (const T *)corr : nullptr;
        if (mask && k == sweeps - 1 && c == 1)
          k_smooth_fine<T, N, FORM, true><<<grid, kBlock, 0, s>>>((T *)x, (const T *)rhs, (const T *)ob, cr, omega,
                                                                g, c, (T *)rt, mask, dirty);
        else
          k_smooth_fine<T, N, FORM, false><<<grid, kBlock, 0, s>>>((T *)x, (const T *)rhs, (const T *)ob, cr, omega,
                                                                 g, c, nullptr, nullptr, MaskDirty{nullptr, 0, 0});
      }
    return 2 * sweeps;
  }
  // color < 0: every node; 0: the first colour only (after smooth() with a mask)
  static int resid(const void *x, const void *rhs, const void *ob, const Geo &g, void *rt, uint8_t *mask,
                   double *rho, int color, const MaskDirty &dirty, cudaStream_t s) {
    const dim3 grid = color < 0 ? row_grid(g.W + 1, g.H + 1) : row_grid((g.W + 2) / 2, g.H + 1);
    k_fine_resid<T, N, FORM><<<grid, kBlock, 0, s>>>((const T *)x, (const T *)rhs, (const T *)ob, g, (T *)rt, mask,
                                                   rho, color, dirty);
    return 1;
  }
  static int restrict0(const void *rt, const Geo &gf, const Geo &gc, const void *op1, void *r1, const LevelLists *L1,
                       cudaStream_t s) {
    const dim3 grid = L1 ? list_grid(L1, L1->cap / N, k_restrict0<T, N>, kTileThreads)
                         : dim3((unsigned)tiles_x(gc), (unsigned)tiles_y(gc));
    k_restrict0<T, N><<<grid, kTileThreads, 0, s>>>((const T *)rt, gf, gc, (const T *)op1, (T *)r1,
                                                  L1 ? L1->tiles : nullptr, L1 ? L1->count + 1 : nullptr);
    return 1;
  }
  static int galerkin0(const uint8_t *mask, const Geo &gf, const Geo &gc, const Galerkin0Table &tab, void *op,
                       const LevelLists *L1, uint8_t *dirty, cudaStream_t s) {
    const dim3 grid((unsigned)tiles_x(gc), (unsigned)tiles_y(gc));
    k_galerkin0<T, N><<<grid, kTileThreads, 0, s>>>(mask, gf, gc, tab, (T *)op, L1 ? L1->flags : nullptr,
                                                  L1 ? L1->items : nullptr, L1 ? L1->tiles : nullptr,
                                                  L1 ? L1->count : nullptr, L1 ? L1->dirty : dirty,
                                                  L1 ? L1->changed : nullptr);
    return 1;
  }
  static int galerkin(const void *opf, const Geo &gf, const Geo &gc, void *opc, const LevelLists *Lf,
                      const LevelLists *Lc, cudaStream_t s) {
    if (Lc) {
      const dim3 grid((unsigned)tiles_x(gc), (unsigned)tiles_y(gc), (unsigned)N);
      k_galerkin_tiled<T, N><<<grid, kTileThreads, 0, s>>>((const T *)opf, gf, gc, (T *)opc, Lf->flags, Lc->flags,
                                                         Lc->items, Lc->count, Lf->changed, Lc->changed);
    } else {
      const PhaseLaunch L = phase_grid(gc.W + 1, gc.H + 1, N);
      k_galerkin<T, N><<<L.grid, L.block, 0, s>>>((const T *)opf, gf, gc, (T *)opc);
    }
    return 1;
  }
  template <bool GS>
  static int coarse_smooth_t(const void *op, const void *r, void *v, void *tmp, const Geo &g, int sweeps,
                             bool zero_start, void **out, const LevelLists *L, cudaStream_t s) {
    const TileList tf = item_list(L);
    void *cur = v;
    int k = 0;
    for (int p = 0; p < sweeps / 2; ++p) {
      if (p == 0 && zero_start) {
        // v is not read: the pair can write it
        constexpr int th = GS ? kGsThreads : kJ2Threads;
        const dim3 grid = tile_grid(g, L, N, k_coarse_pair<T, N, true, GS>, th);
        k_coarse_pair<T, N, true, GS><<<grid, th, 0, s>>>((const T *)op, (const T *)r, (const T *)v, (T *)v, g, tf);
      } else {
        void *nxt = cur == v ? tmp : v;
        constexpr int th = GS ? kGsThreads : kJ2Threads;
        const dim3 grid = tile_grid(g, L, N, k_coarse_pair<T, N, false, GS>, th);
        k_coarse_pair<T, N, false, GS><<<grid, th, 0, s>>>((const T *)op, (const T *)r, (const T *)cur, (T *)nxt, g,
                                                            tf);
        cur = nxt;
      }
      ++k;
    }
    *out = cur;
    return k;
  }
  static int coarse_smooth(const void *op, const void *r, void *v, void *tmp, const Geo &g, int sweeps,
                           bool zero_start, void **out, const LevelLists *L, bool gs, cudaStream_t s) {
    return gs ? coarse_smooth_t<true>(op, r, v, tmp, g, sweeps, zero_start, out, L, s)
              : coarse_smooth_t<false>(op, r, v, tmp, g, sweeps, zero_start, out, L, s);
  }
  // two sweeps from v = 0, then t = r - S v; float: one fused launch (its
  // shared memory is over the static limit in double)
  template <bool GS>
  static int coarse_pre_resid_t(const void *op, const void *r, void *v, void *t, const Geo &g, const LevelLists *L,
                                cudaStream_t s) {
    const TileList tf = item_list(L);
    if constexpr (sizeof(T) == 4) {
      constexpr int th = GS ? kGsThreads : kJ2Threads;
      const dim3 grid = tile_grid(g, L, N, k_coarse_pair_resid<T, N, GS>, th);
      k_coarse_pair_resid<T, N, GS><<<grid, th, 0, s>>>((const T *)op, (const T *)r, (T *)v, (T *)t, g, tf);
      return 1;
    } else {
      constexpr int th = GS ? kGsThreads : kJ2Threads;
      const dim3 grid = tile_grid(g, L, N, k_coarse_pair<T, N, true, GS>, th);
      k_coarse_pair<T, N, true, GS><<<grid, th, 0, s>>>((const T *)op, (const T *)r, (const T *)v, (T *)v, g, tf);
      return 1 + coarse_resid(op, r, v, g, t, L, s);
    }
  }
  static int coarse_pre_resid(const void *op, const void *r, void *v, void *t, const Geo &g, const LevelLists *L,
                              bool gs, cudaStream_t s) {
    return gs ? coarse_pre_resid_t<true>(op, r, v, t, g, L, s) : coarse_pre_resid_t<false>(op, r, v, t, g, L, s);
  }
  static int coarse_solve(const void *op, const void *r, void *v, const Geo &g, int sweeps, cudaStream_t s) {
    const int64_t nc = (int64_t)g.Wn * (g.H + 1);
    const size_t smem = (size_t)6 * N * nc * sizeof(T);
    if (smem <= 48 * 1024) {
      const int threads = (int)std::min<int64_t>(1024, ((N * nc + 31) / 32) * 32);
      k_coarse_solve_smem<T, N><<<1, threads, smem, s>>>((const T *)op, (const T *)r, (T *)v, g, sweeps);
    } else {
      k_coarse_solve_block<T, N><<<1, 1024, 0, s>>>((const T *)op, (const T *)r, (T *)v, g, sweeps);
    }
    return 1;
  }
  static int coarse_resid(const void *op, const void *r, const void *v, const Geo &g, void *t, const LevelLists *Lv,
                          cudaStream_t s) {
    if (Lv) {
      k_coarse_resid_tiled<T, N><<<list_grid(Lv, Lv->cap, k_coarse_resid_tiled<T, N>, kTileThreads), kTileThreads, 0,
                                   s>>>((const T *)op, (const T *)r, (const T *)v, g,
                                                                    (T *)t, item_list(Lv));
    } else {
      const PhaseLaunch L = phase_grid(g.W + 1, g.H + 1, N);
      k_coarse_resid<T, N><<<L.grid, L.block, 0, s>>>((const T *)op, (const T *)r, (const T *)v, g, (T *)t);
    }
    return 1;
  }
  static int restrict_(const void *t, const Geo &gf, const Geo &gc, const void *opc, void *rc, const LevelLists *Lc,
                       cudaStream_t s) {
    if (Lc) {
      k_restrict_tiled<T, N><<<list_grid(Lc, Lc->cap, k_restrict_tiled<T, N>, kTileThreads), kTileThreads, 0, s>>>((const T *)t, gf, gc, (const T *)opc, (T *)rc,
                                                               item_list(Lc));
    } else {
      const PhaseLaunch L = phase_grid(gc.W + 1, gc.H + 1, N);
      k_restrict<T, N><<<L.grid, L.block, 0, s>>>((const T *)t, gf, gc, (const T *)opc, (T *)rc);
    }
    return 1;
  }
  static int prolong_add(const void *vc, const Geo &gf, const Geo &gc, const void *opf, void *vf, const LevelLists *Lf,
                         cudaStream_t s) {
    if (Lf) {
      k_prolong_add_tiled<T, N><<<list_grid(Lf, Lf->cap, k_prolong_add_tiled<T, N>, kTileThreads), kTileThreads, 0,
                                  s>>>((const T *)vc, gf, gc, (const T *)opf, (T *)vf,
                                                                  item_list(Lf));
    } else if ((int64_t)(gf.W + 1) * (gf.H + 1) >= kWideLevelNodes) {
      k_prolong_add<T, N, false><<<row_grid(gf.W + 1, gf.H + 1), kBlock, 0, s>>>((const T *)vc, gf, gc,
                                                                                 (const T *)opf, (T *)vf);
    } else {
      const PhaseLaunch L = phase_grid(gf.W + 1, gf.H + 1, N);
      k_prolong_add<T, N, true><<<L.grid, L.block, 0, s>>>((const T *)vc, gf, gc, (const T *)opf, (T *)vf);
    }
    return 1;
  }
  template <bool GS>
  static int coarse_tail_t(const TailArgs &a, const void *r0, void *v0, int coarse_sweeps, int coarsest_sweeps,
                           size_t smem, cudaStream_t s) {
    // the cap, not this launch's size: the attribute is process-wide and
    // graphs captured for other grids replay launches of other sizes
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_coarse_tail<T, N, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemBytes);
    (void)attr;
    k_coarse_tail<T, N, GS><<<N, kTailThreads, smem, s>>>(a, (const T *)r0, (T *)v0, coarse_sweeps, coarsest_sweeps);
    return 1;
  }
  static int coarse_tail(const TailArgs &a, const void *r0, void *v0, int coarse_sweeps, int coarsest_sweeps,
                         size_t smem, bool gs, cudaStream_t s) {
    return gs ? coarse_tail_t<true>(a, r0, v0, coarse_sweeps, coarsest_sweeps, smem, s)
              : coarse_tail_t<false>(a, r0, v0, coarse_sweeps, coarsest_sweeps, smem, s);
  }
  static int line_search(const void *x, const void *ob, const void *rt, const void *v1, const uint8_t *mask,
                         const Geo &gf, const Geo &gc, void *d, double *part, double *tot, double *omega,
                         cudaStream_t s) {
    const dim3 grid = row_grid(gf.W + 1, gf.H + 1);
    const int blocks = (int)(grid.x * grid.y);
    k_ls_dir<T, N, FORM><<<grid, kBlock, 0, s>>>((const T *)x, (const T *)ob, (const T *)rt, (const T *)v1, mask, gf,
                                               gc, (T *)d, part);
    k_ls_curv<T, N><<<grid, kBlock, 0, s>>>((const T *)d, mask, gf, part + blocks);
    k_colsum<<<1, 1024, 0, s>>>(part, blocks, 1, tot);
    k_colsum<<<1, 1024, 0, s>>>(part + blocks, blocks, 1, tot + 1);
    k_ls_finish<<<1, 32, 0, s>>>(tot, omega);
    return 5;
  }
  static SolverOps table() {
    return SolverOps{(int)sizeof(T), smooth,       resid,        restrict0,   galerkin0,   galerkin,   coarse_smooth,
                     coarse_solve,   coarse_resid, coarse_pre_resid, restrict_, prolong_add, coarse_tail,
                     line_search};
  }
};

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
    k_init_random<N><<<blocks_for(n), kBlock, 0, s>>>(u, n, seed);
    return 1;
  }
  static int means(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
                   double *energy, double eps, double lam, cudaStream_t s) {
    const int64_t n = (int64_t)g.Wn * (g.H + 1);
    const int64_t b = (n + kBlock - 1) / kBlock;
    const int blocks = (int)(b < kMaxPartBlocks ? b : kMaxPartBlocks);
    if (energy) {
      k_means_partial<N, true><<<blocks, kBlock, 0, s>>>(u, mom, g, part);
      k_colsum<<<7 * N, 1024, 0, s>>>(part, blocks, 7 * N, tot);
      k_means_finish<N, true><<<1, 32, 0, s>>>(tot, c, energy, eps, lam);
    } else {
      k_means_partial<N, false><<<blocks, kBlock, 0, s>>>(u, mom, g, part);
      k_colsum<<<4 * N, 1024, 0, s>>>(part, blocks, 4 * N, tot);
      k_means_finish<N, false><<<1, 32, 0, s>>>(tot, c, nullptr, eps, lam);
    }
    return 3;
  }
  static int rhs(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl, double *b,
                 cudaStream_t s) {
    k_rhs<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, mom, c, g, a1, tl, b);
    return 1;
  }
  static int means_df(const double *u, const double *mom, const Geo &g, double *part, double *tot, double *c,
                      double *energy, double eps, double lam, cudaStream_t s) {
    const int64_t n = (int64_t)g.Wn * (g.H + 1);
    const int64_t b = (n + kBlock - 1) / kBlock;
    const int blocks = (int)(b < kMaxPartBlocks ? b : kMaxPartBlocks);
    if (energy) {
      k_means_partial_df<N, true><<<blocks, kBlock, 0, s>>>(u, mom, g, part);
      k_colsum<<<4 * N + 3, 1024, 0, s>>>(part, blocks, 4 * N + 3, tot);
      k_means_finish_df<N><<<1, 32, 0, s>>>(tot, c, energy, eps, lam);
    } else {
      k_means_partial_df<N, false><<<blocks, kBlock, 0, s>>>(u, mom, g, part);
      k_colsum<<<4 * N, 1024, 0, s>>>(part, blocks, 4 * N, tot);
      k_means_finish<N, false><<<1, 32, 0, s>>>(tot, c, nullptr, eps, lam);
    }
    return 3;
  }
  static int rhs_df(const double *u, const double *mom, const double *c, const Geo &g, double a1, double tl,
                    float *b, cudaStream_t s) {
    k_rhs_df<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, mom, c, g, a1, tl, b);
    return 1;
  }
  static int outer_resid(const double *u, const float *b, const Geo &g, float *r32, float *u32, double *rho,
                         bool rho32, cudaStream_t s) {
    if (rho32) {
      static const cudaError_t attr = cudaFuncSetAttribute(
          k_outer_resid_df<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)outer_resid_smem<N>());
      (void)attr;
      k_outer_resid_df<N><<<dim3((g.W + 1 + kOrThreads - 3) / (kOrThreads - 2), (g.H + kOrRows) / kOrRows),
                            kOrThreads, outer_resid_smem<N>(), s>>>(u, b, g, r32, u32, rho);
    }
    else
      k_outer_resid<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, b, g, r32, u32, rho);
    return 1;
  }
  static int outer_update(double *u, const float *delta, const Geo &g, cudaStream_t s) {
    k_outer_update<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, delta, g);
    return 1;
  }
  static int composite(const double *u, const double *c, const Geo &g, int r, int rounded, float *out,
                       cudaStream_t s) {
    k_composite<N><<<row_grid(g.W >> r, g.H >> r), kBlock, 0, s>>>(u, c, g, r, rounded, out);
    return 1;
  }
  static int labels(const double *u, const Geo &g, int r, int8_t *node_lab, int8_t *pix_lab, cudaStream_t s) {
    int k = 0;
    if (node_lab) {
      k_labels<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(u, g, node_lab);
      ++k;
    }
    if (pix_lab) {
      k_pixel_labels<N><<<row_grid(g.W >> r, g.H >> r), kBlock, 0, s>>>(u, g, r, pix_lab);
      ++k;
    }
    return k;
  }
  static int to_split32(const double *in, const Geo &g, float *out, cudaStream_t s) {
    k_to_split32<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(in, g, out);
    return 1;
  }
  static int from_split32(const float *in, const Geo &g, const double *freeset, double *out, cudaStream_t s) {
    k_from_split32<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(in, g, freeset, out);
    return 1;
  }
  static int adj_prepare(const double *up, const double *g, int64_t n, double *freeset, double *rhs, cudaStream_t s) {
    k_adj_prepare<N><<<blocks_for(n), kBlock, 0, s>>>(up, g, n, freeset, rhs);
    return 1;
  }
  static int adj_accum(const double *w, const double *u, const double *up, const double *mom, const double *c,
                       const Geo &g, double tau, double eps, double lam, double *gm, double *part, double *tot,
                       double *scal, cudaStream_t s) {
    const dim3 grid = row_grid(g.W + 1, g.H + 1);
    const int blocks = (int)(grid.x * grid.y);
    k_adj_accum<N><<<grid, kBlock, 0, s>>>(w, u, up, mom, c, g, tau, eps, lam, gm, part);
    k_colsum<<<2 + 3 * N, 1024, 0, s>>>(part, blocks, 2 + 3 * N, tot);
    k_adj_scalars<<<1, 32, 0, s>>>(tot, scal);
    return 3;
  }
  static int adj_back(const double *w, const double *u, const double *mom, const double *c, const double *tot,
                      const double *mass, const Geo &g, double a1, double *gout, double *gm, cudaStream_t s) {
    k_adj_back<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(w, u, mom, c, tot, mass, g, a1, gout, gm);
    return 1;
  }
  static int adj_image(const double *gm, const double *img, const Geo &g, double *gimg, cudaStream_t s) {
    k_adj_image<<<row_grid(g.W, g.H), kBlock, 0, s>>>(gm, img, g, gimg);
    return 1;
  }
  static int tangent_apply(const double *p, const double *f, const Geo &g, double *q, cudaStream_t s) {
    k_tangent_apply<N><<<row_grid(g.W + 1, g.H + 1), kBlock, 0, s>>>(p, f, g, q);
    return 1;
  }
  static int dot2(const double *a0, const double *b0, const double *a1, const double *b1, int64_t count,
                  double *part, double *tot, cudaStream_t s) {
    k_dot2<<<kMaxPartBlocks, kBlock, 0, s>>>(a0, b0, a1, b1, count, part);
    k_colsum<<<2, 1024, 0, s>>>(part, kMaxPartBlocks, 2, tot);
    return 2;
  }
  static int fcg_step(double *x, double *r, const double *p, const double *q, double alpha, int64_t count,
                      cudaStream_t s) {
    k_fcg_step<<<blocks_for(count), kBlock, 0, s>>>(x, r, p, q, alpha, count);
    return 1;
  }
  static int fcg_dir(double *p, const double *z, double beta, int64_t count, cudaStream_t s) {
    k_fcg_dir<<<blocks_for(count), kBlock, 0, s>>>(p, z, beta, count);
    return 1;
  }
  static int absmax(const double *v, int64_t count, double *out, cudaStream_t s) {
    k_absmax<<<kMaxPartBlocks, kBlock, 0, s>>>(v, count, out);
    return 1;
  }
  static int project(const double *y, double *x, int64_t count, cudaStream_t s) {
    if (count <= 0) return 0;
    k_project<N><<<blocks_for(count), kBlock, 0, s>>>(y, x, count);
    return 1;
  }
  static const Ops *table() {
    static const Ops t = {N,
                          moments_f32,
                          moments_f64,
                          init_random,
                          means,
                          rhs,
                          means_df,
                          rhs_df,
                          outer_resid,
                          outer_update,
                          labels,
                          composite,
                          project,
                          SolverLaunch<double, N, kDirect>::table(),
                          SolverLaunch<float, N, kShifted>::table(),
                          SolverLaunch<double, N, kTangent>::table(),
                          SolverLaunch<float, N, kTangent>::table(),
                          to_split32,
                          from_split32,
                          adj_prepare,
                          adj_accum,
                          adj_back,
                          adj_image,
                          absmax,
                          tangent_apply,
                          dot2,
                          fcg_step,
                          fcg_dir};
    return &t;
  }
};

}  // namespace ac
