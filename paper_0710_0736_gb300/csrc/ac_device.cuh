// ac_device.cuh -- device-side building blocks of libac (sm_103a).
//
// Mesh: W x H pixels of side 1, nodes at pixel corners (x, y), node index
// n = y*(W+1) + x, each pixel split along its (x,y)-(x+1,y+1) diagonal
// (P1 finite elements, Sec. 3.1 of Kay & Tomasi).  On that triangulation:
//   lumped mass  Mhat_n = (#incident triangles)/6 : 1 inside, 1/2 on edges,
//                1/3 at (0,0) and (W,H), 1/6 at (W,0) and (0,H);
//   stiffness    A = 5-point graph Laplacian with weight 1 on interior axis
//                edges, 1/2 on boundary axis edges and 0 on the diagonals
//                (their opposite angles are right angles).
// The step matrix is S = Mhat + tau*eps*A (Sec. 3.2, Eq. alpha).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "ac_df64.cuh"

namespace ac {

// Geometry of one level, passed by value to kernels.  Node classes are
// cls = cy*3 + cx with cx = 0 (x == 0), 2 (x == W), 1 otherwise, cy alike:
// the lumped mass and the diagonal of S depend only on the class.
struct Geo {
  int W, H;        // cells
  int Wn;          // W + 1, the row stride in nodes
  double te;       // tau * eps
  double m0[9];    // Mhat by class
  double D[9];     // S_nn by class
  double invD[9];  // 1 / S_nn by class
  int64_t half;    // ((W + 1)(H + 1) + 1) / 2: colour-split stride of the FP32 fine arrays
  float tef, Df[9], invDf[9];  // te, D, invD rounded to float (FP32 kernels do no FP64 conversions)
  float teh, tel, m0h[9], m0l[9];  // te and Mhat as double-floats h + l (the defect correction's residual)
};

// Tiles of the coarse levels: kJ2X x kJ2Y nodes of one phase plane, the unit
// of the fused l1-Jacobi kernels and of the live flags below.
constexpr int kJ2X = 32, kJ2Y = 16;

// Live flags of the tiled coarse levels (the levels above the one-launch
// coarse tail): one byte per (tile, phase), at tf[(i * tiles_y + ty) *
// tiles_x + tx].  Bit kLiveNow: some row of phase i in the tile has a
// nonzero diagonal in this cycle's truncated operator; bit kLivePrev: so it
// had in the previous cycle.  The level's producers (Galerkin product,
// restriction, l1-Jacobi pairs, residual, prolongation) work on live tiles
// only, write zeros into a tile once, in the cycle it stops being live
// (kLivePrev without kLiveNow), and skip it while it stays dead.  So every
// array of a tiled level (operator, r, v, t) holds exact zeros on tiles that
// are not live, which is what a dense level would hold there: readers of
// halos and neighbours need no flags.  The producer derives kLivePrev from
// the kLiveNow it finds, so a new, re-scheduled or newly tiled level starts
// with kLiveNow set everywhere: its first cycle then writes every tile.
constexpr uint8_t kLiveNow = 1, kLivePrev = 2;

__host__ __device__ __forceinline__ int tiles_x(const Geo &g) { return (g.W + kJ2X) / kJ2X; }
__host__ __device__ __forceinline__ int tiles_y(const Geo &g) { return (g.H + kJ2Y) / kJ2Y; }

// The flag byte of the tile holding node (x, y), phase i.
__device__ __forceinline__ uint8_t tile_flag(const uint8_t *__restrict__ tf, const Geo &g, int x, int y, int i) {
  return __ldg(tf + ((int64_t)i * tiles_y(g) + y / kJ2Y) * tiles_x(g) + x / kJ2X);
}

// Changes of the fine free mask, for the first coarse level's operator: it
// depends on the fine masks in the 6x6-node boxes of its nodes only, so a
// first-level tile whose boxes saw no change keeps its operator.  The kernels
// that write the mask set p[ty * tx + tx'] for every first-level tile whose
// boxes hold a node whose mask byte changed (fine x in [2 kJ2X tx - 2,
// 2 kJ2X tx + 2 kJ2X + 1], y alike); the first level's Galerkin kernel
// clears them.  p == null: no tracking.
struct MaskDirty {
  uint8_t *p;
  int tx, ty;  // tiles of the first coarse level
};

__device__ __forceinline__ void mark_dirty(const MaskDirty &d, int x, int y) {
  constexpr int SX = 2 * kJ2X, SY = 2 * kJ2Y;  // fine nodes per tile
  const int x0 = x - (SX + 1) <= 0 ? 0 : (x - (SX + 1) + SX - 1) / SX, x1 = min(d.tx - 1, (x + 2) / SX);
  const int y0 = y - (SY + 1) <= 0 ? 0 : (y - (SY + 1) + SY - 1) / SY, y1 = min(d.ty - 1, (y + 2) / SY);
  for (int ty = y0; ty <= y1; ++ty)
    for (int tx = x0; tx <= x1; ++tx) d.p[(int64_t)ty * d.tx + tx] = 1;
}

// te, S_nn, 1/S_nn in a kernel's scalar type.
template <typename T>
__host__ __device__ __forceinline__ T geo_te(const Geo &g) {
  if constexpr (sizeof(T) == 4) return g.tef; else return g.te;
}
template <typename T>
__host__ __device__ __forceinline__ T geo_D(const Geo &g, int cls) {
  if constexpr (sizeof(T) == 4) return g.Df[cls]; else return g.D[cls];
}
template <typename T>
__host__ __device__ __forceinline__ T geo_invD(const Geo &g, int cls) {
  if constexpr (sizeof(T) == 4) return g.invDf[cls]; else return g.invD[cls];
}

// The line-search step omega is kept as a double followed by its float
// rounding (two doubles of storage); a kernel reads it in its scalar type.
template <typename T>
__device__ __forceinline__ T omega_t(const double *omega) {
  if constexpr (sizeof(T) == 4) return reinterpret_cast<const float *>(omega + 1)[0]; else return omega[0];
}

__host__ __device__ __forceinline__ int node_class(const Geo &g, int x, int y) {
  int cx = x == 0 ? 0 : (x == g.W ? 2 : 1);
  int cy = y == 0 ? 0 : (y == g.H ? 2 : 1);
  return cy * 3 + cx;
}

// Storage slot of fine node (x, y) in an array of element type T.  FP32
// arrays (the mixed form's correction solve) are split by red-black colour:
// colour c = (x + y) & 1 holds its nodes at c * half + ((y Wn + x) >> 1),
// which is one-to-one within a colour for any row stride, so one colour's
// sweep reads and writes contiguous memory only.  FP64 arrays keep the plain
// node order y Wn + x.
template <typename T>
__host__ __device__ __forceinline__ int64_t fslot(const Geo &g, int x, int y) {
  const int64_t n = (int64_t)y * g.Wn + x;
  if constexpr (sizeof(T) == 4)
    return (((x + y) & 1) ? g.half : 0) + (n >> 1);
  else
    return n;
}

// Stiffness weights of the four axis edges at (x, y): east, west, north, south.
struct Weights { float e, w, n, s; };

__host__ __device__ __forceinline__ Weights edge_weights(const Geo &g, int x, int y) {
  float vy = 0.5f * (float)((y < g.H) + (y > 0));  // rows above/below the horizontal edge
  float vx = 0.5f * (float)((x < g.W) + (x > 0));
  Weights w;
  w.e = x < g.W ? vy : 0.f;
  w.w = x > 0 ? vy : 0.f;
  w.n = y < g.H ? vx : 0.f;
  w.s = y > 0 ? vx : 0.f;
  return w;
}

// ---- asynchronous global -> shared copies (cp.async) ------------------------
// B bytes (4, 8 or 16; both addresses B-aligned) from global to shared memory
// without passing through registers, cached in L1; completion is awaited per
// commit group with cp_async_wait<K>() (all but the K most recent groups).
template <int B>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// ---- vector loads / stores of one node's N values ------------------------

template <typename T, int N>
__device__ __forceinline__ void ldn(const T *__restrict__ p, T (&v)[N]) {
  if constexpr (sizeof(T) * N % 16 == 0) {
    constexpr int K = 16 / sizeof(T);
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
#pragma unroll
    for (int j = 0; j < N / K; ++j) {
      V t = __ldg(reinterpret_cast<const V *>(p) + j);
      if constexpr (sizeof(T) == 8) {
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
      } else {
        v[4 * j] = t.x;
        v[4 * j + 1] = t.y;
        v[4 * j + 2] = t.z;
        v[4 * j + 3] = t.w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

// Plain (non read-only-path) load, for arrays written by the same kernel.
template <typename T, int N>
__device__ __forceinline__ void ldn_rw(const T *p, T (&v)[N]) {
  if constexpr (sizeof(T) * N % 16 == 0) {
    constexpr int K = 16 / sizeof(T);
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
#pragma unroll
    for (int j = 0; j < N / K; ++j) {
      V t = reinterpret_cast<const V *>(p)[j];
      if constexpr (sizeof(T) == 8) {
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
      } else {
        v[4 * j] = t.x;
        v[4 * j + 1] = t.y;
        v[4 * j + 2] = t.z;
        v[4 * j + 3] = t.w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

template <typename T, int N>
__device__ __forceinline__ void stn(T *p, const T (&v)[N]) {
  if constexpr (sizeof(T) * N % 16 == 0) {
    constexpr int K = 16 / sizeof(T);
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
#pragma unroll
    for (int j = 0; j < N / K; ++j) {
      V t;
      if constexpr (sizeof(T) == 8) {
        t.x = v[2 * j];
        t.y = v[2 * j + 1];
      } else {
        t.x = v[4 * j];
        t.y = v[4 * j + 1];
        t.z = v[4 * j + 2];
        t.w = v[4 * j + 3];
      }
      reinterpret_cast<V *>(p)[j] = t;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

// 1/k for the small integers 1..8 without a division.
template <typename T>
__device__ __forceinline__ T rcp_small(int k) {
  return k == 1 ? T(1) : k == 2 ? T(0.5) : k == 3 ? T(1.0 / 3.0) : k == 4 ? T(0.25)
       : k == 5 ? T(0.2) : k == 6 ? T(1.0 / 6.0) : k == 7 ? T(1.0 / 7.0) : T(0.125);
}

// Constraint forms of a multigrid solve.
enum Form { kDirect = 0, kShifted = 1, kTangent = 2 };

// Nodal projection of the solve's form, in place, in registers:
//   kDirect  : Euclidean projection onto x_i >= 0, sum_i x_i = 1 (the Gibbs simplex)
//   kShifted : onto x_i >= -ob_i, sum_i x_i = 0 (corrections delta with u + delta
//              on the simplex, ob = u)
//   kTangent : orthogonal projection onto the tangent space of a frozen active
//              set, ob_i = 1 for the free phases (at least two) and 0 otherwise:
//              x_i = z_i - mean_free(z) on the free phases, 0 elsewhere
// For the first two the kept set starts full; theta = (sum of kept z + sum of
// dropped bounds - total)/|kept|; components with z_i - theta at or below their
// bound leave the set; repeat until none leaves (at most N passes).  This is
// the clamp-and-redistribute loop of Sec. 3.3 written with the threshold theta
// (Michelot's form of the same iteration).  In the shifted form the result is
// computed as a difference from the bound, so it keeps the relative precision
// of the correction itself.
template <typename T, int N, int FORM>
__device__ __forceinline__ void proj_box(T (&z)[N], const T (&ob)[N]) {
  if constexpr (FORM == kTangent) {
    T s = T(0);
    int k = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (ob[i] != T(0)) {
        s += z[i];
        ++k;
      }
    const T mean = k >= 2 ? s * rcp_small<T>(k) : T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) z[i] = (k >= 2 && ob[i] != T(0)) ? z[i] - mean : T(0);
    return;
  } else {
    constexpr bool SH = FORM == kShifted;
    const T total = SH ? T(0) : T(1);
    unsigned keep = (1u << N) - 1u;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) s += z[i];
    T theta = (s - total) * rcp_small<T>(N);
#pragma unroll 1
    for (int pass = 1; pass < N; ++pass) {
      unsigned drop = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const T lo = SH ? -ob[i] : T(0);
        if (((keep >> i) & 1u) && z[i] - theta <= lo) drop |= 1u << i;
      }
      // in exact arithmetic some kept component stays above its bound; if
      // rounding drops them all, keep the last set and its theta
      if (!drop || drop == keep) break;
      keep &= ~drop;
      s = T(0);
      T L = T(0);
      int k = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if ((keep >> i) & 1u) {
          s += z[i];
          ++k;
        } else if (SH) {
          L -= ob[i];
        }
      }
      theta = (s + L - total) * rcp_small<T>(k);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) z[i] = ((keep >> i) & 1u) ? z[i] - theta : (SH ? -ob[i] : T(0));
  }
}

// Free set (bit i: component i above its bound) of the shifted-form
// projection of z with bounds -ob, by the same iteration as proj_box; z and ob
// are not changed.
template <typename T, int N>
__device__ __forceinline__ unsigned shifted_free_set(const T (&z)[N], const T (&ob)[N]) {
  unsigned keep = (1u << N) - 1u;
  T s = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) s += z[i];
  T theta = s * rcp_small<T>(N);
#pragma unroll 1
  for (int pass = 1; pass < N; ++pass) {
    unsigned drop = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (((keep >> i) & 1u) && z[i] - theta <= -ob[i]) drop |= 1u << i;
    if (!drop || drop == keep) break;
    keep &= ~drop;
    s = T(0);
    int k = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if ((keep >> i) & 1u) {
        s += z[i];
        ++k;
      } else {
        s -= ob[i];
      }
    }
    theta = s * rcp_small<T>(k);
  }
  return keep;
}

// Shifted-form projection of z (bounds -ob, sum 0) in FP64 given a candidate
// free set from a float pass: theta from that set, then the optimality
// conditions (free components above their bound, the others at or below it)
// are checked in FP64.  If they hold, z becomes the projection (the
// conditions characterise it) and true is returned; otherwise z is unchanged
// and false is returned.
template <int N>
__device__ __forceinline__ bool shifted_proj_on_set(double (&z)[N], const double (&ob)[N], unsigned keep) {
  double s = 0.0, L = 0.0;
  int k = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if ((keep >> i) & 1u) {
      s += z[i];
      ++k;
    } else {
      L -= ob[i];
    }
  }
  if (k == 0) return false;
  const double theta = (s + L) * rcp_small<double>(k);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const bool above = z[i] - theta > -ob[i];
    ok = ok && (above == (((keep >> i) & 1u) != 0u));
  }
  if (!ok) return false;
#pragma unroll
  for (int i = 0; i < N; ++i) z[i] = ((keep >> i) & 1u) ? z[i] - theta : -ob[i];
  return true;
}

// Projection onto the Gibbs simplex (direct form).
template <typename T, int N>
__device__ __forceinline__ void proj_simplex(T (&y)[N]) {
  const T none[N] = {};
  proj_box<T, N, kDirect>(y, none);
}

// Weighted sum of the four axis neighbours' values, acc = sum_m w_nm u_m (u
// in the storage order of fslot<T>).
template <typename T, int N>
__device__ __forceinline__ void nbr_sum(const T *u, const Geo &g, int x, int y, T (&acc)[N]) {
  T t[N];
  if (x > 0 && x < g.W && y > 0 && y < g.H) {
    ldn_rw<T, N>(u + fslot<T>(g, x + 1, y) * N, acc);
    ldn_rw<T, N>(u + fslot<T>(g, x - 1, y) * N, t);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += t[i];
    ldn_rw<T, N>(u + fslot<T>(g, x, y + 1) * N, t);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += t[i];
    ldn_rw<T, N>(u + fslot<T>(g, x, y - 1) * N, t);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] += t[i];
  } else {
    Weights w = edge_weights(g, x, y);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = T(0);
    if (w.e > 0.f) {
      ldn_rw<T, N>(u + fslot<T>(g, x + 1, y) * N, t);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] += T(w.e) * t[i];
    }
    if (w.w > 0.f) {
      ldn_rw<T, N>(u + fslot<T>(g, x - 1, y) * N, t);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] += T(w.w) * t[i];
    }
    if (w.n > 0.f) {
      ldn_rw<T, N>(u + fslot<T>(g, x, y + 1) * N, t);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] += T(w.n) * t[i];
    }
    if (w.s > 0.f) {
      ldn_rw<T, N>(u + fslot<T>(g, x, y - 1) * N, t);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] += T(w.s) * t[i];
    }
  }
}

// P1 interpolation weight of coarse node L at fine node b (fine coordinates),
// for nested right-diagonal meshes: 1 at 2L, 1/2 at the six neighbours of 2L
// along the coarse edges (E, W, N, S, NE, SW), 0 elsewhere.
__host__ __device__ __forceinline__ double hat_weight(int dx, int dy) {
  if (dx == 0 && dy == 0) return 1.0;
  if ((dx == 1 || dx == -1) && dy == 0) return 0.5;
  if (dx == 0 && (dy == 1 || dy == -1)) return 0.5;
  if ((dx == 1 && dy == 1) || (dx == -1 && dy == -1)) return 0.5;
  return 0.0;
}

// Entry S_ab of the fine step matrix S = Mhat + tau eps A for b = a + (ddx, ddy),
// (ddx, ddy) in {0, E, W, N, S}, both nodes inside the level.
__host__ __device__ __forceinline__ double fine_S(const Geo &g, int ax, int ay, int ddx, int ddy) {
  if (ddx == 0 && ddy == 0) return g.D[node_class(g, ax, ay)];
  Weights w = edge_weights(g, ax, ay);
  float ww = ddx == 1 ? w.e : ddx == -1 ? w.w : ddy == 1 ? w.n : w.s;
  return -g.te * (double)ww;
}

// The same entry in the scalar type of a solve (float kernels must not spend
// GB300's scarce FP64 issue slots on it).
template <typename T>
__device__ __forceinline__ T fine_S_t(const Geo &g, int ax, int ay, int ddx, int ddy) {
  if (ddx == 0 && ddy == 0) return geo_D<T>(g, node_class(g, ax, ay));
  Weights w = edge_weights(g, ax, ay);
  float ww = ddx == 1 ? w.e : ddx == -1 ? w.w : ddy == 1 ? w.n : w.s;
  return -geo_te<T>(g) * (T)ww;
}

template <typename T>
__host__ __device__ __forceinline__ T hat_weight_t(int dx, int dy) {
  if (dx == 0 && dy == 0) return T(1);
  if ((dx == 1 || dx == -1) && dy == 0) return T(0.5);
  if (dx == 0 && (dy == 1 || dy == -1)) return T(0.5);
  if ((dx == 1 && dy == 1) || (dx == -1 && dy == -1)) return T(0.5);
  return T(0);
}

// Untruncated first-level Galerkin entries (C, E, N, NE) of P'SP by coarse-node
// class: x class 0, 1, 2 (interior), 3, 4 for X = 0, 1, other, Wc-1, Wc (y
// alike), index cy*5 + cx.
struct Galerkin0Table {
  double v[25][4];
  float vf[25][4];  // the same entries rounded to float (FP32 solves)
};

__host__ __device__ __forceinline__ int g0_class(int X, int Wc) {
  return X == 0 ? 0 : X == 1 ? 1 : X == Wc ? 4 : X == Wc - 1 ? 3 : 2;
}

// The first-level Galerkin entry (K, K + (lx, ly)) of P' M S M P, where M keeps
// the fine nodes whose bit `bit` is set in mask(x, y) (mask == nullptr: all).
template <class MaskF>
__host__ __device__ inline double galerkin0_entry(const Geo &gf, const Geo &gc, int X, int Y, int lx, int ly,
                                                  MaskF free_at) {
  const int sx[7] = {0, 1, -1, 0, 0, 1, -1};
  const int sy[7] = {0, 0, 0, 1, -1, 1, -1};
  const int ox[5] = {0, 1, -1, 0, 0};
  const int oy[5] = {0, 0, 0, 1, -1};
  const int LX = X + lx, LY = Y + ly;
  if (LX > gc.W || LY > gc.H) return 0.0;
  double acc = 0.0;
  for (int s = 0; s < 7; ++s) {
    const int ax = 2 * X + sx[s], ay = 2 * Y + sy[s];
    if (ax < 0 || ax > gf.W || ay < 0 || ay > gf.H || !free_at(ax, ay)) continue;
    const double pa = s == 0 ? 1.0 : 0.5;
    for (int o = 0; o < 5; ++o) {
      const int bx = ax + ox[o], by = ay + oy[o];
      if (bx < 0 || bx > gf.W || by < 0 || by > gf.H || !free_at(bx, by)) continue;
      acc += pa * fine_S(gf, ax, ay, ox[o], oy[o]) * hat_weight(bx - 2 * LX, by - 2 * LY);
    }
  }
  return acc;
}

// Block-wide reductions (blockDim.x a multiple of 32, <= 1024).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// max that propagates a NaN held in either argument.
template <typename T>
__device__ __forceinline__ T nanmax(T a, T b) { return (a != a || b <= a) ? a : b; }

template <typename T>
__device__ __forceinline__ T warp_nanmax(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax<T>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Non-negative doubles (and NaN) order like their bit patterns as unsigned.
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace ac
