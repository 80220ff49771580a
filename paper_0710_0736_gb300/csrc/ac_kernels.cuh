// ac_kernels.cuh -- the sm_103a kernels of libac, templated on the phase
// count N, the scalar type T of a multigrid solve and its constraint form
// FORM (see proj_box).  Instantiated once per N in ac_inst_n<N>.cu; the host
// driver (ac_api.cu) calls them through the Ops table of ac_ops.h.
//
// Three solves share these kernels:
//   FP64 form : T = double, kDirect,  unknown x = u, right-hand side b.
//   mixed form: T = float,  kShifted, unknown x = delta (a correction of the
//               FP64 state u), right-hand side r = b - S u (computed in FP64),
//               obstacle ob = u rounded to float (delta_i >= -u_i, sum 0).
//   adjoint   : T = double, kTangent, unknown x = w, right-hand side Pi g,
//               ob = the frozen free set of u^{t+1} (1/0 per phase).
//
// Data layout in HBM:
//   fine level (node-major, phase innermost, n x N): x, rhs, ob, rt, d;
//     mask n bytes (bit i: phase i free at the node); mom n x 4 (m1 RGB, m2)
//   coarse level k (phase-major, so a thread per node reads coalesced rows):
//     op[(c*N + i)*n_k + node], c in {C, E, N, NE} (W, S, SW are the
//     neighbours' E, N, NE); r, v, t [i*n_k + node].
#pragma once
#include "ac_device.cuh"
#include "ac_ops.h"

namespace ac {

constexpr int kBlock = 256;
// Kernels that work on kJ2X x kJ2Y tiles of a coarse level: kTileThreads
// threads per block, kTileRows rows of the tile per thread.
constexpr int kTileThreads = 256, kTileRows = kJ2X * kJ2Y / kTileThreads;

// A list of the (tile, phase) items of a tiled level that are live or died
// this cycle (see kLiveNow), appended by the kernel that computes the level's
// flags: item = tile | phase << 32 | dying << 40 (tile = ty * tiles_x + tx).
// Kernels driven by it run a fixed grid that strides over the count; with
// items == null they run one block per tile and phase instead (a dense
// level).  Every item writes its own tile only, so the order of the list does
// not change any result.
struct TileList {
  const uint64_t *items;
  const int *count;
};
constexpr uint64_t kItemDying = 1ull << 40;
__device__ __forceinline__ uint64_t tile_item(int64_t tile, int phase, bool dying) {
  return (uint64_t)tile | ((uint64_t)phase << 32) | (dying ? kItemDying : 0ull);
}

// Run body(tx, ty, i, dying) for the block's tiles: the grid's tile and phase
// (dense) or the list's items in block-strided order.
template <class F>
__device__ __forceinline__ void for_each_tile(const TileList &L, const Geo &g, F &&body) {
  if (!L.items) {
    body((int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, false);
    return;
  }
  const int cnt = *L.count, ntx = tiles_x(g);
  for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
    const uint64_t e = L.items[w];
    const int tile = (int)(e & 0xffffffffull), i = (int)((e >> 32) & 0xffull);
    __syncthreads();  // the previous item's shared-memory tiles are no longer read
    body(tile % ntx, tile / ntx, i, (e & kItemDying) != 0ull);
  }
}


// m1 (RGB) and m2 of one node as two 16-byte loads.
__device__ __forceinline__ double4 ld_mom(const double *p) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of K values per thread; threads k < K write
// the block's totals to dst[k].
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double *dst) {
  __shared__ double sm[kBlock / 32][K];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm[wid][k] = v[k];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][k];
    dst[k] = s;
  }
}

// Block maximum (NaN-propagating) of non-negative values in the kernel's
// scalar type, folded into *rho by one atomic per block (the conversion of a
// float maximum to double is exact).
template <typename T>
__device__ __forceinline__ void block_max_atomic(T e, double *rho) {
  __shared__ T sm[kBlock / 32];
  e = warp_nanmax<T>(e);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x < 32) {
    T v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : T(0);
    v = warp_nanmax<T>(v);
    if (threadIdx.x == 0) atomic_max_nonneg(rho, (double)v);
  }
}

// Block sum of one value per thread in the kernel's scalar type; thread 0
// stores the block's total as a double (FP32 kernels keep the FP64 pipe
// free; the totals across blocks are summed in FP64).
template <typename T>
__device__ __forceinline__ void block_sum_store1(T v, double *dst) {
  __shared__ T sm[kBlock / 32];
  v = warp_sum<T>(v);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : T(0);
    t = warp_sum<T>(t);
    if (threadIdx.x == 0) *dst = (double)t;
  }
}

// Column sums of a rows x cols row-major matrix of block partials; one block
// per column (any blockDim that is a multiple of 32, <= 1024), four
// independent accumulators per thread, fixed summation order (bit-reproducible
// for a fixed grid and block size).
static __global__ void __launch_bounds__(1024) k_colsum(const double *__restrict__ part, int rows, int cols,
                                                        double *__restrict__ out) {
  __shared__ double sm[32];
  const int c = blockIdx.x, B = blockDim.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int r = threadIdx.x;
  for (; r + 3 * B < rows; r += 4 * B) {
    s0 += part[(int64_t)r * cols + c];
    s1 += part[(int64_t)(r + B) * cols + c];
    s2 += part[(int64_t)(r + 2 * B) * cols + c];
    s3 += part[(int64_t)(r + 3 * B) * cols + c];
  }
  for (; r < rows; r += B) s0 += part[(int64_t)r * cols + c];
  double v = warp_sum((s0 + s1) + (s2 + s3));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (int)threadIdx.x < (B >> 5) ? sm[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[c] = v;
  }
}

// ---------------------------------------------------------------------------
// a1: image moments, projection by simplex (Sec. 4.2).  A node collects 1/6
// of the value of each incident triangle: twice from pixels (x,y) and
// (x-1,y-1), once from (x-1,y) and (x,y-1) (pixels outside the image omitted).
// ---------------------------------------------------------------------------
template <typename TI>
__global__ void k_moments(const TI *__restrict__ img, Geo g, double *__restrict__ mom) {
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
    const TI *p = img + ((int64_t)py[k] * g.W + px[k]) * 3;
    double r = (double)p[0], gg = (double)p[1], bb = (double)p[2];
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

// ---------------------------------------------------------------------------
// Seeded random point of the simplex per node: normalised exponentials
// -log(U) (a Dirichlet(1,..,1) draw).  U comes from SplitMix64 (Steele, Lea &
// Flood 2014) on the counter n*N + i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int N>
__global__ void k_init_random(double *__restrict__ u, int64_t n, uint64_t seed) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  // -log U in float for a uniform U on the 2^23 midpoints (j + 1/2) 2^-23
  // of (0, 1), exact in float (binary64 logarithms run on GB300's slow FP64
  // pipe), widened exactly and normalised in binary64, so that the node lies
  // on the simplex to binary64 rounding with every component > 0
  double e[N], s = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    uint64_t z = splitmix64(seed ^ splitmix64((uint64_t)(k * N + i)));
    const float U = ((float)(uint32_t)(z >> 41) + 0.5f) * 0x1.0p-23f;
    e[i] = f32_to_f64(-logf(U));
    s += e[i];
  }
  const double inv = 1.0 / s;
#pragma unroll
  for (int i = 0; i < N; ++i) e[i] *= inv;
  stn<double, N>(u + k * N, e);
}

// ---------------------------------------------------------------------------
// a2: colour means (and, with ENERGY, the energy terms), FP64 accumulation.
// Per phase i the block partials hold at index q*N + i:
//   q=0 mass = sum_n u m0        q=1..3 sum_n u m1 (RGB)
//   ENERGY only: q=4 sum_n u m2, q=5 sum_n m0 u (1-u),
//                q=6 sum over axis edges of w (u_a - u_b)^2  (= u_i' A u_i)
// (Eq. VV_fidelity with the RGB fitting of Sec. 4.4; Eq. E.)
// ---------------------------------------------------------------------------
template <int N, bool ENERGY>
__global__ void __launch_bounds__(kBlock) k_means_partial(const double *__restrict__ u, const double *__restrict__ mom,
                                                          Geo g, double *__restrict__ part) {
  constexpr int Q = ENERGY ? 7 : 4;
  double acc[Q * N];
#pragma unroll
  for (int k = 0; k < Q * N; ++k) acc[k] = 0.0;
  const int64_t n = (int64_t)g.Wn * (g.H + 1);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned k32 = (unsigned)k;  // n <= 2^31: 32-bit division suffices
    const int x = (int)(k32 % (unsigned)g.Wn), y = (int)(k32 / (unsigned)g.Wn);
    const double m0 = g.m0[node_class(g, x, y)];
    double uk[N];
    ldn<double, N>(u + k * N, uk);
    const double4 m = ld_mom(mom + k * 4);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      acc[0 * N + i] += uk[i] * m0;
      acc[1 * N + i] += uk[i] * m.x;
      acc[2 * N + i] += uk[i] * m.y;
      acc[3 * N + i] += uk[i] * m.z;
    }
    if constexpr (ENERGY) {
      double t[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        acc[4 * N + i] += uk[i] * m.w;
        acc[5 * N + i] += m0 * uk[i] * (1.0 - uk[i]);
      }
      Weights w = edge_weights(g, x, y);
      if (x < g.W) {
        ldn<double, N>(u + (k + 1) * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[6 * N + i] += (double)w.e * (uk[i] - t[i]) * (uk[i] - t[i]);
      }
      if (y < g.H) {
        ldn<double, N>(u + (k + g.Wn) * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[6 * N + i] += (double)w.n * (uk[i] - t[i]) * (uk[i] - t[i]);
      }
    }
  }
  block_sum_store<Q * N>(acc, part + (int64_t)blockIdx.x * Q * N);
}

// c_i = s_i / mass_i (previous c kept when mass_i == 0).  With ENERGY the
// discrete Eq. (E): sum_i eps/2 u'Au + (1/eps) sum m0 u(1-u) + lambda (U2 - |s|^2/mass).
template <int N, bool ENERGY>
__global__ void k_means_finish(const double *__restrict__ tot, double *__restrict__ c, double *__restrict__ energy,
                               double eps, double lam) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double E = 0.0;
  for (int i = 0; i < N; ++i) {
    const double mass = tot[0 * N + i];
    const double s0 = tot[1 * N + i], s1 = tot[2 * N + i], s2 = tot[3 * N + i];
    if (mass != 0.0) {
      c[i * 3 + 0] = s0 / mass;
      c[i * 3 + 1] = s1 / mass;
      c[i * 3 + 2] = s2 / mass;
    }
    if constexpr (ENERGY) {
      if (mass != 0.0) E += lam * (tot[4 * N + i] - (s0 * s0 + s1 * s1 + s2 * s2) / mass);
      E += tot[5 * N + i] / eps + 0.5 * eps * tot[6 * N + i];
    }
  }
  if (ENERGY && energy) *energy = E;
}

// ---------------------------------------------------------------------------
// a3: right-hand side b = m0 u^t (1 + 2 tau/eps) - tau lambda f(c^t), with
// f_n,i = m2 - 2 c_i.m1 + |c_i|^2 m0  (Eq. alpha multiplied out), FP64.
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_rhs(const double *__restrict__ u, const double *__restrict__ mom, const double *__restrict__ c, Geo g,
                      double a1, double tl, double *__restrict__ b) {
  // per phase, once per block: 2 tau lambda c_i (RGB) and tau lambda |c_i|^2,
  // so that b_i = a1 m0 u_i - tau lambda m2 + (2 tau lambda c_i).m1
  //             - (tau lambda |c_i|^2) m0
  __shared__ double coef[N][4];
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    const double c0 = c[i * 3], c1 = c[i * 3 + 1], c2 = c[i * 3 + 2];
    coef[i][0] = 2.0 * tl * c0;
    coef[i][1] = 2.0 * tl * c1;
    coef[i][2] = 2.0 * tl * c2;
    coef[i][3] = tl * (c0 * c0 + c1 * c1 + c2 * c2);
  }
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t k = (int64_t)y * g.Wn + x;
  const double m0 = g.m0[node_class(g, x, y)];
  const double4 m = ld_mom(mom + k * 4);
  double uk[N], bk[N];
  ldn<double, N>(u + k * N, uk);
  const double base = -tl * m.w, am0 = a1 * m0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    bk[i] = fma(am0, uk[i], base + coef[i][0] * m.x + coef[i][1] * m.y + coef[i][2] * m.z - coef[i][3] * m0);
  stn<double, N>(b + k * N, bk);
}

// ---------------------------------------------------------------------------
// Mixed form: a2 and a3 in double-float arithmetic (GB300's FP64 pipe runs
// at about 1/64 of the FP32 rate; see ac_df64.cuh).  The stored binary64
// phase field and moments are split on the integer pipe.
// k_means_partial_df: per thread, k_means_partial's sums over its nodes
// (same q layout, with ENERGY the energy terms too) as double-float
// accumulators renormalised after every addition, converted to FP64 once
// per thread for the block sums.
// k_rhs_df: b = m0 u (1 + 2 tau/eps) - tau lambda (m2 - 2 c_i.m1 + |c_i|^2 m0)
// as double-floats, stored node-major as N heads followed by N tails (the
// bytes of N doubles); the mixed form's residual reads them as they are.
// Both err by about 2^-46 of the terms' magnitudes.
// ---------------------------------------------------------------------------
template <int N, bool ENERGY>
__global__ void __launch_bounds__(kBlock, 2) k_means_partial_df(const double *__restrict__ u,
                                                             const double *__restrict__ mom, Geo g,
                                                             double *__restrict__ part) {
  // 4N sums per phase (k_means_partial's q = 0..3), and with ENERGY three
  // sums over all phases: u m2, m0 u (1 - u), w (u_a - u_b)^2
  constexpr int QN = ENERGY ? 4 * N + 3 : 4 * N;
  f2 acc[QN];
#pragma unroll
  for (int k = 0; k < QN; ++k) acc[k] = {0.f, 0.f};
  const int64_t n = (int64_t)g.Wn * (g.H + 1);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned k32 = (unsigned)k;  // n <= 2^31: 32-bit division suffices
    const int x = (int)(k32 % (unsigned)g.Wn), y = (int)(k32 / (unsigned)g.Wn);
    const int cls = node_class(g, x, y);
    const double4 m = ld_mom(mom + k * 4);
    float mh[5], ml[5];
    mh[0] = g.m0h[cls];
    ml[0] = g.m0l[cls];
    split_f64(m.x, mh[1], ml[1]);
    split_f64(m.y, mh[2], ml[2]);
    split_f64(m.z, mh[3], ml[3]);
    if constexpr (ENERGY) split_f64(m.w, mh[4], ml[4]);
    float uh[N], ul[N];
    {
      double t[N];
      ldn<double, N>(u + k * N, t);
#pragma unroll
      for (int i = 0; i < N; ++i) split_f64(t[i], uh[i], ul[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const f2 p = mul_f2(uh[i], ul[i], mh[q], ml[q]);
        acc[q * N + i] = add_f2(acc[q * N + i], p.h, p.l);
      }
    }
    if constexpr (ENERGY) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        f2 p = mul_f2(uh[i], ul[i], mh[4], ml[4]);  // u m2
        acc[4 * N] = add_f2(acc[4 * N], p.h, p.l);
        f2 v = two_sum(1.f, -uh[i]);  // 1 - u
        v.l -= ul[i];
        p = mul_f2(uh[i], ul[i], v.h, v.l);
        p = fast_two_sum(p.h, p.l);
        p = mul_f2(mh[0], ml[0], p.h, p.l);  // m0 u (1 - u)
        acc[4 * N + 1] = add_f2(acc[4 * N + 1], p.h, p.l);
      }
      // w (u_a - u_b)^2 over the east and north axis edges of the node
      const Weights w = edge_weights(g, x, y);
      auto edge = [&](int64_t nb, float we) {
        double t[N];
        ldn<double, N>(u + nb * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float h, l;
          split_f64(t[i], h, l);
          f2 d = two_sum(uh[i], -h);
          d = fast_two_sum(d.h, d.l + (ul[i] - l));
          const f2 p = mul_f2(d.h, d.l, d.h, d.l);
          acc[4 * N + 2] = add_f2(acc[4 * N + 2], we * p.h, we * p.l);
        }
      };
      if (x < g.W) edge(k + 1, w.e);
      if (y < g.H) edge(k + g.Wn, w.n);
    }
  }
  double v[QN];
#pragma unroll
  for (int k = 0; k < QN; ++k) v[k] = f32_to_f64(acc[k].h) + f32_to_f64(acc[k].l);
  block_sum_store<QN>(v, part + (int64_t)blockIdx.x * QN);
}

// c_i as k_means_finish; with energy the discrete Eq. (E) from the 4N + 3
// totals of k_means_partial_df<N, true>: lambda (sum u m2 - sum_i |s_i|^2 /
// mass_i) + (1/eps) sum m0 u (1 - u) + eps/2 sum u'Au (a phase of zero mass
// is 0 everywhere, so its u m2 term is 0 as in k_means_finish).
template <int N>
__global__ void k_means_finish_df(const double *__restrict__ tot, double *__restrict__ c, double *__restrict__ energy,
                                  double eps, double lam) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double fit = 0.0;
  for (int i = 0; i < N; ++i) {
    const double mass = tot[0 * N + i];
    const double s0 = tot[1 * N + i], s1 = tot[2 * N + i], s2 = tot[3 * N + i];
    if (mass != 0.0) {
      c[i * 3 + 0] = s0 / mass;
      c[i * 3 + 1] = s1 / mass;
      c[i * 3 + 2] = s2 / mass;
      fit += (s0 * s0 + s1 * s1 + s2 * s2) / mass;
    }
  }
  if (energy) *energy = lam * (tot[4 * N] - fit) + tot[4 * N + 1] / eps + 0.5 * eps * tot[4 * N + 2];
}

template <int N>
__global__ void k_rhs_df(const double *__restrict__ u, const double *__restrict__ mom, const double *__restrict__ c,
                         Geo g, double a1, double tl, float *__restrict__ b) {
  // per phase, once per block: 2 tau lambda c_i (RGB) and tau lambda |c_i|^2
  // as double-floats; a1 = 1 + 2 tau/eps and tau lambda likewise
  __shared__ float coef[N][4][2];
  __shared__ float sc[2][2];
  if (threadIdx.x < N) {
    const int i = threadIdx.x;
    const double c0 = c[i * 3], c1 = c[i * 3 + 1], c2 = c[i * 3 + 2];
    split_f64(2.0 * tl * c0, coef[i][0][0], coef[i][0][1]);
    split_f64(2.0 * tl * c1, coef[i][1][0], coef[i][1][1]);
    split_f64(2.0 * tl * c2, coef[i][2][0], coef[i][2][1]);
    split_f64(tl * (c0 * c0 + c1 * c1 + c2 * c2), coef[i][3][0], coef[i][3][1]);
  }
  if (threadIdx.x == 32) {
    split_f64(a1, sc[0][0], sc[0][1]);
    split_f64(tl, sc[1][0], sc[1][1]);
  }
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t k = (int64_t)y * g.Wn + x;
  const int cls = node_class(g, x, y);
  const float m0h = g.m0h[cls], m0l = g.m0l[cls];
  const double4 m = ld_mom(mom + k * 4);
  float mh[4], ml[4];
  split_f64(m.x, mh[0], ml[0]);
  split_f64(m.y, mh[1], ml[1]);
  split_f64(m.z, mh[2], ml[2]);
  split_f64(m.w, mh[3], ml[3]);
  f2 am0 = mul_f2(sc[0][0], sc[0][1], m0h, m0l);
  am0 = fast_two_sum(am0.h, am0.l);
  const f2 base = mul_f2(sc[1][0], sc[1][1], mh[3], ml[3]);  // tau lambda m2
  double t[N];
  ldn<double, N>(u + k * N, t);
  float bh[N], bl[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float uh, ul;
    split_f64(t[i], uh, ul);
    f2 p = mul_f2(am0.h, am0.l, uh, ul);
    f2 s = fast_two_sum(p.h, p.l);
    s = add_f2(s, -base.h, -base.l);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      p = mul_f2(coef[i][q][0], coef[i][q][1], mh[q], ml[q]);
      s = add_f2(s, p.h, p.l);
    }
    p = mul_f2(coef[i][3][0], coef[i][3][1], m0h, m0l);
    s = add_f2(s, -p.h, -p.l);
    bh[i] = s.h;
    bl[i] = s.l;
  }
  stn<float, N>(b + k * 2 * N, bh);
  stn<float, N>(b + k * 2 * N + N, bl);
}

// ---------------------------------------------------------------------------
// Mixed form, outer defect correction.
// b is the double-float right-hand side of k_rhs_df (N heads, N tails per
// node).
// k_outer_resid: r = b - S u in FP64, shifted per node by max_i r_i; stores r
// rounded to float and u's truncated head (f64_head, 0 <= head <= u: the
// right-hand side and obstacle of the FP32 correction solve) and the natural
// residual max_n |P_G(u_n + z_n) - u_n|,
// z = r/S_nn, computed in FP64 as a correction by the shifted projection
// (free set found in float, theta and the optimality conditions checked in
// FP64).  This is the FP64 check that ac_residual reports.
// k_outer_resid_df: the same residual in double-float arithmetic, the one
// the mixed solve runs (below).
// k_outer_update: u <- P_G(u + delta) in FP64 (components on their bound
// exactly 0).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kBlock) k_outer_resid(const double *__restrict__ u, const float *__restrict__ b, Geo g,
                                                        float *__restrict__ r32, float *__restrict__ u32,
                                                        double *__restrict__ rho) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  double e = 0.0;
  if (x <= g.W) {
    const int64_t n = (int64_t)y * g.Wn + x;
    double acc[N], uk[N], bk[N];
    nbr_sum<double, N>(u, g, x, y, acc);
    ldn<double, N>(u + n * N, uk);
    {
      float bh[N], bl[N];  // b as k_rhs_df stores it
      ldn<float, N>(b + n * 2 * N, bh);
      ldn<float, N>(b + n * 2 * N + N, bl);
#pragma unroll
      for (int i = 0; i < N; ++i) bk[i] = (double)bh[i] + (double)bl[i];
    }
    const int cls = node_class(g, x, y);
    const double D = g.D[cls], invD = g.invD[cls];
    float rf[N], uf[N];
    double z[N], r[N], mu = -INFINITY;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      r[i] = bk[i] + g.te * acc[i] - D * uk[i];
      mu = fmax(mu, r[i]);
    }
    // r carries the node's simplex multiplier, O(1) even at the solution: at
    // the minimiser the free phases share max_i r_i and the others lie below.
    // A per-node constant changes neither problem, so subtract the maximum
    // before rounding to float; the free phases' residuals stay small.
#pragma unroll
    for (int i = 0; i < N; ++i) {
      r[i] -= mu;
      rf[i] = (float)r[i];
      uf[i] = f64_head(uk[i]);  // the float obstacle: u's truncated head, which k_outer_update tests against
      z[i] = r[i] * invD;
    }
    const int64_t sl = fslot<float>(g, x, y);
    stn<float, N>(r32 + sl * N, rf);
    stn<float, N>(u32 + sl * N, uf);
    // the free set from a float pass, then theta and the optimality
    // conditions on that set in FP64 (one pass instead of the iteration);
    // the full FP64 iteration only where the conditions fail (near ties)
    float zf[N];
    const float invDf = g.invDf[cls];
#pragma unroll
    for (int i = 0; i < N; ++i) zf[i] = rf[i] * invDf;
    const unsigned keep = shifted_free_set<float, N>(zf, uf);
    if (!shifted_proj_on_set<N>(z, uk, keep)) proj_box<double, N, kShifted>(z, uk);
#pragma unroll
    for (int i = 0; i < N; ++i) e = nanmax<double>(e, fabs(z[i]));
    if (!(uk[0] == uk[0])) e = uk[0];
  }
  block_max_atomic(e, rho);
}

// The mixed solve's residual.  u is read as binary64 bit patterns and split
// into float heads and tails on the integer pipe (split_f64), b comes as
// the double-float pairs of k_rhs_df, and
//   r = b - Mhat u + tau eps sum_m w_nm (u_m - u)
// (the same S u, since S = Mhat + tau eps A and A's rows sum to zero) is
// formed in double-float arithmetic: the differences u_m - u and their
// weighted sum by two-sums, the products by mul_f2.  Its error is about
// 2^-46 of the terms' magnitudes (|b|, Mhat |u|, tau eps |u_m - u|), far
// below the float rounding of the shifted residual it produces; the FP64
// pipe sees one conversion per block.  Shift, float rounding of r, the
// heads of u as the obstacle and the natural residual in float (accurate to
// a few float ulps of rho near the solution, see solve_mixed) as in the FP64
// kernel.
// Each block walks kOrRows rows of a strip of kOrThreads columns (one
// column per thread, kOrThreads - 2 output columns plus one halo column on
// each side), so every value of u is loaded and split once (the halo columns
// and rows by two blocks): a thread keeps
// the split rows y - 1, y, y + 1 of its column in registers and finds its
// west and east neighbours in shared memory.
// 64-column strips: at 128 registers a thread, eight blocks of two warps per
// SM wait at their own per-row barriers (256 columns, two blocks of eight
// warps: 0.99 against 0.93 ms per launch of the defect-correction class at
// 4096^2, N = 8)
#ifndef AC_OR_THREADS
#define AC_OR_THREADS 64
#endif
#ifndef AC_OR_ROWS
#define AC_OR_ROWS 16
#endif
constexpr int kOrRows = AC_OR_ROWS, kOrThreads = AC_OR_THREADS;
// blocks per SM: 128 registers a thread at most
constexpr int kOrMinBlocks = 65536 / (128 * kOrThreads);
static_assert(kOrThreads % 32 == 0 && kOrThreads <= kBlock && kOrThreads >= 64, "outer residual block");

template <int N>
__device__ __forceinline__ void or_load_row(const double *__restrict__ u, const Geo &g, bool col, int x, int y,
                                            float (&h)[N], float (&l)[N]) {
  if (col && y >= 0 && y <= g.H) {
    double t[N];
    ldn<double, N>(u + ((int64_t)y * g.Wn + x) * N, t);
#pragma unroll
    for (int i = 0; i < N; ++i) split_f64(t[i], h[i], l[i]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) h[i] = l[i] = 0.f;
  }
}

// sum_m w_nm (u_m - u) for one neighbour m, heads by two-sums, tails and
// errors in float
template <int N>
__device__ __forceinline__ void or_add(const float (&mh)[N], const float (&ml)[N], const float (&uh)[N],
                                       const float (&ul)[N], float w, float (&sh)[N], float (&sl)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const f2 d = two_sum(mh[i], -uh[i]);
    const f2 s = two_sum(sh[i], w * d.h);
    sh[i] = s.h;
    sl[i] += s.l + w * (d.l + (ml[i] - ul[i]));
  }
}

// One output node (x, y) of k_outer_resid_df: r from the split rows (west
// and east neighbours from the shared row, north and south from the thread's
// own registers), r32 and u32 stored, and the node's natural-residual term
// returned (NaN if u is).
// Float j (0 .. 2N - 1) of this thread's node in a b slot of
// k_outer_resid_df (read when it is used, to spare registers).
template <int N>
__device__ __forceinline__ float or_bval(const unsigned char *slot, int tx, int j) {
  constexpr int B = (N % 2 == 0) ? 16 : 8, K = B / 4;
  return reinterpret_cast<const float *>(slot + ((size_t)(j / K) * kOrThreads + tx) * B)[j % K];
}

template <int N>
__device__ __forceinline__ float or_node(const unsigned char *bslot, const Geo &g, int x, int y,
                                         const float (&rh_s)[N][kOrThreads], const float (&rl_s)[N][kOrThreads],
                                         int tx, const float (&ph)[N], const float (&pl)[N], const float (&uh)[N],
                                         const float (&ul)[N], const float (&nh)[N],
                                         const float (&nl)[N], float *__restrict__ r32, float *__restrict__ u32) {
  float sh[N], sl[N];
  {
    float eh[N], el[N], wh[N], wl[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      eh[i] = rh_s[i][tx + 1];
      el[i] = rl_s[i][tx + 1];
      wh[i] = rh_s[i][tx - 1];
      wl[i] = rl_s[i][tx - 1];
      sh[i] = 0.f;
      sl[i] = 0.f;
    }
    if (x > 0 && x < g.W && y > 0 && y < g.H) {
      // (u_E + u_W + u_N + u_S) - 4 u: the heads summed by two-sums, 4 u_h
      // exactly, the tails and the two-sum errors in float
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const f2 a = two_sum(eh[i], wh[i]);
        const f2 b = two_sum(nh[i], ph[i]);
        const f2 c = two_sum(a.h, b.h);
        const f2 d = two_sum(c.h, -4.f * uh[i]);
        sh[i] = d.h;
        sl[i] = d.l + (c.l + (a.l + b.l)) + (((el[i] + wl[i]) + (nl[i] + pl[i])) - 4.f * ul[i]);
      }
    } else {
      const Weights w = edge_weights(g, x, y);
      if (w.e > 0.f) or_add<N>(eh, el, uh, ul, w.e, sh, sl);
      if (w.w > 0.f) or_add<N>(wh, wl, uh, ul, w.w, sh, sl);
      if (w.n > 0.f) or_add<N>(nh, nl, uh, ul, w.n, sh, sl);
      if (w.s > 0.f) or_add<N>(ph, pl, uh, ul, w.s, sh, sl);
    }
  }
  const int64_t n = (int64_t)y * g.Wn + x;
  const int cls = node_class(g, x, y);
  const float m0h = g.m0h[cls], m0l = g.m0l[cls];
  // r_i = rh_i + rl_i, not renormalised: rh_i the rounded sum of the heads
  float rh[N], rl[N], mu = -INFINITY;
  {
    // b as k_rhs_df stores it: N heads, then N tails
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const f2 p = mul_f2(g.teh, g.tel, sh[i], sl[i]);  // tau eps sum_m w_nm (u_m - u)
      const f2 q = mul_f2(m0h, m0l, uh[i], ul[i]);      // Mhat u
      const f2 s1 = two_sum(or_bval<N>(bslot, tx, i), -q.h);
      const f2 s2 = two_sum(s1.h, p.h);
      rh[i] = s2.h;
      rl[i] = s1.l + s2.l + ((or_bval<N>(bslot, tx, N + i) - q.l) + p.l);
      mu = fmaxf(mu, rh[i]);
    }
  }
  // shift by the largest head (any per-node constant serves, see above)
  float rf[N], zf[N], of[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const f2 a = two_sum(rh[i], -mu);
    rf[i] = a.h + (a.l + rl[i]);
    of[i] = uh[i];  // the float obstacle: u's truncated head
  }
  const int64_t slot = fslot<float>(g, x, y);
  stn<float, N>(r32 + slot * N, rf);
  stn<float, N>(u32 + slot * N, of);
  const float invDf = g.invDf[cls];
#pragma unroll
  for (int i = 0; i < N; ++i) zf[i] = rf[i] * invDf;
  proj_box<float, N, kShifted>(zf, of);
  float e = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) e = nanmax<float>(e, fabsf(zf[i]));
  return uh[0] == uh[0] ? e : __int_as_float(0x7fc00000);
}

// The rows of u a thread needs next (two ahead) and the b of its next node
// are copied to shared memory with cp.async while the thread works on the
// current row, so the loads' latency overlaps the double-float arithmetic.
// A node's 8N bytes (N doubles of u, or the 2N floats of b) go as OrCopy<N>::C
// pieces of B bytes, stored piece-major ([piece][thread]) so that a warp's
// shared-memory reads are conflict-free.
template <int N>
struct OrCopy {
  static constexpr int B = (N % 2 == 0) ? 16 : 8, C = 8 * N / B;
  static constexpr int kSlotBytes = 8 * N * kOrThreads;  // one row of the strip
};
// Shared memory of k_outer_resid_df beyond its static arrays: two u slots and
// two b slots.
template <int N>
constexpr size_t outer_resid_smem() { return 4 * (size_t)OrCopy<N>::kSlotBytes; }

template <int N>
__device__ __forceinline__ void or_issue(unsigned char *slot, const void *gsrc, int tx) {
  using O = OrCopy<N>;
#pragma unroll
  for (int c = 0; c < O::C; ++c)
    cp_async<O::B>(slot + ((size_t)c * kOrThreads + tx) * O::B, static_cast<const unsigned char *>(gsrc) + c * O::B);
}

// The thread's 8N bytes back from its slot, as T values (double: u, float: b).
template <int N, typename T, int M>
__device__ __forceinline__ void or_read(const unsigned char *slot, int tx, T (&v)[M]) {
  using O = OrCopy<N>;
  static_assert(M * sizeof(T) == 8 * N, "one node's bytes");
#pragma unroll
  for (int c = 0; c < O::C; ++c) {
    const unsigned char *q = slot + ((size_t)c * kOrThreads + tx) * O::B;
    constexpr int K = O::B / sizeof(T);
#pragma unroll
    for (int j = 0; j < K; ++j) v[c * K + j] = reinterpret_cast<const T *>(q)[j];
  }
}

// Split a node's u (binary64) into heads and tails; the heads (the
// significands truncated to 24 bits) are also the inner solve's obstacle.
template <int N>
__device__ __forceinline__ void or_split(const double (&t)[N], float (&h)[N], float (&l)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) split_f64(t[i], h[i], l[i]);
}

template <int N>
__global__ void __launch_bounds__(kOrThreads, kOrMinBlocks) k_outer_resid_df(const double *__restrict__ u,
                                                               const float *__restrict__ b, Geo g,
                                                               float *__restrict__ r32, float *__restrict__ u32,
                                                               double *__restrict__ rho) {
  __shared__ float s_h[2][N][kOrThreads], s_l[2][N][kOrThreads];
  extern __shared__ __align__(16) unsigned char or_ring[];
  // slots: u of rows in flight at [0, 2), b at [2, 4)
  auto uslot = [&](int q) { return or_ring + q * OrCopy<N>::kSlotBytes; };
  auto bslot = [&](int q) { return or_ring + (2 + q) * OrCopy<N>::kSlotBytes; };
  const int tx = threadIdx.x;
  const int x = blockIdx.x * (kOrThreads - 2) - 1 + tx;
  const int y0 = blockIdx.y * kOrRows;
  const bool col = x >= 0 && x <= g.W;
  const bool out = col && tx >= 1 && tx <= kOrThreads - 2;
  auto u_ok = [&](int y) { return col && y >= 0 && y <= g.H; };
  auto u_row = [&](int y) { return u + ((int64_t)y * g.Wn + x) * N; };
  auto b_row = [&](int y) { return b + ((int64_t)y * g.Wn + x) * 2 * N; };
  float ph[N], pl[N], ch[N], cl[N];
  or_load_row<N>(u, g, col, x, y0 - 1, ph, pl);
  or_load_row<N>(u, g, col, x, y0, ch, cl);
  // the first group: u of row y0 + 1, b of row y0
  if (u_ok(y0 + 1)) or_issue<N>(uslot(0), u_row(y0 + 1), tx);
  if (out && y0 <= g.H) or_issue<N>(bslot(0), b_row(y0), tx);
  cp_async_commit();
  float e = 0.f;
  for (int k = 0; k < kOrRows; ++k) {
    const int y = y0 + k;
    if (y > g.H) break;  // the same for every thread of the block
    // the next group: u of row y + 2 (the north row of the next iteration)
    // and b of row y + 1, into the slots this thread emptied last iteration
    const int nxt = (k + 1) & 1, cur = k & 1;
    if (k + 1 < kOrRows) {
      if (u_ok(y + 2)) or_issue<N>(uslot(nxt), u_row(y + 2), tx);
      if (out && y + 1 <= g.H) or_issue<N>(bslot(nxt), b_row(y + 1), tx);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this iteration's group (u of row y + 1, b of row y) has landed
    float nh[N], nl[N];
    if (u_ok(y + 1)) {
      double t[N];
      or_read<N>(uslot(cur), tx, t);
      or_split<N>(t, nh, nl);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) nh[i] = nl[i] = 0.f;
    }
    const int buf = k & 1;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      s_h[buf][i][tx] = ch[i];
      s_l[buf][i][tx] = cl[i];
    }
    __syncthreads();  // with two buffers, one barrier per row
    if (out)
      e = nanmax<float>(e, or_node<N>(bslot(cur), g, x, y, s_h[buf], s_l[buf], tx, ph, pl, ch, cl, nh, nl, r32,
                                      u32));
#pragma unroll
    for (int i = 0; i < N; ++i) {
      ph[i] = ch[i];
      pl[i] = cl[i];
      ch[i] = nh[i];
      cl[i] = nl[i];
    }
  }
  cp_async_wait<0>();
  block_max_atomic(e, rho);
}

// One thread per node; the node's update is outer_update_node (ac_df64.cuh),
// its warp-wide skips of binary64 operations by __reduce_or_sync.
template <int N>
__global__ void k_outer_update(double *__restrict__ u, const float *__restrict__ delta, Geo g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const unsigned lanes = __activemask();
  const int64_t k = (int64_t)y * g.Wn + x;
  double uk[N];
  float dk[N];
  ldn_rw<double, N>(u + k * N, uk);
  ldn<float, N>(delta + fslot<float>(g, x, y) * N, dk);
  const int path = outer_update_node<N>(uk, dk, [lanes](unsigned m) { return __reduce_or_sync(lanes, m); });
  if (path == 2) proj_simplex<double, N>(uk);
  stn<double, N>(u + k * N, uk);
}

// ---------------------------------------------------------------------------
// a4/a5: one colour of the projected block Gauss-Seidel sweep on the fine
// level (Sec. 3.1: nodal sub-problems in red-black order; Sec. 3.3: each
// nodal N-vector projected onto the simplex).  Nodes with (x + y) % 2 ==
// color are independent given the other colour:
//   z_n = (rhs_n + tau eps sum_m w_nm x_m) / S_nn,   x_n <- P(z_n).
// ---------------------------------------------------------------------------
// MASK: the last pass of a smoothing sequence (its own instantiation, so the
// other passes keep their register budget).
// With corr != null (first colour of the first sweep after a coarse
// correction) the neighbours are read as x + omega d: that is exactly the
// pending update x += omega d, because this pass overwrites its own colour
// and the next pass overwrites the other one without reading old values.
template <typename T, int N, int FORM, bool MASK>
__global__ void __launch_bounds__(kBlock) k_smooth_fine(T *__restrict__ x, const T *__restrict__ rhs,
                                                        const T *__restrict__ ob, const T *__restrict__ corr,
                                                        const double *__restrict__ omega, Geo g, int color,
                                                        T *__restrict__ rt, uint8_t *__restrict__ mask,
                                                        MaskDirty dirty) {
  const int y = blockIdx.y;
  const int xx = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((y + color) & 1);
  if (xx > g.W) return;
  const int64_t n = fslot<T>(g, xx, y);
  // the mask byte this pass replaces, loaded first so its latency overlaps
  const uint8_t old_mask = (MASK && dirty.p) ? mask[(int64_t)y * g.Wn + xx] : (uint8_t)0;
  T acc[N], bk[N], o[N];
  nbr_sum<T, N>(x, g, xx, y, acc);
  if (corr) {
    const T w = omega_t<T>(omega);
    if (w != T(0)) {
      T dc[N];
      nbr_sum<T, N>(corr, g, xx, y, dc);
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] += w * dc[i];
    }
  }
  ldn<T, N>(rhs + n * N, bk);
  if constexpr (FORM != kDirect) ldn<T, N>(ob + n * N, o);
  const int cls = node_class(g, xx, y);
  const T te = geo_te<T>(g), invD = geo_invD<T>(g, cls);
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = (bk[i] + te * acc[i]) * invD;
  proj_box<T, N, FORM>(acc, o);
  stn<T, N>(x + n * N, acc);
  if constexpr (MASK) {
    // last pass of a smoothing sequence: this node's nodal problem is solved
    // exactly, so its natural residual is 0 and its residual is constant on
    // the free phases (tangent part 0); store the free mask (and rt = 0 when
    // rt != null) here, and k_fine_resid visits the other colour only
    int cnt = 0;
    unsigned pos = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const bool fr = FORM == kTangent ? o[i] != T(0) : acc[i] > (FORM == kShifted ? -o[i] : T(0));
      if (fr) {
        pos |= 1u << i;
        ++cnt;
      }
    }
    const uint8_t nm = (uint8_t)(cnt >= 2 ? pos : 0u);
    if (dirty.p && old_mask != nm) mark_dirty(dirty, xx, y);
    mask[(int64_t)y * g.Wn + xx] = nm;
    if (rt) {
      T z[N];
#pragma unroll
      for (int i = 0; i < N; ++i) z[i] = T(0);
      stn<T, N>(rt + n * N, z);
    }
  }
}
// ---------------------------------------------------------------------------
// a6/a9: fine residual r = rhs - S x, natural residual rho = max |x - P(z)|
// (z = x + r/S_nn), free-phase mask and the tangent projection of r:
//   free_n,i = x_n,i above its bound, and at least two phases of node n free;
//   rt_n,i   = r_n,i - mean_{free j} r_n,j for free i, 0 otherwise.
// A node at a vertex of the simplex has no free phase.  rt and mask may be
// null (residual only).  After a red-black smoothing sequence only the first
// colour needs this kernel: see k_smooth_fine.  With a mask, the number of
// visited nodes with a free phase is added to the integer that follows *rho
// (the host picks the coarse correction's form from it).
// ---------------------------------------------------------------------------
template <typename T, int N, int FORM>
__global__ void __launch_bounds__(kBlock) k_fine_resid(const T *__restrict__ x, const T *__restrict__ rhs,
                                                       const T *__restrict__ ob, Geo g, T *__restrict__ rt,
                                                       uint8_t *__restrict__ mask, double *__restrict__ rho,
                                                       int color, MaskDirty dirty) {
  // color < 0: every node; color 0 or 1: the nodes of that colour only (the
  // other colour's share was stored by the last smoothing pass)
  const int y = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int xx = color < 0 ? t : 2 * t + ((y + color) & 1);
  T e = T(0);
  int nfree = 0;
  if (xx <= g.W) {
    const int64_t n = (int64_t)y * g.Wn + xx, sl = fslot<T>(g, xx, y);
    // the mask byte this kernel replaces, loaded first so its latency overlaps
    const uint8_t old_mask = (rt && dirty.p) ? mask[n] : (uint8_t)0;
    T acc[N], xk[N], bk[N], r[N], o[N];
    nbr_sum<T, N>(x, g, xx, y, acc);
    ldn<T, N>(x + sl * N, xk);
    ldn<T, N>(rhs + sl * N, bk);
    if constexpr (FORM != kDirect) ldn<T, N>(ob + sl * N, o);
    const int cls = node_class(g, xx, y);
    const T D = geo_D<T>(g, cls), invD = geo_invD<T>(g, cls), te = geo_te<T>(g);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      r[i] = bk[i] + te * acc[i] - D * xk[i];
      acc[i] = (bk[i] + te * acc[i]) * invD;
    }
    proj_box<T, N, FORM>(acc, o);
    int cnt = 0;
    unsigned pos = 0;
    T et = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      et = nanmax<T>(et, fabs(xk[i] - acc[i]));
      // free: above the bound (direct, shifted), or in the frozen set (tangent)
      const bool fr = FORM == kTangent ? o[i] != T(0) : xk[i] > (FORM == kShifted ? -o[i] : T(0));
      if (fr) {
        pos |= 1u << i;
        ++cnt;
      }
    }
    e = et;
    if (!(xk[0] == xk[0])) e = xk[0];
    if (rt) {
      const unsigned fr = cnt >= 2 ? pos : 0u;
      nfree = fr != 0u;
      T s = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i)
        if ((fr >> i) & 1u) s += r[i];
      const T mean = cnt >= 2 ? s * rcp_small<T>(cnt) : T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) r[i] = ((fr >> i) & 1u) ? r[i] - mean : T(0);
      stn<T, N>(rt + sl * N, r);
      if (dirty.p && old_mask != (uint8_t)fr) mark_dirty(dirty, xx, y);
      mask[n] = (uint8_t)fr;
    }
  }
  if (rt) {
    const int c = __syncthreads_count(nfree);
    if (threadIdx.x == 0 && c) atomicAdd(reinterpret_cast<unsigned long long *>(rho + 1), (unsigned long long)c);
  }
  block_max_atomic<T>(e, rho);
}

// ---------------------------------------------------------------------------
// Restriction r_c(K) = sum_a P_aK t(a) over the 7 fine nodes of the support
// of the coarse basis function (weights 1 at 2K, 1/2 at E, W, N, S, NE, SW).
// k_restrict0: fine (node-major) -> first coarse level (phase-major);
// k_restrict : coarse -> coarser (both phase-major).
// A coarse row with a zero diagonal in the coarse operator opc has no free
// (or active) fine node of its phase in its support, where t = 0: r_c = 0
// without reading t.
// ---------------------------------------------------------------------------
// One kJ2X x kJ2Y tile of coarse nodes per block (kTileRows rows per
// thread), all phases per node: the grid's tiles (a dense level), or the
// first level's tile list (tile | now << 32 | written << 40): phases live
// now are computed, the ones that just died are zeroed, and tiles dead in
// both cycles are not in the list (see kLiveNow).
template <typename T, int N>
__device__ __forceinline__ void restrict0_tile(const T *__restrict__ t, const Geo &gf, const Geo &gc,
                                               const T *__restrict__ opc, T *__restrict__ rc, int tx, int ty,
                                               unsigned now, unsigned wr);

template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_restrict0(const T *__restrict__ t, Geo gf, Geo gc,
                                                            const T *__restrict__ opc, T *__restrict__ rc,
                                                            const uint64_t *__restrict__ tiles,
                                                            const int *__restrict__ count) {
  if (!tiles) {
    restrict0_tile<T, N>(t, gf, gc, opc, rc, (int)blockIdx.x, (int)blockIdx.y, (1u << N) - 1u, (1u << N) - 1u);
    return;
  }
  const int cnt = *count, ntx = tiles_x(gc);
  for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
    const uint64_t e = tiles[w];
    const int tile = (int)(e & 0xffffffffull);
    restrict0_tile<T, N>(t, gf, gc, opc, rc, tile % ntx, tile / ntx, (unsigned)((e >> 32) & 0xffull),
                         (unsigned)((e >> 40) & 0xffull));
  }
}

template <typename T, int N>
__device__ __forceinline__ void restrict0_tile(const T *__restrict__ t, const Geo &gf, const Geo &gc,
                                               const T *__restrict__ opc, T *__restrict__ rc, int tx, int ty,
                                               unsigned now, unsigned wr) {
  constexpr int dx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int dy[7] = {0, 0, 0, 1, -1, 1, -1};
  const int64_t nc = (int64_t)gc.Wn * (gc.H + 1);
  const int X = tx * kJ2X + (int)(threadIdx.x % kJ2X);
#pragma unroll 1
  for (int q = 0; q < kTileRows; ++q) {
    const int Y = ty * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
    if (X > gc.W || Y > gc.H) continue;
    const int64_t K = (int64_t)Y * gc.Wn + X;
    unsigned live = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if ((now >> i) & 1u) live |= (opc[i * nc + K] > T(0)) ? 1u << i : 0u;
    T acc[N], v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = T(0);
    if (live) {
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        const int ax = 2 * X + dx[s], ay = 2 * Y + dy[s];
        if (ax < 0 || ax > gf.W || ay < 0 || ay > gf.H) continue;
        const T p = s == 0 ? T(1) : T(0.5);
        ldn<T, N>(t + fslot<T>(gf, ax, ay) * N, v);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] += p * v[i];
      }
    }
    // a row with a zero diagonal has no free fine node of its phase under it
    // (rt = 0 there): r = 0
#pragma unroll
    for (int i = 0; i < N; ++i)
      if ((wr >> i) & 1u) rc[i * nc + K] = ((live >> i) & 1u) ? acc[i] : T(0);
  }
}

// One coarse row (node, phase) of the restriction between coarse levels.
template <typename T, int N>
__device__ __forceinline__ void restrict_row(const T *__restrict__ t, const Geo &gf, const Geo &gc,
                                             const T *__restrict__ opc, T *__restrict__ rc, int X, int Y, int i) {
  constexpr int dx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int dy[7] = {0, 0, 0, 1, -1, 1, -1};
  const int64_t nf = (int64_t)gf.Wn * (gf.H + 1), nc = (int64_t)gc.Wn * (gc.H + 1);
  if (!(opc[i * nc + (int64_t)Y * gc.Wn + X] > T(0))) {
    rc[i * nc + (int64_t)Y * gc.Wn + X] = T(0);
    return;
  }
  const T *ti = t + i * nf;
  T acc = T(0);
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    const int ax = 2 * X + dx[s], ay = 2 * Y + dy[s];
    if (ax < 0 || ax > gf.W || ay < 0 || ay > gf.H) continue;
    const T p = s == 0 ? T(1) : T(0.5);
    acc += p * ti[(int64_t)ay * gf.Wn + ax];
  }
  rc[i * nc + (int64_t)Y * gc.Wn + X] = acc;
}

// The restriction onto a tiled level, driven by the coarse level's list:
// live tiles computed, dying ones zeroed (see kLiveNow).
template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_restrict_tiled(const T *__restrict__ t, Geo gf, Geo gc,
                                                                 const T *__restrict__ opc, T *__restrict__ rc,
                                                                 TileList L) {
  for_each_tile(L, gc, [&](int tx, int ty, int i, bool dying) {
    const int64_t nc = (int64_t)gc.Wn * (gc.H + 1);
    const int X = tx * kJ2X + (int)(threadIdx.x % kJ2X);
#pragma unroll
    for (int q = 0; q < kTileRows; ++q) {
      const int Y = ty * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
      if (X > gc.W || Y > gc.H) continue;
      if (dying)
        rc[i * nc + (int64_t)Y * gc.Wn + X] = T(0);
      else
        restrict_row<T, N>(t, gf, gc, opc, rc, X, Y, i);
    }
  });
}

template <typename T, int N>
__global__ void k_restrict(const T *__restrict__ t, Geo gf, Geo gc, const T *__restrict__ opc, T *__restrict__ rc) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y, i = blockIdx.z;
  if (X > gc.W) return;
  constexpr int dx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int dy[7] = {0, 0, 0, 1, -1, 1, -1};
  const int64_t nf = (int64_t)gf.Wn * (gf.H + 1), nc = (int64_t)gc.Wn * (gc.H + 1);
  if (!(opc[i * nc + (int64_t)Y * gc.Wn + X] > T(0))) {
    rc[i * nc + (int64_t)Y * gc.Wn + X] = T(0);
    return;
  }
  const T *ti = t + i * nf;
  T acc = T(0);
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    const int ax = 2 * X + dx[s], ay = 2 * Y + dy[s];
    if (ax < 0 || ax > gf.W || ay < 0 || ay > gf.H) continue;
    const T p = s == 0 ? T(1) : T(0.5);
    acc += p * ti[(int64_t)ay * gf.Wn + ax];
  }
  rc[i * nc + (int64_t)Y * gc.Wn + X] = acc;
}

// ---------------------------------------------------------------------------
// Truncated Galerkin operator of the first coarse level, per phase i:
//   S_1,i = P' M_i S M_i P,  M_i = diag(free_n,i)  (truncated prolongation).
// Stored as the C, E, N, NE entries of each coarse node.  Phases free on the
// whole neighbourhood take the untruncated product from a per-class table;
// phases free nowhere get 0; only phases free on part of it are summed here
// (at most 35 products of dyadic weights with S entries).
// ---------------------------------------------------------------------------
// One coarse node of the truncated first-level operator.  The 6x6 box of fine
// masks around the node is loaded once (0 outside the grid: such nodes drop
// out of every product) and the sums over the 7 fine nodes a of the coarse
// hat and their 5 stencil neighbours b unroll completely, so hat weights and
// offsets are compile-time constants.  INTERIOR (2 <= X <= Wc-2,
// 2 <= Y <= Hc-2): every box node is in the grid and every a, b is an interior
// fine node (S_aa = D[interior], S_ab = -tau eps), so range tests and
// stencil lookups drop out.
// The 6x6 box of fine masks around coarse node (X, Y): the mask of fine node
// (2X - 2 + i, 2Y - 2 + j), 0 outside the grid, is byte i of the packed row
// words pk[j][0] (i < 4) and pk[j][1] (i = 4, 5).  all / any: the phases free
// at every / some box node inside the grid (any is a superset of the phases
// whose row of the truncated operator is nonzero).
template <int N, bool INTERIOR>
__device__ __forceinline__ void galerkin0_box(const uint8_t *__restrict__ mask, const Geo &gf, int X, int Y,
                                              unsigned (&pk)[6][2], unsigned &all, unsigned &any) {
  all = (1u << N) - 1u;
  any = 0u;
  const int64_t row0 = (int64_t)(2 * Y - 2) * gf.Wn + (2 * X - 2);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    pk[j][0] = pk[j][1] = 0u;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int fx = 2 * X - 2 + i, fy = 2 * Y - 2 + j;
      const bool v = INTERIOR || (fx >= 0 && fx <= gf.W && fy >= 0 && fy <= gf.H);
      const unsigned b = v ? (unsigned)mask[row0 + (int64_t)j * gf.Wn + i] : 0u;
      pk[j][i >> 2] |= b << (8 * (i & 3));
      if (v) {
        all &= b;
        any |= b;
      }
    }
  }
}

// The operator entries of coarse node (X, Y) from its box, for the phases in
// wmask (the others are not written).
template <typename T, int N, bool INTERIOR>
__device__ __forceinline__ void galerkin0_node(const unsigned (&pk)[6][2], unsigned all, unsigned any,
                                               unsigned wmask, const Geo &gf, const Geo &gc,
                                               const Galerkin0Table &tab, int cls, int X, int Y,
                                               T *__restrict__ op) {
  constexpr int sx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int sy[7] = {0, 0, 0, 1, -1, 1, -1};
  constexpr int ox[5] = {0, 1, -1, 0, 0};
  constexpr int oy[5] = {0, 0, 0, 1, -1};
  constexpr int lx[4] = {0, 1, 0, 1};
  constexpr int ly[4] = {0, 0, 1, 1};
  auto m = [&](int j, int i) -> unsigned { return (pk[j][i >> 2] >> (8 * (i & 3))) & 0xffu; };
  const int64_t nc = (int64_t)gc.Wn * (gc.H + 1), K = (int64_t)Y * gc.Wn + X;
  const unsigned partial = any & ~all;
  T tvT[4];  // the table entries of this node's class in T
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    if constexpr (sizeof(T) == 4)
      tvT[l] = tab.vf[cls][l];
    else
      tvT[l] = tab.v[cls][l];
  }
  if (!partial) {
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
      for (int i = 0; i < N; ++i)
        if ((wmask >> i) & 1u) op[(l * N + i) * nc + K] = ((all >> i) & 1u) ? tvT[l] : T(0);
    return;
  }
  if constexpr (INTERIOR) {
    // one phase at a time (4 live accumulators), products with compile-time
    // hat weights and the interior stencil constants
    const T Daa = geo_D<T>(gf, 4), Sab = -geo_te<T>(gf);
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      if (!((wmask >> i) & 1u)) continue;
      T c4[4] = {T(0), T(0), T(0), T(0)};
      if ((partial >> i) & 1u) {
#pragma unroll
        for (int s = 0; s < 7; ++s) {
          const T pa = s == 0 ? T(1) : T(0.5);
          const unsigned ma = (m(2 + sy[s], 2 + sx[s]) >> i) & 1u;
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const bool on = (ma & (m(2 + sy[s] + oy[o], 2 + sx[s] + ox[o]) >> i)) != 0u;
            const T sab = o == 0 ? Daa : Sab;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const T q = hat_weight_t<T>(sx[s] + ox[o] - 2 * lx[l], sy[s] + oy[o] - 2 * ly[l]);
              if (q == T(0)) continue;
              c4[l] += on ? pa * sab * q : T(0);
            }
          }
        }
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) op[(l * N + i) * nc + K] = ((all >> i) & 1u) ? tvT[l] : c4[l];
    }
  } else {
    // boundary nodes: one phase at a time (few registers), stencil entries by
    // node class
    bool lval[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) lval[l] = (lx[l] == 0 || X < gc.W) && (ly[l] == 0 || Y < gc.H);
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      if (!((wmask >> i) & 1u)) continue;
      T c4[4] = {T(0), T(0), T(0), T(0)};
      if (((partial >> i) & 1u)) {
#pragma unroll
        for (int s = 0; s < 7; ++s) {
          const T pa = s == 0 ? T(1) : T(0.5);
          const unsigned ma = (m(2 + sy[s], 2 + sx[s]) >> i) & 1u;
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const unsigned mm = ma & (m(2 + sy[s] + oy[o], 2 + sx[s] + ox[o]) >> i);
            if (!(mm & 1u)) continue;
            const T sab = fine_S_t<T>(gf, 2 * X + sx[s], 2 * Y + sy[s], ox[o], oy[o]);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const T q = hat_weight_t<T>(sx[s] + ox[o] - 2 * lx[l], sy[s] + oy[o] - 2 * ly[l]);
              if (q == T(0) || !lval[l]) continue;
              c4[l] += pa * sab * q;
            }
          }
        }
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) op[(l * N + i) * nc + K] = ((all >> i) & 1u) ? tvT[l] : c4[l];
    }
  }
}

// One block per kJ2X x kJ2Y tile of coarse nodes, kTileThreads threads with
// kTileRows rows of nodes each.  With live flags (tf != null, a tiled first
// level) the block first ORs the fine masks over the union of its nodes' 6x6
// boxes (the phases with a free fine node near the tile) into the tile's
// flags, then writes the entries of the phases live now or in the previous
// cycle only (zeros for the latter, see kLiveNow): a tile that stays dead
// costs the OR alone.
// The tiles of the first level are also appended to its lists: each (tile,
// phase) live or dying to items, and each tile with phases to write to tiles
// as tile | now << 32 | written << 40 (phase masks).
// A tile whose boxes saw no mask change since its last computation (dirty
// byte clear) keeps its operator and its live phases: only its flags and list
// entries are renewed.  changed[tile] tells the next level whether the
// tile's operator was rewritten this cycle.  A dense first level (tf null)
// with dirty flags skips its clean tiles the same way.
template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_galerkin0(const uint8_t *__restrict__ mask, Geo gf, Geo gc,
                                                            Galerkin0Table tab, T *__restrict__ op,
                                                            uint8_t *__restrict__ tf, uint64_t *__restrict__ items,
                                                            uint64_t *__restrict__ tiles, int *__restrict__ count,
                                                            uint8_t *__restrict__ dirty,
                                                            uint8_t *__restrict__ changed) {
  __shared__ unsigned s_now, s_prev;
  __shared__ int s_base, s_dirty;
  unsigned wmask = (1u << N) - 1u;
  if (!tf && dirty) {
    // dense level: a tile whose boxes saw no mask change keeps its operator
    const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) s_dirty = dirty[tile];
    __syncthreads();
    if (!s_dirty) return;
    __syncthreads();  // every thread has read the flag before it is cleared
    if (threadIdx.x == 0) dirty[tile] = 0;
  }
  if (tf) {
    const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) s_dirty = dirty[tile];
    __syncthreads();
    if (!s_dirty) {
      // the operator stands: the phases live before stay live (one lane per
      // phase of the first warp)
      if (threadIdx.x < 32u) {
        const unsigned lane = threadIdx.x;
        unsigned live = 0u;
        uint8_t *f = tf + ((int64_t)lane * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (lane < (unsigned)N) {
          live = *f & kLiveNow;
          *f = (uint8_t)(live ? (kLiveNow | kLivePrev) : 0u);
        }
        const unsigned now = __ballot_sync(0xffffffffu, live != 0u);
        if (now) {
          int base = 0;
          if (lane == 0) {
            base = atomicAdd(count, __popc(now));
            tiles[atomicAdd(count + 1, 1)] = (uint64_t)tile | ((uint64_t)now << 32) | ((uint64_t)now << 40);
          }
          base = __shfl_sync(0xffffffffu, base, 0);
          if (live) items[base + __popc(now & ((1u << lane) - 1u))] = tile_item(tile, (int)lane, false);
        }
        if (lane == 0) changed[tile] = 0;
      }
      return;
    }
    if (threadIdx.x == 0) {
      dirty[tile] = 0;
      changed[tile] = 1;
    }
    if (threadIdx.x == 0) s_now = s_prev = 0u;
    __syncthreads();
    // fine nodes 2X - 2 .. 2X + 3 over the tile's X range (rows alike), a
    // (2 kJ2X + 4) x (2 kJ2Y + 4) box clamped to the grid; the loops have
    // compile-time trip counts, so every load issues before the first OR
    constexpr int BX = 2 * kJ2X + 4, BY = 2 * kJ2Y + 4, WARPS = kTileThreads / 32;
    const int fx0 = 2 * (int)blockIdx.x * kJ2X - 2, fy0 = 2 * (int)blockIdx.y * kJ2Y - 2;
    unsigned a = 0u;
#pragma unroll
    for (int j = 0; j < (BY + WARPS - 1) / WARPS; ++j)
#pragma unroll
      for (int c = 0; c < (BX + 31) / 32; ++c) {
        const int by = j * WARPS + (int)(threadIdx.x / 32u), bx = c * 32 + (int)(threadIdx.x & 31u);
        const int fx = fx0 + bx, fy = fy0 + by;
        if (by < BY && bx < BX && fx >= 0 && fx <= gf.W && fy >= 0 && fy <= gf.H)
          a |= mask[(int64_t)fy * gf.Wn + fx];
      }
    a = __reduce_or_sync(0xffffffffu, a);
    if ((threadIdx.x & 31u) == 0u && a) atomicOr(&s_now, a);
    __syncthreads();
    if (threadIdx.x < (unsigned)N) {
      uint8_t *f = tf + ((int64_t)threadIdx.x * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      const unsigned old = *f, now = (s_now >> threadIdx.x) & 1u;
      *f = (uint8_t)(now | ((old & kLiveNow) ? kLivePrev : 0u));
      if (old & kLiveNow) atomicOr(&s_prev, 1u << threadIdx.x);
    }
    __syncthreads();
    wmask = s_now | s_prev;
    // one atomic per list and block: the block's items go to consecutive slots
    if (threadIdx.x == 0 && wmask) {
      s_base = atomicAdd(count, __popc(wmask));
      tiles[atomicAdd(count + 1, 1)] = (uint64_t)tile | ((uint64_t)s_now << 32) | ((uint64_t)wmask << 40);
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)N && ((wmask >> threadIdx.x) & 1u))
      items[s_base + __popc(wmask & ((1u << threadIdx.x) - 1u))] =
          tile_item(tile, (int)threadIdx.x, !((s_now >> threadIdx.x) & 1u));
  }
  if (!wmask) return;
#pragma unroll 1
  for (int q = 0; q < kTileRows; ++q) {
    const int X = blockIdx.x * kJ2X + (int)(threadIdx.x % kJ2X);
    const int Y = blockIdx.y * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
    if (X > gc.W || Y > gc.H) continue;
    unsigned pk[6][2], all, any;
    if (X >= 2 && X <= gc.W - 2 && Y >= 2 && Y <= gc.H - 2) {
      galerkin0_box<N, true>(mask, gf, X, Y, pk, all, any);
      galerkin0_node<T, N, true>(pk, all, any, wmask, gf, gc, tab, 2 * 5 + 2, X, Y, op);
    } else {
      galerkin0_box<N, false>(mask, gf, X, Y, pk, all, any);
      galerkin0_node<T, N, false>(pk, all, any, wmask, gf, gc, tab, g0_class(Y, gc.H) * 5 + g0_class(X, gc.W), X,
                                  Y, op);
    }
  }
}


// S entry (K, K + d) of a stored coarse operator, d in the 7-point pattern
// (a compile-time direction once unrolled): C, E, N, NE are stored at the
// node, W, S, SW at the neighbour.
template <typename T, int N>
__device__ __forceinline__ T op_entry_k(const T *op, int64_t Wn, int64_t nc, int64_t K, int ddx, int ddy, int i) {
  if (ddx == 0 && ddy == 0) return op[(0 * N + i) * nc + K];
  if (ddx == 1 && ddy == 0) return op[(1 * N + i) * nc + K];
  if (ddx == 0 && ddy == 1) return op[(2 * N + i) * nc + K];
  if (ddx == 1 && ddy == 1) return op[(3 * N + i) * nc + K];
  if (ddx == -1 && ddy == 0) return op[(1 * N + i) * nc + K - 1];
  if (ddx == 0 && ddy == -1) return op[(2 * N + i) * nc + K - Wn];
  return op[(3 * N + i) * nc + K - Wn - 1];  // SW
}

// One phase of the Galerkin product S_c = P' S_f P at coarse node (X, Y):
// the C, E, N, NE entries.  The loops over the 7 fine nodes a of the coarse
// hat and their 7 stencil neighbours b unroll completely, so the hat weights
// and stencil directions are compile-time constants and each phase's ~20 loads
// issue together.  INTERIOR (1 <= X <= Wc-1, 1 <= Y <= Hc-1) drops the range
// predicates that the boundary rows need.
template <typename T, int N, bool INTERIOR>
__device__ __forceinline__ void galerkin_phase(const T *__restrict__ opf, const Geo &gf, const Geo &gc, int64_t nf,
                                               int X, int Y, int i, T (&c4)[4]) {
  constexpr int sx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int sy[7] = {0, 0, 0, 1, -1, 1, -1};
  constexpr int lx[4] = {0, 1, 0, 1};
  constexpr int ly[4] = {0, 0, 1, 1};
  bool lval[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) lval[l] = INTERIOR || ((lx[l] == 0 || X < gc.W) && (ly[l] == 0 || Y < gc.H));
  const int64_t a0 = (int64_t)(2 * Y) * gf.Wn + 2 * X;
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    const int ax = 2 * X + sx[s], ay = 2 * Y + sy[s];
    const bool va = INTERIOR || (ax >= 0 && ax <= gf.W && ay >= 0 && ay <= gf.H);
    const int64_t a = a0 + (int64_t)sy[s] * gf.Wn + sx[s];
    const T pa = s == 0 ? T(1) : T(0.5);
#pragma unroll
    for (int o = 0; o < 7; ++o) {
      T q[4];
      bool anyq = false;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        q[l] = hat_weight_t<T>(sx[s] + sx[o] - 2 * lx[l], sy[s] + sy[o] - 2 * ly[l]);
        anyq |= q[l] != T(0);
      }
      if (!anyq) continue;
      const int bx = ax + sx[o], by = ay + sy[o];
      const bool vb = INTERIOR || (va && bx >= 0 && bx <= gf.W && by >= 0 && by <= gf.H);
      if (!vb) continue;
      const T sab = pa * op_entry_k<T, N>(opf, gf.Wn, nf, a, sx[o], sy[o], i);
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (q[l] != T(0) && lval[l]) c4[l] += sab * q[l];
    }
  }
}

// Galerkin product of a stored 7-point operator: S_c = P' S_f P, one thread
// per (coarse node, phase) (phase = blockIdx.z; phase-major arrays).
template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_galerkin(const T *__restrict__ opf, Geo gf, Geo gc, T *__restrict__ opc) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y, i = blockIdx.z;
  if (X > gc.W) return;
  const int64_t nf = (int64_t)gf.Wn * (gf.H + 1), nc = (int64_t)gc.Wn * (gc.H + 1);
  const int64_t K = (int64_t)Y * gc.Wn + X;
  T c4[4] = {T(0), T(0), T(0), T(0)};
  // the coarse row is zero when every fine row under the coarse hat (2X, 2Y
  // and its E, W, N, S, NE, SW neighbours) is zero
  bool live = false;
  {
    constexpr int sx[7] = {0, 1, -1, 0, 0, 1, -1};
    constexpr int sy[7] = {0, 0, 0, 1, -1, 1, -1};
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      const int ax = 2 * X + sx[s], ay = 2 * Y + sy[s];
      if (ax >= 0 && ax <= gf.W && ay >= 0 && ay <= gf.H) live |= opf[i * nf + (int64_t)ay * gf.Wn + ax] > T(0);
    }
  }
  if (live) {
    if (X >= 1 && X <= gc.W - 1 && Y >= 1 && Y <= gc.H - 1)
      galerkin_phase<T, N, true>(opf, gf, gc, nf, X, Y, i, c4);
    else
      galerkin_phase<T, N, false>(opf, gf, gc, nf, X, Y, i, c4);
  }
#pragma unroll
  for (int l = 0; l < 4; ++l) opc[(l * N + i) * nc + K] = c4[l];
}

// The same product onto a tiled level (live flags tfc) from a tiled level
// (flags tff): one block per (kJ2X x kJ2Y tile, phase), one thread per node.
// The fine tiles under the coarse tile and its one-node halo are looked up
// first: if none is live for the phase, no coarse row of the tile can be
// nonzero and no fine operator entry is read.
// With changed_f (whether each fine tile's operator was rewritten this
// cycle) a coarse tile over fine tiles that all kept theirs keeps its own
// operator and live phases; changed_c records the same for this level.
template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_galerkin_tiled(const T *__restrict__ opf, Geo gf, Geo gc,
                                                                 T *__restrict__ opc, const uint8_t *__restrict__ tff,
                                                                 uint8_t *__restrict__ tfc, uint64_t *__restrict__ items,
                                                                 int *__restrict__ count,
                                                                 const uint8_t *__restrict__ changed_f,
                                                                 uint8_t *__restrict__ changed_c) {
  __shared__ int s_fine, s_changed;
  __shared__ unsigned s_prev;
  const int i = blockIdx.z;
  const int64_t nf = (int64_t)gf.Wn * (gf.H + 1), nc = (int64_t)gc.Wn * (gc.H + 1);
  {
    // fine nodes 2X - 1 .. 2X + 1 over the tile's X range (rows alike): fine
    // tiles 2 tx - 1 .. 2 tx + 1 (ty alike), one flag per thread of the first 9
    bool f = false, c = false;
    if (threadIdx.x < 9u) {
      const int fx = 2 * (int)blockIdx.x - 1 + (int)(threadIdx.x % 3u), fy = 2 * (int)blockIdx.y - 1 + (int)(threadIdx.x / 3u);
      if (fx >= 0 && fx < tiles_x(gf) && fy >= 0 && fy < tiles_y(gf)) {
        f = (tff[((int64_t)i * tiles_y(gf) + fy) * tiles_x(gf) + fx] & kLiveNow) != 0;
        c = changed_f[(int64_t)fy * tiles_x(gf) + fx] != 0;
      }
    }
    const int any = __syncthreads_or(f);
    const int chg = __syncthreads_or(c);
    if (threadIdx.x == 0) {
      s_fine = any;
      s_changed = chg;
    }
  }
  __syncthreads();
  const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  if (!s_changed) {
    // the fine operator under the tile stands, and so does this one
    if (threadIdx.x == 0) {
      uint8_t *f = tfc + ((int64_t)i * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      const unsigned live = *f & kLiveNow;
      *f = (uint8_t)(live ? (kLiveNow | kLivePrev) : 0u);
      if (live) items[atomicAdd(count, 1)] = tile_item(tile, i, false);
      if (changed_c && i == 0) changed_c[tile] = 0;
    }
    return;
  }
  if (changed_c && threadIdx.x == 0 && i == 0) changed_c[tile] = 1;
  // the rows of this thread: a row is live when a fine row under its hat is
  unsigned live = 0u;
  const int X = blockIdx.x * kJ2X + (int)(threadIdx.x % kJ2X);
  if (s_fine) {
#pragma unroll
    for (int q = 0; q < kTileRows; ++q) {
      const int Y = blockIdx.y * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
      if (X > gc.W || Y > gc.H) continue;
      constexpr int sx[7] = {0, 1, -1, 0, 0, 1, -1};
      constexpr int sy[7] = {0, 0, 0, 1, -1, 1, -1};
      bool lq = false;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const int ax = 2 * X + sx[k], ay = 2 * Y + sy[k];
        if (ax >= 0 && ax <= gf.W && ay >= 0 && ay <= gf.H) lq |= opf[i * nf + (int64_t)ay * gf.Wn + ax] > T(0);
      }
      live |= lq ? 1u << q : 0u;
    }
  }
  const int now = __syncthreads_or(live != 0u);
  if (threadIdx.x == 0) {
    uint8_t *f = tfc + ((int64_t)i * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const unsigned old = *f;
    s_prev = old & kLiveNow;
    *f = (uint8_t)((now ? kLiveNow : 0u) | (s_prev ? kLivePrev : 0u));
    if (now || s_prev) items[atomicAdd(count, 1)] = tile_item((int64_t)blockIdx.y * gridDim.x + blockIdx.x, i, !now);
  }
  __syncthreads();
  if (!now && !s_prev) return;
#pragma unroll 1
  for (int q = 0; q < kTileRows; ++q) {
    const int Y = blockIdx.y * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
    if (X > gc.W || Y > gc.H) continue;
    const int64_t K = (int64_t)Y * gc.Wn + X;
    T c4[4] = {T(0), T(0), T(0), T(0)};
    if ((live >> q) & 1u) {
      if (X >= 1 && X <= gc.W - 1 && Y >= 1 && Y <= gc.H - 1)
        galerkin_phase<T, N, true>(opf, gf, gc, nf, X, Y, i, c4);
      else
        galerkin_phase<T, N, false>(opf, gf, gc, nf, X, Y, i, c4);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) opc[(l * N + i) * nc + K] = c4[l];
  }
}

// (S v)_K - S_KK v_K for phase i of a stored operator (phase-major arrays).
template <typename T, int N>
__device__ __forceinline__ T op_offdiag(const T *op, const T *v, const Geo &g, int64_t nc, int x, int y, int i) {
  const int64_t K = (int64_t)y * g.Wn + x;
  const T *oE = op + (1 * N + i) * nc, *oN = op + (2 * N + i) * nc, *oNE = op + (3 * N + i) * nc;
  const T *vi = v + i * nc;
  T s = T(0);
  if (x < g.W) s += oE[K] * vi[K + 1];
  if (x > 0) s += oE[K - 1] * vi[K - 1];
  if (y < g.H) s += oN[K] * vi[K + g.Wn];
  if (y > 0) s += oN[K - g.Wn] * vi[K - g.Wn];
  if (x < g.W && y < g.H) s += oNE[K] * vi[K + g.Wn + 1];
  if (x > 0 && y > 0) s += oNE[K - g.Wn - 1] * vi[K - g.Wn - 1];
  return s;
}

// a7: l1-Jacobi smoothing on a coarse level, vout = vin + (r - S vin) / l1,
// l1 = sum_j |S_Kj| (convergent for any symmetric positive definite S).
// Rows with a zero diagonal stay 0.  ZERO_IN: vin = 0 (the first sweep of a
// V-cycle level), so the first sweep gives r / l1 and vin is not read.  The
// phases of a coarse level are independent systems.
// Two l1-Jacobi sweeps fused, one kJ2X x kJ2Y tile of one phase plane per
// block (phase = blockIdx.z).  The operator and vin on the tile plus a halo
// of 2, and r on the tile plus a halo of 1, are staged in shared memory
// (nodes outside the grid as 0: their coefficients are 0, so they drop out of
// every sum); the first sweep runs on the tile plus a halo of 1, the second on
// the tile, which is then written once.  Each node's sums run in the fixed
// order C, E, W, N, S, NE, SW, so the halo nodes recomputed by neighbouring
// tiles agree bit for bit; one read and one write of the level per pair of
// sweeps, and no neighbour loads through L1/L2.  The first sweep keeps each
// node's 1 / l1 in shared memory for the second.  vout must not alias vin
// unless ZERO_IN (vin unread).
constexpr int kJ2Threads = 256;

// Zeros into the tile (tx, ty) of phase plane a (and b when not null): a tile
// that stopped being live this cycle (see kLiveNow).
template <typename T>
__device__ __forceinline__ void tile_zero(const Geo &g, int tx, int ty, T *__restrict__ a, T *__restrict__ b) {
  for (int t = threadIdx.x; t < kJ2X * kJ2Y; t += blockDim.x) {
    const int x = tx * kJ2X + t % kJ2X, y = ty * kJ2Y + t / kJ2X;
    if (x <= g.W && y <= g.H) {
      a[(int64_t)y * g.Wn + x] = T(0);
      if (b) b[(int64_t)y * g.Wn + x] = T(0);
    }
  }
}

template <typename T, int N, bool ZERO_IN>
__device__ __forceinline__ void jacobi2_tile(const T *__restrict__ op, const T *__restrict__ r, const T *vin,
                                             T *vout, const Geo &g, int bxt, int byt, int i) {
  constexpr int AX = kJ2X + 4, AY = kJ2Y + 4;  // tile + halo 2
  constexpr int BX = kJ2X + 2, BY = kJ2Y + 2;  // tile + halo 1
  __shared__ T sC[AY][AX], sE[AY][AX], sN[AY][AX], sNE[AY][AX], sV[AY][AX];
  __shared__ T sR[BY][BX], sV1[BY][BX], sI[BY][BX];
  const int64_t nc = (int64_t)g.Wn * (g.H + 1);
  const T *C = op + (0 * N + i) * nc, *E = op + (1 * N + i) * nc, *Nn = op + (2 * N + i) * nc,
          *NE = op + (3 * N + i) * nc, *ri = r + i * nc, *vi = vin + i * nc;
  T *vo = vout + i * nc;
  const int x0 = bxt * kJ2X - 2, y0 = byt * kJ2Y - 2;  // grid position of [0][0] of the A arrays
  // A tile whose rows all have a zero diagonal (no free fine node of this
  // phase under any of them) has vout = 0 whatever vin: write the zeros and
  // stop.  After phase separation most tiles of a phase are like that.
  int live = 0;
  for (int t = threadIdx.x; t < AX * AY; t += kJ2Threads) {
    const int ax = t % AX, ay = t / AX, x = x0 + ax, y = y0 + ay;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    const T c = in ? C[in ? (int64_t)y * g.Wn + x : 0] : T(0);
    sC[ay][ax] = c;
    live |= (ax >= 2 && ax < 2 + kJ2X && ay >= 2 && ay < 2 + kJ2Y && c > T(0)) ? 1 : 0;
  }
  if (!__syncthreads_or(live)) {
    for (int t = threadIdx.x; t < kJ2X * kJ2Y; t += kJ2Threads) {
      const int x = x0 + 2 + t % kJ2X, y = y0 + 2 + t / kJ2X;
      if (x <= g.W && y <= g.H) vo[(int64_t)y * g.Wn + x] = T(0);
    }
    return;
  }
  for (int t = threadIdx.x; t < AX * AY; t += kJ2Threads) {
    const int ax = t % AX, ay = t / AX, x = x0 + ax, y = y0 + ay;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    const int64_t K = in ? (int64_t)y * g.Wn + x : 0;
    sE[ay][ax] = in ? E[K] : T(0);
    sN[ay][ax] = in ? Nn[K] : T(0);
    sNE[ay][ax] = in ? NE[K] : T(0);
    sV[ay][ax] = (!ZERO_IN && in) ? vi[K] : T(0);
  }
  for (int t = threadIdx.x; t < BX * BY; t += kJ2Threads) {
    const int bx = t % BX, by = t / BX, x = x0 + 1 + bx, y = y0 + 1 + by;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    sR[by][bx] = in ? ri[(int64_t)y * g.Wn + x] : T(0);
  }
  __syncthreads();
  // first sweep on the tile + halo 1: B (bx, by) is A (bx + 1, by + 1)
  for (int t = threadIdx.x; t < BX * BY; t += kJ2Threads) {
    const int bx = t % BX, by = t / BX, ax = bx + 1, ay = by + 1;
    const T d = sC[ay][ax];
    T sv = ZERO_IN ? T(0) : d * sV[ay][ax], l1 = fabs(d), c;
    c = sE[ay][ax]; if (!ZERO_IN) sv += c * sV[ay][ax + 1]; l1 += fabs(c);
    c = sE[ay][ax - 1]; if (!ZERO_IN) sv += c * sV[ay][ax - 1]; l1 += fabs(c);
    c = sN[ay][ax]; if (!ZERO_IN) sv += c * sV[ay + 1][ax]; l1 += fabs(c);
    c = sN[ay - 1][ax]; if (!ZERO_IN) sv += c * sV[ay - 1][ax]; l1 += fabs(c);
    c = sNE[ay][ax]; if (!ZERO_IN) sv += c * sV[ay + 1][ax + 1]; l1 += fabs(c);
    c = sNE[ay - 1][ax - 1]; if (!ZERO_IN) sv += c * sV[ay - 1][ax - 1]; l1 += fabs(c);
    const T v0 = ZERO_IN ? T(0) : sV[ay][ax];
    const T inv = d > T(0) ? T(1) / l1 : T(0);  // 1 / l1, kept for the second sweep
    sI[by][bx] = inv;
    sV1[by][bx] = d > T(0) ? v0 + (sR[by][bx] - sv) * inv : T(0);
  }
  __syncthreads();
  // second sweep on the tile: tile (tx, ty) is B (tx + 1, ty + 1), A (tx + 2, ty + 2)
  for (int t = threadIdx.x; t < kJ2X * kJ2Y; t += kJ2Threads) {
    const int tx = t % kJ2X, ty = t / kJ2X, x = x0 + 2 + tx, y = y0 + 2 + ty;
    if (x > g.W || y > g.H) continue;
    const int bx = tx + 1, by = ty + 1, ax = tx + 2, ay = ty + 2;
    T sv = sC[ay][ax] * sV1[by][bx];
    sv += sE[ay][ax] * sV1[by][bx + 1];
    sv += sE[ay][ax - 1] * sV1[by][bx - 1];
    sv += sN[ay][ax] * sV1[by + 1][bx];
    sv += sN[ay - 1][ax] * sV1[by - 1][bx];
    sv += sNE[ay][ax] * sV1[by + 1][bx + 1];
    sv += sNE[ay - 1][ax - 1] * sV1[by - 1][bx - 1];
    vo[(int64_t)y * g.Wn + x] = sV1[by][bx] + (sR[by][bx] - sv) * sI[by][bx];
  }
}

// ---- 3-colour Gauss-Seidel on a tile (coarse levels) -------------------------
// The 7-point pattern (E, W, N, S, NE, SW) is 3-coloured by (x + y) mod 3:
// every neighbour of a node differs from it by +-1 or +-2 in x + y.  A block
// stages its tile with a halo in shared memory and sweeps it colour by
// colour, so each update sees the newest values of its neighbours inside the
// block; values outside the block's region are those at the launch.  The
// first sweep covers the tile and a ring, the second the tile (and, for the
// pre-smoothing, a ring for the residual), so one launch does two sweeps,
// and blocks agree wherever their regions overlap only up to that boundary
// information -- a smoother with overlapping blocks (every block's sweep is
// Gauss-Seidel on its own region).  The second sweep runs the colours in
// reverse (symmetric Gauss-Seidel).  Rows with a zero diagonal (no free fine
// node of the phase under them) keep 0.

// The blocks' work is spread over threads by horizontal triplets: a thread
// owns three consecutive nodes of a row of the first sweep's region -- one
// of each colour -- and keeps their operator entries, 1/d and r in registers
// for both sweeps and the residual; only the iterate is in shared memory.
// Each row's triplets start on a node of colour 0, so a thread's node q has
// colour q and the pass of colour q updates node q at a compile-time offset.
// kGsTrip triplets per row (one more than the widest region needs, for the
// row's shift) and kGsThreads threads per block.
constexpr int kGsTrip = 13, kGsThreads = 288;
enum { kGsPost = 0, kGsZero = 1, kGsPreResid = 2 };

__device__ __forceinline__ float rcp_t(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double rcp_t(double d) { return __drcp_rn(d); }

// Two Gauss-Seidel sweeps on a tile of phase i, colours forward then
// backward (see above).  MODE kGsPost: from vin, the first sweep on the tile
// + 1, the second on the tile, v written.  kGsZero: the same from v = 0 (vin
// is not read).  kGsPreResid: from v = 0, the first sweep on the tile + 2,
// the second on the tile + 1, then v and the residual t = r - S v written on
// the tile (k_coarse_resid's arithmetic order).  Rows with a zero diagonal
// keep 0 in v and t.  INTERIOR: every node the block reads lies in the grid
// (no range tests).
template <int MODE>
struct GsShape {
  static constexpr int H1 = MODE == kGsPreResid ? 2 : 1;        // halo of the first sweep's region
  static constexpr int W1 = kJ2X + 2 * H1, R1 = kJ2Y + 2 * H1;  // its width and height
  // shared columns cx <-> grid x = xs + cx: the region is cx in [3, 2 + W1]
  // (a ring at 2 and 3 + W1); rows cy <-> y = ys + cy: the region is [1, R1]
  static constexpr int X1 = 3, AX = 3 * kGsTrip + 4, AY = R1 + 2;
};

template <typename T, int N, int MODE, bool INTERIOR>
__device__ __forceinline__ void gs_tile_body(const T *__restrict__ op, const T *__restrict__ r, const T *vin, T *vout,
                                             T *__restrict__ tout, const Geo &g, int i, int xs, int ys,
                                             T (&sV)[GsShape<MODE>::AY][GsShape<MODE>::AX]) {
  using S = GsShape<MODE>;
  constexpr int H1 = S::H1, W1 = S::W1, R1 = S::R1, X1 = S::X1, AX = S::AX, AY = S::AY;
  // rows of triplets fit the block; with the row shift sh <= 2 the triplets
  // cover columns [1 + sh, 3 kGsTrip + sh] (a region [3, 2 + W1]) and touch
  // [sh, 3 kGsTrip + sh + 1] < AX
  static_assert(R1 * kGsTrip <= kGsThreads && 3 * kGsTrip >= X1 - 1 + W1 && 3 * kGsTrip + 3 < AX, "triplet grid");
  const int64_t nc = (int64_t)g.Wn * (g.H + 1);
  const T *C = op + (0 * N + i) * nc, *E = op + (1 * N + i) * nc, *Nn = op + (2 * N + i) * nc,
          *NE = op + (3 * N + i) * nc, *ri = r + i * nc;
  const int row = (int)threadIdx.x / kGsTrip, trip = (int)threadIdx.x - row * kGsTrip;
  const bool owner = row < R1;
  const int cy = row + 1, y = ys + cy;
  int sh = -(xs + 1 + y) % 3;  // shift so that node 0 (cx0) has colour 0
  sh += sh < 0 ? 3 : 0;
  const int cx0 = 1 + sh + 3 * trip, x0 = xs + cx0;
  // node q: in the first region, the second, the tile (where v and t are
  // written), the grid
  unsigned in1 = 0u, in2 = 0u, inT = 0u, grid = 0u;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int cx = cx0 + q;
    if (owner && cx >= X1 && cx <= X1 + W1 - 1) in1 |= 1u << q;
    if (owner && cx >= X1 + 1 && cx <= X1 + W1 - 2 && cy >= 2 && cy <= R1 - 1) in2 |= 1u << q;
    if (owner && cx >= X1 + H1 && cx <= X1 + H1 + kJ2X - 1 && cy >= 1 + H1 && cy <= H1 + kJ2Y) inT |= 1u << q;
    if (owner && (INTERIOR || (x0 + q >= 0 && x0 + q <= g.W && y >= 0 && y <= g.H))) grid |= 1u << q;
  }
  const int64_t K0 = (int64_t)y * g.Wn + x0;
  // every load of the tile first (one round trip of latency): the
  // operator entries and r of the triplet into registers, the iterate --
  // vin (kGsPost) or 0 -- on the region, its ring and the spare columns
  T cD[3], cI[3], cR[3], cE[3], cW[3], cN[3], cS[3], cNE[3], cSW[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool on = (grid >> q) & 1u;
    const bool w = on && (INTERIOR || x0 + q > 0), s = on && (INTERIOR || y > 0);
    cD[q] = on ? C[K0 + q] : T(0);
    cR[q] = on ? ri[K0 + q] : T(0);
    cE[q] = on ? E[K0 + q] : T(0);
    cN[q] = on ? Nn[K0 + q] : T(0);
    cNE[q] = on ? NE[K0 + q] : T(0);
    cW[q] = w ? E[K0 + q - 1] : T(0);
    cS[q] = s ? Nn[K0 + q - g.Wn] : T(0);
    cSW[q] = w && s ? NE[K0 + q - g.Wn - 1] : T(0);
  }
  const T *vi = MODE == kGsPost ? vin + i * nc : nullptr;
  for (int t = threadIdx.x; t < AX * AY; t += kGsThreads) {
    const int bx = t % AX, by = t / AX, gx = xs + bx, gy = ys + by;
    T v = T(0);
    if (MODE == kGsPost && (INTERIOR || (gx >= 0 && gx <= g.W && gy >= 0 && gy <= g.H)))
      v = vi[(int64_t)gy * g.Wn + gx];
    sV[by][bx] = v;
  }
  int live = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    live |= ((inT >> q) & 1u) && cD[q] > T(0) ? 1 : 0;
    cI[q] = cD[q] > T(0) ? rcp_t(cD[q]) : T(0);
  }
  if (!__syncthreads_or(live)) {
    // a tile with no live row: v (and t) are 0 whatever vin
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (((inT & grid) >> q) & 1u) {
        vout[i * nc + K0 + q] = T(0);
        if (MODE == kGsPreResid) tout[i * nc + K0 + q] = T(0);
      }
    return;
  }
  T *const sv = &sV[owner ? cy : 1][cx0];  // node 0 of the thread's triplet (read only by owners)
#define AC_GS_UPDATE(q)                                          \
  do {                                                           \
    T s_ = cE[q] * sv[(q) + 1];                                  \
    s_ += cW[q] * sv[(q)-1];                                     \
    s_ += cN[q] * sv[(q) + AX];                                  \
    s_ += cS[q] * sv[(q)-AX];                                    \
    s_ += cNE[q] * sv[(q) + AX + 1];                             \
    s_ += cSW[q] * sv[(q)-AX - 1];                               \
    sv[q] = (cR[q] - s_) * cI[q];                                \
  } while (0)
  if (in1 & 1u) AC_GS_UPDATE(0);
  __syncthreads();
  if (in1 & 2u) AC_GS_UPDATE(1);
  __syncthreads();
  if (in1 & 4u) AC_GS_UPDATE(2);
  __syncthreads();
  if (in2 & 4u) AC_GS_UPDATE(2);
  __syncthreads();
  if (in2 & 2u) AC_GS_UPDATE(1);
  __syncthreads();
  if (in2 & 1u) AC_GS_UPDATE(0);
  __syncthreads();
#undef AC_GS_UPDATE
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (!(((inT & grid) >> q) & 1u)) continue;
    const T vk = sv[q];
    vout[i * nc + K0 + q] = vk;
    if constexpr (MODE == kGsPreResid) {
      T s = T(0);
      s += cE[q] * sv[q + 1];
      s += cW[q] * sv[q - 1];
      s += cN[q] * sv[q + AX];
      s += cS[q] * sv[q - AX];
      s += cNE[q] * sv[q + AX + 1];
      s += cSW[q] * sv[q - AX - 1];
      tout[i * nc + K0 + q] = cD[q] > T(0) ? cR[q] - cD[q] * vk - s : T(0);
    }
  }
}

template <typename T, int N, int MODE>
__device__ __forceinline__ void gs_tile_rt(const T *__restrict__ op, const T *__restrict__ r, const T *vin, T *vout,
                                           T *__restrict__ tout, const Geo &g, int bxt, int byt, int i) {
  using S = GsShape<MODE>;
  __shared__ T sV[S::AY][S::AX];
  const int xs = bxt * kJ2X - S::H1 - S::X1, ys = byt * kJ2Y - S::H1 - 1;
  // every node the block can read: columns xs - 1 .. xs + AX - 1 (a west
  // neighbour of the first triplet), rows ys - 1 .. ys + AY - 1
  if (xs >= 1 && xs + S::AX <= g.W && ys >= 1 && ys + S::AY <= g.H)
    gs_tile_body<T, N, MODE, true>(op, r, vin, vout, tout, g, i, xs, ys, sV);
  else
    gs_tile_body<T, N, MODE, false>(op, r, vin, vout, tout, g, i, xs, ys, sV);
}

// (the register bound keeps as many blocks per SM as the shared memory
// allows: eight in float, five in double; the Gauss-Seidel tiles hold their
// triplets' operator entries in registers: four blocks of 288 threads in
// float, two in double, without spills)
constexpr int j2_min_blocks(int elem) { return elem == 4 ? 8 : 5; }
#ifndef AC_GS_BLOCKS
#define AC_GS_BLOCKS 4
#endif
constexpr int pair_min_blocks(int elem, bool gs) { return gs ? (elem == 4 ? AC_GS_BLOCKS : 2) : j2_min_blocks(elem); }
// Two smoothing sweeps per tile of a coarse level: 3-colour Gauss-Seidel
// (GS) or l1-Jacobi.
template <typename T, int N, bool ZERO_IN, bool GS>
__global__ void __launch_bounds__(GS ? kGsThreads : kJ2Threads, pair_min_blocks(sizeof(T), GS)) k_coarse_pair(const T *__restrict__ op, const T *__restrict__ r,
                                                                  const T *vin, T *vout, Geo g, TileList L) {
  for_each_tile(L, g, [&](int tx, int ty, int i, bool dying) {
    const int64_t nc = (int64_t)g.Wn * (g.H + 1);
    if (dying)
      tile_zero<T>(g, tx, ty, vout + i * nc, (T *)nullptr);
    else if constexpr (GS)
      gs_tile_rt<T, N, ZERO_IN ? kGsZero : kGsPost>(op, r, vin, vout, (T *)nullptr, g, tx, ty, i);
    else
      jacobi2_tile<T, N, ZERO_IN>(op, r, vin, vout, g, tx, ty, i);
  });
}

// The pre-smoothing pair of a coarse level (two l1-Jacobi sweeps from v = 0)
// fused with the level's residual t = r - S v: the operator is staged on the
// tile plus a halo of 3 and r on the tile plus a halo of 2, the first sweep
// runs on the tile plus 2, the second on the tile plus 1, and the residual
// on the tile, so one launch writes v and t of the tile (k_coarse_resid's
// arithmetic and order; rows with a zero diagonal give 0 for both).
template <typename T, int N>
__device__ __forceinline__ void jacobi2_resid_tile(const T *__restrict__ op, const T *__restrict__ r,
                                                   T *__restrict__ vout, T *__restrict__ tout, const Geo &g, int bxt,
                                                   int byt, int i) {
  constexpr int AX = kJ2X + 6, AY = kJ2Y + 6;  // tile + halo 3 (operator)
  constexpr int BX = kJ2X + 4, BY = kJ2Y + 4;  // tile + halo 2 (r, first sweep)
  constexpr int CX = kJ2X + 2, CY = kJ2Y + 2;  // tile + halo 1 (second sweep)
  __shared__ T sC[AY][AX], sE[AY][AX], sN[AY][AX], sNE[AY][AX];
  __shared__ T sR[BY][BX], sV1[BY][BX], sI[BY][BX], sV2[CY][CX];
  const int64_t nc = (int64_t)g.Wn * (g.H + 1);
  const T *C = op + (0 * N + i) * nc, *E = op + (1 * N + i) * nc, *Nn = op + (2 * N + i) * nc,
          *NE = op + (3 * N + i) * nc, *ri = r + i * nc;
  T *vo = vout + i * nc, *to = tout + i * nc;
  const int x0 = bxt * kJ2X - 3, y0 = byt * kJ2Y - 3;  // grid position of [0][0] of the A arrays
  int live = 0;
  for (int t = threadIdx.x; t < AX * AY; t += kJ2Threads) {
    const int ax = t % AX, ay = t / AX, x = x0 + ax, y = y0 + ay;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    const T c = in ? C[in ? (int64_t)y * g.Wn + x : 0] : T(0);
    sC[ay][ax] = c;
    live |= (ax >= 3 && ax < 3 + kJ2X && ay >= 3 && ay < 3 + kJ2Y && c > T(0)) ? 1 : 0;
  }
  if (!__syncthreads_or(live)) {
    for (int t = threadIdx.x; t < kJ2X * kJ2Y; t += kJ2Threads) {
      const int x = x0 + 3 + t % kJ2X, y = y0 + 3 + t / kJ2X;
      if (x <= g.W && y <= g.H) {
        vo[(int64_t)y * g.Wn + x] = T(0);
        to[(int64_t)y * g.Wn + x] = T(0);
      }
    }
    return;
  }
  for (int t = threadIdx.x; t < AX * AY; t += kJ2Threads) {
    const int ax = t % AX, ay = t / AX, x = x0 + ax, y = y0 + ay;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    const int64_t K = in ? (int64_t)y * g.Wn + x : 0;
    sE[ay][ax] = in ? E[K] : T(0);
    sN[ay][ax] = in ? Nn[K] : T(0);
    sNE[ay][ax] = in ? NE[K] : T(0);
  }
  for (int t = threadIdx.x; t < BX * BY; t += kJ2Threads) {
    const int bx = t % BX, by = t / BX, x = x0 + 1 + bx, y = y0 + 1 + by;
    const bool in = x >= 0 && x <= g.W && y >= 0 && y <= g.H;
    sR[by][bx] = in ? ri[(int64_t)y * g.Wn + x] : T(0);
  }
  __syncthreads();
  // first sweep from zero on the tile + 2: B (bx, by) is A (bx + 1, by + 1)
  for (int t = threadIdx.x; t < BX * BY; t += kJ2Threads) {
    const int bx = t % BX, by = t / BX, ax = bx + 1, ay = by + 1;
    const T d = sC[ay][ax];
    T l1 = fabs(d);
    l1 += fabs(sE[ay][ax]);
    l1 += fabs(sE[ay][ax - 1]);
    l1 += fabs(sN[ay][ax]);
    l1 += fabs(sN[ay - 1][ax]);
    l1 += fabs(sNE[ay][ax]);
    l1 += fabs(sNE[ay - 1][ax - 1]);
    const T inv = d > T(0) ? T(1) / l1 : T(0);
    sI[by][bx] = inv;
    sV1[by][bx] = d > T(0) ? (sR[by][bx] - T(0)) * inv : T(0);
  }
  __syncthreads();
  // second sweep on the tile + 1: C (cx, cy) is B (cx + 1, cy + 1), A (cx + 2, cy + 2)
  for (int t = threadIdx.x; t < CX * CY; t += kJ2Threads) {
    const int cx = t % CX, cy = t / CX, bx = cx + 1, by = cy + 1, ax = cx + 2, ay = cy + 2;
    T sv = sC[ay][ax] * sV1[by][bx];
    sv += sE[ay][ax] * sV1[by][bx + 1];
    sv += sE[ay][ax - 1] * sV1[by][bx - 1];
    sv += sN[ay][ax] * sV1[by + 1][bx];
    sv += sN[ay - 1][ax] * sV1[by - 1][bx];
    sv += sNE[ay][ax] * sV1[by + 1][bx + 1];
    sv += sNE[ay - 1][ax - 1] * sV1[by - 1][bx - 1];
    sV2[cy][cx] = sV1[by][bx] + (sR[by][bx] - sv) * sI[by][bx];
  }
  __syncthreads();
  // v and the residual on the tile: C (tx + 1, ty + 1), B (tx + 2, ty + 2), A (tx + 3, ty + 3)
  for (int t = threadIdx.x; t < kJ2X * kJ2Y; t += kJ2Threads) {
    const int tx = t % kJ2X, ty = t / kJ2X, x = x0 + 3 + tx, y = y0 + 3 + ty;
    if (x > g.W || y > g.H) continue;
    const int cx = tx + 1, cy = ty + 1, bx = tx + 2, by = ty + 2, ax = tx + 3, ay = ty + 3;
    const T d = sC[ay][ax], vk = sV2[cy][cx];
    T s = T(0);
    s += sE[ay][ax] * sV2[cy][cx + 1];
    s += sE[ay][ax - 1] * sV2[cy][cx - 1];
    s += sN[ay][ax] * sV2[cy + 1][cx];
    s += sN[ay - 1][ax] * sV2[cy - 1][cx];
    s += sNE[ay][ax] * sV2[cy + 1][cx + 1];
    s += sNE[ay - 1][ax - 1] * sV2[cy - 1][cx - 1];
    const int64_t K = (int64_t)y * g.Wn + x;
    vo[K] = vk;
    to[K] = d > T(0) ? sR[by][bx] - d * vk - s : T(0);
  }
}

template <typename T, int N, bool GS>
__global__ void __launch_bounds__(GS ? kGsThreads : kJ2Threads, pair_min_blocks(sizeof(T), GS)) k_coarse_pair_resid(const T *__restrict__ op,
                                                                        const T *__restrict__ r, T *__restrict__ vout,
                                                                        T *__restrict__ tout, Geo g, TileList L) {
  for_each_tile(L, g, [&](int tx, int ty, int i, bool dying) {
    const int64_t nc = (int64_t)g.Wn * (g.H + 1);
    if (dying)
      tile_zero<T>(g, tx, ty, vout + i * nc, tout + i * nc);
    else if constexpr (GS)
      gs_tile_rt<T, N, kGsPreResid>(op, r, (const T *)nullptr, vout, tout, g, tx, ty, i);
    else
      jacobi2_resid_tile<T, N>(op, r, vout, tout, g, tx, ty, i);
  });
}

// Whole-level Gauss-Seidel in one block for small coarsest grids: `sweeps`
// passes over 3 colours ((x + y) % 3 is a valid colouring of the 7-point
// E, W, N, S, NE, SW pattern) with a barrier between colours.
template <typename T, int N>
__global__ void __launch_bounds__(1024) k_coarse_solve_block(const T *__restrict__ op, const T *__restrict__ r,
                                                             T *__restrict__ v, Geo g, int sweeps) {
  const int64_t nc = (int64_t)g.Wn * (g.H + 1);
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 3; ++color) {
      for (int64_t k = threadIdx.x; k < nc; k += blockDim.x) {
        const int x = (int)(k % g.Wn), y = (int)(k / g.Wn);
        if ((x + y) % 3 != color) continue;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const T d = op[i * nc + k];
          v[i * nc + k] = d > T(0) ? (r[i * nc + k] - op_offdiag<T, N>(op, v, g, nc, x, y, i)) / d : T(0);
        }
      }
      __syncthreads();
    }
}

// The same Gauss-Seidel for coarsest grids that fit in shared memory: the
// operator, right-hand side and iterate are staged on chip and each thread
// updates (node, phase) items of the current colour.  Dynamic shared memory:
// 6 N nc values of T.
template <typename T, int N>
__global__ void __launch_bounds__(1024) k_coarse_solve_smem(const T *__restrict__ op, const T *__restrict__ r,
                                                            T *__restrict__ v, Geo g, int sweeps) {
  extern __shared__ unsigned char smem_raw[];
  T *sop = reinterpret_cast<T *>(smem_raw);
  const int nc = g.Wn * (g.H + 1);
  T *sr = sop + 4 * N * nc, *sv = sr + N * nc;
  for (int t = threadIdx.x; t < 4 * N * nc; t += blockDim.x) sop[t] = op[t];
  for (int t = threadIdx.x; t < N * nc; t += blockDim.x) {
    sr[t] = r[t];
    sv[t] = T(0);
  }
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 3; ++color) {
      for (int t = threadIdx.x; t < N * nc; t += blockDim.x) {
        const int i = t / nc, k = t - i * nc;
        const int x = k % g.Wn, y = k / g.Wn;
        if ((x + y) % 3 != color) continue;
        const T d = sop[i * nc + k];
        sv[t] = d > T(0) ? (sr[t] - op_offdiag<T, N>(sop, sv, g, nc, x, y, i)) / d : T(0);
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < N * nc; t += blockDim.x) v[t] = sv[t];
}

// ---------------------------------------------------------------------------
// The bottom of the coarse V-cycle in one launch.  Below some level k0 the
// levels are small (at most a few thousand nodes) and each of their kernels
// is latency-bound, about 7 us for tiny grids.  One block per phase stages
// the operators of levels k0 .. depth-1 and r of level k0 in shared memory
// and runs the same cycle there: kCoarseSweeps l1-Jacobi sweeps from zero,
// residual, restriction, ..., Gauss-Seidel on the coarsest level,
// prolongation and kCoarseSweeps l1-Jacobi sweeps back up.  v of level k0
// is written once.  Only W, H of each level and its operator are needed.
// ---------------------------------------------------------------------------
constexpr int kTailThreads = 1024;

// Shared-memory view of one level of one phase.
template <typename T>
struct TailLevel {
  int W, H, Wn, n;
  T *C, *E, *Nn, *NE, *r, *v, *t;
};

// sum over the six off-diagonal neighbours (E, W, N, S, NE, SW) of S_Km v_m
template <typename T>
__device__ __forceinline__ T tail_offdiag(const TailLevel<T> &L, const T *v, int k, int x, int y, T &l1) {
  T s = T(0), c;
  if (x < L.W) { c = L.E[k]; s += c * v[k + 1]; l1 += fabs(c); }
  if (x > 0) { c = L.E[k - 1]; s += c * v[k - 1]; l1 += fabs(c); }
  if (y < L.H) { c = L.Nn[k]; s += c * v[k + L.Wn]; l1 += fabs(c); }
  if (y > 0) { c = L.Nn[k - L.Wn]; s += c * v[k - L.Wn]; l1 += fabs(c); }
  if (x < L.W && y < L.H) { c = L.NE[k]; s += c * v[k + L.Wn + 1]; l1 += fabs(c); }
  if (x > 0 && y > 0) { c = L.NE[k - L.Wn - 1]; s += c * v[k - L.Wn - 1]; l1 += fabs(c); }
  return s;
}

// one l1-Jacobi sweep vout = vin + (r - S vin) / l1 (vin = 0 when null);
// rows with a zero diagonal give 0
template <typename T>
__device__ __forceinline__ void tail_jacobi(const TailLevel<T> &L, const T *vin, T *vout) {
  for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
    const T d = L.C[k];
    if (!(d > T(0))) {
      vout[k] = T(0);
      continue;
    }
    const int x = k % L.Wn, y = k / L.Wn;
    T l1 = fabs(d), sv = T(0);
    if (vin) {
      sv = d * vin[k] + tail_offdiag(L, vin, k, x, y, l1);
    } else {
      if (x < L.W) l1 += fabs(L.E[k]);
      if (x > 0) l1 += fabs(L.E[k - 1]);
      if (y < L.H) l1 += fabs(L.Nn[k]);
      if (y > 0) l1 += fabs(L.Nn[k - L.Wn]);
      if (x < L.W && y < L.H) l1 += fabs(L.NE[k]);
      if (x > 0 && y > 0) l1 += fabs(L.NE[k - L.Wn - 1]);
    }
    vout[k] = (vin ? vin[k] : T(0)) + (L.r[k] - sv) / l1;
  }
}

// t = r - S v (0 on rows with a zero diagonal)
template <typename T>
__device__ __forceinline__ void tail_resid(const TailLevel<T> &L) {
  for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
    const T d = L.C[k];
    if (!(d > T(0))) {
      L.t[k] = T(0);
      continue;
    }
    const int x = k % L.Wn, y = k / L.Wn;
    T l1 = T(0);
    L.t[k] = L.r[k] - d * L.v[k] - tail_offdiag(L, L.v, k, x, y, l1);
  }
}

// r_c = P' t (weights 1 at 2K, 1/2 at its E, W, N, S, NE, SW fine
// neighbours; 0 on coarse rows with a zero diagonal)
template <typename T>
__device__ __forceinline__ void tail_restrict(const TailLevel<T> &F, const TailLevel<T> &Cc) {
  constexpr int dx[7] = {0, 1, -1, 0, 0, 1, -1};
  constexpr int dy[7] = {0, 0, 0, 1, -1, 1, -1};
  for (int K = threadIdx.x; K < Cc.n; K += blockDim.x) {
    if (!(Cc.C[K] > T(0))) {
      Cc.r[K] = T(0);
      continue;
    }
    const int X = K % Cc.Wn, Y = K / Cc.Wn;
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      const int ax = 2 * X + dx[s], ay = 2 * Y + dy[s];
      if (ax < 0 || ax > F.W || ay < 0 || ay > F.H) continue;
      acc += (s == 0 ? T(1) : T(0.5)) * F.t[ay * F.Wn + ax];
    }
    Cc.r[K] = acc;
  }
}

// v_f += P v_c on rows with a nonzero diagonal (odd-odd fine nodes sit on
// the coarse SW-NE diagonal)
template <typename T>
__device__ __forceinline__ void tail_prolong(const TailLevel<T> &F, const TailLevel<T> &Cc) {
  for (int k = threadIdx.x; k < F.n; k += blockDim.x) {
    if (!(F.C[k] > T(0))) continue;
    const int x = k % F.Wn, y = k / F.Wn;
    const int K0 = (y >> 1) * Cc.Wn + (x >> 1);
    T p = Cc.v[K0];
    if ((x & 1) || (y & 1)) p = T(0.5) * (p + Cc.v[K0 + (x & 1) + (y & 1) * Cc.Wn]);
    F.v[k] += p;
  }
}

// Gauss-Seidel in three colours ((x + y) % 3 colours the 7-point pattern)
// from v = 0 on the coarsest level
template <typename T>
__device__ __forceinline__ void tail_gs(const TailLevel<T> &L, int sweeps) {
  for (int k = threadIdx.x; k < L.n; k += blockDim.x) L.v[k] = T(0);
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 3; ++color) {
      for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
        const int x = k % L.Wn, y = k / L.Wn;
        if ((x + y) % 3 != color) continue;
        const T d = L.C[k];
        T l1 = T(0);
        L.v[k] = d > T(0) ? (L.r[k] - tail_offdiag(L, L.v, k, x, y, l1)) / d : T(0);
      }
      __syncthreads();
    }
}

// `sweeps` Gauss-Seidel sweeps on v in place, the colours forward (0, 1, 2)
// in even sweeps and backward in odd ones (as the tiles of k_coarse_pair)
template <typename T>
__device__ __forceinline__ void tail_sgs(const TailLevel<T> &L, int sweeps) {
  for (int s = 0; s < sweeps; ++s)
    for (int q = 0; q < 3; ++q) {
      const int color = (s & 1) ? 2 - q : q;
      for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
        const int x = k % L.Wn, y = k / L.Wn;
        if ((x + y) % 3 != color) continue;
        const T d = L.C[k];
        if (!(d > T(0))) continue;
        T l1 = T(0);
        L.v[k] = (L.r[k] - tail_offdiag(L, L.v, k, x, y, l1)) / d;
      }
      __syncthreads();
    }
}

// one block per phase (blockIdx.x); dynamic shared memory
// kTailArrays * sum_l n_l values of T.  GS: the levels' smoothing sweeps are
// Gauss-Seidel (tail_sgs), else l1-Jacobi.
template <typename T, int N, bool GS>
__global__ void __launch_bounds__(kTailThreads) k_coarse_tail(TailArgs a, const T *__restrict__ r0, T *__restrict__ v0,
                                                              int coarse_sweeps, int coarsest_sweeps) {
  extern __shared__ unsigned char smem_raw[];
  T *base = reinterpret_cast<T *>(smem_raw);
  const int i = blockIdx.x;
  TailLevel<T> lv[kTailMaxLevels];
  int off = 0;
  for (int l = 0; l < a.levels; ++l) {
    TailLevel<T> &L = lv[l];
    L.W = a.W[l];
    L.H = a.H[l];
    L.Wn = L.W + 1;
    L.n = L.Wn * (L.H + 1);
    L.C = base + off;
    L.E = L.C + L.n;
    L.Nn = L.E + L.n;
    L.NE = L.Nn + L.n;
    L.r = L.NE + L.n;
    L.v = L.r + L.n;
    L.t = L.v + L.n;
    off += kTailArrays * L.n;
    const T *op = static_cast<const T *>(a.op[l]);
    for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
      L.C[k] = op[(0 * N + i) * L.n + k];
      L.E[k] = op[(1 * N + i) * L.n + k];
      L.Nn[k] = op[(2 * N + i) * L.n + k];
      L.NE[k] = op[(3 * N + i) * L.n + k];
    }
  }
  for (int k = threadIdx.x; k < lv[0].n; k += blockDim.x) lv[0].r[k] = r0[(int64_t)i * lv[0].n + k];
  __syncthreads();
  const int last = a.levels - 1;
  for (int l = 0; l < last; ++l) {
    const TailLevel<T> &L = lv[l];
    if constexpr (GS) {
      for (int k = threadIdx.x; k < L.n; k += blockDim.x) L.v[k] = T(0);
      __syncthreads();
      tail_sgs(L, coarse_sweeps);
    } else {
      // coarse_sweeps (even) sweeps from zero, alternating t and v, ending in v
      for (int s = 0; s < coarse_sweeps; ++s) {
        if (s & 1)
          tail_jacobi(L, L.t, L.v);
        else
          tail_jacobi(L, s == 0 ? (const T *)nullptr : L.v, L.t);
        __syncthreads();
      }
    }
    tail_resid(L);
    __syncthreads();
    tail_restrict(L, lv[l + 1]);
    __syncthreads();
  }
  tail_gs(lv[last], coarsest_sweeps);
  for (int l = last - 1; l >= 0; --l) {
    const TailLevel<T> &L = lv[l];
    tail_prolong(L, lv[l + 1]);
    __syncthreads();
    if constexpr (GS) {
      tail_sgs(L, coarse_sweeps);
    } else {
      for (int s = 0; s < coarse_sweeps; ++s) {
        if (s & 1)
          tail_jacobi(L, L.t, L.v);
        else
          tail_jacobi(L, L.v, L.t);
        __syncthreads();
      }
    }
  }
  for (int k = threadIdx.x; k < lv[0].n; k += blockDim.x) v0[(int64_t)i * lv[0].n + k] = lv[0].v[k];
}

// t = r - S v on a coarse level, one thread per (node, phase) (interior
// nodes branch-free; the same arithmetic and order as op_offdiag).  The
// float forms fuse it into the pre-smoothing pair (k_coarse_pair_resid).
template <typename T, int N>
__device__ __forceinline__ void coarse_resid_row(const T *__restrict__ op, const T *__restrict__ r,
                                                 const T *__restrict__ v, const Geo &g, T *__restrict__ t, int x, int y,
                                                 int i);

template <typename T, int N>
__global__ void k_coarse_resid(const T *__restrict__ op, const T *__restrict__ r, const T *__restrict__ v, Geo g,
                               T *__restrict__ t) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, i = blockIdx.z;
  if (x > g.W) return;
  coarse_resid_row<T, N>(op, r, v, g, t, x, y, i);
}

// The same on a tiled level, driven by its list (dying tiles zeroed).
template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_coarse_resid_tiled(const T *__restrict__ op, const T *__restrict__ r,
                                                                     const T *__restrict__ v, Geo g, T *__restrict__ t,
                                                                     TileList L) {
  for_each_tile(L, g, [&](int tx, int ty, int i, bool dying) {
    const int x = tx * kJ2X + (int)(threadIdx.x % kJ2X);
#pragma unroll
    for (int q = 0; q < kTileRows; ++q) {
      const int y = ty * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
      if (x > g.W || y > g.H) continue;
      if (dying)
        t[i * ((int64_t)g.Wn * (g.H + 1)) + (int64_t)y * g.Wn + x] = T(0);
      else
        coarse_resid_row<T, N>(op, r, v, g, t, x, y, i);
    }
  });
}

template <typename T, int N>
__device__ __forceinline__ void coarse_resid_row(const T *__restrict__ op, const T *__restrict__ r,
                                                 const T *__restrict__ v, const Geo &g, T *__restrict__ t, int x, int y,
                                                 int i) {
  const int64_t nc = (int64_t)g.Wn * (g.H + 1), K = (int64_t)y * g.Wn + x;
  // a row with a zero diagonal is zero, and so is its r (no free fine node of
  // the phase under it): t = 0 without reading the row
  if (!(op[i * nc + K] > T(0))) {
    t[i * nc + K] = T(0);
    return;
  }
  if (x > 0 && x < g.W && y > 0 && y < g.H) {
    const T *oE = op + (1 * N + i) * nc, *oN = op + (2 * N + i) * nc, *oNE = op + (3 * N + i) * nc;
    const T *vi = v + i * nc;
    T s = T(0);
    s += oE[K] * vi[K + 1];
    s += oE[K - 1] * vi[K - 1];
    s += oN[K] * vi[K + g.Wn];
    s += oN[K - g.Wn] * vi[K - g.Wn];
    s += oNE[K] * vi[K + g.Wn + 1];
    s += oNE[K - g.Wn - 1] * vi[K - g.Wn - 1];
    t[i * nc + K] = r[i * nc + K] - op[i * nc + K] * vi[K] - s;
    return;
  }
  t[i * nc + K] = r[i * nc + K] - op[i * nc + K] * v[i * nc + K] - op_offdiag<T, N>(op, v, g, nc, x, y, i);
}

// P1 prolongation of phase-major coarse values to fine node (x, y) (nested
// right-diagonal meshes: odd-odd fine nodes sit on the coarse SW-NE diagonal).
template <typename T, int N>
__device__ __forceinline__ void prolong_at(const T *vc, const Geo &gc, int x, int y, T (&o)[N]) {
  const int64_t nc = (int64_t)gc.Wn * (gc.H + 1);
  const int64_t K0 = (int64_t)(y >> 1) * gc.Wn + (x >> 1);
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = vc[i * nc + K0];
  if ((x & 1) == 0 && (y & 1) == 0) return;
  const int64_t K1 = K0 + (x & 1) + (int64_t)(y & 1) * gc.Wn;
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = T(0.5) * (o[i] + vc[i * nc + K1]);
}

// v_f += P v_c (coarse levels, phase-major), the arithmetic of prolong_at.
// PHASES_IN_Z: one thread per (node, phase), phase = blockIdx.z (narrow
// levels, where latency dominates); otherwise one thread per node doing all
// phases (wide levels, fewer blocks for the same bytes).  Rows of the fine
// level's operator opf with a zero diagonal are skipped: the smoothing that
// follows sets them to 0 whatever they hold (and their coefficients are 0),
// and the pre-smoothing left them 0.
template <typename T, int N, bool PHASES_IN_Z>
__global__ void k_prolong_add(const T *__restrict__ vc, Geo gf, Geo gc, const T *__restrict__ opf,
                              T *__restrict__ vf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > gf.W) return;
  const int64_t nc = (int64_t)gc.Wn * (gc.H + 1), nf = (int64_t)gf.Wn * (gf.H + 1);
  const int64_t K0 = (int64_t)(y >> 1) * gc.Wn + (x >> 1), a = (int64_t)y * gf.Wn + x;
  const bool mid = (x & 1) || (y & 1);
  const int64_t K1 = K0 + (x & 1) + (int64_t)(y & 1) * gc.Wn;
  constexpr int I = PHASES_IN_Z ? 1 : N;
#pragma unroll
  for (int j = 0; j < I; ++j) {
    const int i = PHASES_IN_Z ? (int)blockIdx.z : j;
    if (!(opf[i * nf + a] > T(0))) continue;
    const T *vi = vc + i * nc;
    T p = vi[K0];
    if (mid) p = T(0.5) * (p + vi[K1]);
    vf[i * nf + a] += p;
  }
}

// The same onto a tiled level, driven by that level's list: the live tiles
// only (a dying tile's v is 0 and stays 0, see kLiveNow).
template <typename T, int N>
__global__ void __launch_bounds__(kTileThreads) k_prolong_add_tiled(const T *__restrict__ vc, Geo gf, Geo gc,
                                                                    const T *__restrict__ opf, T *__restrict__ vf,
                                                                    TileList L) {
  for_each_tile(L, gf, [&](int tx, int ty, int i, bool dying) {
    if (dying) return;
    const int64_t nc = (int64_t)gc.Wn * (gc.H + 1), nf = (int64_t)gf.Wn * (gf.H + 1);
    const int x = tx * kJ2X + (int)(threadIdx.x % kJ2X);
    const T *vi = vc + i * nc;
#pragma unroll
    for (int q = 0; q < kTileRows; ++q) {
      const int y = ty * kJ2Y + (int)(threadIdx.x / kJ2X) + q * (kTileThreads / kJ2X);
      if (x > gf.W || y > gf.H) continue;
      const int64_t a = (int64_t)y * gf.Wn + x;
      if (!(opf[i * nf + a] > T(0))) continue;
      const int64_t K0 = (int64_t)(y >> 1) * gc.Wn + (x >> 1);
      T p = vi[K0];
      if ((x & 1) || (y & 1)) p = T(0.5) * (p + vi[K0 + (x & 1) + (int64_t)(y & 1) * gc.Wn]);
      vf[i * nf + a] += p;
    }
  });
}

// ---------------------------------------------------------------------------
// a8: coarse correction on the fine level with a feasible line search.
//   w   = tangent projection (over the free phases) of the truncated
//         prolongation M_i (P v)_i,
//   d   = P(x + w) - x  (feasible direction: the constraint set is convex),
//   omega = clamp(rt'd / d'Sd, 0, 1) minimises the step energy on [x, x + d].
// k_ls_dir writes d and the block partials of rt'd; k_ls_curv the partials of
// d'Sd; k_ls_finish computes omega; the next smoothing pass applies
// x += omega d (see k_smooth_fine).
// ---------------------------------------------------------------------------
template <typename T, int N, int FORM>
__global__ void __launch_bounds__(kBlock) k_ls_dir(const T *__restrict__ x, const T *__restrict__ ob,
                                                   const T *__restrict__ rt, const T *__restrict__ v1,
                                                   const uint8_t *__restrict__ mask, Geo gf, Geo gc,
                                                   T *__restrict__ d, double *__restrict__ part) {
  const int xx = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  T dot = T(0);
  if (xx <= gf.W) {
    const int64_t n = (int64_t)y * gf.Wn + xx, sl = fslot<T>(gf, xx, y);
    const unsigned fr = mask[n];
    T dn[N];
    if (fr) {
      T w[N], xk[N], r[N], o[N];
      prolong_at<T, N>(v1, gc, xx, y, w);
      T s = T(0);
      int cnt = 0;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if ((fr >> i) & 1u) {
          s += w[i];
          ++cnt;
        }
      const T mean = s * rcp_small<T>(cnt);
      ldn<T, N>(x + sl * N, xk);
      if constexpr (FORM != kDirect) ldn<T, N>(ob + sl * N, o);
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = xk[i] + (((fr >> i) & 1u) ? w[i] - mean : T(0));
      proj_box<T, N, FORM>(w, o);
      ldn<T, N>(rt + sl * N, r);
      T loc = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        dn[i] = w[i] - xk[i];
        loc += r[i] * dn[i];
      }
      dot = loc;
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) dn[i] = T(0);
    }
    stn<T, N>(d + sl * N, dn);
  }
  block_sum_store1<T>(dot, part + blockIdx.y * gridDim.x + blockIdx.x);
}

// d'Sd = sum_n S_nn |d_n|^2 - 2 tau eps sum over axis edges (n, m) of
// w_nm d_n . d_m, each edge counted once at its west / south end: three
// node reads per thread (own, east, north) instead of the five of S d.  A
// node with no free phase has d_n = 0 (k_ls_dir), so its terms vanish and
// only its mask byte is read.
template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_ls_curv(const T *__restrict__ d, const uint8_t *__restrict__ mask, Geo g,
                                                    double *__restrict__ part) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  T dot = T(0);
  if (x <= g.W && mask[(int64_t)y * g.Wn + x]) {
    T dk[N], t[N];
    ldn<T, N>(d + fslot<T>(g, x, y) * N, dk);
    const Weights w = edge_weights(g, x, y);
    T sq = T(0), cross = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) sq += dk[i] * dk[i];
    if (x < g.W) {
      ldn<T, N>(d + fslot<T>(g, x + 1, y) * N, t);
      T e = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) e += dk[i] * t[i];
      cross += T(w.e) * e;
    }
    if (y < g.H) {
      ldn<T, N>(d + fslot<T>(g, x, y + 1) * N, t);
      T e = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) e += dk[i] * t[i];
      cross += T(w.n) * e;
    }
    dot = geo_D<T>(g, node_class(g, x, y)) * sq - T(2) * geo_te<T>(g) * cross;
  }
  block_sum_store1<T>(dot, part + blockIdx.y * gridDim.x + blockIdx.x);
}

static __global__ void k_ls_finish(const double *__restrict__ tot, double *__restrict__ omega) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rd = tot[0], dsd = tot[1];
  double w = 0.0;
  if (dsd > 0.0 && rd > 0.0) w = fmin(1.0, rd / dsd);
  omega[0] = w;
  reinterpret_cast<float *>(omega + 1)[0] = (float)w;
}

// ---------------------------------------------------------------------------
// a13: adjoint of a time step (the step map differentiated with the active
// set of u^{t+1} frozen; see ac_adjoint_backward).  With w the solution of
// (Pi S Pi) w = Pi g in the tangent space V of u^{t+1}: dL/db = w and
// dL/dS = -w u^{t+1}'.  FP64 throughout.
// ---------------------------------------------------------------------------

// Frozen free set of u^{t+1} as 1/0 per phase (free: u > 0 at a node with at
// least two such phases) and the right-hand side Pi g.
template <int N>
__global__ void k_adj_prepare(const double *__restrict__ up, const double *__restrict__ g, int64_t n,
                              double *__restrict__ freeset, double *__restrict__ rhs) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double uk[N], gk[N], f[N];
  ldn<double, N>(up + k * N, uk);
  ldn<double, N>(g + k * N, gk);
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) cnt += uk[i] > 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) f[i] = (cnt >= 2 && uk[i] > 0.0) ? 1.0 : 0.0;
  proj_box<double, N, kTangent>(gk, f);
  stn<double, N>(freeset + k * N, f);
  stn<double, N>(rhs + k * N, gk);
}

// Per-node parts of the parameter gradients, block partials of
//   [0] dL/dlambda = sum w . (-tau f)
//   [1] dL/deps    = sum w . m0 u^t (-2 tau/eps^2) - tau sum w . A u^{t+1}
//   [2 + 3i + ch]  G_i = dL/dc_i = 2 tau lambda sum w_i (m1 - c_i m0)
// and the moment gradients gm (dL/dm1 RGB, dL/dm2) accumulated in place:
//   dL/dm2 += -tau lambda sum_i w_i,  dL/dm1 += 2 tau lambda sum_i w_i c_i.
template <int N>
__global__ void __launch_bounds__(kBlock) k_adj_accum(const double *__restrict__ w, const double *__restrict__ u,
                                                      const double *__restrict__ up, const double *__restrict__ mom,
                                                      const double *__restrict__ c, Geo g, double tau, double eps,
                                                      double lam, double *__restrict__ gm, double *__restrict__ part) {
  double acc[2 + 3 * N];
#pragma unroll
  for (int k = 0; k < 2 + 3 * N; ++k) acc[k] = 0.0;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x <= g.W) {
    const int64_t n = (int64_t)y * g.Wn + x;
    const double m0 = g.m0[node_class(g, x, y)];
    const double4 m = ld_mom(mom + n * 4);
    double wk[N], uk[N], upk[N], nb[N];
    ldn<double, N>(w + n * N, wk);
    ldn<double, N>(u + n * N, uk);
    ldn<double, N>(up + n * N, upk);
    nbr_sum<double, N>(up, g, x, y, nb);
    const Weights wt = edge_weights(g, x, y);
    const double wsum = (double)wt.e + (double)wt.w + (double)wt.n + (double)wt.s;
    double sw = 0.0, swc[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double c0 = c[i * 3], c1 = c[i * 3 + 1], c2 = c[i * 3 + 2];
      const double f = m.w - 2.0 * (c0 * m.x + c1 * m.y + c2 * m.z) + (c0 * c0 + c1 * c1 + c2 * c2) * m0;
      acc[0] += wk[i] * (-tau * f);
      acc[1] += wk[i] * m0 * uk[i] * (-2.0 * tau / (eps * eps)) - tau * wk[i] * (wsum * upk[i] - nb[i]);
      acc[2 + 3 * i + 0] += 2.0 * tau * lam * wk[i] * (m.x - c0 * m0);
      acc[2 + 3 * i + 1] += 2.0 * tau * lam * wk[i] * (m.y - c1 * m0);
      acc[2 + 3 * i + 2] += 2.0 * tau * lam * wk[i] * (m.z - c2 * m0);
      sw += wk[i];
      swc[0] += wk[i] * c0;
      swc[1] += wk[i] * c1;
      swc[2] += wk[i] * c2;
    }
    double *gk = gm + n * 4;
    gk[0] += 2.0 * tau * lam * swc[0];
    gk[1] += 2.0 * tau * lam * swc[1];
    gk[2] += 2.0 * tau * lam * swc[2];
    gk[3] += -tau * lam * sw;
  }
  block_sum_store<2 + 3 * N>(acc, part + (int64_t)(blockIdx.y * gridDim.x + blockIdx.x) * (2 + 3 * N));
}

// dL/du^t = m0 a1 w + sum_ch G_i,ch (m1_ch - c_i,ch m0) / M_i, and
// dL/dm1 += sum_i G_i u^t_i / M_i (c_i = s_i/M_i); phases of zero mass kept
// their previous mean and contribute no c-term.  G at tot[2 + 3i + ch], M_i at
// mass[i].
template <int N>
__global__ void k_adj_back(const double *__restrict__ w, const double *__restrict__ u, const double *__restrict__ mom,
                           const double *__restrict__ c, const double *__restrict__ tot,
                           const double *__restrict__ mass, Geo g, double a1, double *__restrict__ gout,
                           double *__restrict__ gm) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t n = (int64_t)y * g.Wn + x;
  const double m0 = g.m0[node_class(g, x, y)];
  const double4 m = ld_mom(mom + n * 4);
  double wk[N], uk[N], o[N], add[3] = {0, 0, 0};
  ldn<double, N>(w + n * N, wk);
  ldn<double, N>(u + n * N, uk);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double v = m0 * a1 * wk[i];
    const double M = mass[i];
    if (M != 0.0) {
      const double G0 = tot[2 + 3 * i], G1 = tot[3 + 3 * i], G2 = tot[4 + 3 * i];
      v += (G0 * (m.x - c[i * 3] * m0) + G1 * (m.y - c[i * 3 + 1] * m0) + G2 * (m.z - c[i * 3 + 2] * m0)) / M;
      add[0] += G0 * uk[i] / M;
      add[1] += G1 * uk[i] / M;
      add[2] += G2 * uk[i] / M;
    }
    o[i] = v;
  }
  stn<double, N>(gout + n * N, o);
  double *gk = gm + n * 4;
  gk[0] += add[0];
  gk[1] += add[1];
  gk[2] += add[2];
}

// Adjoint of the moment gather (Sec. 4.2): pixel p feeds nodes (px,py) and
// (px+1,py+1) with weight 2/6 and (px+1,py), (px,py+1) with 1/6, through
// m1 (I) and m2 (|I|^2): dL/dI_p = sum_n w_np (dL/dm1_n + 2 I_p dL/dm2_n).
static __global__ void k_adj_image(const double *__restrict__ gm, const double *__restrict__ img, Geo g,
                            double *__restrict__ gimg) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= g.W) return;
  const int64_t n00 = (int64_t)py * g.Wn + px;
  const int64_t nodes[4] = {n00, n00 + 1, n00 + g.Wn, n00 + g.Wn + 1};
  const double wts[4] = {2.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 2.0 / 6.0};
  const double *I = img + ((int64_t)py * g.W + px) * 3;
  double out[3] = {0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double *gk = gm + nodes[q] * 4;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) out[ch] += wts[q] * (gk[ch] + 2.0 * I[ch] * gk[3]);
  }
  double *o = gimg + ((int64_t)py * g.W + px) * 3;
  o[0] = out[0];
  o[1] = out[1];
  o[2] = out[2];
}

// acc[0..1] += tot[0..1] (the lambda and eps gradients of one step).
static __global__ void k_adj_scalars(const double *__restrict__ tot, double *__restrict__ acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    acc[0] += tot[0];
    acc[1] += tot[1];
  }
}

// max_k |v_k| over count values (atomic max of non-negative doubles).
// a13, Krylov acceleration of the adjoint solve (flexible CG with the
// truncated V-cycle as preconditioner).  q = Pi (S p) with the frozen free set
// f (1/0 per phase): the adjoint system's operator Pi S Pi on a tangent p.
template <int N>
__global__ void k_tangent_apply(const double *__restrict__ p, const double *__restrict__ f, Geo g,
                                double *__restrict__ q) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t n = (int64_t)y * g.Wn + x;
  double acc[N], pk[N], fk[N];
  nbr_sum<double, N>(p, g, x, y, acc);
  ldn<double, N>(p + n * N, pk);
  ldn<double, N>(f + n * N, fk);
  const double D = g.D[node_class(g, x, y)], te = g.te;
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = D * pk[i] - te * acc[i];
  proj_box<double, N, kTangent>(acc, fk);
  stn<double, N>(q + n * N, acc);
}

// Block partials of two dot products a0.b0 and a1.b1 over `count` doubles
// (a1 == nullptr: the first only); fixed order for a fixed grid.
static __global__ void __launch_bounds__(kBlock) k_dot2(const double *__restrict__ a0, const double *__restrict__ b0,
                                                        const double *__restrict__ a1, const double *__restrict__ b1,
                                                        int64_t count, double *__restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    acc[0] += a0[k] * b0[k];
    if (a1) acc[1] += a1[k] * b1[k];
  }
  block_sum_store<2>(acc, part + (int64_t)blockIdx.x * 2);
}

// x += alpha p, r -= alpha q.
static __global__ void k_fcg_step(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                  const double *__restrict__ q, double alpha, int64_t count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  x[k] += alpha * p[k];
  r[k] -= alpha * q[k];
}

// p = z + beta p.
static __global__ void k_fcg_dir(double *__restrict__ p, const double *__restrict__ z, double beta, int64_t count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  p[k] = z[k] + beta * p[k];
}

static __global__ void k_absmax(const double *__restrict__ v, int64_t count, double *__restrict__ out) {
  double e = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    e = nanmax<double>(e, fabs(v[k]));
  block_max_atomic(e, out);
}

// ---------------------------------------------------------------------------
// a10: labels and the composite image (Sec. 4.3), on the pixels of the image
// (the solve grid may be the pixel grid refined r times).
// ---------------------------------------------------------------------------
// Pixel integrals (times 6) of u_i on the right-diagonal split, summed over
// the 2^r x 2^r cells of pixel (px, py) of the refined grid (r = 0: the cell
// itself): v_i = sum (2 u00 + u10 + u01 + 2 u11).
template <int N>
__device__ __forceinline__ void pixel_integrals(const double *__restrict__ u, const Geo &g, int r, int px, int py,
                                                double (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = 0.0;
  const int side = 1 << r;
  for (int b = 0; b < side; ++b)
    for (int a = 0; a < side; ++a) {
      const int64_t n = (int64_t)((py << r) + b) * g.Wn + ((px << r) + a);
      double a0[N], b10[N], b01[N], b11[N];
      ldn<double, N>(u + n * N, a0);
      ldn<double, N>(u + (n + 1) * N, b10);
      ldn<double, N>(u + (n + g.Wn) * N, b01);
      ldn<double, N>(u + (n + g.Wn + 1) * N, b11);
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] += 2.0 * a0[i] + b10[i] + b01[i] + 2.0 * b11[i];
    }
}

// argmax with the lowest index on ties.
template <int N>
__device__ __forceinline__ int argmax_low(const double (&v)[N]) {
  int best = 0;
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (v[i] > v[best]) best = i;
  return best;
}

// Composite (Sec. 4.3): per pixel sum_i c_i ubar_i, ubar_i = the pixel mean
// of u_i (pixel_integrals / (6 4^r)); rounded: c of the pixel's label (argmax
// of ubar, lowest index on ties), the rounded composite.  Output
// (H >> r) x (W >> r) x 3 float, pixels of the image.
template <int N>
__global__ void k_composite(const double *__restrict__ u, const double *__restrict__ c, Geo g, int r, int rounded,
                            float *__restrict__ out) {
  const int W0 = g.W >> r, H0 = g.H >> r;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W0 || y >= H0) return;
  double v[N];
  pixel_integrals<N>(u, g, r, x, y, v);
  const int best = argmax_low<N>(v);
  const double scale = 1.0 / (6.0 * (double)(1 << (2 * r)));
  double rgb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double m = v[i] * scale;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) rgb[ch] += c[i * 3 + ch] * m;
  }
  float *o = out + ((int64_t)y * W0 + x) * 3;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) o[ch] = (float)(rounded ? c[best * 3 + ch] : rgb[ch]);
}

// Node label = argmax_i u_n,i (lowest index on ties), on the solve grid.
template <int N>
__global__ void k_labels(const double *__restrict__ u, Geo g, int8_t *__restrict__ node_lab) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t n = (int64_t)y * g.Wn + x;
  double a[N];
  ldn<double, N>(u + n * N, a);
  node_lab[n] = (int8_t)argmax_low<N>(a);
}

// Pixel label = argmax_i of the pixel integral of u_i, (2 u00 + u10 + u01 +
// 2 u11) per cell of the right-diagonal split, summed over the pixel's 4^r
// cells; lowest index on ties.  Output (H >> r) x (W >> r).
template <int N>
__global__ void k_pixel_labels(const double *__restrict__ u, Geo g, int r, int8_t *__restrict__ pix_lab) {
  const int W0 = g.W >> r, H0 = g.H >> r;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W0 || y >= H0) return;
  if (r == 0) {
    // A float filter first (GB300 runs FP64 arithmetic at 1/64 of its FP32
    // rate): the heads of the four corners' u (binary64 significands
    // truncated to 24 bits on the integer pipe, |error| <= 2^-23 for u in
    // [0, 1]) summed in float, |v_f - v| <= 6 2^-23 + 3 2^-22 < 1.5e-6.  When
    // the float argmax leads every other phase by more than 4e-6 (the
    // difference of two floats that close is exact), the binary64 sums have
    // the same unique argmax; otherwise (near-ties, NaN) they decide.
    const int64_t n = (int64_t)y * g.Wn + x;
    const double *p00 = u + n * N, *p10 = u + (n + 1) * N, *p01 = u + (n + g.Wn) * N, *p11 = u + (n + g.Wn + 1) * N;
    double c[N];
    float vf[N];
    ldn<double, N>(p00, c);
#pragma unroll
    for (int i = 0; i < N; ++i) vf[i] = 2.0f * f64_head(c[i]);
    ldn<double, N>(p10, c);
#pragma unroll
    for (int i = 0; i < N; ++i) vf[i] += f64_head(c[i]);
    ldn<double, N>(p01, c);
#pragma unroll
    for (int i = 0; i < N; ++i) vf[i] += f64_head(c[i]);
    ldn<double, N>(p11, c);
#pragma unroll
    for (int i = 0; i < N; ++i) vf[i] += 2.0f * f64_head(c[i]);
    int best = 0;
#pragma unroll
    for (int i = 1; i < N; ++i)
      if (vf[i] > vf[best]) best = i;
    float second = -1.0f;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i != best) second = fmaxf(second, vf[i]);
    if (vf[best] - second > 4e-6f) {
      pix_lab[(int64_t)y * W0 + x] = (int8_t)best;
      return;
    }
  }
  double v[N];
  pixel_integrals<N>(u, g, r, x, y, v);
  pix_lab[(int64_t)y * W0 + x] = (int8_t)argmax_low<N>(v);
}

// A binary64 node array in node order (N values per node) to the colour-split
// float layout of the FP32 solves (fslot), rounded to nearest on the integer
// pipe, and a float one back, widened exactly: the adjoint's FP32
// preconditioner takes the FCG residual and returns its correction this way.
template <int N>
__global__ void k_to_split32(const double *__restrict__ in, Geo g, float *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  double v[N];
  ldn<double, N>(in + ((int64_t)y * g.Wn + x) * N, v);
  float f[N];
#pragma unroll
  for (int i = 0; i < N; ++i) f[i] = f64_to_f32_rn(v[i]);
  stn<float, N>(out + fslot<float>(g, x, y) * N, f);
}

// With freeset != null the widened values are projected onto the frozen
// tangent space in binary64 (proj_box's kTangent form: the mean over the free
// phases removed, the others zeroed): the FP32 solve keeps that space only to
// float precision, and the CG's solution would accumulate the difference.
template <int N>
__global__ void k_from_split32(const float *__restrict__ in, Geo g, const double *__restrict__ freeset,
                               double *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x > g.W) return;
  const int64_t n = (int64_t)y * g.Wn + x;
  float f[N];
  ldn<float, N>(in + fslot<float>(g, x, y) * N, f);
  double v[N];
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = f32_to_f64(f[i]);
  if (freeset) {
    double fr[N];
    ldn<double, N>(freeset + n * N, fr);
    proj_box<double, N, kTangent>(v, fr);
  }
  stn<double, N>(out + n * N, v);
}

// Kernel-level projection of count independent N-vectors onto the simplex.
template <int N>
__global__ void k_project(const double *y, double *x, int64_t count) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  double v[N];
  ldn_rw<double, N>(y + k * N, v);
  proj_simplex<double, N>(v);
  stn<double, N>(x + k * N, v);
}

}  // namespace ac
