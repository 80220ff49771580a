/*
 * ac_oracle.c -- plain, slow, sequential FP64 CPU oracle for one time step of
 * the vector-valued Allen-Cahn colour segmentation of Kay & Tomasi
 * ("Colour Image Segmentation by the Vector-valued Allen-Cahn Phase-field
 * Model: a Multigrid Solution").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Conventions (the paper is silent on them; the readings are listed in the
 * design notes of the repository):
 *   - the image is W x H pixels of side h = 1, piecewise constant per pixel
 *     (Sec. 4.1); eps and tau are measured in pixels;
 *   - nodes are pixel corners (x, y), 0 <= x <= W, 0 <= y <= H, index
 *     n = y*(W+1) + x; the phase field is stored u[n*N + i];
 *   - pixel (px, py) is split along its (px,py)-(px+1,py+1) diagonal into
 *     T_lo = {(px,py),(px+1,py),(px+1,py+1)} and T_up = {(px,py),(px,py+1),(px+1,py+1)};
 *   - P1 finite elements on that triangulation (Sec. 3.1), natural boundary
 *     conditions (the weak form holds for all test functions, Sec. 3.1);
 *   - the stiffness sign is +eps*A with A positive semi-definite (the printed
 *     "-eps A" in Eq. (alpha) cannot be: it makes the step matrix indefinite),
 *     and the eps*A*u^k term of Eq. (alpha) carries the time step delta t.
 *
 * Step problem (Sec. 3.2, Eq. (alpha) with the readings above): given u^t on
 * the Gibbs simplex at every node,
 *     c_i   = sum_n u_{n,i} m1_n / sum_n u_{n,i} m0_n            (Eq. VV_fidelity, Sec. 4.4)
 *     f_n,i = integral of eta_n |I - c_i|^2 = m2_n - 2 c_i.m1_n + |c_i|^2 m0_n
 *     S     = Mhat + tau*eps*A
 *     b_n,i = Mhat_n u^t_n,i (1 + 2 tau/eps) - tau*lambda*f_n,i
 *     u^{t+1} = argmin over the product of simplices of sum_i (1/2 u_i'S u_i - b_i'u_i).
 * The tangent projection T of Eq. (projection_operator_T) shifts every
 * phase's right-hand side at a node by the same amount, which cannot change
 * the minimiser on the simplex, so it is not applied.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 16
#define OR_ROW 7 /* a P1 node on this triangulation couples to itself and 6 neighbours */

/* ------------------------------------------------------------------------ */
/* Triangulation and P1 matrices (Sec. 3.1)                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int W, H;
  int64_t n;
  double *mhat;  /* lumped mass <eta_n, 1>, length n */
  int *col;      /* sparse stiffness rows, OR_ROW slots per node */
  double *val;
  int *cnt;
} or_mesh;

static int64_t nid(int W, int x, int y) { return (int64_t)y * (W + 1) + x; }

/* The two triangles of pixel (px, py); vertices as (x, y) pairs. */
static void pixel_triangles(int px, int py, int tri[2][3][2]) {
  int lo[3][2] = {{px, py}, {px + 1, py}, {px + 1, py + 1}};
  int up[3][2] = {{px, py}, {px, py + 1}, {px + 1, py + 1}};
  memcpy(tri[0], lo, sizeof lo);
  memcpy(tri[1], up, sizeof up);
}

static void row_add(or_mesh *m, int64_t r, int c, double v) {
  for (int k = 0; k < m->cnt[r]; ++k)
    if (m->col[r * OR_ROW + k] == c) {
      m->val[r * OR_ROW + k] += v;
      return;
    }
  int k = m->cnt[r]++;
  m->col[r * OR_ROW + k] = c;
  m->val[r * OR_ROW + k] = v;
}

/* Assemble Mhat_n = <eta_n, 1> and A_nm = <grad eta_n, grad eta_m> triangle
 * by triangle: on a triangle of area |T| the barycentric gradients are the
 * rotated opposite edges over 2|T|, and a linear function integrates to
 * |T| times its vertex mean (Sec. 3.1). */
static int mesh_build(or_mesh *m, int W, int H) {
  m->W = W;
  m->H = H;
  m->n = (int64_t)(W + 1) * (H + 1);
  m->mhat = calloc(m->n, sizeof(double));
  m->col = calloc(m->n * OR_ROW, sizeof(int));
  m->val = calloc(m->n * OR_ROW, sizeof(double));
  m->cnt = calloc(m->n, sizeof(int));
  if (!m->mhat || !m->col || !m->val || !m->cnt) return -1;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tri[2][3][2];
      pixel_triangles(px, py, tri);
      for (int t = 0; t < 2; ++t) {
        double x0 = tri[t][0][0], y0 = tri[t][0][1];
        double x1 = tri[t][1][0], y1 = tri[t][1][1];
        double x2 = tri[t][2][0], y2 = tri[t][2][1];
        double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        double area = 0.5 * fabs(det);
        double g[3][2] = {{(y1 - y2) / det, (x2 - x1) / det},
                          {(y2 - y0) / det, (x0 - x2) / det},
                          {(y0 - y1) / det, (x1 - x0) / det}};
        for (int a = 0; a < 3; ++a) {
          int64_t ra = nid(W, tri[t][a][0], tri[t][a][1]);
          m->mhat[ra] += area / 3.0;
          for (int b = 0; b < 3; ++b) {
            int64_t cb = nid(W, tri[t][b][0], tri[t][b][1]);
            row_add(m, ra, (int)cb, area * (g[a][0] * g[b][0] + g[a][1] * g[b][1]));
          }
        }
      }
    }
  return 0;
}

static void mesh_free(or_mesh *m) {
  free(m->mhat);
  free(m->col);
  free(m->val);
  free(m->cnt);
}

/* (S v)_r for one phase, S = Mhat + tau*eps*A, v strided by N. */
static double S_row(const or_mesh *m, double te, int64_t r, const double *v, int N, int i) {
  double s = m->mhat[r] * v[r * N + i];
  for (int k = 0; k < m->cnt[r]; ++k) s += te * m->val[r * OR_ROW + k] * v[(int64_t)m->col[r * OR_ROW + k] * N + i];
  return s;
}

static double S_diag(const or_mesh *m, double te, int64_t r) {
  double d = m->mhat[r];
  for (int k = 0; k < m->cnt[r]; ++k)
    if (m->col[r * OR_ROW + k] == r) d += te * m->val[r * OR_ROW + k];
  return d;
}

/* Export of the assembled matrices, for the tests: mhat (n), and A as rows of
 * OR_ROW (col, val) slots with cnt entries used. */
int or_assemble(int W, int H, double *mhat, int *col, double *val, int *cnt) {
  or_mesh m;
  if (W < 1 || H < 1 || mesh_build(&m, W, H)) return -1;
  memcpy(mhat, m.mhat, m.n * sizeof(double));
  memcpy(col, m.col, m.n * OR_ROW * sizeof(int));
  memcpy(val, m.val, m.n * OR_ROW * sizeof(double));
  memcpy(cnt, m.cnt, m.n * sizeof(int));
  mesh_free(&m);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Data projection by simplex (Sec. 4.2)                                     */
/* ------------------------------------------------------------------------ */

/* Per-node image moments, integrated triangle by triangle with the image
 * constant on each pixel:  m0_n = <eta_n, 1>, m1_n = <eta_n, I> (3 channels),
 * m2_n = <eta_n, |I|^2>.  On a triangle t, <eta_n, 1>_t = |t|/3.
 * Output m[n*5 + {0,1,2,3,4}] = m0, m1r, m1g, m1b, m2. img is H x W x 3. */
int or_moments(int W, int H, const double *img, double *m) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  memset(m, 0, n * 5 * sizeof(double));
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const double *I = img + ((int64_t)py * W + px) * 3;
      double I2 = I[0] * I[0] + I[1] * I[1] + I[2] * I[2];
      int tri[2][3][2];
      pixel_triangles(px, py, tri);
      for (int t = 0; t < 2; ++t)
        for (int a = 0; a < 3; ++a) {
          double *mm = m + nid(W, tri[t][a][0], tri[t][a][1]) * 5;
          double w = 0.5 / 3.0; /* area 1/2 over 3 vertices */
          mm[0] += w;
          mm[1] += w * I[0];
          mm[2] += w * I[1];
          mm[3] += w * I[2];
          mm[4] += w * I2;
        }
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Data projection by node (Sec. 4.2)                                        */
/* ------------------------------------------------------------------------ */

/* Projection by node takes one image value I_n per node and the standard
 * (consistent) mass matrix M_nm = <eta_n, eta_m>: the fitting term of phase i
 * at node n is sum_m M_nm |I_m - c_i|^2 and c_i = (M I . u_i) / (M 1 . u_i),
 * i.e. the moments of the P1 interpolant I_h = sum_m I_m eta_m:
 *     m0_n = sum_m M_nm, m1_n = sum_m M_nm I_m, m2_n = sum_m M_nm |I_m|^2.
 * The nodes sit at pixel corners, where a pixelwise-constant image has no
 * value; following the paper's rule for nodes without data (each takes the
 * value of a neighbour, never an interpolated one), node (x, y) takes the
 * value of pixel (min(x, W-1), min(y, H-1)), the pixel whose lower-left
 * corner it is (the last column and row of nodes take the last pixels). */
static const double *node_value(int W, int H, const double *img, int x, int y) {
  int px = x < W ? x : W - 1, py = y < H ? y : H - 1;
  return img + ((int64_t)py * W + px) * 3;
}

/* M assembled triangle by triangle: on a triangle of area |t| the P1 basis
 * functions give <eta_a, eta_b>_t = |t| (1 + delta_ab) / 12. */
int or_moments_node(int W, int H, const double *img, double *m) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  memset(m, 0, n * 5 * sizeof(double));
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tri[2][3][2];
      pixel_triangles(px, py, tri);
      for (int t = 0; t < 2; ++t)
        for (int a = 0; a < 3; ++a) {
          double *ma = m + nid(W, tri[t][a][0], tri[t][a][1]) * 5;
          for (int b = 0; b < 3; ++b) {
            const double *I = node_value(W, H, img, tri[t][b][0], tri[t][b][1]);
            double w = 0.5 * (a == b ? 2.0 : 1.0) / 12.0;
            ma[0] += w;
            ma[1] += w * I[0];
            ma[2] += w * I[1];
            ma[3] += w * I[2];
            ma[4] += w * (I[0] * I[0] + I[1] * I[1] + I[2] * I[2]);
          }
        }
    }
  return 0;
}

/* The moments of either projection: 0 by simplex, 1 by node. */
static int moments_of(int W, int H, const double *img, int projection, double *m) {
  return projection == 1 ? or_moments_node(W, H, img, m) : or_moments(W, H, img, m);
}

/* ------------------------------------------------------------------------ */
/* Colour means, fitting term, right-hand side, energy (Sec. 2.3, 4.4)       */
/* ------------------------------------------------------------------------ */

/* c_i = int u_i I / int u_i per channel (Eq. VV_fidelity and the
 * multichannel form of Sec. 4.4).  A phase with zero mass keeps c_prev.
 * mass_out (nullable) receives int u_i. */
int or_means(int W, int H, int N, const double *u, const double *m, const double *c_prev, double *c,
             double *mass_out) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  for (int i = 0; i < N; ++i) {
    double mass = 0, s[3] = {0, 0, 0};
    for (int64_t k = 0; k < n; ++k) {
      mass += u[k * N + i] * m[k * 5 + 0];
      for (int ch = 0; ch < 3; ++ch) s[ch] += u[k * N + i] * m[k * 5 + 1 + ch];
    }
    for (int ch = 0; ch < 3; ++ch) c[i * 3 + ch] = (mass == 0.0) ? (c_prev ? c_prev[i * 3 + ch] : 0.0) : s[ch] / mass;
    if (mass_out) mass_out[i] = mass;
  }
  return 0;
}

/* f_n,i = int eta_n |I - c_i|^2 = m2 - 2 c_i.m1 + |c_i|^2 m0 (exact for a
 * piecewise-constant image), and the right-hand side of the step problem
 * b = Mhat u^t (1 + 2 tau/eps) - tau lambda f (Eq. alpha multiplied out). */
int or_rhs(int W, int H, int N, const double *ut, const double *m, const double *c, double eps, double lam,
           double tau, double *b) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  for (int64_t k = 0; k < n; ++k)
    for (int i = 0; i < N; ++i) {
      const double *ci = c + i * 3;
      const double *mk = m + k * 5;
      double cm1 = ci[0] * mk[1] + ci[1] * mk[2] + ci[2] * mk[3];
      double cc = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
      double f = mk[4] - 2.0 * cm1 + cc * mk[0];
      b[k * N + i] = mk[0] * ut[k * N + i] * (1.0 + 2.0 * tau / eps) - tau * lam * f;
    }
  return 0;
}

/* Discrete energy of Eq. (E): sum_i [ eps/2 u_i'A u_i + (1/eps) sum_n Mhat_n u_n,i (1 - u_n,i)
 * + lambda sum_n u_n,i f_n,i(c(u)) ], with c(u) the colour means of u. */
double or_energy(int W, int H, int N, const double *u, const double *m, double eps, double lam) {
  or_mesh mesh;
  if (mesh_build(&mesh, W, H)) return NAN;
  double c[OR_MAXN * 3];
  or_means(W, H, N, u, m, NULL, c, NULL);
  double E = 0;
  for (int i = 0; i < N; ++i) {
    const double *ci = c + i * 3;
    double cc = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
    for (int64_t k = 0; k < mesh.n; ++k) {
      double Au = 0;
      for (int s = 0; s < mesh.cnt[k]; ++s) Au += mesh.val[k * OR_ROW + s] * u[(int64_t)mesh.col[k * OR_ROW + s] * N + i];
      double uk = u[k * N + i];
      const double *mk = m + k * 5;
      double f = mk[4] - 2.0 * (ci[0] * mk[1] + ci[1] * mk[2] + ci[2] * mk[3]) + cc * mk[0];
      E += 0.5 * eps * uk * Au + mesh.mhat[k] * uk * (1.0 - uk) / eps + lam * uk * f;
    }
  }
  mesh_free(&mesh);
  return E;
}

/* ------------------------------------------------------------------------ */
/* Gibbs constraint: clamp and redistribute (Sec. 3.3)                       */
/* ------------------------------------------------------------------------ */

/* Closest point to z in { a : sum_i a_i = total, a_i >= lo_i }, computed by
 * the paper's loop: take the trial that already has the right sum; every
 * component below its bound is raised to the bound, the total raise is taken
 * in equal parts from the k components still free, and the check is repeated
 * on those free components only.  Each pass removes at least one component,
 * so there are at most N passes.  Returns the number of passes. */
static int clamp_redistribute(int N, const double *z, const double *lo, double total, double *a) {
  int free_[OR_MAXN];
  double sz = 0;
  for (int i = 0; i < N; ++i) sz += z[i];
  for (int i = 0; i < N; ++i) {
    a[i] = z[i] - (sz - total) / N;
    free_[i] = 1;
  }
  int k = N, passes = 0;
  for (;;) {
    ++passes;
    double raise = 0;
    int removed = 0;
    for (int i = 0; i < N; ++i)
      if (free_[i] && a[i] < lo[i]) {
        raise += lo[i] - a[i];
        a[i] = lo[i];
        free_[i] = 0;
        ++removed;
      }
    if (!removed) break;
    k -= removed;
    if (k == 0) break;
    for (int i = 0; i < N; ++i)
      if (free_[i]) a[i] -= raise / k;
  }
  return passes;
}

/* Projection onto the Gibbs simplex G^N (Eq. Gibbs_simplex) by the same loop.
 * passes (nullable) receives the pass count. */
int or_project_simplex(int N, const double *y, double *x, int *passes) {
  double lo[OR_MAXN] = {0};
  int p = clamp_redistribute(N, y, lo, 1.0, x);
  if (passes) *passes = p;
  return 0;
}

/* Batched form for the tests: count vectors of length N. */
int or_project_simplex_batch(int N, int64_t count, const double *y, double *x, int *passes) {
  for (int64_t k = 0; k < count; ++k) or_project_simplex(N, y + k * N, x + k * N, passes ? passes + k : NULL);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Nodal problems, natural residual, plain projected Gauss-Seidel (Sec. 3.1) */
/* ------------------------------------------------------------------------ */

/* Unconstrained nodal minimiser with all other nodes frozen:
 * y_n = (b_n - sum_{m != n} S_nm u_m) / S_nn. */
static void nodal_y(const or_mesh *m, double te, int N, int64_t r, const double *u, const double *b, double *y) {
  double d = S_diag(m, te, r);
  for (int i = 0; i < N; ++i) {
    double off = 0;
    for (int k = 0; k < m->cnt[r]; ++k) {
      int64_t c = m->col[r * OR_ROW + k];
      if (c != r) off += te * m->val[r * OR_ROW + k] * u[c * N + i];
    }
    y[i] = (b[r * N + i] - off) / d;
  }
}

/* rho(u) = max_n || u_n - P_G(y_n(u)) ||_inf: zero exactly at the solution of
 * the step problem (the nodal variational inequalities of Eq. E_fe hold). */
static double residual_mesh(const or_mesh *m, double te, int N, const double *u, const double *b) {
  double rho = 0, y[OR_MAXN], p[OR_MAXN];
  for (int64_t r = 0; r < m->n; ++r) {
    nodal_y(m, te, N, r, u, b, y);
    or_project_simplex(N, y, p, NULL);
    for (int i = 0; i < N; ++i) {
      double e = fabs(u[r * N + i] - p[i]);
      if (e > rho) rho = e;
    }
  }
  return rho;
}

double or_natural_residual(int W, int H, int N, const double *u, const double *b, double eps, double tau) {
  or_mesh m;
  if (mesh_build(&m, W, H)) return NAN;
  double rho = residual_mesh(&m, tau * eps, N, u, b);
  mesh_free(&m);
  return rho;
}

/* ------------------------------------------------------------------------ */
/* Successive subspace correction over all multigrid levels (Sec. 3.2)       */
/* ------------------------------------------------------------------------ */

/* Nested triangulations: the pixel grid is coarsened by halving the cell
 * counts while both are even and the smaller one stays >= coarse_min after
 * halving.  Returns the number of levels (1 = fine grid only). */
int or_num_levels(int W, int H, int coarse_min) {
  int L = 1;
  while (W % 2 == 0 && H % 2 == 0 && (W < H ? W : H) / 2 >= coarse_min) {
    W /= 2;
    H /= 2;
    ++L;
  }
  return L;
}

/* The P1 hat function of a node of the uniform right-diagonal mesh, in units
 * of that mesh's spacing: it is 1 at the node, 0 at the six neighbours
 * (E, W, N, S, NE, SW) and linear on each of the six triangles around it. */
static double hat(double s, double t) {
  double a = fabs(s), b = fabs(t), c = fabs(s - t);
  double mx = a > b ? a : b;
  mx = mx > c ? mx : c;
  return mx < 1.0 ? 1.0 - mx : 0.0;
}

/* One subspace correction along the level-k basis function of coarse node
 * (X, Y), written out on the fine grid (Fig. basis_fn: the coarse basis
 * function projected onto the finest grid):
 *   d = eta'S eta, g_i = eta'(b_i - S u_i), and u <- u + eta (x) alpha with
 *   alpha = argmin 1/2 d |alpha|^2 - g.alpha  subject to  sum_i alpha_i = 0
 *   (Sec. 3.3) and u + eta alpha_i >= 0 on every affected node, i.e.
 *   alpha_i >= -min_q u_q,i / eta(q).
 * The minimiser is the clamp-and-redistribute projection of g/d. */
static void ssc_update(const or_mesh *m, double te, int N, int k, int X, int Y, double *u, const double *b,
                       int64_t *sq, double *sw) {
  int W = m->W, H = m->H, s = 1 << k;
  int cx = X * s, cy = Y * s;
  int ns = 0;
  for (int y = cy - s + 1; y <= cy + s - 1; ++y) {
    if (y < 0 || y > H) continue;
    for (int x = cx - s + 1; x <= cx + s - 1; ++x) {
      if (x < 0 || x > W) continue;
      double w = hat((double)(x - cx) / s, (double)(y - cy) / s);
      if (w > 0) {
        sq[ns] = nid(W, x, y);
        sw[ns] = w;
        ++ns;
      }
    }
  }
  /* d = sum_q eta(q) (S eta)(q), with eta evaluated at every matrix column. */
  double d = 0;
  for (int j = 0; j < ns; ++j) {
    int64_t r = sq[j];
    double Seta = m->mhat[r] * sw[j];
    for (int e = 0; e < m->cnt[r]; ++e) {
      int64_t c = m->col[r * OR_ROW + e];
      int xc = (int)(c % (W + 1)), yc = (int)(c / (W + 1));
      Seta += te * m->val[r * OR_ROW + e] * hat((double)(xc - cx) / s, (double)(yc - cy) / s);
    }
    d += sw[j] * Seta;
  }
  double lo[OR_MAXN] = {0}, z[OR_MAXN] = {0}, a[OR_MAXN];
  for (int i = 0; i < N; ++i) {
    double gi = 0, li = INFINITY;
    for (int j = 0; j < ns; ++j) {
      int64_t r = sq[j];
      gi += sw[j] * (b[r * N + i] - S_row(m, te, r, u, N, i));
      double l = u[r * N + i] / sw[j];
      if (l < li) li = l;
    }
    lo[i] = -li;
    z[i] = gi / d;
  }
  clamp_redistribute(N, z, lo, 0.0, a);
  for (int j = 0; j < ns; ++j)
    for (int i = 0; i < N; ++i) u[sq[j] * N + i] += sw[j] * a[i];
}

/* One lexicographic pass over the basis functions of level k.  On the finest
 * level (k = 0) a basis function is a single node, and the correction along
 * it equals u_n <- P_G(y_n) in exact arithmetic; it is computed in that nodal
 * form so that rounding cannot let sum_i u_n,i drift away from 1 (updates
 * with sum_i alpha_i = 0 only preserve whatever sum the node already has). */
static void ssc_level_pass(const or_mesh *m, double te, int N, int k, double *u, const double *b, int64_t *sq,
                           double *sw) {
  int Wk = m->W >> k, Hk = m->H >> k;
  double y[OR_MAXN];
  for (int Y = 0; Y <= Hk; ++Y)
    for (int X = 0; X <= Wk; ++X) {
      if (k == 0) {
        int64_t r = nid(m->W, X, Y);
        nodal_y(m, te, N, r, u, b, y);
        or_project_simplex(N, y, u + r * N, NULL);
      } else {
        ssc_update(m, te, N, k, X, Y, u, b, sq, sw);
      }
    }
}

/* Solve the step problem by SSC iterations.  One iteration visits the levels
 * in V(nu1, nu2) order: fine to coarse with nu1 lexicographic passes per
 * level, then back up with nu2 passes (the level order does not change the
 * fixed point).  Stops when rho(u) <= tol or after max_iter iterations.
 * Returns 0 on convergence, 1 if max_iter was reached. */
int or_ssc_solve(int W, int H, int N, double *u, const double *b, double eps, double tau, double tol, int max_iter,
                 int nu1, int nu2, int coarse_min, int *iters, double *rho_out) {
  or_mesh m;
  if (N < 2 || N > OR_MAXN || mesh_build(&m, W, H)) return -1;
  double te = tau * eps;
  int L = or_num_levels(W, H, coarse_min);
  int smax = 1 << (L - 1);
  int64_t cap = (int64_t)(2 * smax + 1) * (2 * smax + 1);
  int64_t *sq = malloc(cap * sizeof(int64_t));
  double *sw = malloc(cap * sizeof(double));
  int it = 0, status = 1;
  double rho = residual_mesh(&m, te, N, u, b);
  while (rho > tol && it < max_iter) {
    for (int k = 0; k < L; ++k)
      for (int p = 0; p < nu1; ++p) ssc_level_pass(&m, te, N, k, u, b, sq, sw);
    for (int k = L - 2; k >= 0; --k)
      for (int p = 0; p < nu2; ++p) ssc_level_pass(&m, te, N, k, u, b, sq, sw);
    ++it;
    rho = residual_mesh(&m, te, N, u, b);
  }
  if (rho <= tol) status = 0;
  if (iters) *iters = it;
  if (rho_out) *rho_out = rho;
  free(sq);
  free(sw);
  mesh_free(&m);
  return status;
}

/* Plain projected Gauss-Seidel on the fine level only, lexicographic node
 * order: u_n <- P_G(y_n(u)) (Sec. 3.1: the nodal sub-problems solved one
 * after another).  Same stopping rule as or_ssc_solve. */
int or_pgs_solve(int W, int H, int N, double *u, const double *b, double eps, double tau, double tol, int max_sweeps,
                 int *sweeps, double *rho_out) {
  or_mesh m;
  if (N < 2 || N > OR_MAXN || mesh_build(&m, W, H)) return -1;
  double te = tau * eps, y[OR_MAXN];
  int it = 0;
  double rho = residual_mesh(&m, te, N, u, b);
  while (rho > tol && it < max_sweeps) {
    for (int64_t r = 0; r < m.n; ++r) {
      nodal_y(&m, te, N, r, u, b, y);
      or_project_simplex(N, y, u + r * N, NULL);
    }
    ++it;
    rho = residual_mesh(&m, te, N, u, b);
  }
  if (sweeps) *sweeps = it;
  if (rho_out) *rho_out = rho;
  mesh_free(&m);
  return rho <= tol ? 0 : 1;
}

/* One time step (Sec. 3.2): c^t and b from u^t, then solve for u^{t+1}.
 * method 0 = SSC over all levels, 1 = plain projected Gauss-Seidel.
 * c (N x 3) holds the previous means on entry (used for phases of zero mass)
 * and the means c^t of u^t on exit. */
int or_step(int W, int H, int N, double *u, const double *m, double *c, double eps, double lam, double tau, double tol,
            int method, int max_iter, int nu1, int nu2, int coarse_min, int *iters, double *rho_out) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  double cprev[OR_MAXN * 3];
  if (N < 2 || N > OR_MAXN) return -1;
  memcpy(cprev, c, N * 3 * sizeof(double));
  or_means(W, H, N, u, m, cprev, c, NULL);
  double *b = malloc(n * N * sizeof(double));
  if (!b) return -1;
  or_rhs(W, H, N, u, m, c, eps, lam, tau, b);
  int st = method == 0 ? or_ssc_solve(W, H, N, u, b, eps, tau, tol, max_iter, nu1, nu2, coarse_min, iters, rho_out)
                       : or_pgs_solve(W, H, N, u, b, eps, tau, tol, max_iter, iters, rho_out);
  free(b);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Rounded composite (Sec. 4.3)                                              */
/* ------------------------------------------------------------------------ */

/* Node labels: the phase with the largest value (lowest index on ties).
 * Pixel labels: the phase with the largest pixel integral; over the two
 * triangles of a pixel that integral is (2 u00 + u10 + u01 + 2 u11)/6, and
 * the comparison uses 2 u00 + u10 + u01 + 2 u11 summed in that order. */
int or_labels(int W, int H, int N, const double *u, int8_t *node_lab, int8_t *pix_lab) {
  int64_t n = (int64_t)(W + 1) * (H + 1);
  if (node_lab)
    for (int64_t k = 0; k < n; ++k) {
      int best = 0;
      for (int i = 1; i < N; ++i)
        if (u[k * N + i] > u[k * N + best]) best = i;
      node_lab[k] = (int8_t)best;
    }
  if (pix_lab)
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        const double *u00 = u + nid(W, px, py) * N, *u10 = u + nid(W, px + 1, py) * N;
        const double *u01 = u + nid(W, px, py + 1) * N, *u11 = u + nid(W, px + 1, py + 1) * N;
        int best = 0;
        double bv = 0;
        for (int i = 0; i < N; ++i) {
          double v = 2.0 * u00[i] + u10[i] + u01[i] + 2.0 * u11[i];
          if (i == 0 || v > bv) {
            bv = v;
            best = i;
          }
        }
        pix_lab[(int64_t)py * W + px] = (int8_t)best;
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of T time steps (gradients of a loss on u^T)                      */
/* ------------------------------------------------------------------------ */

/* The step map u^t -> u^{t+1} of Sec. 3.2 is differentiated with the active
 * set of u^{t+1} frozen.  At the minimiser the free phases of a node n (those
 * with u > 0, when there are at least two) satisfy (S u - b)_n,i = mu_n, the
 * other phases are 0, so du lies in the tangent space V (free phases only,
 * sum zero per node) and solves  Pi S du = Pi (db - dS u), Pi the orthogonal
 * projection onto V.  Hence for a loss L with g = dL/du^{t+1}:
 *     w = (Pi S Pi)^+ Pi g   (w in V),   dL/db = w,   dL/dS = -w u'.
 * b = Mhat u^t (1 + 2 tau/eps) - tau lambda f(c), f_i = m2 - 2 c_i.m1 + |c_i|^2 m0,
 * c_i = s_i / M_i (s_i = sum u_i m1, M_i = sum u_i m0) and S = Mhat + tau eps A
 * (tau held fixed) give the chain rule below. */

/* v -> Pi v over the free set of u (free: u > 0 at nodes with >= 2 such). */
static void tangent_project(int64_t n, int N, const double *u, const double *v, double *out) {
  for (int64_t k = 0; k < n; ++k) {
    int cnt = 0;
    double s = 0;
    for (int i = 0; i < N; ++i)
      if (u[k * N + i] > 0) {
        ++cnt;
        s += v[k * N + i];
      }
    for (int i = 0; i < N; ++i)
      out[k * N + i] = (cnt >= 2 && u[k * N + i] > 0) ? v[k * N + i] - s / cnt : 0.0;
  }
}

static double dotv(int64_t m, const double *a, const double *b) {
  double s = 0;
  for (int64_t k = 0; k < m; ++k) s += a[k] * b[k];
  return s;
}

/* Conjugate gradients for (Pi S Pi) w = Pi g in V, from w = 0, until the
 * residual norm is below rtol times that of Pi g, or p'q <= 0: in exact
 * arithmetic that means p = 0 (converged); in floating point it is CG past
 * its rounding floor, where conjugacy is lost and further steps can grow the
 * iterate without bound. */
static int tangent_cg(const or_mesh *m, double te, int N, const double *up, const double *g, double *w, double rtol) {
  int64_t nn = m->n * N;
  double *r = calloc(nn, sizeof(double)), *p = calloc(nn, sizeof(double)), *q = calloc(nn, sizeof(double)),
         *t = calloc(nn, sizeof(double));
  if (!r || !p || !q || !t) return -1;
  tangent_project(m->n, N, up, g, r);
  memset(w, 0, nn * sizeof(double));
  memcpy(p, r, nn * sizeof(double));
  double rr = dotv(nn, r, r), r0 = sqrt(rr);
  int it = 0;
  while (sqrt(rr) > rtol * r0 && rr > 0 && it < 20 * nn) {
    for (int64_t k = 0; k < m->n; ++k)
      for (int i = 0; i < N; ++i) t[k * N + i] = S_row(m, te, k, p, N, i);
    tangent_project(m->n, N, up, t, q);
    const double pq = dotv(nn, p, q);
    if (!(pq > 0)) break;
    double a = rr / pq;
    for (int64_t k = 0; k < nn; ++k) {
      w[k] += a * p[k];
      r[k] -= a * q[k];
    }
    double rr2 = dotv(nn, r, r);
    for (int64_t k = 0; k < nn; ++k) p[k] = r[k] + (rr2 / rr) * p[k];
    rr = rr2;
    ++it;
  }
  free(r);
  free(p);
  free(q);
  free(t);
  return it;
}

/* states: (T+1) x n x N forward states u^0..u^T produced by or_step with the
 * same parameters; gT = dL/du^T.  Outputs dL/dlambda, dL/deps (tau fixed),
 * dL/dI (H x W x 3) and dL/du^0 (n x N, nullable). */
int or_adjoint(int W, int H, int N, const double *img, const double *states, int T, double eps, double lam, double tau,
               const double *gT, double *g_lam, double *g_eps, double *g_img, double *g_u0, double cg_rtol,
               int projection) {
  or_mesh mesh;
  if (N < 2 || N > OR_MAXN || T < 0 || mesh_build(&mesh, W, H)) return -1;
  const int64_t n = mesh.n, nn = n * N;
  const double te = tau * eps, a1 = 1.0 + 2.0 * tau / eps;
  double *m = malloc(n * 5 * sizeof(double)), *c = malloc((size_t)(T + 1) * N * 3 * sizeof(double));
  double *g = malloc(nn * sizeof(double)), *gn = malloc(nn * sizeof(double)), *w = malloc(nn * sizeof(double));
  double *gm = calloc(n * 4, sizeof(double)); /* dL/dm1 (3), dL/dm2 */
  if (!m || !c || !g || !gn || !w || !gm) return -1;
  moments_of(W, H, img, projection, m);
  /* the means the forward used at each step (empty phases keep the previous) */
  double cprev[OR_MAXN * 3] = {0};
  for (int t = 0; t < T; ++t) {
    or_means(W, H, N, states + (int64_t)t * nn, m, cprev, c + (int64_t)t * N * 3, NULL);
    memcpy(cprev, c + (int64_t)t * N * 3, N * 3 * sizeof(double));
  }
  memcpy(g, gT, nn * sizeof(double));
  double glam = 0, geps = 0;
  for (int t = T - 1; t >= 0; --t) {
    const double *u = states + (int64_t)t * nn, *up = states + (int64_t)(t + 1) * nn, *ct = c + (int64_t)t * N * 3;
    if (tangent_cg(&mesh, te, N, up, g, w, cg_rtol) < 0) return -1;
    double G[OR_MAXN][3] = {{0}}, M[OR_MAXN] = {0};
    for (int i = 0; i < N; ++i)
      for (int64_t k = 0; k < n; ++k) M[i] += u[k * N + i] * m[k * 5];
    for (int64_t k = 0; k < n; ++k) {
      const double *mk = m + k * 5;
      for (int i = 0; i < N; ++i) {
        const double *ci = ct + i * 3;
        const double wk = w[k * N + i];
        double f = mk[4] - 2.0 * (ci[0] * mk[1] + ci[1] * mk[2] + ci[2] * mk[3]) +
                   (ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2]) * mk[0];
        glam += wk * (-tau * f);
        geps += wk * mk[0] * u[k * N + i] * (-2.0 * tau / (eps * eps));
        geps += -tau * wk * (S_row(&mesh, te, k, up, N, i) - mesh.mhat[k] * up[k * N + i]) / te;
        for (int ch = 0; ch < 3; ++ch) G[i][ch] += 2.0 * tau * lam * wk * (mk[1 + ch] - ci[ch] * mk[0]);
        gm[k * 4 + 3] += -tau * lam * wk;
        for (int ch = 0; ch < 3; ++ch) gm[k * 4 + ch] += 2.0 * tau * lam * wk * ci[ch];
      }
    }
    for (int64_t k = 0; k < n; ++k) {
      const double *mk = m + k * 5;
      for (int i = 0; i < N; ++i) {
        const double *ci = ct + i * 3;
        double v = mk[0] * a1 * w[k * N + i];
        if (M[i] != 0.0)
          for (int ch = 0; ch < 3; ++ch) {
            v += G[i][ch] * (mk[1 + ch] - ci[ch] * mk[0]) / M[i];
            gm[k * 4 + ch] += G[i][ch] * u[k * N + i] / M[i];
          }
        gn[k * N + i] = v;
      }
    }
    memcpy(g, gn, nn * sizeof(double));
  }
  /* adjoint of the triangle-by-triangle moment assembly (Sec. 4.2) */
  memset(g_img, 0, (size_t)W * H * 3 * sizeof(double));
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tri[2][3][2];
      pixel_triangles(px, py, tri);
      for (int tt = 0; tt < 2; ++tt)
        for (int a = 0; a < 3; ++a) {
          const double *gk = gm + nid(W, tri[tt][a][0], tri[tt][a][1]) * 4;
          if (projection == 1) {
            /* m_a gathers w_ab (I_b, |I_b|^2) from the triangle's nodes b,
             * each carrying the value of the pixel it copies */
            for (int b = 0; b < 3; ++b) {
              int bx = tri[tt][b][0], by = tri[tt][b][1];
              int sx = bx < W ? bx : W - 1, sy = by < H ? by : H - 1;
              const double *I = img + ((int64_t)sy * W + sx) * 3;
              double *gI = g_img + ((int64_t)sy * W + sx) * 3;
              double w = 0.5 * (a == b ? 2.0 : 1.0) / 12.0;
              for (int ch = 0; ch < 3; ++ch) gI[ch] += w * (gk[ch] + 2.0 * I[ch] * gk[3]);
            }
          } else {
            const double *I = img + ((int64_t)py * W + px) * 3;
            double *gI = g_img + ((int64_t)py * W + px) * 3;
            for (int ch = 0; ch < 3; ++ch) gI[ch] += (0.5 / 3.0) * (gk[ch] + 2.0 * I[ch] * gk[3]);
          }
        }
    }
  *g_lam = glam;
  *g_eps = geps;
  if (g_u0) memcpy(g_u0, g, nn * sizeof(double));
  free(m);
  free(c);
  free(g);
  free(gn);
  free(w);
  free(gm);
  mesh_free(&mesh);
  return 0;
}
