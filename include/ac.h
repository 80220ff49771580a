/*
 * ac.h -- C ABI of libac, the GB300 (sm_103a) solver for the time steps of
 * the vector-valued Allen-Cahn colour segmentation of Kay & Tomasi
 * ("Colour Image Segmentation by the Vector-valued Allen-Cahn Phase-field
 * Model: a Multigrid Solution").
 *
 * Problem (Sec. 2.3, Eq. E and Eq. VV_fidelity with the RGB fitting of
 * Sec. 4.4): an N-phase field u on the P1 finite-element space of the pixel
 * grid (nodes at pixel corners, every pixel split along its
 * (x,y)-(x+1,y+1) diagonal, Sec. 3.1), held on the Gibbs simplex at every
 * node (Eq. Gibbs_simplex).  One time step (Sec. 3.2, Eq. alpha; stiffness
 * taken with the sign that makes the step matrix positive definite):
 *     c_i     = int u_i I / int u_i                       (colour means)
 *     b_n,i   = Mhat_n u_n,i (1 + 2 tau/eps) - tau lambda int eta_n |I - c_i|^2
 *     u^{t+1} = argmin over the simplices of sum_i 1/2 u_i'(Mhat + tau eps A) u_i - b_i'u_i
 * solved to a natural residual max_n |u_n - P_G(y_n(u))| <= tol by a
 * truncated monotone multigrid V(nu1,nu2) cycle whose smoother is the
 * projected block Gauss-Seidel of Sec. 3.1 / Sec. 3.3 in red-black order.
 *
 * Layouts.  Image: H x W x 3 (row y, column x, RGB), values in [0, 1].
 * Phase field: (H+1)(W+1) nodes x N phases, node index n = y*(W+1) + x,
 * phase innermost (u[n*N + i]), FP64 at the ABI.  Labels: int8.
 * eps and tau are in pixel units (pixel side 1, Sec. 4.1).
 *
 * Ownership.  The context owns all device memory it allocates (in
 * ac_create).  Caller buffers are only read or written during the call.
 * "is_device" = 1 means the pointer is CUDA device memory of the current
 * device, 0 means host memory.  All work is ordered on params.stream (a
 * cudaStream_t; NULL = the legacy default stream).  Calls that return data
 * to host memory synchronise that stream.
 *
 * Errors.  Every int-returning call returns AC_OK (0) or a negative AC_ERR_*
 * code and never throws; ac_last_error() describes the last failure of the
 * calling thread.  A context that saw AC_ERR_CUDA should be destroyed.
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AC_OK = 0,
  AC_ERR_ARG = -1,           /* invalid argument or size */
  AC_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
  AC_ERR_NOT_CONVERGED = -3, /* a step reached max_cycles with residual > tol (the state is still feasible) */
  AC_ERR_NUMERIC = -4,       /* NaN/Inf found in the residual */
  AC_ERR_STATE = -5,         /* call out of order (e.g. ac_step before ac_set_image) */
  AC_ERR_NOMEM = -6          /* device allocation failed */
};

enum { AC_FP64 = 0, AC_MIXED = 1 };

/* Data projection of the image onto the finite-element space (Sec. 4.2). */
enum {
  AC_PROJ_SIMPLEX = 0, /* "projection by simplex": the exact integrals of the pixelwise-constant image
                          against every hat function, m1_n = <eta_n, I>, m2_n = <eta_n, |I|^2> */
  AC_PROJ_NODE = 1     /* "projection by node": one image value I_n per node and the standard (consistent)
                          mass matrix M_nm = <eta_n, eta_m>, m1 = M I, m2 = M |I|^2.  Nodes sit at pixel
                          corners; node (x, y) takes the value of pixel (min(x, W-1), min(y, H-1)) (the
                          paper's rule for nodes without data: copy a neighbour's value, never interpolate) */
};

#define AC_MAX_PHASES 8

typedef struct ac_ctx ac_ctx;

typedef struct {
  int width, height;   /* image size W x H in pixels (>= 1 each) */
  int n_phases;        /* N, 2 <= N <= AC_MAX_PHASES */
  double eps;          /* interface width epsilon (pixels), > 0 */
  double lambda;       /* fitting weight lambda, >= 0 */
  double tau;          /* time step delta t, > 0 */
  double tol;          /* natural-residual tolerance of each step, > 0 */
  int nu1, nu2;        /* pre/post projected smoothing sweeps of the V-cycle, >= 0, nu1+nu2 >= 1 */
  int max_cycles;      /* V-cycle cap per step, >= 1 */
  int coarse_min;      /* coarsen while both cell counts are even and min/2 >= coarse_min (>= 1) */
  int precision;       /* AC_FP64: every array and operation of the solve in FP64.
                          AC_MIXED: FP64 state u and its update; right-hand side, colour
                          means, energy and residual r = b - S u of the defect correction in
                          double-float arithmetic (about 2^-46 of the terms: GB300 runs FP64
                          at 1/64 of its FP32 rate); the correction delta is solved by the
                          same multigrid in FP32 with obstacle -u (u's significand truncated
                          to 24 bits, so u + delta >= 0) and the natural residual is
                          checked in float on that residual shifted per node by its maximum;
                          the image is rounded to bfloat16 on input (ac_set_image only). */
  uint64_t seed;       /* seed of the random simplex initialisation in ac_set_image */
  int refine;          /* r in [0, 4]: solve on the pixel grid refined r times (Sec. 4.1: at least four
                          nodes across an interface): every pixel becomes 2^r x 2^r cells carrying the pixel's
                          colour (data projection by copy, Sec. 4.2), with eps, tau, lambda still in pixel
                          units.  On cells of side 1 this is the plain step with eps' = 2^r eps,
                          tau' = 2^r tau, lambda' = 2^-r lambda (the system is the pixel-unit one times
                          4^r).  Images come in and pixel labels, composites and image gradients go out at
                          W x H; phase fields, node labels and moments are on the refined grid
                          ((2^r W + 1)(2^r H + 1) nodes); energies are in pixel units. */
  int projection;      /* AC_PROJ_SIMPLEX (default) or AC_PROJ_NODE: how the image enters the fitting terms
                          and the colour means (on the refined grid when refine > 0) */
  void *stream;        /* cudaStream_t for all work of this context */
} ac_params;

typedef struct {
  double energy;       /* discrete Eq. (E) at u^t of the last step, with c = c(u^t) */
  double residual;     /* natural residual at the end of the last step */
  int cycles;          /* V-cycles used by the last step */
  int total_cycles;    /* V-cycles over all steps of the call */
  int steps;           /* time steps done by the call */
  int converged;       /* 1 if every step of the call reached tol */
  int64_t fine_sweeps; /* red-black projected sweeps on the fine level over the call */
  int outer;           /* AC_MIXED: defect-correction passes over the call (0 for AC_FP64) */
} ac_stats;

/* Kernel classes of the profile (no counterpart in the paper: instrumentation). */
enum {
  AC_PROF_SMOOTH = 0,  /* fine red-black projected Gauss-Seidel, one launch per colour */
  AC_PROF_RESID,       /* fine residual, natural residual, mask, tangent projection */
  AC_PROF_COARSE,      /* coarse-level smoothing, residuals and coarsest solve */
  AC_PROF_TRANSFER,    /* truncated Galerkin operators, restriction, prolongation */
  AC_PROF_LINESEARCH,  /* coarse-correction direction, line search, update */
  AC_PROF_SETUP,       /* colour means, energy and right-hand side of a step */
  AC_PROF_OUTER,       /* AC_MIXED: residual and update of the defect correction */
  AC_PROF_COUNT
};

typedef struct {
  double ms[AC_PROF_COUNT];        /* summed device time per class (CUDA events on the context's stream) */
  int64_t launches[AC_PROF_COUNT]; /* kernel launches per class while profiling was on */
  double smooth_bytes_per_launch;  /* algorithmic HBM bytes of one smoother launch (one colour): AC_FP64
                                      1.5 n N 8 (b of the colour, u of the other colour read, u of the
                                      colour written), AC_MIXED 2 n N 4 (r and obstacle of the colour,
                                      delta of the other colour read, delta of the colour written) */
  int64_t total_launches;          /* every kernel launched by this context since creation */
  int64_t smooth_corr_launches;    /* smoother launches that also applied a pending coarse correction
                                      x += omega d: they read d of the other colour as well */
  double smooth_corr_extra_bytes;  /* the extra algorithmic bytes of such a launch: 0.5 n N 8 (AC_FP64),
                                      0.5 n N 4 (AC_MIXED) */
  double bytes[AC_PROF_COUNT];     /* algorithmic HBM bytes of the class's launches while profiling was on:
                                      every array element a launch is defined on read once and written once
                                      (dense counts: rows the coarse kernels skip are still counted) */
} ac_profile;

/* Defaults: tol 1e-10, nu1 = nu2 = 2, max_cycles 200, coarse_min 4, AC_FP64,
 * seed 0, stream NULL; size, N, eps, lambda and tau are left 0. */
int ac_default_params(ac_params *p);

/* Validate p and allocate every device buffer of the solver for a W x H image
 * with N phases: the phase field, right-hand side, image moments and the
 * multigrid hierarchy (levels as described for coarse_min).  *out receives
 * the context.  AC_ERR_ARG for invalid parameters, AC_ERR_NOMEM if device
 * memory runs out. */
int ac_create(ac_ctx **out, const ac_params *p);

/* Copy an RGB image in (H x W x 3 float32, values in [0,1]), compute the
 * per-node image moments of params.projection (Sec. 4.2): by simplex m0 =
 * <eta_n,1>, m1 = <eta_n,I>, m2 = <eta_n,|I|^2> (exact for a
 * pixelwise-constant image); by node m1 = M I, m2 = M |I|^2 with nodal
 * values I_n and the consistent mass matrix M (m0 = <eta_n,1> either way)
 * -- and reset u to a seeded random point of the simplex at every node. */
int ac_set_image(ac_ctx *ctx, const float *rgb, int is_device);
/* The same with an FP64 image (used for parity with the FP64 oracle). */
int ac_set_image_f64(ac_ctx *ctx, const double *rgb, int is_device);

/* Advance n_steps >= 0 time steps (Sec. 3.2).  out (nullable) receives the
 * statistics of the call; the energy it reports is evaluated for the last
 * step only when out is not NULL (about one extra read of u and the
 * moments).  Returns AC_ERR_NOT_CONVERGED if some step hit max_cycles (all
 * steps are still taken), AC_ERR_NUMERIC on NaN/Inf. */
int ac_step(ac_ctx *ctx, int n_steps, ac_stats *out);

/* ac_step(n_steps), then write the rounded composite (Sec. 4.3): the pixel
 * label (H x W int8) is the phase with the largest integral over the pixel,
 * lowest phase index on ties.  Same return codes as ac_step. */
int ac_segment(ac_ctx *ctx, int n_steps, int8_t *pixel_labels, int is_device, ac_stats *out);

/* Free every resource of the context (NULL is accepted). */
void ac_destroy(ac_ctx *ctx);

/* ---- state access (tests, checkpoint/resume, adjoint) ------------------ */

/* Replace u ((H+1)(W+1) x N FP64).  Each node must lie on the simplex; the
 * values are used as given.  The colour means of the previous step (used for
 * phases of zero mass) are reset to 0. */
int ac_set_phase(ac_ctx *ctx, const double *u, int is_device);
/* Copy u out ((H+1)(W+1) x N FP64). */
int ac_get_phase(ac_ctx *ctx, double *u, int is_device);
/* Colour means c (N x 3 FP64, host) used by the last step. */
int ac_get_means(ac_ctx *ctx, double *c);
/* Image moments ((H+1)(W+1) x 5 FP64, host): m0, m1 (RGB), m2. */
int ac_get_moments(ac_ctx *ctx, double *m);
/* Right-hand side b ((H+1)(W+1) x N FP64, host) of the last step.  The
 * mixed form (AC_MIXED) holds b as double-float pairs (about 2^-46 of the
 * terms' magnitudes); their sums are returned. */
int ac_get_rhs(ac_ctx *ctx, double *b);
/* Node labels ((H+1)(W+1) int8): argmax of u_n, lowest index on ties. */
int ac_get_node_labels(ac_ctx *ctx, int8_t *labels, int is_device);
/* Composite image (Sec. 4.3, post-processing): per pixel, sum_i c_i ubar_i
 * with c = c(u) the colour means of the current u and ubar_i the pixel mean
 * of u_i on the right-diagonal split, (2 u(x,y) + u(x+1,y) + u(x,y+1) +
 * 2 u(x+1,y+1)) / 6.  rounded != 0: the rounded composite, c of the pixel's
 * label (argmax of ubar, lowest index on ties; the labels of ac_segment).
 * rgb: H x W x 3 float, row-major, host (is_device = 0) or device memory,
 * written on the context's stream (host: the call returns after the copy).
 * Errors: AC_ERR_ARG (NULL), AC_ERR_STATE (no image), AC_ERR_NOMEM,
 * AC_ERR_CUDA. */
int ac_get_composite(ac_ctx *ctx, float *rgb, int rounded, int is_device);
/* Discrete energy Eq. (E) of the current u with c = c(u) (host double). */
int ac_energy(ac_ctx *ctx, double *energy);
/* Natural residual max_n |u_n - P_G(y_n(u))| of the current u against the
 * right-hand side of the last step (host double). */
int ac_residual(ac_ctx *ctx, double *rho);

/* ---- kernel-level entry point ------------------------------------------ */

/* Euclidean projection of count vectors y (count x N FP64, device) onto the
 * Gibbs simplex (Eq. Gibbs_simplex), the closed form max(y - theta, 0) that
 * the clamp-and-redistribute loop of Sec. 3.3 reaches in <= N passes.  x
 * (device, count x N) may alias y.  Ordered on stream. */
int ac_project_simplex(const double *y, double *x, int64_t count, int n_phases, void *stream);

/* ---- coarse-level tiling (no counterpart in the paper) -------------------- */

/* How the coarse corrections treat their first levels.  Dense: every row of
 * every level is visited, the rows of phases with no free fine node under
 * them (exact zeros) at little cost.  Tiled: the large levels are split into
 * 32 x 16-node tiles per phase; a Galerkin kernel marks the tiles with a
 * nonzero row (live) and lists them, and the level's other kernels work on
 * the listed tiles only (tiles that stay dead hold exact zeros and are not
 * visited).  Both forms compute the same numbers; the tiled one pays when
 * few tiles are live, i.e. once the phases have separated.
 *   AC_TILES_AUTO (default): tiled for levels with at least 32 (tile, phase)
 *     pairs per multiprocessor, chosen per V-cycle when fewer than a quarter
 *     of the fine nodes have a free phase;
 *   AC_TILES_NEVER: dense always;
 *   AC_TILES_ALWAYS: tiled on every coarse level above the coarsest and the
 *     one-launch tail, whatever its size (a check of the tiled kernels). */
enum { AC_TILES_AUTO = 0, AC_TILES_NEVER = 1, AC_TILES_ALWAYS = 2 };
int ac_set_coarse_tiling(ac_ctx *ctx, int mode);

/* ---- the coarse levels' smoother --------------------------------------- */

/* The linear V-cycle on the coarse levels (Sec. 3.2: the coarse corrections
 * of the multigrid) smooths each level twice before and twice after its
 * coarse correction, in one launch per pair of sweeps over 32 x 16-node
 * tiles staged in shared memory.
 *   AC_SMOOTH_GS3 (default): Gauss-Seidel in three colours ((x + y) mod 3
 *     colours the 7-point pattern of the coarse operators), forward then
 *     backward; within a tile each update sees its neighbours' newest values,
 *     across tiles the values at the launch (overlapping blocks);
 *   AC_SMOOTH_JACOBI: l1-Jacobi, x += (r - S x) / sum_m |S_nm|, which
 *     converges for any symmetric positive definite operator.
 * The one-block bottom of the cycle runs the same kind of sweeps, and the
 * coarsest level always takes Gauss-Seidel.  Every coarse correction goes
 * through the feasible direction and the exact line search, so either
 * smoother reaches the same minimiser; at 4096^2, N = 8 (mixed, tol 1e-6)
 * Gauss-Seidel needs 8.65 V-cycles per step over the first 20 steps against
 * 9.6, and 7.2 against 8.8 once the phases have separated.
 * AC_ERR_ARG for a NULL context or an unknown mode. */
enum { AC_SMOOTH_GS3 = 0, AC_SMOOTH_JACOBI = 1 };
int ac_set_coarse_smoother(ac_ctx *ctx, int mode);

/* ---- where the V-cycle loop runs (no counterpart in the paper) ----------- */

/* The cycles of a time step repeat until the natural residual reaches tol
 * (Sec. 3.2); a defect-correction pass (AC_MIXED) repeats until the outer
 * residual does.  Those tests can run on the host, which reads rho back
 * after every cycle, or on the device: the whole time step is then one CUDA
 * graph whose WHILE nodes loop over the cycles and passes, with their
 * conditions set by one-thread kernels from rho, and ac_step synchronises
 * once per call.  Both run the same kernels with the same arguments, so the
 * results are bit-identical.
 *   AC_LOOP_AUTO (default): on the device whenever the context can -- it
 *     has a stream (the legacy default stream cannot be captured), profiling
 *     is off (a profiled cycle brackets its kernels with events, which a
 *     conditional body cannot hold), and no coarse level can run tiled
 *     (ac_set_coarse_tiling; with AC_TILES_AUTO that is every image whose
 *     coarse levels are too small for tiles, e.g. 1024^2 and below at N <= 8)
 *     -- and on the host otherwise;
 *   AC_LOOP_HOST: always on the host.
 * If the graph cannot be captured or instantiated (a driver without
 * conditional nodes), the context switches itself to AC_LOOP_HOST and the
 * step runs on the host loop.  ac_get_cycle_loop sets *on_device to 1 if the
 * next ac_step runs the loop on the device.  AC_ERR_ARG for a NULL context or
 * an unknown mode. */
enum { AC_LOOP_AUTO = 0, AC_LOOP_HOST = 1 };
int ac_set_cycle_loop(ac_ctx *ctx, int mode);
int ac_get_cycle_loop(ac_ctx *ctx, int *on_device);

/* ---- instrumentation (no counterpart in the paper) ------------------------ */

/* Turn per-class kernel timing on (1) or off (0) and clear the accumulated
 * profile.  While on, every kernel group is bracketed by CUDA events on the
 * context's stream. */
int ac_set_profiling(ac_ctx *ctx, int enable);
/* Like ac_set_profiling(ctx, class_mask != 0), but only the classes whose bit
 * (1 << AC_PROF_*) is set are bracketed by events; every class's launches are
 * still counted.  Events cost host time after each V-cycle (a replayed graph's
 * events are read back before it runs again), so a timing run that needs one
 * class can ask for that class alone.  Changing the mask re-captures the
 * context's profiled graphs. */
int ac_set_profiling_mask(ac_ctx *ctx, unsigned class_mask);
/* Synchronise the stream and return the profile accumulated since the last
 * ac_set_profiling call (total_launches counts from creation). */
int ac_get_profile(ac_ctx *ctx, ac_profile *out);

/* ---- adjoint: gradients of a loss on u after T steps (not in the paper) -- */

/* Run n_steps time steps from the current u (as ac_step), keeping u at steps
 * 0, k, 2k, ... (k = checkpoint_every, e.g. sqrt(n_steps)) and the colour
 * means entering them, for ac_adjoint_backward.  Leaves u = u^T. */
int ac_adjoint_forward(ac_ctx *ctx, int n_steps, int checkpoint_every);

/* Gradients of a loss L through the steps of the last ac_adjoint_forward,
 * given grad_u = dL/du^T ((H+1)(W+1) x N FP64, device).  Each step (Sec. 3.2)
 * is differentiated with the active set of u^{t+1} frozen: w solves
 * (Pi S Pi) w = Pi g in the tangent space of u^{t+1} (free phases, sum zero
 * per node), by the same truncated V-cycle (FP64, projection Pi in place of
 * P_G, to 1e-13 max|Pi g|), and dL/db = w, dL/dS = -w u^{t+1}'.  The chain
 * rule through b = Mhat u^t (1 + 2 tau/eps) - tau lambda f(c(u^t)) and the
 * image moments then gives dL/dlambda, dL/deps (tau held fixed) (host
 * doubles), dL/dI (H x W x 3 FP64, device; with respect to the image the
 * moments used, i.e. after the bfloat16 rounding in AC_MIXED) and dL/du^0
 * (device, nullable).  Each segment between checkpoints is recomputed from
 * its checkpoint.  Leaves u = u^T.  AC_ERR_STATE without a forward. */
int ac_adjoint_backward(ac_ctx *ctx, const double *grad_u, double *grad_lambda, double *grad_eps, double *grad_image,
                        double *grad_u0);

/* The adjoint's tangent solve (ac_adjoint_backward) is flexible CG in FP64
 * preconditioned by two truncated V-cycles from zero.  AC_ADJ_PRECOND_F32
 * (default) runs those V-cycles in FP32 on the residual rounded to float (the
 * CG recurrence, residual, stopping test and gradients stay FP64; GB300 runs
 * FP64 at 1/64 of its FP32 rate), AC_ADJ_PRECOND_F64 in FP64.  Takes effect at
 * the next ac_adjoint_forward.  AC_ERR_ARG for a NULL context or another value. */
enum { AC_ADJ_PRECOND_F32 = 0, AC_ADJ_PRECOND_F64 = 1 };
int ac_set_adjoint_preconditioner(ac_ctx *ctx, int precision);

/* Check of the checkpointing (no counterpart in the paper): *count receives
 * the number of components at which a segment recomputed by the last
 * ac_adjoint_backward ended on a state that differs, bit for bit, from the
 * forward's own state there (the next checkpoint, or u^T for the last
 * segment), summed over the segments.  Each segment's first step starts its
 * correction from zero in both passes (AC_MIXED), so the recomputation repeats
 * the forward's arithmetic and the count is 0; a nonzero count means that the
 * backward pass differentiated states other than those the forward visited.
 * 0 before any backward pass.  AC_ERR_ARG for NULL arguments. */
int ac_adjoint_recompute_diff(ac_ctx *ctx, int64_t *count);

/* ---- batches of independent images (no counterpart in the paper) -------- */

/* A batch runs many independent images (uneven sizes and phase counts) at
 * once: one context per image, each with its own CUDA-graph V-cycles, spread
 * over n_streams CUDA streams (longest-processing-time first on
 * (W+1)(H+1)N) and advanced by one host worker thread per stream.  Each
 * image's results are bit-identical to a single-image context with the same
 * parameters and schedule. */
typedef struct ac_batch ac_batch;

typedef struct {
  int images;             /* images in the batch */
  int steps;              /* time steps per image done by the call */
  int converged_images;   /* images whose every step reached tol */
  int64_t total_cycles;   /* V-cycles over all images and steps */
  int64_t fine_sweeps;    /* fine-level red-black sweeps over all images and steps */
  int64_t nodes;          /* sum over images of (W+1)(H+1) */
  int64_t dof;            /* sum over images of N (W+1)(H+1) */
  double dof_sweeps;      /* sum over images of N (W+1)(H+1) x fine sweeps (for GDOF/s) */
} ac_batch_stats;

/* params[k] describes image k; its stream field is ignored.  AC_ERR_ARG if
 * count < 1, n_streams < 1 or any params[k] is invalid. */
int ac_batch_create(ac_batch **out, const ac_params *params, int count, int n_streams);
/* ac_set_image / ac_set_phase / ac_get_phase of image k. */
int ac_batch_set_image(ac_batch *b, int k, const float *rgb, int is_device);
int ac_batch_set_phase(ac_batch *b, int k, const double *u, int is_device);
int ac_batch_get_phase(ac_batch *b, int k, double *u, int is_device);
/* Pixel labels (rounded composite, Sec. 4.3) of image k's current field. */
int ac_batch_segment(ac_batch *b, int k, int8_t *labels, int is_device);
/* Advance every image n_steps time steps (Sec. 3.2).  Returns the first
 * error of any image (AC_ERR_NOT_CONVERGED only if nothing worse happened). */
int ac_batch_step(ac_batch *b, int n_steps, ac_batch_stats *out);
/* Autotuner: per group of images with equal size, N and model parameters,
 * time trial_steps steps of every candidate schedule -- the coarse smoother
 * (AC_SMOOTH_GS3, AC_SMOOTH_JACOBI: the colouring of the coarse sweeps),
 * (nu1, nu2) in {(1,1),(2,1),(1,2),(2,2)} and multigrid depth in {all levels,
 * 5} -- on the group's first image (its state is restored after each trial)
 * and give the whole group the fastest candidate that converged.  chosen
 * (nullable, count x 4 ints) receives nu1, nu2, depth and the coarse smoother
 * per image.  Every image needs its image set first. */
int ac_batch_tune(ac_batch *b, int trial_steps, int *chosen);
/* How ac_batch_step launches the images' work.
 *   AC_BATCH_STREAMS (default): one host worker thread per stream advances
 *     its images one after the other (ac_step on each image's own stream);
 *   AC_BATCH_ONE_GRAPH: one CUDA graph holds a time step of every image --
 *     each image an independent chain with its V-cycle loop on the device
 *     (see ac_set_cycle_loop), whatever the images' own loop setting -- and
 *     is launched once per time step on the first stream, with one
 *     synchronisation per call.  Needs every image able to run its loop on
 *     the device: no coarse level that can run tiled (AC_ERR_STATE from
 *     ac_batch_step otherwise).  The graph is captured on the first
 *     ac_batch_step and again after ac_batch_tune.
 * Both give every image the results of a single-image context, bit for bit.
 * The images of a batch start with AC_LOOP_HOST (ac_batch_set_cycle_loop
 * changes it): in the stream pool the host loop measured faster.
 * AC_ERR_ARG for a NULL batch or an unknown mode. */
enum { AC_BATCH_STREAMS = 0, AC_BATCH_ONE_GRAPH = 1 };
int ac_batch_set_launch(ac_batch *b, int mode);
/* ac_set_cycle_loop on every image of the batch. */
int ac_batch_set_cycle_loop(ac_batch *b, int mode);
/* Free the batch (NULL is accepted). */
void ac_batch_destroy(ac_batch *b);

/* ---- colour means without device allocation (no counterpart in the paper) -- */

/* Colour means c_i = int u_i I / int u_i (N x 3 FP64, device) of a phase field
 * u ((H+1)(W+1) x N FP64, device, the ac_get_phase layout) on an RGB image
 * (H x W x 3 float32, device), for callers that cannot call cudaMalloc (for
 * example real-time pipelines that forbid allocation once running, or code
 * under a framework's fixed device-memory budget).  It allocates nothing: its
 * reduction scratch is a file-scope __device__ array of 132 KiB (512 blocks x
 * 32 partial sums plus 32 totals), held by every GPU that loads the library
 * until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every slot the call reads is written
 * earlier in the same call, so nothing needs clearing, but all calls share
 * the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Ordered on stream.
 * A phase of zero mass gets c_i = 0.  AC_ERR_ARG for NULL pointers, W or H
 * < 1, more than 2^31 nodes, or n_phases outside [2, AC_MAX_PHASES] (the
 * scratch holds 4 sums for at most 8 phases per block). */
int ac_colour_means_static(const double *u, const float *rgb, int width, int height, int n_phases, double *c,
                           void *stream);

/* Description of the last error on the calling thread ("" if none). */
const char *ac_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */
