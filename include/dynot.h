/*
 * dynot.h -- C ABI of the GB300 dynamic optimal-transport solver.
 *
 * The library solves the discrete dynamic optimal-transport problem of
 * Fitschen, Laus & Steidl, "Dynamic Optimal Transport with Mixed Boundary
 * Conditions for Color Image Processing" (arXiv 1501.04840):
 *
 *   minimise ||J(u, v)||_1  s.t.  S_M m = u,  S_F f + f_b^+ = v,
 *                                (D_M | D_F)(m, f) = f_b^-          (section 2)
 *
 * with the primal-dual iteration of Algorithm 1 (section 3), on a staggered grid
 * of one to three spatial axes (x, y, colour) with Neumann or periodic boundary
 * conditions per axis and P time intervals:
 *   - RGB images: n = {n1, n2, 3}, bc = {NEUMANN, NEUMANN, PERIODIC} (section 1,
 *     Remark 2: the 4D Poisson problem with periodic colour);
 *   - hue histograms: ndim = 1, n = {bins}, bc = {PERIODIC} (section 5);
 *   - grey images / 1D signals: ndim = 2 or 1 with Neumann axes (section 1);
 *   - any axis of a 2- or 3-axis grid may be periodic (kappa = 0 in section 2):
 *     periodic x and y axes use the real Fourier basis instead of the DCT.
 *
 * Array conventions (all float32, C order, slowest index first):
 *   densities f0, f1 : [c][y][x]               (S = n1*n2*C values per problem)
 *   path f           : [t][c][y][x], t = 1..P-1 (f at time t/P; section 2)
 *   path m_k         : [t][c][y][x] with axis k holding n_k - kappa_k faces,
 *                      t = 1..P (half-times (t-1/2)/P).  Face index i along
 *                      axis k is the paper's face j = i + kappa_k at position
 *                      j/n_k: for Neumann axes (kappa = 1) the face right of
 *                      cell i, for periodic axes (kappa = 0) the face left of
 *                      cell i (section 2, "Discretization").
 *   packed path      : m_0 | m_1 | ... | m_{d-1} | f   (the vector (m, f)).
 *   packed dual      : b_m0 | ... | b_m{d-1} | b_f, each P*S cells [t][c][y][x].
 * A batch of B problems of one size is stored problem after problem.
 *
 * Pointers: every array argument may be host or device memory (unified virtual
 * addressing; copies use cudaMemcpyDefault).  The caller owns its buffers; the
 * plan owns its device workspace.  All work is ordered on the plan's stream;
 * every call returns after its results are in the caller's buffers.
 *
 * Errors: every entry point returns an ot_status; ot_last_error() gives a
 * thread-local message for the last failure on the calling thread.  No C++
 * exception crosses this interface: a failed host allocation inside a call
 * returns OT_ENOMEM, any other internal exception OT_ECUDA.
 */
#ifndef DYNOT_H
#define DYNOT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OT_ABI_VERSION 2

typedef struct ot_plan_s* ot_plan_t;

typedef enum {
  OT_OK = 0,
  OT_EINVAL = 1,       /* bad argument or unsupported grid */
  OT_EMASS = 2,        /* negative / non-finite density or ||f0||_1 != ||f1||_1 */
  OT_ENOMEM = 3,       /* device or host allocation failed */
  OT_ECUDA = 4,        /* a CUDA call failed (message in ot_last_error) */
  OT_ETIMEOUT = 5,     /* reserved: a device wait exceeded its limit */
  OT_ENUMERIC = 6,     /* NaN or Inf in a residual */
  OT_ENOTCONV = 7,     /* iteration budget spent before the tolerance; results valid */
  OT_EUNSUPPORTED = 8  /* grid shape outside what the kernels implement */
} ot_status;

typedef enum { OT_BC_PERIODIC = 0, OT_BC_NEUMANN = 1 } ot_bc; /* kappa of section 2 */

typedef enum {
  OT_PREC_MIXED = 0, /* FP32 stencils/transforms/prox; FP64 low-mode divide and reductions */
  OT_PREC_FP32 = 1,  /* as MIXED but every eigenvalue divide in FP32 */
  OT_PREC_FP64 = 2   /* every kernel in FP64 */
} ot_precision;

typedef struct {
  int ndim;              /* spatial axes: 1 (hue / 1D), 2 (grey), 3 (x, y, colour) */
  int n[3];              /* cells per axis; unused axes are ignored */
  int bc[3];             /* ot_bc per axis */
  int P;                 /* time intervals p (2..64) */
  double sigma;          /* step 2 parameter; 0 selects the default 0.3 */
  double tau;            /* step 1 parameter, tau*sigma < 1 (Algorithm 1); 0 => 0.99/sigma */
  double axis_scale[3];  /* factor of D_n per axis; 0 => n[k] (the unit cube, eq. (cont_model)) */
  int precision;         /* ot_precision */
  int check_every;       /* iterations between residual checks in ot_solve (0 => 10) */
  double lam_fp64;       /* MIXED: eigenvalues below this are divided in FP64 (0 => 64) */
} ot_grid;

typedef struct {
  int iterations;        /* iterations performed */
  double residual;       /* ||b^{r+1} - b^r|| / ||K x^{r+1} + (0, f_b^+)|| at the last check */
  double energy;         /* (1/#cells) sum J(u, v) in the caller's density units */
  double mass_drift;     /* max_t |sum_x f(t) - M| / M over the interior times */
  double elapsed_ms;     /* device time of the call (CUDA events) */
  double dual_value;     /* dual objective at p = sigma b of the last check, caller units (see below) */
  double gap;            /* primal-dual gap |energy - dual_value| / max(|energy|, |dual_value|) */
} ot_solve_stats;
/*
 * The dual value (no counterpart in the paper; a convergence measure beside
 * the residual): the problem's Lagrangian dual function at p = sigma b,
 *   D = sigma (<b_m, S_M m0> + <b_f, S_F f0 + f_b^+>) / #cells,
 * where (m0, f0) = Pi_{C_d}(0) is the least-norm path that meets the continuity
 * constraint.  Step 2 keeps sigma b in the subdifferential of J (so J*(p) = 0)
 * and D takes the infimum of <K^T p, x> over C_d at x0, which is exact once
 * K^T p lies in the range of A^T.  At a saddle point D equals the energy, so
 * the gap tends to zero with the iteration.  Residual, energy and dual sums
 * are formed from per-thread compensated sums in the working precision and
 * summed across threads in FP64.
 */

/* Fill *g with the defaults for an RGB grid n1 x n2 x 3 with P time intervals. */
void ot_grid_rgb(ot_grid* g, int n1, int n2, int P);
/* Fill *g with the defaults for a periodic hue histogram of `bins` bins. */
void ot_grid_hue(ot_grid* g, int bins, int P);

/*
 * Create a plan for `batch` problems of the shape *g, ordered on `cuda_stream`
 * (a cudaStream_t; NULL => the plan creates its own stream).  Allocates the
 * device workspace on the current device.  Returns OT_EINVAL / OT_EUNSUPPORTED
 * for grids the kernels do not cover, OT_ENOMEM when allocation fails.  The
 * kernels cover 2 <= P <= 64, axes of at most 4096 cells (hue: 8192 bins), a
 * colour axis of at most 4, fewer than 2^31 cells P n1 n2 C per problem and
 * batch * P <= 65535.
 */
ot_status ot_plan(const ot_grid* g, int batch, void* cuda_stream, ot_plan_t* out);

/* Release the plan and its device memory.  NULL is ignored. */
void ot_destroy(ot_plan_t p);

/*
 * Solve Algorithm 1 for the pairs (f0, f1) (batch x S values each).
 * Validates f >= 0, finite, and | ||f0||_1 - ||f1||_1 | <= 1e-6 max(...) per pair
 * (section 2 requires equal masses; section 4 rescales images to reach it),
 * otherwise returns OT_EMASS.  Internally every pair is rescaled to mean
 * density 1 and the path is scaled back by the mean of the two masses over S.
 * Starts from x = 0, b = bbar = 0 (Algorithm 1) or, if init_path != NULL, from
 * x = init_path (packed path in the caller's units) with b = bbar = 0.
 * Runs until the residual of the last check is <= tol or `iters` iterations
 * are done (OT_ENOTCONV with valid results in the latter case when tol > 0).
 * `g` may be NULL (use the plan's grid) or must match the plan's sizes; its
 * sigma, tau and check_every then apply to this call.  stats may be NULL.
 */
ot_status ot_solve(ot_plan_t p, const float* f0, const float* f1, const ot_grid* g, int iters, double tol,
                   const float* init_path, ot_solve_stats* stats);

/*
 * ot_solve from a warm start x0 = init_path (required; packed path in the
 * caller's units, host or device).  The first step of Algorithm 1 projects
 * x0 - tau sigma K^T bbar0 onto the continuity constraint, so x0 need not
 * satisfy it.  The dual starts from
 *   - init_dual != NULL: b = bbar = init_dual (the packed dual layout of
 *     ot_state_get; the dual is a velocity and has no density units);
 *   - otherwise dual_init = 0: b = bbar = 0 (as ot_solve does);
 *   - otherwise dual_init = 1: the dual of a fixed point of step 2 for x0,
 *     b = bbar = grad J(y) / sigma at y = K x0 + (0, f_b^+), where
 *     grad J(u, v) = (w, -|w|^2 / 2) with the velocity w = u / v (J of
 *     section 2; v is clamped below at 1e-3 of the mean density and |w| above
 *     at the domain's diameter, which no optimal path exceeds), in cells whose
 *     density (in units of the mean density) is at least dual_support, and
 *     b = 0 in the others, where an optimal path does not determine its dual.
 * fallback_residual > 0: when the residual at the first check exceeds it, the
 * call restarts from the cold start of Algorithm 1 and sets *used_cold = 1
 * (used_cold may be NULL); the iterations already spent count towards `iters`
 * and stats->iterations.  The paper has no warm start; this serves learned or
 * reused initial paths.
 */
ot_status ot_solve_warm(ot_plan_t p, const float* f0, const float* f1, const ot_grid* g, int iters, double tol,
                        const float* init_path, const float* init_dual, int dual_init, double dual_support,
                        double fallback_residual, ot_solve_stats* stats, int* used_cold);

/*
 * Copy the primal path x of the last iteration into caller buffers (any of
 * them may be NULL): f, and m along axes 0, 1, 2 (in the layout above, caller
 * units).  For ndim < 3 the unused m pointers are ignored.
 */
ot_status ot_path(ot_plan_t p, float* f, float* m0, float* m1, float* m2);

/* Number of floats of the packed path and packed dual per batch (all problems). */
size_t ot_path_size(ot_plan_t p);
size_t ot_dual_size(ot_plan_t p);

/*
 * Checkpoint / resume of the iteration state (x, b, bbar) of Algorithm 1 in
 * solver units, with the boundary densities f0, f1 used as given (no mass
 * rescaling).  bbar may be NULL on set (=> bbar = b).
 */
ot_status ot_state_set(ot_plan_t p, const float* f0, const float* f1, const float* x_packed,
                       const float* b_packed, const float* bbar_packed);
ot_status ot_state_get(ot_plan_t p, float* x_packed, float* b_packed, float* bbar_packed);

/* Run `iters` iterations of Algorithm 1 from the current state; stats may be NULL. */
ot_status ot_iterate(ot_plan_t p, int iters, ot_solve_stats* stats);

/*
 * Step 1 of Algorithm 1 alone: x = Pi_{C_d}(a) = a - A^T (A A^T)^+ (A a - f_b^-)
 * (section 3), for a packed path a and boundary densities f0, f1 used as given.
 * phi (P*S per problem, NULL allowed) receives (A A^T)^+ (A a - f_b^-).
 */
ot_status ot_project(ot_plan_t p, const float* f0, const float* f1, const float* a_packed, float* x_packed,
                     float* phi);

/*
 * Step 2 of Algorithm 1 alone: for each of `count` cells,
 *   (u, v) = argmin |u|^2/(2v) + sigma/2 |u - a_m|^2 + sigma/2 (v - a_f)^2
 * (section 3).  a_m holds ncomp (1..3) components of `count` values each
 * (component-major), u likewise; FP32 on the device.
 */
ot_status ot_prox(int count, int ncomp, double sigma, const float* a_m, const float* a_f, float* u, float* v);

/*
 * The same map with the cubic's root in closed form (Cardano's formula, which
 * section 3 names as the alternative to Newton's method) instead of Newton
 * iterations; for comparing the two in FP32.  Same arguments as ot_prox.
 */
ot_status ot_prox_cardano(int count, int ncomp, double sigma, const float* a_m, const float* a_f, float* u,
                          float* v);

/*
 * Measurement: run `iters` iterations with CUDA events around every kernel and
 * return the mean device time per launch in ms: ms[0..3] = the four kernels of
 * an iteration (rhs + forward x/t transform, y/colour solve, inverse x/t
 * transform, update), ms[4] = one whole iteration replayed from a CUDA graph.
 * The state advances.  `names` (may be NULL) receives a static string naming
 * the kernels.
 */
ot_status ot_profile(ot_plan_t p, int iters, double ms[5], const char** names);

/*
 * ot_project for hue histograms without any device allocation (the paper has
 * no counterpart; this serves callers that cannot call cudaMalloc, such as
 * hosts that reserve all device memory up front or forbid allocation after
 * start-up).  Computes, for `batch` problems of `bins` periodic bins and P
 * time intervals, x = a - A^T (A A^T)^+ (A a - f_b^-) and phi = (A A^T)^+ (A a - f_b^-),
 * the operator of a hue plan's ot_project (results within 1e-5 of it; eigenvalues
 * below 64 divided in double as the plan does), with axis_scale == 0 meaning `bins`
 * (a negative, infinite or NaN axis_scale returns OT_EINVAL).
 * All pointers are DEVICE memory: f0, f1 [batch][bins]; a_packed, x_packed
 * [batch][packed path]; phi [batch][P][bins].  The work is queued on cuda_stream
 * (NULL = legacy default stream) and the call returns without waiting for it:
 * order later work and reads of x_packed and phi after it on that stream.
 * Working memory is a fixed file-scope device array of 4,194,304 floats
 * (16 MiB) held by every GPU that loads the library until exit; a call needs
 * batch * 2 * bins * P floats of it and returns OT_EINVAL above that.  The
 * first call on each device resolves the array's device address (make that
 * first call before any stream capture).  All calls share the array: calls
 * whose kernels overlap on the GPU race and must not be issued.
 */
ot_status ot_hue_project_noalloc(int bins, int P, int batch, double axis_scale, const float* f0, const float* f1,
                                 const float* a_packed, float* x_packed, float* phi, void* cuda_stream);

/*
 * Mixed-size batches (many problems of different shapes solved together).
 * Problems whose grids are identical share one batched plan; every such group
 * runs on its own stream and whole iterations of all groups are captured into
 * one CUDA graph, so that small problems fill the GPU side by side.  Each
 * problem follows Algorithm 1 exactly as ot_solve would.
 *
 * ot_batch_create: `count` grids (sizes and parameters per problem), ordered on
 *   cuda_stream (NULL => own stream).  Allocates one workspace per group.
 * ot_batch_solve: f0[i], f1[i] are problem i's densities (host or device,
 *   layout of ot_solve, same validation and mass rescaling).  All problems run
 *   in lockstep for up to `iters` iterations; every `check_every` iterations
 *   (0 => 10) the residuals are read and the batch stops once every problem's
 *   residual is <= tol (OT_ENOTCONV with valid results otherwise, when tol > 0).
 *   stats (may be NULL) receives `count` entries; elapsed_ms is the whole batch.
 * ot_batch_path: problem i's path, as ot_path.
 */
typedef struct ot_batch_s* ot_batch_t;
ot_status ot_batch_create(const ot_grid* grids, int count, void* cuda_stream, ot_batch_t* out);
ot_status ot_batch_solve(ot_batch_t b, const float* const* f0, const float* const* f1, int iters, double tol,
                         int check_every, ot_solve_stats* stats);
ot_status ot_batch_path(ot_batch_t b, int i, float* f, float* m0, float* m1, float* m2);
int ot_batch_groups(ot_batch_t b);
void ot_batch_destroy(ot_batch_t b);

/*
 * Warm-start network kernels (a learned initial path for Algorithm 1; the
 * paper has no network).  A 3D U-Net over (t, y, x) maps the boundary densities
 * of an RGB pair to an initial path x0 for Algorithm 1 (ot_solve's init_path).
 * All pointers are DEVICE memory; work is ordered on `stream` (cudaStream_t,
 * NULL = legacy default stream) and the calls return without synchronising.
 * Activations are channels-last [N][T][Y][X][channels] in bf16; a tensor is
 * addressed by its channel stride (xs, ys) and first channel (xo, yo), so that
 * concatenations are channel slices.  Weights are [cout][27][cin] bf16 (tap =
 * 9 (dt+1) + 3 (dy+1) + (dx+1)), bias fp32.
 *
 * ot_nn_conv3d: y = relu?(conv3x3x3(x, w) + bias), zero padding; cin % 16 == 0,
 *   cout % 8 == 0; out_f32 selects an fp32 output.  Tensor cores (bf16, fp32 accumulate):
 *   tcgen05 with the accumulator in tensor memory and operands staged by bulk tensor copies
 *   where cout % 16 == 0 (16 <= cout <= 256; 32 or more when X < 128), the input slice starts
 *   on 16 bytes, the output rows hold 16-byte vectors and X divides 128 (or 128 divides X);
 *   mma.sync otherwise.
 * ot_nn_check: waits for `stream` and returns OT_ETIMEOUT (once) if a bounded device wait of
 *   the tcgen05 convolution ran out since the last check (that launch wrote NaN), else OT_OK.
 * ot_nn_conv3d_wgrad: dw (fp32 [cout][27][cin]) += sum_v dy[v] x[v + tap]; db (fp32,
 *   may be NULL) += sum_v dy[v]; cin, cout % 16 == 0.  Tensor cores: tcgen05 (both operands
 *   staged by bulk tensor copies, fp32 sums in tensor memory, per-CTA partials added in a fixed
 *   order) where 32 <= cin <= 128, 32 <= cout <= 64, X is 16, 32, 64 or 128 and the slices
 *   start on 16 bytes; mma.sync otherwise.  The data gradient is
 *   ot_nn_conv3d with ot_nn_rotate_weights(w) (wr[ci][tap][co] = w[co][26-tap][ci]).
 * ot_nn_relu_grad: g *= (y > 0).  ot_nn_pool / ot_nn_upsample: 2x2 average pooling
 *   and nearest upsampling over (y, x) (Yc, Xc = coarse sizes), forward or backward.
 * ot_nn_add_slice: y[:, yo:yo+C] += x[:, xo:xo+C].
 * ot_nn_mse: loss (fp32, accumulated) += mean over M voxels x Cv channels of
 *   (out - target)^2 (out fp32 with channel stride os, target bf16 [M][Cv]);
 *   g (bf16, gs channels) = its gradient, zero in channels Cv..gs-1.
 * ot_nn_adamw: AdamW step `step` (1-based) on fp32 master weights p with fp32 grads g;
 *   pb (bf16 copy, may be NULL) is refreshed.  ot_nn_to_bf16: fp32 -> bf16.
 * ot_nn_make_input: network input [N][P][Y][X][Cp] (Cp >= 10) from densities f0, f1
 *   ([N][3][Y][X] fp32) times scale[n] (device, NULL = 1): channels f0 (3), f1 (3),
 *   (1 - tau) f0 + tau f1 at tau = (t + 1)/P (3), (t + 1/2)/P, zeros.
 * ot_nn_path_channels: packed path (the ABI layout of ot_path / init_path, N problems)
 *   <-> 12 cell-aligned fp32 channels [N][P][Y][X][cs] (cs >= 12; faces to the right of
 *   each cell for m_x, m_y, m_c, then f; zero where the model has no variable; channels
 *   12..cs-1 are not touched).
 *   to_channels: ch = scale[n] (packed - L); otherwise packed = ch / scale[n] + L,
 *   where L is zero for m and, when f0/f1 (same units as packed) are given, the
 *   linear interpolation (1 - tau) f0 + tau f1 of the densities for f.
 * ot_nn_dual_channels: packed dual (the layout of ot_state_get's b: per problem
 *   b_mx, b_my, b_mc, b_f, each [P][3][Y][X]) <-> channels co + 3k + c of
 *   [N][P][Y][X][cs].
 */
ot_status ot_nn_conv3d(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo, const void* w,
                       const float* bias, void* y, int ys, int yo, int relu, int out_f32, void* stream);
ot_status ot_nn_check(void* stream);
ot_status ot_nn_conv3d_wgrad(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo,
                             const void* dy, int dys, int dyo, float* dw, float* db, void* stream);
ot_status ot_nn_rotate_weights(int Cin, int Cout, const void* w, void* wr, void* stream);
ot_status ot_nn_relu_grad(long long M, int C, void* g, int gs, int go, const void* y, int ys, int yo, void* stream);
ot_status ot_nn_pool(int N, int T, int Yc, int Xc, int C, const void* x, int xs, int xo, void* y, int ys, int yo,
                     int backward, void* stream);
ot_status ot_nn_upsample(int N, int T, int Yc, int Xc, int C, const void* x, int xs, int xo, void* y, int ys, int yo,
                         int backward, void* stream);
ot_status ot_nn_add_slice(long long M, int C, const void* x, int xs, int xo, void* y, int ys, int yo, void* stream);
ot_status ot_nn_mse(long long M, int Cv, const float* out, int os, const void* target, void* g, int gs, float* loss,
                    void* stream);
ot_status ot_nn_adamw(long long n, float* p, const float* g, float* m, float* v, void* pb, float lr, float b1,
                      float b2, float eps, float wd, int step, void* stream);
ot_status ot_nn_to_bf16(long long n, const float* x, void* y, void* stream);
ot_status ot_nn_make_input(int N, int P, int Y, int X, int Cp, const float* f0, const float* f1, const float* scale,
                           void* out, void* stream);
ot_status ot_nn_path_channels(int N, int Y, int X, int P, int to_channels, const float* scale, const float* f0,
                              const float* f1, float* packed, float* ch, int cs, void* stream);
ot_status ot_nn_dual_channels(int N, int Y, int X, int P, int to_channels, float* packed, float* ch, int cs, int co,
                              void* stream);

/*
 * Hue image pipeline (section 5): two images that differ only in hue are
 * morphed by transporting the hue histogram with the periodic OT of the
 * paper (ot_solve on an ot_grid_hue grid) and specifying the source hues to
 * each intermediate histogram, keeping saturation and value.  All pointers
 * are DEVICE memory; work is ordered on `stream` (cudaStream_t, NULL = legacy
 * default stream).
 *
 * ot_rgb_to_hsv / ot_hsv_to_rgb: rgb is [3][npix] in [0, 1]; hue in [0, 1)
 *   (hexcone model), saturation, value.  Asynchronous.
 * ot_hue_histogram: hist[bins] = fraction of the pixels whose hue lies in
 *   [b / bins, (b + 1) / bins) (mass 1); 1 <= npix < 2^24.  Asynchronous.
 * ot_hue_specify: h_out = the hues h re-assigned so that their histogram is
 *   exactly `target` (bins values; negative entries count as 0 and the rest is
 *   renormalised to mass 1; integer counts by largest remainders).  The paper cites its circular specification method without
 *   printing it; the reading implemented: pixels ranked by (hue, index), rank
 *   r gets target rank (r - s) mod npix, where the cyclic shift s has the least
 *   squared circular distance of all npix shifts (exhaustive search, ties to the
 *   smaller shift; for sorted points on the circle an optimal matching under a
 *   cost convex in the distance is such a shift), and target rank q in bin b
 *   gets the hue (b + (q - C_b + 1/2) / c_b) / bins.  Allocates its workspace
 *   and synchronises `stream`; 1 <= npix <= 2^21 (the search costs npix^2 terms).
 */
ot_status ot_rgb_to_hsv(int npix, const float* rgb, float* h, float* s, float* v, void* stream);
ot_status ot_hsv_to_rgb(int npix, const float* h, const float* s, const float* v, float* rgb, void* stream);
ot_status ot_hue_histogram(int npix, const float* h, int bins, float* hist, void* stream);
ot_status ot_hue_specify(int npix, const float* h, int bins, const float* target, float* h_out, void* stream);

/* Thread-local description of the last error on this thread ("" if none). */
const char* ot_last_error(void);

/* Version of this ABI (OT_ABI_VERSION). */
int ot_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DYNOT_H */
