/*
 * claire.h -- C ABI of a B300 (sm_103a) implementation of the hot path of
 * CLAIRE's diffeomorphic image registration (arXiv 2401.17493): the RK2
 * semi-Lagrangian transport solves inside an inexact Gauss-Newton-Krylov
 * optimiser for a stationary velocity v, composed into the reduced gradient
 * and the Hessian matvec.
 *
 * Conventions (every entry point):
 *  - Grids are periodic, nx x ny x nz nodes on [-pi, pi)^3, spacing
 *    h_i = 2 pi / n_i, node x_l = l h along increasing index (Sec. 2.5.1).
 *  - Scalar fields are float32 arrays [nx][ny][nz], nz fastest.  Vector
 *    fields are SoA float32 [3][nx][ny][nz].
 *  - Pointer arguments are CALLER-OWNED DEVICE pointers unless the name ends
 *    in _host.  The library never frees them and never keeps them past the
 *    call (claire_set_images copies the images).
 *  - The context owns all workspace (histories, departure points, FFT plans,
 *    reduction scratch); it is allocated in claire_create.
 *  - Calls are synchronous with respect to the stream given in the options
 *    (default: the legacy default stream) and return a claire_status.  They
 *    never abort, exit or trap; claire_last_error() gives a message.
 *  - A context is not thread-safe; separate contexts are independent.
 */
#ifndef CLAIRE_H
#define CLAIRE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct claire_ctx claire_ctx;

typedef enum {
  CLAIRE_OK = 0,
  CLAIRE_EINVAL = 1,       /* bad argument: shape, nt, null pointer, option range   */
  CLAIRE_ENOMEM = 2,       /* device allocation failed                              */
  CLAIRE_ECUDA = 3,        /* a CUDA / cuFFT call failed                            */
  CLAIRE_ENONFINITE = 4,   /* NaN or Inf met in J, g or a PCG scalar                */
  CLAIRE_ENOTCONV = 5,     /* max_newton reached before the gradient tolerance      */
  CLAIRE_ENEGCURV = 6,     /* PCG met <s, H s> <= 0 (previous iterate kept)         */
  CLAIRE_ELINESEARCH = 7,  /* Armijo failed after max halvings                      */
  CLAIRE_ETIMEOUT = 8,     /* a bounded device wait ran out                         */
  CLAIRE_EORDER = 9        /* hessian_matvec before any objective_gradient          */
} claire_status;

typedef struct {
  int precision;        /* 0: FP32 storage (default). 1: mixed (16-bit field storage,
                           FP32 math and coordinates, FP64 reductions)               */
  int hessian;          /* 0: Gauss-Newton (default, Sec. 2.5.5). 1: full Newton (eq.
                           matvec with the lam terms: sources div(lam^j vt) in the
                           incremental adjoint and sum_j w_j lam^j grad m~^j); needs
                           precision 0 and (nt + 2) N more floats; PCG ends on
                           negative curvature as in Sec. 2.5.5                      */
  double beta_w;        /* divergence-penalty weight of the near-incompressible model
                           (Appendix); 0 = plain H1 seminorm (default)             */
  double eps_opt;       /* relative gradient tolerance, default 5e-2 (Sec. 2.6)      */
  int max_newton;       /* outer iteration cap, default 50                           */
  int max_pcg;          /* PCG iteration cap per Newton step, default 100            */
  int fixed_iters;      /* 1: run exactly max_newton x max_pcg iterations (parity)   */
  int forcing;          /* 0: superlinear eta = min(1/2, sqrt(rel g)), 1: quadratic  */
  void* stream;         /* cudaStream_t to run on; NULL = legacy default stream      */
  int verbose;          /* 1: one line per Newton iteration on stderr                */
  double gnorm0;        /* > 0: denominator of the relative gradient; <= 0: use
                           ||g(v = 0)||_inf computed by the solver (reading C-10)    */
  int autotune;         /* 1: time the tile-shape variants on the first evaluation of a
                           solve and keep the fastest for this context (default 0)   */
  int graphs;           /* 1: replay the parts of PCG (start, H s and update, next
                           direction) as captured CUDA graphs, the two-level nested CG
                           inside them as a conditional while node; bitwise the same
                           results as launch by launch (0, the default)              */
  int precond;          /* PCG preconditioner (Sec. 2.5.6).  0: spectral, (beta_v L)^-1
                           with the zero symbol set to one.  1: two-level
                           zero-velocity H0: R^-1/2 M^-1 R^-1/2 with R = beta_v L, M^-1
                           the coarse (n/2) solve of I + R^-1/2 (grad m (x) grad m)
                           R^-1/2 at the current m(1) plus the high-frequency part;
                           needs every n_i % 4 == 0 (EINVAL otherwise).  2 (default):
                           two-level when every n_i % 4 == 0, else spectral -- the
                           paper's default preconditioner where it applies (Sec. 2.6) */
  int max_inner;        /* nested CG iteration cap of precond 1 (default 50)          */
  double inner_rtol;    /* > 0: fixed relative tolerance of the nested CG; <= 0: one
                           tenth of the outer PCG's relative tolerance (Sec. 2.6)    */
  int distance;         /* 0: 1/2 ||m(1) - m1||^2 (default, eq. varopt-claire).  1: NCC,
                           1 - <m(1), m1>^2 / (||m1||^2 ||m(1)||^2) (Appendix), which
                           changes lam(1) and lam~(1); needs precision 0             */
  int warm_check;       /* 1: in claire_solve* and claire_solve_batch a nonzero initial
                           guess v0 is kept only if J(v0) <= J(0), the distance of the
                           template (the regulariser vanishes at v = 0); otherwise the
                           solve restarts from v = 0 (the fallback of a learned warm
                           start).  An accepted v0's evaluation is the solver's first
                           one, so the check costs no extra PDE solve unless it
                           rejects.  Default 0                                        */
} claire_options;

typedef struct {
  int newton_iters, pcg_iters, matvecs, pde_solves, linesearch_halvings;
  double J0, J, mismatch_rel, grad_rel, gnorm0;
  double detF_min, detF_max, detF_mean;
  double seconds;       /* device time of the call (CUDA events)                    */
  int status;
  int inner_iters;      /* nested CG iterations of the two-level preconditioner       */
  int warm_fallback;    /* 1: options.warm_check rejected the initial guess            */
} claire_stats;

/* Fill *opt with the defaults listed above.  EINVAL on NULL. */
claire_status claire_default_options(claire_options* opt);

/* Create a context for an nx x ny x nz grid with nt time steps, regularisation
 * weight beta_v (alpha in Sec. 2.2) and operator exponent gamma
 * (L = (-Laplacian)^gamma, gamma = 1: H1 seminorm).  Sizes must be even and
 * >= 16 with 3 nx ny nz < 2^31 (the largest cube is 894^3), nt >= 1,
 * beta_v > 0, gamma > 0, else EINVAL.  Allocates the whole workspace
 * (ENOMEM / ECUDA on failure, *out left NULL). */
claire_status claire_create(int nx, int ny, int nz, int nt, double beta_v, double gamma,
                            claire_ctx** out);
claire_status claire_set_options(claire_ctx* ctx, const claire_options* opt);
claire_status claire_get_options(const claire_ctx* ctx, claire_options* opt);
/* Change beta_v (continuation, Sec. 2.6).  Invalidates the stored evaluation. */
claire_status claire_set_beta(claire_ctx* ctx, double beta_v);
/* Bytes of device memory the context holds (workspace high-water mark). */
size_t claire_workspace_bytes(const claire_ctx* ctx);

/* Copy template m0 and reference m1 (device, [nx][ny][nz]) into the context. */
claire_status claire_set_images(claire_ctx* ctx, const float* m0, const float* m1);

/* m(1) of the state equation (eq. transport, Sec. 2.2) for velocity v:
 * RK2 departure points (Sec. 2.5.2) and nt homogeneous SL steps.  In the mixed
 * form (options.precision = 1) the state between the steps is stored in FP16
 * with the images' power-of-two scale, as in the solver; m1_out is FP32.  The
 * state history of the last evaluation is left untouched. */
claire_status claire_transport(claire_ctx* ctx, const float* v, float* m1_out);

/* Objective J (eq. varopt-claire) and reduced gradient g (eq. rgrad, plus the
 * near-incompressible projection when beta_w > 0) at v.  J is a host double;
 * g may be NULL.  Stores the state for claire_hessian_matvec. */
claire_status claire_objective_gradient(claire_ctx* ctx, const float* v, double* J_host,
                                        float* g);

/* H vt (eq. matvec; Gauss-Newton unless options.hessian = 1) at the v of the
 * last claire_objective_gradient / claire_solve.  EORDER if there is none. */
claire_status claire_hessian_matvec(claire_ctx* ctx, const float* vt, float* Hvt);

/* Inexact Gauss-Newton-Krylov solve (Algorithms 1 and 2) from the initial
 * guess in v_inout; the result overwrites it.  stats may be NULL.  Returns
 * OK, ENOTCONV, ELINESEARCH or ENONFINITE (v_inout then holds the last
 * accepted iterate), or an argument/CUDA error. */
claire_status claire_solve(claire_ctx* ctx, float* v_inout, claire_stats* stats);

/* Parameter continuation (Sec. 2.6): solve for betas[0], betas[1], ... in
 * turn, each level warm-started from the previous one; the relative-gradient
 * denominator is ||g(v = 0)||_inf for every level (g(0) has no regularisation
 * term).  The context's beta_v ends at betas[nlevels - 1].  stats accumulate
 * over the levels. */
claire_status claire_solve_continuation(claire_ctx* ctx, const double* betas, int nlevels,
                                        float* v_inout, claire_stats* stats);

/* claire_solve / claire_solve_continuation with HOST buffers: copies m0, m1
 * and the initial v in, solves (betas == NULL: one level at the context's
 * beta_v; else nlevels continuation levels), copies v out, all on the
 * context's stream.  Pageable or pinned host memory ([nx][ny][nz] images,
 * [3][nx][ny][nz] v).  The images replace those of claire_set_images. */
claire_status claire_solve_host(claire_ctx* ctx, const float* m0_host, const float* m1_host,
                                const double* betas, int nlevels, float* v_inout_host,
                                claire_stats* stats);

claire_status claire_destroy(claire_ctx* ctx);
const char* claire_last_error(const claire_ctx* ctx);

/* ---- single steps of the path (for step-by-step parity checks) ---------- */

/* RK2 departure points (Sec. 2.5.2) of v as displacements in grid units:
 * d_fwd = (y - x) / h for transport along +v (state, incremental state),
 * d_bwd for transport along -v (adjoint, incremental adjoint).  [3][N] each;
 * either output may be NULL. */
claire_status claire_trace(claire_ctx* ctx, const float* v, float* d_fwd, float* d_bwd);

/* out(x) = u(x + d(x)) by periodic tricubic Lagrange interpolation
 * (Sec. 2.5.4); d is a displacement in grid units [3][N]. */
claire_status claire_interp(claire_ctx* ctx, const float* u, const float* d, float* out);

/* FD8 gradient [N] -> [3][N] and divergence [3][N] -> [N] (Sec. 2.5.3). */
claire_status claire_grad8(claire_ctx* ctx, const float* u, float* grad_u);
claire_status claire_div8(claire_ctx* ctx, const float* w, float* div_w);

/* Spectral operators on a vector field [3][N] (Sec. 2.5.3, 2.5.6, Appendix):
 * op 0: L = (-Laplacian)^gamma;  1: (beta_v L)^-1 with the zero symbol set to
 * one;  2: P_par (gradient part of the Leray decomposition);  3: c(kappa) P_par
 * (near-incompressible term with options.beta_w);  4: (beta_v L)^-1/2 with the
 * zero symbol set to one (the smoother of the two-level preconditioner). */
enum { CLAIRE_OP_L = 0, CLAIRE_OP_REG_INV = 1, CLAIRE_OP_LERAY_PAR = 2, CLAIRE_OP_NEAR_INC = 3,
       CLAIRE_OP_REG_INV_SQRT = 4 };
claire_status claire_spectral(claire_ctx* ctx, int op, const float* in, float* out);

/* Regularisation-parameter search with det F bounds (Sec. 2.6, "Parameter
 * Selection", eq. ddgradbound): starting at beta0, beta_v drops by decades
 * until eps_d < min det F1 and max det F1 < 1/eps_d fails (or beta_min is
 * reached), then bisects between the last admissible and the failing value
 * (arithmetic midpoint; stops when the bracket is narrower than rtol times its
 * admissible end or after max_bisect steps).  Each trial is a Gauss-Newton
 * solve (options as set) warm-started from the previous trial.  v_inout
 * (device [3][N]) is the initial guess on entry and the velocity of *beta_out
 * (the smallest admissible value found) on return; *beta_out = 0 when beta0
 * already violates the bound (v_inout then holds that trial's velocity).
 * Up to max_trials (beta, min det F1, max det F1) triples go to the host
 * arrays; *ntrials (may be NULL) receives the number of trials.  stats (may
 * be NULL) sums all trials.  0 < eps_d < 1, beta0, beta_min, rtol > 0. */
claire_status claire_beta_search(claire_ctx* ctx, double eps_d, double beta0, double beta_min,
                                 double rtol, int max_bisect, float* v_inout, double* beta_out,
                                 double* trial_beta, double* trial_detmin, double* trial_detmax,
                                 int max_trials, int* ntrials, claire_stats* stats);

/* z = M^-1 r (device [3][N]) with the preconditioner of options.precond
 * (Sec. 2.5.6) at the image m(1) of the last claire_objective_gradient
 * (EORDER if there is none).  For precond 1 the nested CG runs to
 * options.inner_rtol (1e-3 when that is <= 0) or options.max_inner
 * iterations; *inner_iters (may be NULL) receives the count. */
claire_status claire_precondition(claire_ctx* ctx, const float* r, float* z, int* inner_iters);

/* det F1 of the deformation-gradient transport (Appendix, eq. def-grad) for
 * velocity v: min / max / mean into minmaxmean_host[3]; det_out ([N]) may be NULL. */
claire_status claire_det_deformation_gradient(claire_ctx* ctx, const float* v,
                                              double* minmaxmean_host, float* det_out);

/* ---- allocation-free transport --------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory.  Every other call works through a context
 * whose workspace comes from cudaMalloc.  Callers whose device memory is
 * reserved up front by another allocator (a framework's caching allocator, a
 * fixed pool sized to the GPU) cannot add driver allocations without failing
 * or fragmenting that pool, and some cannot accept the device-wide
 * synchronisation that cudaMalloc / cudaFree may imply.
 *
 * claire_transport_noalloc computes the same m(1) as claire_transport with the
 * same kernels, without a context and without allocating: no cudaMalloc, no
 * cudaFree, no allocating library routine.  Its scratch (departure
 * displacements and one intermediate field, 16 bytes per voxel) is a
 * file-scope device array sized for CLAIRE_NOALLOC_MAX_VOXELS voxels
 * (2^20, i.e. 16 MiB), which every GPU that loads the library holds until the
 * process exits.  Larger grids are rejected with CLAIRE_EINVAL and a message.
 *
 *  v       device [3][nx][ny][nz] float32 velocity (caller-owned, read only)
 *  m0      device [nx][ny][nz] float32 template (read only)
 *  m1_out  device [nx][ny][nz] float32 output; must not overlap m0 or v
 *  stream  cudaStream_t (NULL = legacy default stream); the call returns after
 *          synchronising that stream, so a stream that is capturing is refused
 *          with CLAIRE_EINVAL before anything is launched
 *  err     optional buffer (may be NULL) that receives a message on failure
 * Sizes must be even and >= 16, 1 <= nt <= 256.  v, m0 and m1_out must be
 * device memory of the current device (checked; CLAIRE_EINVAL otherwise).
 *
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture.  With lazy module loading (the CUDA
 * default) that first lookup is also when the driver loads this part of the
 * library onto the device and commits the 16 MiB array, so a caller whose
 * device memory is reserved afterwards should make one call first; the calls
 * after it commit nothing.  A failed lookup is not cached: the next call
 * retries it.  All calls in the process share the one array per device and
 * it keeps the last call's contents (every call rewrites all of the scratch
 * it reads, so nothing needs clearing); calls that overlap on the same GPU
 * (other streams or threads) race on it, so callers must serialise them. */
#define CLAIRE_NOALLOC_MAX_VOXELS (1LL << 20)
claire_status claire_transport_noalloc(int nx, int ny, int nz, int nt, const float* v,
                                       const float* m0, float* m1_out, void* stream,
                                       char* err, size_t err_len);

/* ---- batched solves --------------------------------------------------------
 * Solves npairs independent registrations, each on its own context (its own
 * grid, images, options), concurrently: up to max_threads host threads
 * (<= 0: one per pair) each drive one context at a time, and each context
 * runs on a stream of its own (a private stream is created for contexts on the
 * legacy default stream), so kernels of different pairs overlap on the GPU.
 * betas == NULL solves every context at its own beta_v, else nlevels
 * continuation levels.  v_inout[i] is pair i's device [3][N] initial guess and
 * result; stats (optional) has npairs entries.  Returns the worst status
 * (ENOTCONV only when nothing worse happened).  A context must not appear
 * twice. */
claire_status claire_solve_batch(claire_ctx** ctxs, int npairs, const double* betas,
                                 int nlevels, float** v_inout, claire_stats* stats,
                                 int max_threads);

/* The same batch with its SL steps, adjoint factors, traces and FD8 history
 * marches launched for several pairs at once: one host thread per pair drives
 * that pair's solve on the pair's stream, and instead of launching those
 * kernels it posts them and waits.  The first post of a round waits until
 * every unfinished pair has posted or wait_us microseconds have passed
 * (wait_us < 0: until every unfinished pair has posted); then one persistent
 * launch per kind walks the (pair, tile) items of all posted ops (the per-tile
 * code of the single launch, so every pair's results are bitwise those of
 * claire_solve_batch and of a solve on its own).  Launches captured into a
 * pair's CUDA graphs (options.graphs) stay in its graphs; the FP16 kernels of
 * precision-1 contexts and all other kernels (cuFFT, reductions, vector
 * updates) run on the pairs' streams as before.  *group_launches and
 * *group_ops (NULL ok) receive the number of grouped launches and of the
 * per-pair launches they replaced.  Same arguments, statuses and rules as
 * claire_solve_batch otherwise. */
claire_status claire_solve_batch_grouped(claire_ctx** ctxs, int npairs, const double* betas,
                                         int nlevels, float** v_inout, claire_stats* stats,
                                         int wait_us, long long* group_launches,
                                         long long* group_ops);

/* ---- autotuner -------------------------------------------------------------
 * Times the compiled tile shapes of the SL gather (the three gather variants, brick
 * depth along x1: 4, 8 or 16 nodes) and of the FD8 history kernels (8, 16, 32 or 64 planes per
 * CTA) on this context's grid and buffers and keeps the fastest for all later
 * calls on the context.  Evaluates J and g at the context's current v first if
 * nothing has been evaluated yet.  The chosen shapes are returned (NULL ok). */
claire_status claire_autotune(claire_ctx* ctx, int* sl_t1, int* march_t1);

/* Sets the tile shapes by hand (kept by options.autotune; drops captured graphs):
 *  sl_gather  0: SL gathers with 64 shared loads per node from a brick staged
 *             by TMA tiled loads, one per brick row (default; bricks whose x3
 *             range wraps around the periodic grid, and grids whose n3 is not
 *             a multiple of 4 or is below 40, are staged as with 2);
 *             1: a per-lane register window of four x1 tap planes (16 shared
 *             loads per node whose displacement floor equals the lane's
 *             reference floor; the other nodes are gathered afterwards by the
 *             whole CTA from the brick);
 *             2: the 64-load gather from a brick staged by the threads'
 *             16-byte cp.async copies.  All three give bitwise the same values
 *             (the FP16 form's interior bricks land by TMA for 0 when
 *             n3 % 8 == 0, else by cp.async);
 *  sl_t1      4, 8 or 16 nodes per thread along x1 (default 8);
 *  march_t1   8, 16, 32 or 64 planes per CTA of the FD8 history kernels (default 64
 *             where that leaves at least four CTAs per multiprocessor, else 32).
 * EINVAL for any other value.  claire_get_tuning reads the current shapes (the
 * autotuner's choice after claire_autotune); NULL outputs are skipped. */
claire_status claire_set_tuning(claire_ctx* ctx, int sl_gather, int sl_t1, int march_t1);
claire_status claire_get_tuning(const claire_ctx* ctx, int* sl_gather, int* sl_t1,
                                int* march_t1);

/* ---- gathers outside the staged brick ---------------------------------------
 * The SL steps stage a brick of the source field around each tile (a halo of 3
 * nodes along x1 and x2, 4 along x3) and interpolate from shared memory; a node
 * whose 4 x 4 x 4 taps leave the brick (floor of the displacement outside
 * [-2, 1] along x1 or x2, [-3, 2] along x3) takes the global-memory gather
 * instead, with the same result.  *fwd / *bwd = the number of such nodes for
 * the forward (state, incremental state) and backward (adjoint, incremental
 * adjoint) departure points of the last evaluation: every SL step in that
 * direction gathers those nodes from global memory.  EORDER before an
 * evaluation.  Synchronises the context's stream. */
claire_status claire_far_nodes(claire_ctx* ctx, long long* fwd, long long* bwd);

/* ---- learned warm start: 3D U-Net kernels --------------------------------------
 * Not part of the paper: a small 3D U-Net predicts an initial velocity from
 * the image pair on a 64^3 grid.  Activations are channels-last BF16 [V][C]
 * (V = batch B x D x H x W voxels, W fastest); weights BF16 [Cout][27][Cin];
 * accumulation FP32.  All convolutions are 3x3x3 with periodic padding and run
 * as implicit GEMMs on the tensor cores.  All pointers are device pointers
 * owned by the caller; calls are asynchronous on the given stream (NULL =
 * legacy default stream) and only report launch errors.
 *
 * Forward: y = act(conv(x, w) + bias); act = ReLU when relu != 0.  cin and cout
 * multiples of 16; y_bf16 ([V][cout] BF16) and / or y_f32 ([V][cout]) may be
 * NULL (not both); bias ([cout]) may be NULL.  V < 2^31 (EINVAL otherwise, here
 * and for the weight gradient). */
claire_status claire_conv3d_forward(const void* x, int B, int D, int H, int W, int cin,
                                    const void* w, const float* bias, int cout, int relu,
                                    void* y_bf16, float* y_f32, void* stream);
/* wf[cin][27][cout] = w[cout][26 - t][cin]: the data gradient of a conv is
 * claire_conv3d_forward of dy with wf (cin and cout swapped, no bias / ReLU). */
claire_status claire_conv3d_flip_weights(const void* w, int cout, int cin, void* wf,
                                         void* stream);
/* Weight gradient dw[cout][27][cin] (FP32) = sum_v dy[v][n] x[nbr_t(v)][c], as at
 * most nsplit partial sums written to partial (room for nsplit x cout x 27 x cin
 * floats) and added in a fixed order.  cin in {16, 32, 48, 64, 96, 128, 192}.
 * On the tcgen05 tensor cores, with min(nsplit, SMs, tiles) persistent CTAs (one
 * partial each): with the output channels as MMA rows where W % 8 == 0,
 * H % 16 == 0 and cin <= cout <= 128 (8 x 16-voxel tiles); else with the input
 * channels as MMA rows where W % 8 == 0, H % 8 == 0 and cout <= 32 or
 * H % 16 != 0 (8 x 8-voxel tiles).  Otherwise on mma.sync over voxel chunks of
 * at least 4096 voxels. */
claire_status claire_conv3d_wgrad(const void* x, int B, int D, int H, int W, int cin,
                                  const void* dy, int cout, float* partial, int nsplit,
                                  float* dw, void* stream);
/* Layer helpers (BF16 channels-last), op:
 *  0 ReLU backward: b (dy) *= (a (y) > 0), V x C elements
 *  1 / 2  2x2x2 average pool forward a -> b / backward a (dy coarse) -> b (dx fine);
 *         (B, D, H, W) = fine grid, C channels
 *  3 / 4  nearest 2x upsampling of a [coarse][C] into channels [c_off, c_off + C)
 *         of b [fine][Cdst] / its adjoint (sum of the 8 children) from a into b;
 *         (B, D, H, W) = coarse grid
 *  5 / 6  copy a [V][C] into channels [c_off, c_off + C) of b [V][Cdst] / back out
 *  7      b += a (V x C elements) */
claire_status claire_unet_op(int op, const void* a, void* b, long long V, int C, int Cdst,
                             int c_off, int B, int D, int H, int W, void* stream);
/* db[c] = sum_v dy[v][c] (FP32 result of a fixed-order FP64 sum: up to nblocks
 * CTAs each sum a contiguous range of voxels for every channel into partial
 * (caller-owned device scratch of nblocks x C doubles), then the partials of a
 * channel are added in a fixed order).  dy 4-byte aligned, C even and <= 512, nblocks >= 1;
 * EINVAL otherwise. */
claire_status claire_unet_bias_grad(const void* dy, long long V, int C, float* db,
                                    double* partial, int nblocks, void* stream);
/* out[v][c] = BF16(scale * f[c][v]) for c < nf, 0 for nf <= c < C. */
claire_status claire_unet_pack(long long V, int nf, const float* f, float scale, int C,
                               void* out, void* stream);
/* On the first 3 channels of y ([V][C] FP32): pred[c][v] = scale y[v][c] (pred
 * may be NULL); with target ([3][V]) also loss = mean squared error (needs
 * partial with nblocks doubles, written to *loss on the device) and its
 * gradient dy ([V][C] BF16, zero in channels >= 3; may be NULL). */
claire_status claire_unet_mse(long long V, int C, const float* y, const float* target,
                              float scale, void* dy, float* pred, double* partial, int nblocks,
                              double* loss, void* stream);
/* Adam step on FP32 master weights p with gradient g and moments m, v (step
 * >= 1 for the bias corrections); pb (BF16 copy of p) may be NULL. */
claire_status claire_unet_adam(long long n, float* p, const float* g, float* m, float* v,
                               float lr, float b1, float b2, float eps, int step, void* pb,
                               void* stream);
/* Bounded waits of the tensor-core and TMA kernels.  Every mbarrier wait of the
 * convolution kernels gives up after 2^22 polls of at most 1 us each; a thread
 * whose wait ran out writes NaN outputs instead of hanging and is counted in a
 * device counter.  The wait for a TMA-staged SL brick gives up after 2^20 polls;
 * its CTA is counted and gathers from global memory instead (same values).
 * claire_wait_status synchronises the device, writes the count
 * since the last call to *timeouts (NULL ok), resets it and returns
 * CLAIRE_ETIMEOUT if it was nonzero, else CLAIRE_OK.
 * claire_wait_selftest runs that failure path on purpose: one CTA of 32 threads
 * polls phase 0 of an mbarrier at most max_polls times (1 <= max_polls <= 2^20,
 * EINVAL otherwise).  With arrive == 0 nothing arrives: every thread gives up,
 * 32 timeouts are counted and the call returns CLAIRE_ETIMEOUT.  With arrive != 0
 * one thread arrives first and the call returns CLAIRE_OK.  No copy or MMA is in
 * flight in that kernel, so giving up leaves nothing behind and the device stays
 * usable.  Synchronises the stream. */
claire_status claire_wait_status(int* timeouts);
claire_status claire_wait_selftest(int max_polls, int arrive, void* stream);
/* Spectral resampling of ncomp planar fields [ncomp][n1][n2][n3] onto an
 * m1 x m2 x m3 grid (Sec. 2.5.6, spectral restriction / prolongation): keeps
 * the Fourier modes with |k_i| < min(n_i, m_i) / 2, zero elsewhere.  Even
 * sizes; ncomp * n1 * n2 * (n3/2+1) < 2^31.  Asynchronous on stream.  The
 * first call for a (device, stream, shapes, ncomp) creates batched cuFFT plans
 * and two spectral buffers that are kept for the process lifetime (the warm
 * start resamples once per registration, and plan creation costs milliseconds);
 * later calls allocate nothing.  The stream must stay valid while it is used. */
claire_status claire_resample(int n1, int n2, int n3, const float* in, int m1, int m2, int m3,
                              float* out, int ncomp, void* stream);

/* ---- launch accounting ---------------------------------------------------
 * The context counts every kernel it launches by class, with the algorithmic
 * bytes each launch moves (each input field read once, each output written
 * once; "cufft" counts one read and one write per transform).  With timing
 * on, each launch is also bracketed by CUDA events on its stream. */
typedef struct {
  const char* name;     /* kernel class: trace, sl_step, adjoint_factor, grad8, div8,
                           sdot_hist, accum_hist, spectral_diag, reduce, vector, detf, cufft */
  long long launches;   /* launches since the last reset                              */
  long long timed;      /* launches with an event-timed duration                     */
  double bytes;         /* algorithmic bytes of those launches                       */
  double ms;            /* summed event-timed duration                               */
  double timed_bytes;   /* algorithmic bytes of the event-timed launches (launches inside
                           captured graphs are counted but not timed)                */
} claire_kernel_stat;

/* Zero the counters; timing != 0 turns per-launch event timing on. */
claire_status claire_profile_reset(claire_ctx* ctx, int timing);
/* Waits for outstanding timing events, writes up to max entries (one per
 * kernel class) and returns how many; with out == NULL returns the number of
 * classes.  -1 on a NULL context or a CUDA error. */
int claire_profile_read(claire_ctx* ctx, claire_kernel_stat* out, int max);

#ifdef __cplusplus
}
#endif

#endif /* CLAIRE_H */
