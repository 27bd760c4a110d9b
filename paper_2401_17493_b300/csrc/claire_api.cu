// Context, reduced-space operators, PCG / Armijo / Gauss-Newton driver and
// the extern "C" entry points declared in include/claire.h.
//
// The host code only sequences kernels and reads FP64 scalars back (J, dot
// products, norms); every field operation runs in the kernels of kernels.cu
// and in cuFFT.  One context = one grid, one stream, one fixed workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/claire.h"
#include "internal.h"

using namespace claire;

struct claire_ctx {
  Grid g{};
  int nt = 4;
  double beta_v = 1e-2, gamma = 1.0;
  claire_options opt{};
  cudaStream_t st = nullptr;
  cufftHandle r2c = 0, c2r = 0;
  bool plans = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // images and the evaluation point
  float *m0 = nullptr, *m1 = nullptr, *v = nullptr, *df = nullptr, *db = nullptr;
  float *D = nullptr, *cf = nullptr, *mhist = nullptr, *lhist = nullptr, *grad = nullptr;
  float *Lv = nullptr, *scr3 = nullptr;
  // matvec and PCG workspace
  float *shist = nullptr, *pp0 = nullptr, *pp1 = nullptr, *lthist = nullptr;
  float *vt = nullptr, *r = nullptr, *z = nullptr, *s = nullptr, *Hs = nullptr;
  float* hs = nullptr;          // beta_v L s, carried by recurrence inside PCG
  // full Newton (options.hessian = 1), allocated on first use: the incremental
  // state history m~^j and e(x) = (h_t/2)(1 + h_t div v(x))
  float *mthist = nullptr, *ef = nullptr;
  float* vbest = nullptr;       // velocity of the last admissible beta (claire_beta_search)
  double* slots = nullptr;      // device FP64 scalars of PCG (see pcg())
  int* dflag = nullptr;         // device flag: negative curvature / non-finite PCG scalar
  unsigned long long* far = nullptr;  // count of claire_far_nodes
  double* hslots = nullptr;     // pinned host mirror of slots + flag
  int partial_blocks = 0;
  // mixed precision (options.precision = 1): FP16 histories, allocated on first use
  __half *mh = nullptr, *lh = nullptr, *sh = nullptr, *lth = nullptr, *ph0 = nullptr,
         *ph1 = nullptr;
  float sig_m = 1.0f;           // power-of-two image scale of the FP16 state / adjoint
  float *vtrial = nullptr, *dtrial = nullptr;
  cufftComplex* cbuf = nullptr;
  double *partial = nullptr, *dres = nullptr, *hres = nullptr;
  int red_blocks = 1184;
  // det F workspace (allocated on first use)
  float* detf = nullptr;
  bool have_eval = false;
  bool lv_spectrum = false;     // cbuf holds the spectrum of L v of the last objective()
  double vLv = 0.0;             // <v, L v> (plain sum) of the last objective()
  double beta_eval = 0.0;       // beta_v of the stored J and g
  double J = 0.0, dist = 0.0;
  // NCC distance (options.distance = 1): <m1, m(1)>, ||m1||^2, ||m(1)||^2 (L2, with h^3)
  // of the last objective evaluation
  double ncc_a = 0.0, ncc_b = 0.0, ncc_c = 0.0;
  std::string err;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Profiler prof;
  Tuning tune;                  // tile shapes for this grid (autotuner)
  bool tuned = false;
  // captured PCG iteration parts (options.graphs), indexed by
  // 4 * (departure-point buffer) + 2 * part + slot parity: the line search swaps
  // the two departure-point buffers, and kernel arguments are fixed at capture
  cudaGraphExec_t graph_exec[9] = {};          // [8]: the PCG start (part S)
  long long graph_launches[9][K_COUNT] = {};
  double graph_bytes[9][K_COUNT] = {};
  float* dbuf0 = nullptr;       // first of the two departure-point buffers
  // two-level preconditioner (options.precond = 1), allocated on first use
  Grid gc{};                    // coarse grid, n_i / 2 points per axis
  cufftHandle tl_r2c1 = 0, tl_c2r1 = 0, tl_r2c3 = 0, tl_c2r3 = 0;
  cufftComplex *tl_cc = nullptr, *cbuf2 = nullptr;
  // nested CG vectors as coarse half spectra [3][Ch], and two real coarse fields
  cufftComplex *tl_sx = nullptr, *tl_sr = nullptr, *tl_sp = nullptr, *tl_sap = nullptr;
  float *tl_gm = nullptr, *tl_mc = nullptr, *tl_q = nullptr, *tl_w = nullptr;
  float2* tl_fw = nullptr;      // per coarse mode: R^-1/2 symbol and Parseval weight
  unsigned* tl_count = nullptr; // block ticket of the nested CG's last-block reductions (0)
  bool tl_ready = false, tl_image = false;
  double tl_rtol = 1e-3;        // nested CG relative tolerance of the current PCG
  int tl_iters = 0;             // nested CG iterations not yet counted in the stats
  // the nested CG as a conditional while node in captured PCG parts: the stream its
  // body is captured on, the launches of one body replay, and whether capturing it
  // failed (part B then runs launch by launch)
  cudaStream_t tl_body = nullptr;
  long long tl_body_launches[K_COUNT] = {};
  double tl_body_bytes[K_COUNT] = {};
  bool tl_nograph = false;
  cudaStream_t own = nullptr;   // private stream for graph capture
  cudaStream_t user = nullptr;  // the stream of the options
  cudaEvent_t e_in = nullptr;   // orders the private stream after the user's stream
};

namespace {

void drop_graphs(claire_ctx* c);

claire_status fail(claire_ctx* c, claire_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CUDA_TRY(ctx, call)                                                           \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, CLAIRE_ECUDA, "%s failed: %s (%s:%d)", #call,                  \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                        \
  } while (0)

#define CUFFT_TRY(ctx, call)                                                          \
  do {                                                                                \
    cufftResult r_ = (call);                                                          \
    if (r_ != CUFFT_SUCCESS)                                                          \
      return fail(ctx, CLAIRE_ECUDA, "%s failed: cufft error %d", #call, (int)r_);    \
  } while (0)

#define TRY(expr)                                  \
  do {                                             \
    claire_status s_ = (expr);                     \
    if (s_ != CLAIRE_OK) return s_;                \
  } while (0)

// Launch errors surface here (asynchronous faults at the next sync).
claire_status check_launch(claire_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, CLAIRE_ECUDA, "kernel launch (%s) failed: %s", what, cudaGetErrorString(e));
  return CLAIRE_OK;
}

claire_status alloc(claire_ctx* c, float** p, int64_t nfloats) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)nfloats * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CLAIRE_ENOMEM, "cudaMalloc of %lld floats failed: %s", (long long)nfloats,
                cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  c->bytes += (size_t)nfloats * sizeof(float);
  *p = (float*)q;
  return CLAIRE_OK;
}

int64_t N_of(const claire_ctx* c) { return c->g.N; }

// Routes the launch accounting of the kernels to this context for one API call.
struct Enter {
  Profiler* prev;
  const Tuning* prev_tune;
  explicit Enter(claire_ctx* c) : prev(tl_prof), prev_tune(tl_tune) {
    tl_prof = c ? &c->prof : nullptr;
    tl_tune = c ? &c->tune : nullptr;
    // with the private (graph) stream, start after the work already queued on
    // the caller's stream; every call ends with a synchronisation of its stream
    if (c && c->own && c->st == c->own && c->e_in) {
      cudaEventRecord(c->e_in, c->user);
      cudaStreamWaitEvent(c->st, c->e_in, 0);
    }
  }
  ~Enter() {
    tl_prof = prev;
    tl_tune = prev_tune;
  }
};
#define ENTER(c) Enter enter_guard_(c)

// NVTX range of one solver phase (shown by profilers that record NVTX, e.g. ncu
// --nvtx; without such a tool attached the calls return at once).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- reductions

claire_status reduce(claire_ctx* c, int64_t n, const float* a, const float* b, int mode,
                     double* out) {
  launch_reduce(n, a, b, mode, c->partial, c->red_blocks, c->dres, c->st);
  TRY(check_launch(c, "reduce"));
  CUDA_TRY(c, cudaMemcpyAsync(c->hres, c->dres, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  *out = c->hres[0];
  return CLAIRE_OK;
}

claire_status dot3(claire_ctx* c, const float* a, const float* b, double* out) {
  return reduce(c, 3 * N_of(c), a, b, RED_DOT, out);
}

// ---------------------------------------------------------------- spectral

// out = op(in) for a vector field; accumulate: out = out_coef * out + op(in) via scr3.
claire_status spectral(claire_ctx* c, int op, const float* in, float* out, double alpha) {
  const double fft_bytes = 3.0 * (4.0 * c->g.N + 8.0 * c->g.n1 * c->g.n2 * (c->g.n3 / 2 + 1));
  {
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    c->lv_spectrum = false;
    CUFFT_TRY(c, cufftExecR2C(c->r2c, (cufftReal*)in, c->cbuf));
  }
  launch_spectral(c->g, c->cbuf, op, (float)alpha, (float)c->gamma, (float)c->opt.beta_w, c->st);
  TRY(check_launch(c, "spectral"));
  {
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    CUFFT_TRY(c, cufftExecC2R(c->c2r, c->cbuf, (cufftReal*)out));
  }
  return CLAIRE_OK;
}

// b <- b - c(kappa) P_par b when beta_w > 0 (near-incompressible model, Appendix).
claire_status project_data_term(claire_ctx* c, float* b) {
  if (c->opt.beta_w <= 0.0) return CLAIRE_OK;
  TRY(spectral(c, CLAIRE_OP_NEAR_INC, b, c->scr3, c->beta_v));
  launch_axpby(3 * N_of(c), -1.0f, c->scr3, 1.0f, b, c->st);
  return check_launch(c, "axpby");
}

// ---------------------------------------------------------------- PDE solves

float ht_of(const claire_ctx* c) { return 1.0f / (float)c->nt; }
bool mixed(const claire_ctx* c) { return c->opt.precision == 1; }
bool grid_div4(const claire_ctx* c) { return c->g.n1 % 4 == 0 && c->g.n2 % 4 == 0 && c->g.n3 % 4 == 0; }
// options.precond 1, or 2 (automatic) on a grid whose sizes are multiples of 4
bool two_level(const claire_ctx* c) {
  return c->opt.precond == 1 || (c->opt.precond == 2 && grid_div4(c));
}

// Slots of the device-side FP64 scalars.
enum { SLOT_RZ0 = 0, SLOT_RZ1 = 1, SLOT_SHS = 2, SLOT_RR = 3, SLOT_MEAN = 4, SLOT_VMAX = 8,
       SLOT_TL_RR0 = 9, SLOT_TL_RR1 = 10, SLOT_TL_PAP = 11, SLOT_ZERO = 12 /* ..14 */,
       SLOT_NCC_AL = 15, SLOT_NCC_GA = 16,
       // nested CG on the device (captured PCG part B): relative tolerance, stop
       // threshold, iterations of the current application, iterations since PCG start
       SLOT_TL_RTOL = 17, SLOT_TL_STOP = 18, SLOT_TL_COUNT = 19, SLOT_TL_ITS = 20,
       NSLOTS = 24 };

// Power-of-two scale that maps max(|m0|, |m1|) into (1/2, 1] (FP16 state range).
claire_status image_scale(claire_ctx* c) {
  double a = 0.0, b = 0.0;
  TRY(reduce(c, N_of(c), c->m0, nullptr, RED_ABSMAX, &a));
  TRY(reduce(c, N_of(c), c->m1, nullptr, RED_ABSMAX, &b));
  const double mx = std::max(a, b);
  if (!std::isfinite(mx)) return fail(c, CLAIRE_ENONFINITE, "images are not finite");
  int e = 0;
  if (mx > 0.0) std::frexp(mx, &e);
  e = std::min(120, std::max(-120, e));
  c->sig_m = std::ldexp(1.0f, -e);
  return CLAIRE_OK;
}

// sum_j w_j lam^j grad m^j (+ base_coef base) into out, FP32 or FP16 histories;
// with vmax the incremental scale 2^-ceil(log2 *vmax) is undone; with partial,
// per-block shares of <dotv, out> (PCG curvature).
claire_status accumulate(claire_ctx* c, const float* lhist, const __half* lh, const float* base,
                         float base_coef, float* out, const double* vmax, const float* dotv,
                         double* partial) {
  if (mixed(c)) {
    const float umul = 1.0f / (c->sig_m * c->sig_m);
    if (!launch_accum_hist_h(c->g, lh, c->mh, c->nt, vmax, umul, base, base_coef, out, dotv,
                             partial, c->st))
      return fail(c, CLAIRE_EINVAL, "mixed precision needs nt in {1, 2, 4, 8}");
  } else {
    launch_accum_hist(c->g, lhist, c->mhist, c->nt, base, base_coef, out, c->st, dotv, partial);
  }
  return check_launch(c, "accumulate");
}

// Full Newton (options.hessian = 1): out += sum_j w_j lam^j grad m~^j, the term of
// eq. (matvec) that Gauss-Newton drops; with partial, per-block shares of
// <dotv, out>.  No-op for Gauss-Newton.
claire_status accumulate_newton(claire_ctx* c, float* out, const float* dotv, double* partial) {
  if (c->opt.hessian != 1) return CLAIRE_OK;
  launch_accum_hist(c->g, c->lhist, c->mthist, c->nt, out, 1.0f, out, c->st, dotv, partial);
  return check_launch(c, "full-Newton accumulate");
}

// The FP32 state, adjoint and incremental histories ((n_t + 1) N floats each),
// allocated on first FP32 use: the mixed-precision form never needs them.
claire_status fp32_histories(claire_ctx* c) {
  if (c->mhist && c->lhist && c->shist && c->lthist) return CLAIRE_OK;
  const int64_t nh = (int64_t)(c->nt + 1) * N_of(c);
  float** hists[] = {&c->mhist, &c->lhist, &c->shist, &c->lthist};
  for (auto p : hists)
    if (!*p) TRY(alloc(c, p, nh));
  return CLAIRE_OK;
}

// m^0 = m0, m^{j+1}(x) = m^j(x + d_f(x))  (eq. transport, homogeneous SL steps)
claire_status state_solve(claire_ctx* c, const float* d) {
  NvtxRange nvtx_("claire.state_solve");
  const int64_t N = N_of(c);
  if (!mixed(c)) TRY(fp32_histories(c));
  if (mixed(c)) {                                  // FP16 history of sig_m m
    launch_axpy_h(N, c->sig_m, c->m0, 0.0f, nullptr, c->mh, c->st);
    for (int j = 0; j < c->nt; ++j)
      launch_sl_h(c->g, c->mh + j * N, d, nullptr, 1.0f, nullptr, 0.0f, c->mh + (j + 1) * N,
                  c->st);
    return check_launch(c, "state_solve");
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->mhist, c->m0, N * sizeof(float), cudaMemcpyDeviceToDevice,
                              c->st));
  for (int j = 0; j < c->nt; ++j)
    launch_sl(c->g, c->mhist + j * N, d, nullptr, 1.0f, nullptr, 0.0f, c->mhist + (j + 1) * N,
              c->st);
  return check_launch(c, "state_solve");
}

// J = 1/2 h^3 sum (m(1) - m1)^2 + beta_v/2 h^3 <v, L v>  (eq. varopt-claire); keeps L v.
claire_status objective(claire_ctx* c, const float* v, double* J) {
  const int64_t N = N_of(c);
  const double h3 = (double)c->g.h1 * c->g.h2 * c->g.h3;
  double sq = 0.0, vLv = 0.0;
  if (mixed(c)) {
    launch_sqdiff_h(N, c->mh + c->nt * N, 1.0f / c->sig_m, c->m1, c->partial, c->red_blocks,
                    c->dres, c->st);
    TRY(check_launch(c, "objective"));
    CUDA_TRY(c, cudaMemcpyAsync(c->hres, c->dres, sizeof(double), cudaMemcpyDeviceToHost,
                                c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    sq = c->hres[0];
  } else if (c->opt.distance == 1) {           // NCC (Appendix)
    const float* m = c->mhist + c->nt * N;
    double a = 0.0, b = 0.0, cc = 0.0;
    TRY(reduce(c, N, m, c->m1, RED_DOT, &a));
    TRY(reduce(c, N, c->m1, nullptr, RED_SQ, &b));
    TRY(reduce(c, N, m, nullptr, RED_SQ, &cc));
    c->ncc_a = h3 * a; c->ncc_b = h3 * b; c->ncc_c = h3 * cc;
    if (!(c->ncc_b > 0.0) || !(c->ncc_c > 0.0))
      return fail(c, CLAIRE_ENONFINITE, "NCC distance of a zero image");
  } else {
    TRY(reduce(c, N, c->mhist + c->nt * N, c->m1, RED_SQDIFF, &sq));
  }
  // <v, L v> by Parseval from the spectrum of v; L v itself is only formed for the
  // point whose gradient is taken (lv_spectrum: cbuf holds L v^ until then)
  {
    const Grid& g = c->g;
    const double fft_bytes = 3.0 * (4.0 * g.N + 8.0 * g.n1 * g.n2 * (g.n3 / 2 + 1));
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    CUFFT_TRY(c, cufftExecR2C(c->r2c, (cufftReal*)v, c->cbuf));
  }
  launch_spectral(c->g, c->cbuf, CLAIRE_OP_L, 1.0f, (float)c->gamma, (float)c->opt.beta_w, c->st,
                  c->partial);
  launch_reduce_final(c->partial, spectral_blocks(c->g), RED_SUM, c->dres, c->st);
  TRY(check_launch(c, "objective"));
  CUDA_TRY(c, cudaMemcpyAsync(c->hres, c->dres, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  vLv = c->hres[0];
  c->vLv = vLv;
  c->lv_spectrum = true;
  c->dist = c->opt.distance == 1 ? 1.0 - c->ncc_a * c->ncc_a / (c->ncc_b * c->ncc_c)
                                  : 0.5 * h3 * sq;
  *J = c->dist + 0.5 * c->beta_v * h3 * vLv;
  if (!std::isfinite(*J)) return fail(c, CLAIRE_ENONFINITE, "objective is not finite (%g)", *J);
  return CLAIRE_OK;
}

// Adjoint solve (eq. adjoint) backward from lam(1) = m1 - m(1), then
// g = beta_v L v + [I - c P_par] sum_j w_j lam^j grad m^j  (eq. rgrad).
claire_status adjoint_and_gradient(claire_ctx* c) {
  NvtxRange nvtx_("claire.adjoint_gradient");
  const int64_t N = N_of(c);
  const Grid& g = c->g;
  if (c->lv_spectrum) {                            // L v of the point objective() evaluated
    const double fft_bytes = 3.0 * (4.0 * g.N + 8.0 * g.n1 * g.n2 * (g.n3 / 2 + 1));
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    CUFFT_TRY(c, cufftExecC2R(c->c2r, c->cbuf, (cufftReal*)c->Lv));
    c->lv_spectrum = false;
  } else {
    TRY(spectral(c, CLAIRE_OP_L, c->v, c->Lv, 1.0));
  }
  launch_trace(g, c->v, nullptr, c->db, ht_of(c), c->st);
  launch_div8(g, c->v, c->D, c->st);
  launch_adjoint_factor(g, c->D, c->db, ht_of(c), c->cf, c->st);
  if (c->opt.hessian == 1) {
    const float ht = ht_of(c);
    launch_affine(N, 0.5f * ht * ht, c->D, 0.5f * ht, c->ef, c->st);
  }
  if (mixed(c)) {                                  // FP16 history of sig_m lam
    launch_axpy_h(N, c->sig_m, c->m1, -1.0f, c->mh + c->nt * N, c->lh + c->nt * N, c->st);
    for (int j = c->nt - 1; j >= 0; --j)
      launch_sl_h(g, c->lh + (j + 1) * N, c->db, c->cf, 1.0f, nullptr, 0.0f, c->lh + j * N,
                  c->st);
  } else {
    if (c->opt.distance == 1) {                  // lam(1) = -d dist_NCC / d m(1)
      const double a = c->ncc_a, b = c->ncc_b, cc = c->ncc_c;
      launch_lincomb(N, (float)(2.0 * a / (b * cc)), c->m1, (float)(-2.0 * a * a / (b * cc * cc)),
                     c->mhist + c->nt * N, c->lhist + c->nt * N, c->st);
    } else {
      launch_lincomb(N, 1.0f, c->m1, -1.0f, c->mhist + c->nt * N, c->lhist + c->nt * N, c->st);
    }
    for (int j = c->nt - 1; j >= 0; --j)
      launch_sl(g, c->lhist + (j + 1) * N, c->db, c->cf, 1.0f, nullptr, 0.0f, c->lhist + j * N,
                c->st);
  }
  TRY(check_launch(c, "adjoint"));
  if (c->opt.beta_w > 0.0) {
    TRY(accumulate(c, c->lhist, c->lh, nullptr, 0.0f, c->grad, nullptr, nullptr, nullptr));
    TRY(project_data_term(c, c->grad));
    launch_axpby(3 * N, (float)c->beta_v, c->Lv, 1.0f, c->grad, c->st);
  } else {
    TRY(accumulate(c, c->lhist, c->lh, c->Lv, (float)c->beta_v, c->grad, nullptr, nullptr,
                   nullptr));
  }
  c->beta_eval = c->beta_v;
  return check_launch(c, "gradient");
}

// The stored evaluation at a new beta_v (continuation, Sec. 2.6): the state, the
// adjoint and the data term b do not depend on beta_v (beta_w = 0), so
// g = beta_v L v + b and J = dist + beta_v/2 h^3 <v, L v> change by the
// regulariser alone.
claire_status rebeta(claire_ctx* c) {
  const double h3 = (double)c->g.h1 * c->g.h2 * c->g.h3;
  launch_axpby(3 * N_of(c), (float)(c->beta_v - c->beta_eval), c->Lv, 1.0f, c->grad, c->st);
  c->J = c->dist + 0.5 * c->beta_v * h3 * c->vLv;
  c->beta_eval = c->beta_v;
  return check_launch(c, "rebeta");
}

// Full evaluation at c->v: trace, state, J, adjoint, g (Algorithm 1, lines 3-6).
claire_status evaluate(claire_ctx* c) {
  NvtxRange nvtx_("claire.evaluate");
  c->have_eval = false;
  launch_trace(c->g, c->v, c->df, nullptr, ht_of(c), c->st);
  TRY(check_launch(c, "trace"));
  TRY(state_solve(c, c->df));
  TRY(objective(c, c->v, &c->J));
  TRY(adjoint_and_gradient(c));
  c->have_eval = true;
  return CLAIRE_OK;
}

// Gauss-Newton H vt (eq. matvec with the lam terms dropped):
//  incremental state along +v with w^j = m~^j - (h_t/2) s^j, s^j = grad m^j . vt:
//    w^0 = -(h_t/2) s^0;  w^{j+1} = w^j(y_f) - h_t s^{j+1};  m~(1) = w^{nt-1}(y_f) - (h_t/2) s^nt
//  incremental adjoint from lam~(1) = -m~(1): lam~^j = c(x) lam~^{j+1}(y_b)
//  H vt = beta_v L vt + [I - c P_par] sum_j w_j lam~^j grad m^j.
claire_status matvec_transport(claire_ctx* c, const float* vt);

claire_status matvec(claire_ctx* c, const float* vt, float* Hvt) {
  NvtxRange nvtx_("claire.matvec");
  if (!c->have_eval)
    return fail(c, CLAIRE_EORDER, "hessian_matvec needs a prior objective_gradient");
  const int64_t N = N_of(c);
  const Grid& g = c->g;
  (void)g;
  const double* vmax = nullptr;
  if (mixed(c)) {                                  // scale of the FP16 incremental fields
    launch_reduce(3 * N, vt, nullptr, RED_ABSMAX, c->partial, c->red_blocks,
                  c->slots + SLOT_VMAX, c->st);
    vmax = c->slots + SLOT_VMAX;
  }
  TRY(matvec_transport(c, vt));
  TRY(spectral(c, CLAIRE_OP_L, vt, c->scr3, 1.0));
  if (c->opt.beta_w > 0.0) {
    TRY(accumulate(c, c->lthist, c->lth, nullptr, 0.0f, Hvt, vmax, nullptr, nullptr));
    TRY(accumulate_newton(c, Hvt, nullptr, nullptr));
    TRY(project_data_term(c, Hvt));
    TRY(spectral(c, CLAIRE_OP_L, vt, c->scr3, 1.0));
    launch_axpby(3 * N, (float)c->beta_v, c->scr3, 1.0f, Hvt, c->st);
  } else {
    TRY(accumulate(c, c->lthist, c->lth, c->scr3, (float)c->beta_v, Hvt, vmax, nullptr,
                   nullptr));
    TRY(accumulate_newton(c, Hvt, nullptr, nullptr));
  }
  return check_launch(c, "matvec accumulate");
}

// ---------------------------------------------------------------- Krylov / Newton

struct Counters {
  int pcg = 0, matvecs = 0, pde = 0, halvings = 0, inner = 0;
};

// Transport part of the Gauss-Newton matvec (incremental state and adjoint):
// fills lthist with lam~^j for direction vt (see matvec()).
claire_status matvec_transport(claire_ctx* c, const float* vt) {
  const int64_t N = N_of(c);
  const Grid& g = c->g;
  const float ht = ht_of(c);
  const int nt = c->nt;
  if (mixed(c)) {                // FP16 incremental fields scaled by sig_m 2^-ceil(log2 |vt|)
    if (!launch_sdot_hist_h(g, c->mh, nt, vt, -0.5f * ht, c->slots + SLOT_VMAX, c->sh, c->st))
      return fail(c, CLAIRE_EINVAL, "mixed precision needs nt in {1, 2, 4, 8}");
    const __half* src = c->sh;
    for (int j = 0; j < nt; ++j) {
      if (j < nt - 1) {
        __half* dst = (j % 2 == 0) ? c->ph0 : c->ph1;
        launch_sl_h(g, src, c->df, nullptr, 1.0f, c->sh + (j + 1) * N, -ht, dst, c->st);
        src = dst;
      } else {
        launch_sl_h(g, src, c->df, nullptr, -1.0f, c->sh + nt * N, 0.5f * ht, c->lth + nt * N,
                    c->st);
      }
    }
    for (int j = nt - 1; j >= 0; --j)
      launch_sl_h(g, c->lth + (j + 1) * N, c->db, c->cf, 1.0f, nullptr, 0.0f, c->lth + j * N,
                  c->st);
    return check_launch(c, "matvec transport");
  }
  const bool newton = c->opt.hessian == 1;
  launch_sdot_hist(g, c->mhist, nt, vt, -0.5f * ht, c->shist, c->st);
  const float* src = c->shist;                       // w^0
  for (int j = 0; j < nt; ++j) {
    if (j < nt - 1) {                                // full Newton keeps every w^j
      float* dst = newton ? c->mthist + (j + 1) * N : ((j % 2 == 0) ? c->pp0 : c->pp1);
      launch_sl(g, src, c->df, nullptr, 1.0f, c->shist + (j + 1) * N, -ht, dst, c->st);
      src = dst;
    } else {                                         // lam~(1) = -m~(1)
      launch_sl(g, src, c->df, nullptr, -1.0f, c->shist + nt * N, 0.5f * ht,
                c->lthist + nt * N, c->st);
    }
  }
  // Full Newton (eq. incadj with the lam terms): m~^0 = 0, m~^j = w^j + (h_t/2) s^j,
  // m~^nt = -(lthist^nt, which holds -m~(1) here)
  if (newton) {
    CUDA_TRY(c, cudaMemsetAsync(c->mthist, 0, N * sizeof(float), c->st));
    for (int j = 1; j < nt; ++j)
      launch_lincomb(N, 1.0f, c->mthist + j * N, 0.5f * ht, c->shist + j * N,
                     c->mthist + j * N, c->st);
    launch_lincomb(N, -1.0f, c->lthist + nt * N, 0.0f, c->lthist + nt * N, c->mthist + nt * N,
                   c->st);
  }
  if (c->opt.distance == 1) {                    // NCC: lam~(1) = -(d^2 dist)[m~(1)]
    const float* m = c->mhist + nt * N;
    float* lt = c->lthist + nt * N;
    launch_reduce(N, c->m1, lt, RED_DOT, c->partial, c->red_blocks, c->slots + SLOT_NCC_AL,
                  c->st);
    launch_reduce(N, m, lt, RED_DOT, c->partial, c->red_blocks, c->slots + SLOT_NCC_GA, c->st);
    launch_ncc_final(N, c->m1, m, lt, c->slots + SLOT_NCC_AL, c->slots + SLOT_NCC_GA, c->ncc_a,
                     c->ncc_b, c->ncc_c, (double)g.h1 * g.h2 * g.h3, c->st);
  }
  if (!newton) {
    for (int j = nt - 1; j >= 0; --j)
      launch_sl(g, c->lthist + (j + 1) * N, c->db, c->cf, 1.0f, nullptr, 0.0f,
                c->lthist + j * N, c->st);
    return check_launch(c, "matvec transport");
  }
  // sources q^j = div8(lam^j vt) (in shist, s no longer needed);
  // lam~^j(x) = c(x) lam~^{j+1}(y) + e(x) q^{j+1}(y) + (h_t/2) q^j(x), the RK2 step
  // of the paper with e = (h_t/2)(1 + h_t div v), as two SL launches.
  for (int j = 0; j <= nt; ++j) launch_div8_prod(g, c->lhist + j * N, vt, c->shist + j * N, c->st);
  for (int j = nt - 1; j >= 0; --j) {
    launch_sl(g, c->lthist + (j + 1) * N, c->db, c->cf, 1.0f, c->shist + j * N, 0.5f * ht,
              c->pp0, c->st);
    launch_sl(g, c->shist + (j + 1) * N, c->db, c->ef, 1.0f, c->pp0, 1.0f, c->lthist + j * N,
              c->st);
  }
  return check_launch(c, "matvec transport");
}

// ---------------------------------------------------------------- two-level preconditioner

claire_status tl_set_streams(claire_ctx* c);

// Coarse grid, cuFFT plans and buffers of the two-level preconditioner.
claire_status tl_setup(claire_ctx* c) {
  if (c->tl_ready) return CLAIRE_OK;
  const Grid& g = c->g;
  if (g.n1 % 4 || g.n2 % 4 || g.n3 % 4)
    return fail(c, CLAIRE_EINVAL, "two-level preconditioner needs every n_i %% 4 == 0");
  Grid& gc = c->gc;
  gc.n1 = g.n1 / 2; gc.n2 = g.n2 / 2; gc.n3 = g.n3 / 2;
  gc.N = (int64_t)gc.n1 * gc.n2 * gc.n3;
  const double tp = 2.0 * M_PI;
  gc.h1 = (float)(tp / gc.n1); gc.h2 = (float)(tp / gc.n2); gc.h3 = (float)(tp / gc.n3);
  gc.inv_h1 = (float)(gc.n1 / tp); gc.inv_h2 = (float)(gc.n2 / tp); gc.inv_h3 = (float)(gc.n3 / tp);
  const int64_t Nc = gc.N;
  const int64_t Ch = (int64_t)gc.n1 * gc.n2 * (gc.n3 / 2 + 1);
  const int64_t Nh = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  // (allocations and plans made by an earlier, failed call are kept)
  float** f3[] = {&c->tl_gm, &c->tl_q, &c->tl_w};
  for (auto p : f3)
    if (!*p) TRY(alloc(c, p, 3 * Nc));
  if (!c->tl_mc) TRY(alloc(c, &c->tl_mc, Nc));
  if (!c->tl_fw) {
    float* q = nullptr;
    TRY(alloc(c, &q, 2 * Ch));
    c->tl_fw = (float2*)q;
  }
  float* p = nullptr;
  cufftComplex** cc3[] = {&c->tl_cc, &c->tl_sx, &c->tl_sr, &c->tl_sp, &c->tl_sap};
  for (auto q : cc3)
    if (!*q) {
      TRY(alloc(c, &p, 3 * Ch * 2));
      *q = (cufftComplex*)p;
    }
  if (!c->cbuf2) {
    TRY(alloc(c, &p, 3 * Nh * 2));
    c->cbuf2 = (cufftComplex*)p;
  }
  if (!c->tl_count) {
    TRY(alloc(c, &p, 1));
    c->tl_count = reinterpret_cast<unsigned*>(p);
    CUDA_TRY(c, cudaMemsetAsync(c->tl_count, 0, sizeof(unsigned), c->st));
  }
  int nc[3] = {gc.n1, gc.n2, gc.n3};
  if ((!c->tl_r2c1 && cufftPlan3d(&c->tl_r2c1, g.n1, g.n2, g.n3, CUFFT_R2C) != CUFFT_SUCCESS) ||
      (!c->tl_c2r1 && cufftPlan3d(&c->tl_c2r1, gc.n1, gc.n2, gc.n3, CUFFT_C2R) != CUFFT_SUCCESS) ||
      (!c->tl_r2c3 && cufftPlanMany(&c->tl_r2c3, 3, nc, nullptr, 1, (int)Nc, nullptr, 1, (int)Ch,
                                    CUFFT_R2C, 3) != CUFFT_SUCCESS) ||
      (!c->tl_c2r3 && cufftPlanMany(&c->tl_c2r3, 3, nc, nullptr, 1, (int)Ch, nullptr, 1, (int)Nc,
                                    CUFFT_C2R, 3) != CUFFT_SUCCESS))
    return fail(c, CLAIRE_ECUDA, "cuFFT plans of the two-level preconditioner");
  CUDA_TRY(c, cudaMemsetAsync(c->slots + SLOT_ZERO, 0, 3 * sizeof(double), c->st));
  c->tl_ready = true;
  return tl_set_streams(c);
}

claire_status tl_set_streams(claire_ctx* c) {
  if (!c->tl_ready) return CLAIRE_OK;
  for (cufftHandle h : {c->tl_r2c1, c->tl_c2r1, c->tl_r2c3, c->tl_c2r3})
    CUFFT_TRY(c, cufftSetStream(h, c->st));
  return CLAIRE_OK;
}

// grad m_c: FD8 gradient of the spectral restriction of m(1) (the last state
// solve) on the coarse grid, the image of the zero-velocity Hessian H0.
claire_status tl_update_image(claire_ctx* c) {
  TRY(tl_setup(c));
  const Grid& g = c->g;
  const int64_t N = g.N;
  const float* m1p = c->mhist + (int64_t)c->nt * N;
  if (mixed(c)) {
    launch_tl_unscale_h(N, c->mh + (int64_t)c->nt * N, 1.0f / c->sig_m, c->scr3, c->st);
    m1p = c->scr3;
  }
  const double bytes = 4.0 * N + 8.0 * g.n1 * g.n2 * (g.n3 / 2 + 1);
  {
    ProfileRange pr(K_CUFFT, bytes, c->st);
    c->lv_spectrum = false;
    CUFFT_TRY(c, cufftExecR2C(c->tl_r2c1, (cufftReal*)m1p, c->cbuf));
  }
  const int64_t Ch = (int64_t)c->gc.n1 * c->gc.n2 * (c->gc.n3 / 2 + 1);
  CUDA_TRY(c, cudaMemsetAsync(c->tl_cc, 0, Ch * sizeof(cufftComplex), c->st));
  launch_tl_split(g, c->cbuf, c->tl_cc, 1, 0, 0.f, 0.f, (float)(1.0 / (double)N), c->st);
  {
    ProfileRange pr(K_CUFFT, bytes / 8, c->st);
    CUFFT_TRY(c, cufftExecC2R(c->tl_c2r1, c->tl_cc, (cufftReal*)c->tl_mc));
  }
  launch_grad8(c->gc, c->tl_mc, c->tl_gm, c->st);
  launch_tl_spec_table(c->gc, (float)c->beta_v, (float)c->gamma, c->tl_fw, c->st);
  if (c->opt.distance == 1) {
    // NCC: the pointwise part of d^2 dist / d m(1)^2 is 2 a^2 / (b c^2) times the identity
    const double w = 2.0 * c->ncc_a * c->ncc_a / (c->ncc_b * c->ncc_c * c->ncc_c);
    const int64_t n3c = 3 * c->gc.N;
    launch_lincomb(n3c, (float)std::sqrt(w), c->tl_gm, 0.0f, c->tl_gm, c->tl_gm, c->st);
  }
  TRY(check_launch(c, "two-level image"));
  c->tl_image = true;
  return CLAIRE_OK;
}

// z = R^-1/2 M^-1 R^-1/2 r and Lz = beta_v L z (Sec. 2.5.6): the low modes of
// R^-1/2 r are restricted to the coarse grid, where nested CG solves
// (I + R^-1/2 (grad m_c (x) grad m_c) R^-1/2) s_c = t_c; s_c is prolonged, the
// high modes are kept, and R^-1/2 is applied again.  With rz_slot >= 0, <r, z>
// goes to slots[rz_slot].
// The nested CG of the two-level preconditioner inside the graph being captured on
// c->st (options.graphs): k_tl_cg_begin sets the condition of a while node whose
// body is one CG iteration ending in k_tl_cg_control, so the loop runs on the
// device with the host loop's stopping decisions and no host round trip.  The
// residual slots keep fixed roles (rr in SLOT_TL_RR0, the new one in SLOT_TL_RR1,
// copied back by the control kernel); an iteration's direction update also runs
// after the last iteration, where p is no longer used.  The iterations of all
// applications since the PCG start add up in SLOT_TL_ITS.
claire_status tl_cg_graph(claire_ctx* c) {
  const Grid& gc = c->gc;
  const int64_t Ch = (int64_t)gc.n1 * gc.n2 * (gc.n3 / 2 + 1);
  const double fft_c = 3.0 * (4.0 * gc.N + 8.0 * Ch);
  const float inv_nc = (float)(1.0 / (double)gc.N);
  if (!c->tl_body) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->tl_body, cudaStreamNonBlocking));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CUDA_TRY(c, cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphConditionalHandle h;
  CUDA_TRY(c, cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
  double* sl = c->slots;
  launch_tl_cg_begin(h, sl + SLOT_TL_RR0, sl + SLOT_TL_RTOL, sl + SLOT_TL_STOP,
                     sl + SLOT_TL_COUNT, c->opt.max_inner, c->st);
  TRY(check_launch(c, "nested cg begin"));
  CUDA_TRY(c, cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CUDA_TRY(c, cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
  CUDA_TRY(c, cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const cudaStream_t bs = c->tl_body;
  Profiler* saved = tl_prof;
  Profiler counter;                                 // launches of one iteration
  tl_prof = &counter;
  CUDA_TRY(c, cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  auto iteration = [&]() -> claire_status {
    CUFFT_TRY(c, cufftSetStream(c->tl_c2r3, bs));
    CUFFT_TRY(c, cufftSetStream(c->tl_r2c3, bs));
    {
      ProfileRange pr(K_CUFFT, fft_c, bs);
      CUFFT_TRY(c, cufftExecC2R(c->tl_c2r3, c->tl_cc, (cufftReal*)c->tl_q));
    }
    launch_tl_outer(gc.N, c->tl_gm, c->tl_q, c->tl_w, bs);
    {
      ProfileRange pr(K_CUFFT, fft_c, bs);
      CUFFT_TRY(c, cufftExecR2C(c->tl_r2c3, (cufftReal*)c->tl_w, c->tl_cc));
    }
    launch_tl_spec_finish(gc, c->tl_fw, c->tl_sp, c->tl_cc, c->tl_sap, inv_nc, c->partial,
                          c->tl_count, sl + SLOT_TL_PAP, bs);
    launch_tl_spec_step(gc, c->tl_fw, sl + SLOT_TL_RR0, sl + SLOT_TL_PAP, c->tl_sx, c->tl_sr,
                        c->tl_sp, c->tl_sap, c->partial, c->tl_count, sl + SLOT_TL_RR1, bs);
    launch_tl_dir_scale(gc, c->tl_fw, sl + SLOT_TL_RR1, sl + SLOT_TL_RR0, c->tl_sr, c->tl_sp,
                        c->tl_cc, bs);
    launch_tl_cg_control(h, sl + SLOT_TL_RR0, sl + SLOT_TL_RR1, sl + SLOT_TL_PAP,
                         sl + SLOT_TL_STOP, sl + SLOT_TL_COUNT, sl + SLOT_TL_ITS,
                         c->opt.max_inner, bs);
    return check_launch(c, "nested cg body");
  };
  claire_status s = iteration();
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(bs, &captured);
  tl_prof = saved;
  const claire_status s2 = tl_set_streams(c);      // the plans back on c->st
  if (s != CLAIRE_OK) return s;
  if (e != cudaSuccess)
    return fail(c, CLAIRE_ECUDA, "nested cg body capture: %s", cudaGetErrorString(e));
  if (s2 != CLAIRE_OK) return s2;
  for (int k = 0; k < K_COUNT; ++k) {
    c->tl_body_launches[k] = counter.launches[k];
    c->tl_body_bytes[k] = counter.bytes[k];
  }
  return CLAIRE_OK;
}

claire_status tl_precondition(claire_ctx* c, const float* r, float* z, float* Lz, int rz_slot) {
  NvtxRange nvtx_("claire.two_level_precondition");
  TRY(tl_setup(c));
  if (!c->tl_image) return fail(c, CLAIRE_EORDER, "two-level preconditioner has no image");
  const Grid& g = c->g;
  const Grid& gc = c->gc;
  const int64_t N = g.N;
  const int64_t Ch = (int64_t)gc.n1 * gc.n2 * (gc.n3 / 2 + 1);
  const double fft_f = 3.0 * (4.0 * N + 8.0 * g.n1 * g.n2 * (g.n3 / 2 + 1));
  const double fft_c = 3.0 * (4.0 * gc.N + 8.0 * Ch);
  const float alpha = (float)c->beta_v, gamma = (float)c->gamma;
  {
    ProfileRange pr(K_CUFFT, fft_f, c->st);
    c->lv_spectrum = false;
    CUFFT_TRY(c, cufftExecR2C(c->r2c, (cufftReal*)r, c->cbuf));
  }
  // right-hand side: the low modes of R^-1/2 r as a coarse spectrum (C2R normalisation)
  CUDA_TRY(c, cudaMemsetAsync(c->tl_cc, 0, 3 * Ch * sizeof(cufftComplex), c->st));
  launch_tl_split(g, c->cbuf, c->tl_cc, 3, 1, alpha, gamma, (float)(1.0 / (double)N), c->st);
  // nested CG on the coarse spectra: x = 0, r = p = b; device scalars, one host
  // read per iteration; two coarse FFTs per operator application
  int cur = SLOT_TL_RR0, nxt = SLOT_TL_RR1;
  launch_tl_spec_init(gc, c->tl_fw, c->tl_cc, c->tl_sx, c->tl_sr, c->tl_sp, c->partial,
                      c->tl_count, c->slots + cur, c->st);
  TRY(check_launch(c, "nested cg"));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CUDA_TRY(c, cudaStreamIsCapturing(c->st, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    TRY(tl_cg_graph(c));
  } else {
  CUDA_TRY(c, cudaMemcpyAsync(c->hres, c->slots + cur, sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  double rr = c->hres[0];
  const double stop2 = c->tl_rtol * c->tl_rtol * rr;
  const float inv_nc = (float)(1.0 / (double)gc.N);
  int it = 0;
  while (it < c->opt.max_inner && rr > stop2 && std::isfinite(rr)) {
    // A p = p + R^-1/2 (grad m_c (grad m_c . R^-1/2 p)) with R^-1/2 diagonal in k;
    // tl_cc holds R^-1/2 p (from the initialisation or the last direction update)
    {
      ProfileRange pr(K_CUFFT, fft_c, c->st);
      CUFFT_TRY(c, cufftExecC2R(c->tl_c2r3, c->tl_cc, (cufftReal*)c->tl_q));
    }
    launch_tl_outer(gc.N, c->tl_gm, c->tl_q, c->tl_w, c->st);
    {
      ProfileRange pr(K_CUFFT, fft_c, c->st);
      CUFFT_TRY(c, cufftExecR2C(c->tl_r2c3, (cufftReal*)c->tl_w, c->tl_cc));
    }
    launch_tl_spec_finish(gc, c->tl_fw, c->tl_sp, c->tl_cc, c->tl_sap, inv_nc, c->partial,
                          c->tl_count, c->slots + SLOT_TL_PAP, c->st);
    launch_tl_spec_step(gc, c->tl_fw, c->slots + cur, c->slots + SLOT_TL_PAP, c->tl_sx,
                        c->tl_sr, c->tl_sp, c->tl_sap, c->partial, c->tl_count, c->slots + nxt,
                        c->st);
    TRY(check_launch(c, "nested cg"));
    CUDA_TRY(c, cudaMemcpyAsync(c->hres, c->slots + SLOT_TL_RR0, 3 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    ++it;
    const double pAp = c->hres[SLOT_TL_PAP - SLOT_TL_RR0];
    if (!(pAp > 0.0) || !std::isfinite(pAp)) break;   // x, r unchanged by this step
    rr = c->hres[nxt - SLOT_TL_RR0];
    if (rr <= stop2) break;
    launch_tl_dir_scale(gc, c->tl_fw, c->slots + nxt, c->slots + cur, c->tl_sr, c->tl_sp,
                        c->tl_cc, c->st);
    std::swap(cur, nxt);
  }
  c->tl_iters += it;
  }
  // prolong the coarse solution (already a spectrum), keep the high modes, R^-1/2
  launch_tl_merge(g, c->cbuf, c->tl_sx, c->cbuf2, alpha, gamma, (float)(1.0 / (double)N), 1.0f,
                  c->st);
  {
    ProfileRange pr(K_CUFFT, 2 * fft_f, c->st);
    CUFFT_TRY(c, cufftExecC2R(c->c2r, c->cbuf, (cufftReal*)z));
    CUFFT_TRY(c, cufftExecC2R(c->c2r, c->cbuf2, (cufftReal*)Lz));
  }
  if (rz_slot >= 0)
    launch_reduce(3 * N, r, z, RED_DOT, c->partial, c->red_blocks, c->slots + rz_slot, c->st);
  return check_launch(c, "two-level preconditioner");
}

// z = M^-1 r with M = beta_v L (zero symbol set to one); <r, z> by Parseval into
// slots[rz_slot] and the component means of r into slots[SLOT_MEAN..+2].
// With options.precond = 1 the two-level preconditioner instead, with
// beta_v L z in scr3.
claire_status precondition(claire_ctx* c, int rz_slot) {
  if (two_level(c)) return tl_precondition(c, c->r, c->z, c->scr3, rz_slot);
  const double fft_bytes = 3.0 * (4.0 * c->g.N + 8.0 * c->g.n1 * c->g.n2 * (c->g.n3 / 2 + 1));
  {
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    c->lv_spectrum = false;
    CUFFT_TRY(c, cufftExecR2C(c->r2c, (cufftReal*)c->r, c->cbuf));
  }
  launch_spectral(c->g, c->cbuf, CLAIRE_OP_REG_INV, (float)c->beta_v, (float)c->gamma,
                  (float)c->opt.beta_w, c->st, c->partial, c->slots + SLOT_MEAN);
  launch_reduce_final(c->partial, spectral_blocks(c->g), RED_SUM, c->slots + rz_slot, c->st);
  TRY(check_launch(c, "precondition"));
  {
    ProfileRange pr(K_CUFFT, fft_bytes, c->st);
    CUFFT_TRY(c, cufftExecC2R(c->c2r, c->cbuf, (cufftReal*)c->z));
  }
  return CLAIRE_OK;
}

// Algorithm 2: PCG for H vt = -g from vt = 0 with M = beta_v L (zero symbol -> 1).
// The scalars kappa and mu stay on the device (FP64 slots); the regularisation
// part of H s is carried by the recurrence beta_v L s = (r - mean r) + mu beta_v L s,
// so each iteration costs one FFT pair (the preconditioner) besides the
// transport solves.  One host synchronisation per iteration reads <s, H s> and
// ||r||^2 for the curvature and stopping tests.
// One PCG iteration is two launch sequences around the host check:
//  part A (slot parity cur): H s (transport solves + accumulation with <s, H s>),
//          the kappa update of vt and r with ||r||^2, and the copy of the FP64
//          slots to pinned host memory;
//  part B (cur -> nxt): z = M^-1 r with <r, z>, the mu update of s and beta_v L s
//          (and ||s||_inf for the FP16 scale in mixed precision).
claire_status pcg_part_a(claire_ctx* c, int cur) {
  const int64_t n3 = 3 * N_of(c);
  const Grid& g = c->g;
  const double* vmax = mixed(c) ? c->slots + SLOT_VMAX : nullptr;
  TRY(matvec_transport(c, c->s));
  const bool newton = c->opt.hessian == 1;
  if (c->opt.beta_w <= 0.0 && march_supported(c->nt)) {
    // <s, H s> fused into the last accumulation
    TRY(accumulate(c, c->lthist, c->lth, c->hs, 1.0f, c->Hs, vmax, newton ? nullptr : c->s,
                   newton ? nullptr : c->partial));
    TRY(accumulate_newton(c, c->Hs, c->s, c->partial));
    launch_reduce_final(c->partial, march_blocks(g), RED_SUM, c->slots + SLOT_SHS, c->st);
  } else {
    TRY(accumulate(c, c->lthist, c->lth, nullptr, 0.0f, c->Hs, vmax, nullptr, nullptr));
    TRY(accumulate_newton(c, c->Hs, nullptr, nullptr));
    TRY(project_data_term(c, c->Hs));
    launch_axpby(n3, 1.0f, c->hs, 1.0f, c->Hs, c->st);
    launch_reduce(n3, c->s, c->Hs, RED_DOT, c->partial, c->red_blocks, c->slots + SLOT_SHS,
                  c->st);
  }
  const int vb = vector_blocks(n3 / 4);
  launch_pcg_update(n3, c->slots + cur, c->slots + SLOT_SHS, c->vt, c->r, c->s, c->Hs,
                    c->partial, vb, c->dflag, c->st);
  launch_reduce_final(c->partial, vb, RED_SUM, c->slots + SLOT_RR, c->st);
  TRY(check_launch(c, "pcg update"));
  CUDA_TRY(c, cudaMemcpyAsync(c->hslots, c->slots, NSLOTS * sizeof(double) + sizeof(int),
                              cudaMemcpyDeviceToHost, c->st));
  return CLAIRE_OK;
}

// beta_v L z for the recurrence of beta_v L s: r - mean(r) for the spectral
// preconditioner, the field computed with z for the two-level one.
const float* lz_source(const claire_ctx* c) { return two_level(c) ? c->scr3 : c->r; }
const double* lz_means(const claire_ctx* c) {
  return c->slots + (two_level(c) ? SLOT_ZERO : SLOT_MEAN);
}

claire_status pcg_part_b(claire_ctx* c, int cur, int nxt) {
  const int64_t N = N_of(c);
  TRY(precondition(c, nxt));
  launch_s_update(N, c->slots + nxt, c->slots + cur, lz_means(c), 0, c->z, lz_source(c), c->s,
                  c->hs, c->st);
  if (mixed(c))
    launch_reduce(3 * N, c->s, nullptr, RED_ABSMAX, c->partial, c->red_blocks,
                  c->slots + SLOT_VMAX, c->st);
  return check_launch(c, "pcg part b");
}

void drop_graphs(claire_ctx* c) {
  for (auto& e : c->graph_exec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
}

claire_status pcg_start(claire_ctx* c);

// Run part A (which = 0) or B (which = 1) for parity p, or the PCG start S
// (which = 2), as a captured CUDA graph when options.graphs is set (captured on
// first use; the kernels inside are counted per replay, not event-timed).
claire_status pcg_part(claire_ctx* c, int which, int cur, int nxt) {
  // with the two-level preconditioner parts S and B hold the nested CG as a
  // conditional while node; if that capture is refused, they run launch by launch
  NvtxRange nvtx_(which == 0 ? "claire.pcg.matvec" : which == 1 ? "claire.pcg.precondition"
                                                    : "claire.pcg.start");
  auto run = [&]() {
    return which == 0 ? pcg_part_a(c, cur) : which == 1 ? pcg_part_b(c, cur, nxt)
                                                        : pcg_start(c);
  };
  if (!c->opt.graphs || (which != 0 && two_level(c) && c->tl_nograph)) return run();
  const int slot = which == 2 ? 8
                              : 4 * (c->df == c->dbuf0 ? 0 : 1) + 2 * which +
                                    (cur == SLOT_RZ0 ? 0 : 1);
  if (!c->graph_exec[slot]) {
    Profiler* saved = tl_prof;
    Profiler counter;                               // counts the captured launches
    tl_prof = &counter;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    claire_status s = run();
    cudaError_t e = cudaStreamEndCapture(c->st, &graph);
    tl_prof = saved;
    if (s == CLAIRE_OK && e == cudaSuccess) {
      e = cudaGraphInstantiate(&c->graph_exec[slot], graph, 0);
      if (e != cudaSuccess) c->graph_exec[slot] = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    if (which != 0 && two_level(c) && (s != CLAIRE_OK || e != cudaSuccess)) {
      // nothing of the failed capture ran: run this part (and later ones) uncaptured
      cudaGetLastError();
      if (c->opt.verbose)
        fprintf(stderr, "[claire] nested CG not captured (%s); PCG parts S and B run uncaptured\n",
                c->err.empty() ? cudaGetErrorString(e) : c->err.c_str());
      c->err.clear();
      c->tl_nograph = true;
      return run();
    }
    if (s != CLAIRE_OK) return s;
    if (e != cudaSuccess) return fail(c, CLAIRE_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    for (int k = 0; k < K_COUNT; ++k) {
      c->graph_launches[slot][k] = counter.launches[k];
      c->graph_bytes[slot][k] = counter.bytes[k];
    }
  }
  if (tl_prof)
    for (int k = 0; k < K_COUNT; ++k) {
      tl_prof->launches[k] += c->graph_launches[slot][k];
      tl_prof->bytes[k] += c->graph_bytes[slot][k];
    }
  CUDA_TRY(c, cudaGraphLaunch(c->graph_exec[slot], c->st));
  return CLAIRE_OK;
}

// Algorithm 2: PCG for H vt = -g from vt = 0 with M = beta_v L (zero symbol -> 1).
// The scalars kappa and mu stay on the device (FP64 slots); the regularisation
// part of H s is carried by the recurrence beta_v L s = (r - mean r) + mu beta_v L s,
// so each iteration costs one FFT pair (the preconditioner) besides the
// transport solves.  One host synchronisation per iteration reads <s, H s> and
// ||r||^2 for the curvature and stopping tests.
// Part S, the start of PCG: vt = 0, r = -g, z = M^-1 r with <r, z>, s = z and
// beta_v L s (and ||s||_inf in mixed precision).
claire_status pcg_start(claire_ctx* c) {
  const int64_t N = N_of(c);
  const int64_t n3 = 3 * N;
  CUDA_TRY(c, cudaMemsetAsync(c->vt, 0, n3 * sizeof(float), c->st));
  CUDA_TRY(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
  CUDA_TRY(c, cudaMemsetAsync(c->slots + SLOT_TL_ITS, 0, sizeof(double), c->st));
  launch_lincomb(n3, -1.0f, c->grad, 0.0f, c->grad, c->r, c->st);    // r = -g
  TRY(precondition(c, SLOT_RZ0));
  launch_s_update(N, c->slots + SLOT_RZ0, c->slots + SLOT_RZ0, lz_means(c), 1, c->z,
                  lz_source(c), c->s, c->hs, c->st);
  if (mixed(c))
    launch_reduce(n3, c->s, nullptr, RED_ABSMAX, c->partial, c->red_blocks,
                  c->slots + SLOT_VMAX, c->st);
  return check_launch(c, "pcg start");
}

claire_status pcg(claire_ctx* c, double tol, Counters& k, claire_status* curv) {
  NvtxRange nvtx_("claire.pcg");
  const int64_t N = N_of(c);
  const int64_t n3 = 3 * N;
  *curv = CLAIRE_OK;
  // nested CG iterations run by captured part-B graphs (a running total on the
  // device): read with the slots after each part A, as every part B is followed
  // by one, and counted with their launches
  int graph_its = 0;
  auto graph_inner = [&]() {
    const int its = (int)c->hslots[SLOT_TL_ITS] - graph_its;
    graph_its += its;
    c->tl_iters += its;
    if (tl_prof)
      for (int kk = 0; kk < K_COUNT; ++kk) {
        tl_prof->launches[kk] += (long long)its * c->tl_body_launches[kk];
        tl_prof->bytes[kk] += its * c->tl_body_bytes[kk];
      }
  };
  int cur = SLOT_RZ0;
  TRY(pcg_part(c, 2, cur, cur));
  for (int it = 1; it <= c->opt.max_pcg; ++it) {
    const int nxt = cur == SLOT_RZ0 ? SLOT_RZ1 : SLOT_RZ0;
    TRY(pcg_part(c, 0, cur, nxt));
    ++k.matvecs;
    k.pde += 2;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    const double sHs = c->hslots[SLOT_SHS], rr = c->hslots[SLOT_RR];
    const int flag = *(const int*)(c->hslots + NSLOTS);
    graph_inner();
    if (flag) {
      if (!std::isfinite(sHs) || !std::isfinite(c->hslots[cur]))
        return fail(c, CLAIRE_ENONFINITE, "PCG scalar not finite");
      *curv = CLAIRE_ENEGCURV;                     // negative curvature (Sec. 2.5.5)
      if (it == 1)
        CUDA_TRY(c, cudaMemcpyAsync(c->vt, c->s, n3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                    c->st));
      return CLAIRE_OK;
    }
    ++k.pcg;
    if (!c->opt.fixed_iters && std::sqrt(rr) < tol) break;
    if (it == c->opt.max_pcg) break;
    TRY(pcg_part(c, 1, cur, nxt));
    cur = nxt;
  }
  return check_launch(c, "pcg");
}

// Armijo backtracking (reading C-9) on J(v + gamma vt); on success the state
// history, departure points and L v belong to the accepted point.
claire_status armijo(claire_ctx* c, Counters& k, double* gamma_out, bool* ok) {
  NvtxRange nvtx_("claire.armijo");
  const int64_t n3 = 3 * N_of(c);
  const double h3 = (double)c->g.h1 * c->g.h2 * c->g.h3;
  double gv = 0.0;
  TRY(dot3(c, c->grad, c->vt, &gv));
  const double slope = h3 * gv;
  const double J0 = c->J;
  double gamma = 1.0;
  *ok = false;
  c->have_eval = false;
  for (int h = 0; h <= 10; ++h) {
    launch_lincomb(n3, 1.0f, c->v, (float)gamma, c->vt, c->vtrial, c->st);
    launch_trace(c->g, c->vtrial, c->dtrial, nullptr, ht_of(c), c->st);
    TRY(check_launch(c, "armijo trace"));
    TRY(state_solve(c, c->dtrial));
    ++k.pde;
    double Jt = 0.0;
    claire_status s = objective(c, c->vtrial, &Jt);
    if (s != CLAIRE_OK && s != CLAIRE_ENONFINITE) return s;
    if (s == CLAIRE_OK && Jt <= J0 + 1e-4 * gamma * slope) {
      std::swap(c->v, c->vtrial);
      std::swap(c->df, c->dtrial);
      c->J = Jt;
      *gamma_out = gamma;
      *ok = true;
      k.halvings += h;
      return CLAIRE_OK;
    }
    gamma *= 0.5;
  }
  k.halvings += 10;
  return CLAIRE_OK;
}

claire_status absmax3(claire_ctx* c, const float* a, double* out) {
  return reduce(c, 3 * N_of(c), a, nullptr, RED_ABSMAX, out);
}

// Autotuner: time each compiled tile shape on this context's own grid and
// buffers (the state history and departure points of the current evaluation)
// with CUDA events, keep the fastest.  For the SL steps the three gather
// variants (64 shared loads per node from a TMA-staged or a cp.async-staged
// brick, register window) at brick depths 4, 8, 16 along x1; planes per CTA
// for the FD8 history kernels (8, 16, 32, 64).
claire_status autotune(claire_ctx* c) {
  if (!c->have_eval) return fail(c, CLAIRE_EORDER, "autotune needs an evaluated state");
  const int64_t N = N_of(c);
  cudaEvent_t a = c->e0, b = c->e1;
  auto time_it = [&](auto&& fn, float* ms) -> claire_status {
    fn();                                           // warm-up (and attribute setup)
    CUDA_TRY(c, cudaEventRecord(a, c->st));
    for (int r = 0; r < 3; ++r) fn();
    CUDA_TRY(c, cudaEventRecord(b, c->st));
    CUDA_TRY(c, cudaEventSynchronize(b));
    CUDA_TRY(c, cudaEventElapsedTime(ms, a, b));
    return check_launch(c, "autotune");
  };
  Profiler* saved = tl_prof;
  tl_prof = nullptr;                                // tuning launches are not counted
  LaunchGroup* saved_group = tl_group;
  tl_group = nullptr;                               // timed on the context's own stream
  struct Restore {
    LaunchGroup* g;
    ~Restore() { tl_group = g; }
  } restore_group{saved_group};
  float best = 1e30f;
  Tuning t = c->tune;
  for (int variant = 0; variant < 9; ++variant) {
    const int t1 = 4 << (variant % 3);
    c->tune.sl_gather = variant / 3;
    c->tune.sl_t1 = t1;
    float ms = 0.f;
    claire_status s = mixed(c)
        ? time_it([&] { launch_sl_h(c->g, c->mh, c->df, nullptr, 1.f, nullptr, 0.f, c->ph0,
                                    c->st); }, &ms)
        : time_it([&] { launch_sl(c->g, c->mhist, c->df, nullptr, 1.f, nullptr, 0.f, c->pp0,
                                  c->st); }, &ms);
    if (s != CLAIRE_OK) { tl_prof = saved; return s; }
    if (ms < best) { best = ms; t.sl_t1 = t1; t.sl_gather = c->tune.sl_gather; }
  }
  c->tune.sl_t1 = t.sl_t1;
  c->tune.sl_gather = t.sl_gather;
  best = 1e30f;
  if (march_supported(c->nt)) {
    for (int m1 : {8, 16, 32, 64}) {
      c->tune.march_t1 = m1;
      float ms = 0.f;
      claire_status s = time_it([&] { (void)accumulate(c, c->lhist, c->lh, c->Lv, 1.0f, c->scr3,
                                                       nullptr, nullptr, nullptr); }, &ms);
      if (s != CLAIRE_OK) { tl_prof = saved; return s; }
      if (ms < best) { best = ms; t.march_t1 = m1; }
    }
  }
  c->tune = t;
  c->tuned = true;
  tl_prof = saved;
  (void)N;
  return CLAIRE_OK;
}

// Algorithm 1 from the iterate in c->v; gnorm0 > 0 fixes the relative-gradient
// denominator (reading C-10), else ||g(v = 0)||_inf is computed first.
claire_status detf_stats(claire_ctx* c, const float* v, double* mmm, float* det_out);

claire_status gauss_newton(claire_ctx* c, double gnorm0, Counters& k, claire_stats* out) {
  NvtxRange nvtx_("claire.gauss_newton");
  const int64_t n3 = 3 * N_of(c);
  double vmax = 0.0;
  TRY(absmax3(c, c->v, &vmax));
  if (gnorm0 <= 0.0 && vmax > 0.0) {
    // g(v = 0) has no regularisation term: evaluate at zero once for the denominator
    CUDA_TRY(c, cudaMemcpyAsync(c->vtrial, c->v, n3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                c->st));
    CUDA_TRY(c, cudaMemsetAsync(c->v, 0, n3 * sizeof(float), c->st));
    TRY(evaluate(c));
    k.pde += 2;
    TRY(absmax3(c, c->grad, &gnorm0));
    std::swap(c->v, c->vtrial);
    c->have_eval = false;                          // the evaluation belongs to v = 0
  }
  if (c->have_eval && c->opt.beta_w <= 0.0) {
    // continuation: the previous level ended evaluated at this v
    if (c->beta_eval != c->beta_v) TRY(rebeta(c));
  } else {
    TRY(evaluate(c));
    k.pde += 2;
  }
  if (c->opt.autotune && !c->tuned) TRY(autotune(c));
  double gn = 0.0;
  TRY(absmax3(c, c->grad, &gn));
  if (!std::isfinite(gn)) return fail(c, CLAIRE_ENONFINITE, "gradient is not finite");
  if (gnorm0 <= 0.0) gnorm0 = gn;
  if (out->newton_iters == 0 && out->J0 == 0.0) out->J0 = c->J;
  out->gnorm0 = gnorm0;
  claire_status result = CLAIRE_OK;
  int iters = 0;
  while (iters < c->opt.max_newton) {
    if (!c->opt.fixed_iters && (gn <= c->opt.eps_opt * gnorm0 || gn <= 1e-6)) break;
    NvtxRange nvtx_it("claire.newton_iteration");
    const double ratio = gn / gnorm0;
    const double eta = std::fmin(0.5, c->opt.forcing == 0 ? std::sqrt(ratio) : ratio);
    double gg = 0.0;
    TRY(dot3(c, c->grad, c->grad, &gg));
    claire_status curv = CLAIRE_OK;
    if (two_level(c)) {
      // H0 at the current m(1); nested tolerance a tenth of the outer one (Sec. 2.6)
      TRY(tl_update_image(c));
      c->tl_rtol = c->opt.inner_rtol > 0.0 ? c->opt.inner_rtol : 0.1 * eta;
      launch_set_scalar(c->slots + SLOT_TL_RTOL, c->tl_rtol, c->st);   // for captured parts
      c->tl_iters = 0;
    }
    TRY(pcg(c, eta * std::sqrt(gg), k, &curv));
    k.inner += c->tl_iters;
    c->tl_iters = 0;
    double gamma = 0.0;
    bool ok = false;
    TRY(armijo(c, k, &gamma, &ok));
    if (!ok) {
      result = fail(c, CLAIRE_ELINESEARCH, "Armijo line search failed after 10 halvings");
      // restore the stored evaluation at the last accepted v
      TRY(evaluate(c));
      k.pde += 2;
      break;
    }
    TRY(adjoint_and_gradient(c));
    ++k.pde;
    c->have_eval = true;
    ++iters;
    ++out->newton_iters;
    TRY(absmax3(c, c->grad, &gn));
    if (!std::isfinite(gn)) return fail(c, CLAIRE_ENONFINITE, "gradient is not finite");
    if (c->opt.verbose)
      fprintf(stderr, "[claire] beta_v %.3e  it %2d  J %.6e  |g|/|g0| %.3e  pcg %d  step %.3g\n",
              c->beta_v, out->newton_iters, c->J, gn / gnorm0, k.pcg, gamma);
  }
  out->J = c->J;
  out->grad_rel = gn / gnorm0;
  if (result == CLAIRE_OK && !c->opt.fixed_iters && gn > c->opt.eps_opt * gnorm0 && gn > 1e-6)
    result = fail(c, CLAIRE_ENOTCONV, "max_newton reached at relative gradient %.3e",
                  gn / gnorm0);
  return result;
}

bool valid_dims(int nx, int ny, int nz) {
  auto ok = [](int n) { return n >= 16 && n % 2 == 0; };
  if (!ok(nx) || !ok(ny) || !ok(nz)) return false;
  const double N = (double)nx * ny * nz;
  return 3.0 * N < 2147483647.0;
}

// The distance of the template, dist(m0, m1): J at v = 0, where m(1) = m0 and the
// regulariser vanishes (eq. varopt-claire; the NCC form of the Appendix).
claire_status distance_at_zero(claire_ctx* c, double* out) {
  const int64_t N = N_of(c);
  *out = 0.0;
  if (c->opt.distance == 1) {
    double a = 0.0, b = 0.0, cc = 0.0;
    TRY(reduce(c, N, c->m0, c->m1, RED_DOT, &a));
    TRY(reduce(c, N, c->m1, nullptr, RED_SQ, &b));
    TRY(reduce(c, N, c->m0, nullptr, RED_SQ, &cc));
    if (b > 0.0 && cc > 0.0) *out = 1.0 - a * a / (b * cc);
    return CLAIRE_OK;
  }
  double sq = 0.0;
  TRY(reduce(c, N, c->m0, c->m1, RED_SQDIFF, &sq));
  *out = 0.5 * (double)c->g.h1 * c->g.h2 * c->g.h3 * sq;
  return CLAIRE_OK;
}

// options.warm_check: keep a nonzero initial guess only if J(v0) <= J(0).  The
// state solve and J at v0 come first; an accepted guess then gets its adjoint
// and gradient, which the first Gauss-Newton level reuses as its evaluation.
// Without a given denominator the evaluation at v = 0 provides both
// ||g(0)||_inf and J(0).
static claire_status warm_start_check(claire_ctx* c, double* gnorm0, Counters& k,
                                      claire_stats* out) {
  double vmax = 0.0;
  TRY(absmax3(c, c->v, &vmax));
  if (vmax == 0.0) return CLAIRE_OK;
  double J0 = 0.0;
  if (*gnorm0 <= 0.0) {
    const size_t b3 = 3 * N_of(c) * sizeof(float);
    CUDA_TRY(c, cudaMemcpyAsync(c->vtrial, c->v, b3, cudaMemcpyDeviceToDevice, c->st));
    CUDA_TRY(c, cudaMemsetAsync(c->v, 0, b3, c->st));
    TRY(evaluate(c));
    k.pde += 2;
    TRY(absmax3(c, c->grad, gnorm0));
    J0 = c->J;
    std::swap(c->v, c->vtrial);
    c->have_eval = false;
  } else {
    TRY(distance_at_zero(c, &J0));
  }
  launch_trace(c->g, c->v, c->df, nullptr, ht_of(c), c->st);
  TRY(check_launch(c, "trace"));
  TRY(state_solve(c, c->df));
  TRY(objective(c, c->v, &c->J));
  ++k.pde;
  if (c->J > J0) {                                 // the guess raises the objective
    CUDA_TRY(c, cudaMemsetAsync(c->v, 0, 3 * N_of(c) * sizeof(float), c->st));
    out->warm_fallback = 1;
    return CLAIRE_OK;
  }
  TRY(adjoint_and_gradient(c));
  ++k.pde;
  c->have_eval = true;
  return CLAIRE_OK;
}

claire_status finish_stats(claire_ctx* c, claire_stats* st, const Counters& k, float ms,
                           claire_status s) {
  if (!st) return s;
  st->pcg_iters = k.pcg;
  st->matvecs = k.matvecs;
  st->pde_solves = k.pde;
  st->linesearch_halvings = k.halvings;
  st->inner_iters = k.inner;
  double mis0 = 0.0;
  if (distance_at_zero(c, &mis0) == CLAIRE_OK && mis0 > 0.0) st->mismatch_rel = c->dist / mis0;
  st->seconds = ms * 1e-3;
  st->status = (int)s;
  return s;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

claire_status claire_default_options(claire_options* o) {
  if (!o) return CLAIRE_EINVAL;
  memset(o, 0, sizeof *o);
  o->precision = 0;
  o->hessian = 0;
  o->beta_w = 0.0;
  o->eps_opt = 5e-2;
  o->max_newton = 50;
  o->max_pcg = 100;
  o->fixed_iters = 0;
  o->forcing = 0;
  o->stream = nullptr;
  o->verbose = 0;
  o->precond = 2;
  o->max_inner = 50;
  o->inner_rtol = 0.0;
  o->distance = 0;
  o->warm_check = 0;
  o->gnorm0 = 0.0;
  o->autotune = 0;
  o->graphs = 0;
  return CLAIRE_OK;
}

claire_status claire_destroy(claire_ctx* c) {
  if (!c) return CLAIRE_OK;
  c->prof.release();
  drop_graphs(c);
  if (c->own) cudaStreamDestroy(c->own);
  if (c->tl_body) cudaStreamDestroy(c->tl_body);
  if (c->plans) {
    cufftDestroy(c->r2c);
    cufftDestroy(c->c2r);
  }
  for (cufftHandle h : {c->tl_r2c1, c->tl_c2r1, c->tl_r2c3, c->tl_c2r3})
    if (h) cufftDestroy(h);
  for (void* p : c->allocs) cudaFree(p);
  if (c->detf) cudaFree(c->detf);
  if (c->hres) cudaFreeHost(c->hres);
  if (c->hslots) cudaFreeHost(c->hslots);
  if (c->e0) cudaEventDestroy(c->e0);
  if (c->e1) cudaEventDestroy(c->e1);
  if (c->e_in) cudaEventDestroy(c->e_in);
  delete c;
  return CLAIRE_OK;
}

claire_status claire_create(int nx, int ny, int nz, int nt, double beta_v, double gamma,
                            claire_ctx** out) {
  if (!out) return CLAIRE_EINVAL;
  *out = nullptr;
  if (!valid_dims(nx, ny, nz) || nt < 1 || nt > 256 || !(beta_v > 0.0) || !(gamma > 0.0))
    return CLAIRE_EINVAL;
  claire_ctx* c = new claire_ctx();
  claire_default_options(&c->opt);
  Grid& g = c->g;
  g.n1 = nx; g.n2 = ny; g.n3 = nz;
  g.N = (int64_t)nx * ny * nz;
  const double tp = 2.0 * M_PI;
  g.h1 = (float)(tp / nx); g.h2 = (float)(tp / ny); g.h3 = (float)(tp / nz);
  g.inv_h1 = (float)(nx / tp); g.inv_h2 = (float)(ny / tp); g.inv_h3 = (float)(nz / tp);
  c->nt = nt;
  c->beta_v = beta_v;
  c->gamma = gamma;
  c->tune.march_t1 = default_march_t1(g);
  const int64_t N = g.N;
  claire_status s = CLAIRE_OK;
  float** fields1[] = {&c->m0, &c->m1, &c->D, &c->cf, &c->pp0, &c->pp1};
  float** fields3[] = {&c->v, &c->df, &c->db, &c->grad, &c->Lv, &c->scr3, &c->vt, &c->r,
                       &c->z, &c->s, &c->Hs, &c->hs, &c->vtrial, &c->dtrial};
  for (auto p : fields1) if (s == CLAIRE_OK) s = alloc(c, p, N);
  for (auto p : fields3) if (s == CLAIRE_OK) s = alloc(c, p, 3 * N);
  c->dbuf0 = c->df;
  const int64_t Nc = (int64_t)nx * ny * (nz / 2 + 1);
  if (s == CLAIRE_OK) {
    float* cb = nullptr;
    s = alloc(c, &cb, 3 * Nc * 2);
    c->cbuf = (cufftComplex*)cb;
  }
  if (s == CLAIRE_OK) {
    // per-block partial sums of every fused reduction share one buffer
    int pb = c->red_blocks;
    pb = std::max(pb, spectral_blocks(g));
    pb = std::max(pb, march_blocks_max(g));        // any tunable depth
    pb = std::max(pb, vector_blocks(3 * N / 4));
    c->partial_blocks = pb;
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)(pb + 8 + NSLOTS + 4) * sizeof(double)) != cudaSuccess) {
      s = CLAIRE_ENOMEM;
    } else {
      c->allocs.push_back(p);
      c->partial = (double*)p;
      c->dres = c->partial + pb;
      c->slots = c->dres + 8;
      c->dflag = (int*)(c->slots + NSLOTS);
      c->far = (unsigned long long*)(c->slots + NSLOTS + 2);
      if (cudaMemset(c->far, 0, sizeof *c->far) != cudaSuccess) s = CLAIRE_ECUDA;
      c->bytes += (size_t)(pb + 8 + NSLOTS + 4) * sizeof(double);
    }
  }
  if (s == CLAIRE_OK && cudaMallocHost(&c->hres, 8 * sizeof(double)) != cudaSuccess)
    s = CLAIRE_ENOMEM;
  if (s == CLAIRE_OK && cudaMallocHost(&c->hslots, (NSLOTS + 4) * sizeof(double)) != cudaSuccess)
    s = CLAIRE_ENOMEM;
  if (s == CLAIRE_OK) {
    int n[3] = {nx, ny, nz};
    if (cufftPlanMany(&c->r2c, 3, n, nullptr, 1, (int)N, nullptr, 1, (int)Nc, CUFFT_R2C, 3) !=
            CUFFT_SUCCESS ||
        cufftPlanMany(&c->c2r, 3, n, nullptr, 1, (int)Nc, nullptr, 1, (int)N, CUFFT_C2R, 3) !=
            CUFFT_SUCCESS)
      s = CLAIRE_ECUDA;
    else
      c->plans = true;
  }
  if (s == CLAIRE_OK && (cudaEventCreate(&c->e0) != cudaSuccess ||
                         cudaEventCreate(&c->e1) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->e_in, cudaEventDisableTiming) !=
                             cudaSuccess))
    s = CLAIRE_ECUDA;
  if (s == CLAIRE_OK) {
    cudaMemset(c->m0, 0, N * sizeof(float));
    cudaMemset(c->m1, 0, N * sizeof(float));
    if (cudaDeviceSynchronize() != cudaSuccess) s = CLAIRE_ECUDA;
  }
  if (s != CLAIRE_OK) {
    cudaGetLastError();
    claire_destroy(c);
    return s;
  }
  *out = c;
  return CLAIRE_OK;
}

claire_status claire_set_options(claire_ctx* c, const claire_options* o) {
  if (!c || !o) return CLAIRE_EINVAL;
  if (o->precision < 0 || o->precision > 1 || o->hessian < 0 || o->hessian > 1 ||
      !(o->beta_w >= 0.0) || !(o->eps_opt > 0.0) || o->max_newton < 0 || o->max_pcg < 1 ||
      o->forcing < 0 || o->forcing > 1 || o->precond < 0 || o->precond > 2 ||
      (o->precond != 0 && o->max_inner < 1) || !std::isfinite(o->inner_rtol) ||
      o->distance < 0 || o->distance > 1 || o->warm_check < 0 || o->warm_check > 1)
    return fail(c, CLAIRE_EINVAL, "invalid option value");
  if (o->distance == 1 && o->precision != 0)
    return fail(c, CLAIRE_EINVAL, "the NCC distance needs FP32 storage (precision 0)");
  if (o->precond == 1 && (c->g.n1 % 4 || c->g.n2 % 4 || c->g.n3 % 4))
    return fail(c, CLAIRE_EINVAL, "two-level preconditioner needs every n_i %% 4 == 0");
  if (o->hessian == 1 && o->precision != 0)
    return fail(c, CLAIRE_EINVAL, "full Newton needs FP32 storage (precision 0)");
  if (o->precision == 0) TRY(fp32_histories(c));
  if (o->hessian == 1 && c->mthist == nullptr) {   // full-Newton buffers on first use
    TRY(alloc(c, &c->mthist, (int64_t)(c->nt + 1) * N_of(c)));
    TRY(alloc(c, &c->ef, N_of(c)));
  }
  if (o->precision == 1 && !march_supported(c->nt))
    return fail(c, CLAIRE_EINVAL, "mixed precision needs nt in {1, 2, 4, 8}");
  if (o->precision == 1 && c->mh == nullptr) {   // FP16 histories on first use
    const int64_t N = N_of(c);
    const int64_t nh = 4 * (int64_t)(c->nt + 1) * N + 2 * N;
    float* p = nullptr;
    TRY(alloc(c, &p, (nh + 1) / 2));
    __half* h = reinterpret_cast<__half*>(p);
    c->mh = h;
    c->lh = h + (c->nt + 1) * N;
    c->sh = h + 2 * (c->nt + 1) * N;
    c->lth = h + 3 * (c->nt + 1) * N;
    c->ph0 = h + 4 * (c->nt + 1) * N;
    c->ph1 = c->ph0 + N;
  }
  // captured graphs bake the launch configuration, the stream and the kernel
  // arguments; options read only on the host (tolerances, caps of the outer
  // loops, gnorm0, warm_check, verbose) leave them valid
  const claire_options& a = c->opt;
  if (o->precision != a.precision || o->hessian != a.hessian || o->beta_w != a.beta_w ||
      o->graphs != a.graphs || o->precond != a.precond || o->max_inner != a.max_inner ||
      o->distance != a.distance || o->stream != a.stream || o->autotune != a.autotune)
    drop_graphs(c);
  c->opt = *o;
  c->user = (cudaStream_t)o->stream;
  if (o->graphs && c->own == nullptr)
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
  // graphs are captured on the private stream (the legacy default stream
  // cannot be captured); calls order it after / before the user's stream
  c->st = o->graphs ? c->own : c->user;
  CUFFT_TRY(c, cufftSetStream(c->r2c, c->st));
  CUFFT_TRY(c, cufftSetStream(c->c2r, c->st));
  if (o->precond == 1 || (o->precond == 2 && grid_div4(c))) TRY(tl_setup(c));
  TRY(tl_set_streams(c));
  c->have_eval = false;
  c->tl_image = false;
  return CLAIRE_OK;
}

claire_status claire_get_options(const claire_ctx* c, claire_options* o) {
  if (!c || !o) return CLAIRE_EINVAL;
  *o = c->opt;
  return CLAIRE_OK;
}

claire_status claire_set_beta(claire_ctx* c, double beta_v) {
  if (!c || !(beta_v > 0.0)) return CLAIRE_EINVAL;
  if (beta_v != c->beta_v) drop_graphs(c);
  c->beta_v = beta_v;
  c->have_eval = false;
  return CLAIRE_OK;
}

size_t claire_workspace_bytes(const claire_ctx* c) { return c ? c->bytes : 0; }

const char* claire_last_error(const claire_ctx* c) { return c ? c->err.c_str() : "null context"; }

claire_status claire_set_images(claire_ctx* c, const float* m0, const float* m1) {
  ENTER(c);
  if (!c || !m0 || !m1) return CLAIRE_EINVAL;
  const size_t b = N_of(c) * sizeof(float);
  CUDA_TRY(c, cudaMemcpyAsync(c->m0, m0, b, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->m1, m1, b, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->have_eval = false;
  return image_scale(c);
}

claire_status claire_transport(claire_ctx* c, const float* v, float* m1_out) {
  ENTER(c);
  if (!c || !v || !m1_out) return CLAIRE_EINVAL;
  const int64_t N = N_of(c);
  launch_trace(c->g, v, c->dtrial, nullptr, ht_of(c), c->st);
  if (mixed(c)) {
    // the mixed form's own m(1): FP16 storage of sig_m m between the steps (the
    // work fields of the matvec; the evaluation's histories are left as they are)
    launch_axpy_h(N, c->sig_m, c->m0, 0.0f, nullptr, c->ph0, c->st);
    const __half* hsrc = c->ph0;
    for (int j = 0; j < c->nt; ++j) {
      __half* hdst = (j % 2 == 0) ? c->ph1 : c->ph0;
      launch_sl_h(c->g, hsrc, c->dtrial, nullptr, 1.0f, nullptr, 0.0f, hdst, c->st);
      hsrc = hdst;
    }
    launch_h2f(N, 1.0f / c->sig_m, hsrc, m1_out, c->st);
  } else {
    const float* src = c->m0;
    for (int j = 0; j < c->nt; ++j) {
      float* dst = (j == c->nt - 1) ? m1_out : ((j % 2 == 0) ? c->pp0 : c->pp1);
      launch_sl(c->g, src, c->dtrial, nullptr, 1.0f, nullptr, 0.0f, dst, c->st);
      src = dst;
    }
  }
  TRY(check_launch(c, "transport"));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_objective_gradient(claire_ctx* c, const float* v, double* J, float* g) {
  ENTER(c);
  if (!c || !v || !J) return CLAIRE_EINVAL;
  const size_t b3 = 3 * N_of(c) * sizeof(float);
  CUDA_TRY(c, cudaMemcpyAsync(c->v, v, b3, cudaMemcpyDeviceToDevice, c->st));
  TRY(evaluate(c));
  *J = c->J;
  if (g) CUDA_TRY(c, cudaMemcpyAsync(g, c->grad, b3, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_hessian_matvec(claire_ctx* c, const float* vt, float* Hvt) {
  ENTER(c);
  if (!c || !vt || !Hvt) return CLAIRE_EINVAL;
  TRY(matvec(c, vt, Hvt));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

// Continuation over nlev values of beta_v (Sec. 2.6), each level warm-started
// from the previous one.  v_in / v_out are device pointers, or NULL to use the
// iterate already held in c->v.
static claire_status solve_levels(claire_ctx* c, const double* betas, int nlev, const float* v_in,
                                  float* v_out, claire_stats* st) {
  NvtxRange nvtx_("claire.solve");
  if (!c || nlev < 1) return CLAIRE_EINVAL;
  ENTER(c);
  for (int i = 0; i < nlev; ++i)
    if (!(betas[i] > 0.0)) return CLAIRE_EINVAL;
  claire_stats local{};
  claire_stats* out = st ? st : &local;
  memset(out, 0, sizeof *out);
  Counters k;
  const size_t b3 = 3 * N_of(c) * sizeof(float);
  if (c->st != c->user) {                          // private stream: start after the user's work
    CUDA_TRY(c, cudaEventRecord(c->e1, c->user));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->e1, 0));
  }
  CUDA_TRY(c, cudaEventRecord(c->e0, c->st));
  if (v_in) CUDA_TRY(c, cudaMemcpyAsync(c->v, v_in, b3, cudaMemcpyDeviceToDevice, c->st));
  c->have_eval = false;                            // evaluated afresh at the initial guess
  double gnorm0 = c->opt.gnorm0;
  claire_status s = CLAIRE_OK;
  for (int i = 0; i < nlev; ++i) {
    if (betas[i] != c->beta_v) drop_graphs(c);
    c->beta_v = betas[i];
    if (i == 0 && c->opt.warm_check) TRY(warm_start_check(c, &gnorm0, k, out));
    s = gauss_newton(c, gnorm0, k, out);
    gnorm0 = out->gnorm0;
    if (s != CLAIRE_OK && s != CLAIRE_ENOTCONV) break;
  }
  cudaError_t e = cudaSuccess;
  if (v_out) e = cudaMemcpyAsync(v_out, c->v, b3, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = cudaEventRecord(c->e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->e1);
  if (e == cudaSuccess && c->st != c->user) e = cudaStreamWaitEvent(c->user, c->e1, 0);
  if (e != cudaSuccess) return fail(c, CLAIRE_ECUDA, "solve epilogue: %s", cudaGetErrorString(e));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->e0, c->e1);
  return finish_stats(c, out, k, ms, s);
}

claire_status claire_solve(claire_ctx* c, float* v_inout, claire_stats* st) {
  if (!c || !v_inout) return CLAIRE_EINVAL;
  const double b = c->beta_v;
  return solve_levels(c, &b, 1, v_inout, v_inout, st);
}

claire_status claire_solve_continuation(claire_ctx* c, const double* betas, int nlevels,
                                        float* v_inout, claire_stats* st) {
  if (!c || !betas || !v_inout || nlevels < 1) return CLAIRE_EINVAL;
  return solve_levels(c, betas, nlevels, v_inout, v_inout, st);
}

claire_status claire_solve_host(claire_ctx* c, const float* m0_host, const float* m1_host,
                                const double* betas, int nlevels, float* v_inout_host,
                                claire_stats* st) {
  if (!c || !m0_host || !m1_host || !v_inout_host) return CLAIRE_EINVAL;
  if (betas != nullptr && nlevels < 1) return CLAIRE_EINVAL;
  ENTER(c);
  const size_t b = N_of(c) * sizeof(float);
  CUDA_TRY(c, cudaMemcpyAsync(c->m0, m0_host, b, cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->m1, m1_host, b, cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->v, v_inout_host, 3 * b, cudaMemcpyHostToDevice, c->st));
  c->have_eval = false;
  TRY(image_scale(c));
  const double beta = c->beta_v;
  claire_status s = betas ? solve_levels(c, betas, nlevels, nullptr, nullptr, st)
                          : solve_levels(c, &beta, 1, nullptr, nullptr, st);
  if (s != CLAIRE_OK && s != CLAIRE_ENOTCONV && s != CLAIRE_ELINESEARCH) return s;
  CUDA_TRY(c, cudaMemcpyAsync(v_inout_host, c->v, 3 * b, cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return s;
}

claire_status claire_trace(claire_ctx* c, const float* v, float* d_fwd, float* d_bwd) {
  ENTER(c);
  if (!c || !v) return CLAIRE_EINVAL;
  launch_trace(c->g, v, d_fwd, d_bwd, ht_of(c), c->st);
  TRY(check_launch(c, "trace"));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_interp(claire_ctx* c, const float* u, const float* d, float* out) {
  ENTER(c);
  if (!c || !u || !d || !out) return CLAIRE_EINVAL;
  launch_sl(c->g, u, d, nullptr, 1.0f, nullptr, 0.0f, out, c->st);
  TRY(check_launch(c, "interp"));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_grad8(claire_ctx* c, const float* u, float* gu) {
  ENTER(c);
  if (!c || !u || !gu) return CLAIRE_EINVAL;
  launch_grad8(c->g, u, gu, c->st);
  TRY(check_launch(c, "grad8"));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_div8(claire_ctx* c, const float* w, float* dw) {
  ENTER(c);
  if (!c || !w || !dw) return CLAIRE_EINVAL;
  launch_div8(c->g, w, dw, c->st);
  TRY(check_launch(c, "div8"));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_spectral(claire_ctx* c, int op, const float* in, float* out) {
  ENTER(c);
  if (!c || !in || !out || op < 0 || op > 4) return CLAIRE_EINVAL;
  if (op == CLAIRE_OP_NEAR_INC && !(c->opt.beta_w > 0.0))
    return fail(c, CLAIRE_EINVAL, "near-incompressible operator needs options.beta_w > 0");
  TRY(spectral(c, op, in, out, c->beta_v));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_precondition(claire_ctx* c, const float* r, float* z, int* inner_iters) {
  ENTER(c);
  if (!c || !r || !z) return CLAIRE_EINVAL;
  if (inner_iters) *inner_iters = 0;
  if (!two_level(c)) {
    TRY(spectral(c, CLAIRE_OP_REG_INV, r, z, c->beta_v));
  } else {
    if (!c->have_eval)
      return fail(c, CLAIRE_EORDER, "precondition needs a prior objective_gradient");
    TRY(tl_update_image(c));
    c->tl_rtol = c->opt.inner_rtol > 0.0 ? c->opt.inner_rtol : 1e-3;
    c->tl_iters = 0;
    TRY(tl_precondition(c, r, z, c->scr3, -1));
    if (inner_iters) *inner_iters = c->tl_iters;
    c->tl_iters = 0;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

claire_status claire_det_deformation_gradient(claire_ctx* c, const float* v, double* mmm,
                                              float* det_out) {
  ENTER(c);
  if (!c || !v || !mmm) return CLAIRE_EINVAL;
  return detf_stats(c, v, mmm, det_out);
}

claire_status claire_beta_search(claire_ctx* c, double eps_d, double beta0, double beta_min,
                                 double rtol, int max_bisect, float* v_inout, double* beta_out,
                                 double* trial_beta, double* trial_detmin, double* trial_detmax,
                                 int max_trials, int* ntrials, claire_stats* st) {
  ENTER(c);
  if (!c || !v_inout || !beta_out || !(eps_d > 0.0 && eps_d < 1.0) || !(beta0 > 0.0) ||
      !(beta_min > 0.0) || !(rtol > 0.0) || max_bisect < 0 || max_trials < 0 ||
      (max_trials > 0 && (!trial_beta || !trial_detmin || !trial_detmax)))
    return CLAIRE_EINVAL;
  const int64_t N = N_of(c);
  const size_t b3 = 3 * N * sizeof(float);
  if (!c->vbest) TRY(alloc(c, &c->vbest, 3 * N));
  claire_stats local{};
  claire_stats* out = st ? st : &local;
  memset(out, 0, sizeof *out);
  Counters k;
  if (ntrials) *ntrials = 0;
  *beta_out = 0.0;
  if (c->st != c->user) {
    CUDA_TRY(c, cudaEventRecord(c->e1, c->user));
    CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->e1, 0));
  }
  CUDA_TRY(c, cudaEventRecord(c->e0, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->v, v_inout, b3, cudaMemcpyDeviceToDevice, c->st));
  c->have_eval = false;
  double gnorm0 = c->opt.gnorm0;
  int n = 0;
  // one trial: solve at beta from the current v (the previous trial's result), then
  // test eps_d < det F1 < 1 / eps_d (eq. ddgradbound)
  auto trial = [&](double beta, bool* ok) -> claire_status {
    if (beta != c->beta_v) drop_graphs(c);
    c->beta_v = beta;
    claire_status s = gauss_newton(c, gnorm0, k, out);
    gnorm0 = out->gnorm0;
    if (s != CLAIRE_OK && s != CLAIRE_ENOTCONV) return s;
    double mmm[3] = {0.0, 0.0, 0.0};
    TRY(detf_stats(c, c->v, mmm, nullptr));
    *ok = eps_d < mmm[0] && mmm[1] < 1.0 / eps_d;
    if (n < max_trials) {
      trial_beta[n] = beta;
      trial_detmin[n] = mmm[0];
      trial_detmax[n] = mmm[1];
    }
    ++n;
    if (*ok) CUDA_TRY(c, cudaMemcpyAsync(c->vbest, c->v, b3, cudaMemcpyDeviceToDevice, c->st));
    return CLAIRE_OK;
  };
  claire_status s = CLAIRE_OK;
  double beta = beta0, ok_beta = 0.0;
  bool ok = false;
  for (;;) {                                       // decades
    s = trial(beta, &ok);
    if (s != CLAIRE_OK || !ok) break;
    ok_beta = beta;
    if (beta / 10.0 < beta_min * (1.0 - 1e-9)) break;
    beta /= 10.0;
  }
  if (s == CLAIRE_OK && ok_beta > 0.0 && !ok) {    // bisection (reading C-17)
    double lo = beta, hi = ok_beta;
    for (int i = 0; i < max_bisect && hi - lo > rtol * hi && s == CLAIRE_OK; ++i) {
      const double mid = 0.5 * (lo + hi);
      s = trial(mid, &ok);
      if (s == CLAIRE_OK) (ok ? hi : lo) = mid;
    }
    ok_beta = hi;
  }
  if (ntrials) *ntrials = n;
  if (s == CLAIRE_OK && ok_beta > 0.0) {
    *beta_out = ok_beta;
    if (ok_beta != c->beta_v) drop_graphs(c);
    c->beta_v = ok_beta;
    CUDA_TRY(c, cudaMemcpyAsync(c->v, c->vbest, b3, cudaMemcpyDeviceToDevice, c->st));
  }
  c->have_eval = false;
  cudaError_t e = cudaMemcpyAsync(v_inout, c->v, b3, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = cudaEventRecord(c->e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->e1);
  if (e == cudaSuccess && c->st != c->user) e = cudaStreamWaitEvent(c->user, c->e1, 0);
  if (e != cudaSuccess) return fail(c, CLAIRE_ECUDA, "search epilogue: %s", cudaGetErrorString(e));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->e0, c->e1);
  return finish_stats(c, out, k, ms, s);
}

}  // extern "C"

namespace {

// det F1 of velocity v (Appendix, eq. def-grad): min, max and mean into mmm, the
// field into det_out when not NULL; synchronises the stream.
claire_status detf_stats(claire_ctx* c, const float* v, double* mmm, float* det_out) {
  const int64_t N = N_of(c);
  if (!c->detf) {
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)37 * N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CLAIRE_ENOMEM, "det F workspace allocation failed");
    }
    c->detf = (float*)p;
    c->bytes += (size_t)37 * N * sizeof(float);
  }
  float* F = c->detf;
  float* Fn = F + 9 * N;
  float* A = Fn + 9 * N;
  float* Ay = A + 9 * N;
  float* det = Ay + 9 * N;
  launch_trace(c->g, v, c->dtrial, nullptr, ht_of(c), c->st);
  launch_detf(c->g, v, c->dtrial, c->nt, F, Fn, A, Ay, det, c->st);
  TRY(check_launch(c, "detF"));
  double mn = 0.0, mx = 0.0, sum = 0.0;
  TRY(reduce(c, N, det, nullptr, RED_MIN, &mn));
  TRY(reduce(c, N, det, nullptr, RED_MAX, &mx));
  TRY(reduce(c, N, det, nullptr, RED_SUM, &sum));
  mmm[0] = mn;
  mmm[1] = mx;
  mmm[2] = sum / (double)N;
  if (det_out) CUDA_TRY(c, cudaMemcpyAsync(det_out, det, N * sizeof(float),
                                           cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return CLAIRE_OK;
}

}  // namespace

namespace claire {

// Combiner of a grouped batch.  Each worker posts one op at a time and blocks
// until it has been launched.  The first op of a round makes its poster the
// round's leader: it waits until every live worker has posted or until
// wait_us microseconds have passed since its own post (wait_us < 0: no time
// limit), whichever comes first, and then launches everything posted so far,
// one persistent grouped launch per kind, on the group's stream.  Workers that
// post later go into the next round, so a pair busy with other work (cuFFT, a
// host synchronisation) does not hold the others back for long.  Ordering: a
// poster records an event on its pair's stream and makes the group's stream
// wait for it before posting (a wait that lands between the launches of a
// concurrent flush only delays them); the flushing thread records `done`
// behind the grouped launches and makes each flushed pair's stream wait for it
// while it holds the lock, so no event is re-recorded before its waits are
// enqueued.
class LaunchGroup {
 public:
  LaunchGroup(int live, cudaStream_t gst, cudaEvent_t done, int wait_us)
      : live_(live), wait_us_(wait_us), gst_(gst), done_(done) {}

  void post(const GroupOp& op, cudaStream_t st, cudaEvent_t ev) {
    note(cudaEventRecord(ev, st));
    note(cudaStreamWaitEvent(gst_, ev, 0));
    std::unique_lock<std::mutex> lk(mu_);
    pending_.push_back(op);
    streams_.push_back(st);
    const uint64_t my = epoch_;
    if ((int)pending_.size() >= live_) {
      flush_locked();
      return;
    }
    if (pending_.size() == 1) {                     // this round's leader
      auto ready = [&] { return epoch_ != my || (int)pending_.size() >= live_; };
      if (wait_us_ < 0) cv_.wait(lk, ready);
      else cv_.wait_until(lk, std::chrono::steady_clock::now() +
                                  std::chrono::microseconds(wait_us_), ready);
      if (epoch_ == my) flush_locked();
      return;
    }
    cv_.wait(lk, [&] { return epoch_ != my; });
  }

  // The calling worker posts nothing more.
  void leave() {
    std::lock_guard<std::mutex> lk(mu_);
    --live_;
    if (live_ > 0 && !pending_.empty() && (int)pending_.size() >= live_) flush_locked();
    cv_.notify_all();                               // a leader may now have everyone
  }

  cudaError_t error() {
    std::lock_guard<std::mutex> lk(err_mu_);
    return err_;
  }
  long long ops() const { return ops_; }
  long long launches() const { return launches_; }

 private:
  void note(cudaError_t e) {
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(err_mu_);
      if (err_ == cudaSuccess) err_ = e;
    }
  }

  void flush_locked() {
    std::vector<SlOpArgs> sl[2];
    std::vector<TraceOpArgs> tr;
    std::vector<std::pair<int, MarchOpArgs>> mh;   // (mode * 16 + nf, args)
    for (const GroupOp& op : pending_) {
      if (op.kind == GOP_SL0 || op.kind == GOP_SL1) sl[op.kind].push_back(op.sl);
      else if (op.kind == GOP_TRACE) tr.push_back(op.tr);
      else mh.emplace_back(op.mode * 16 + op.nf, op.mh);
    }
    for (int m = 0; m < 2; ++m)
      if (!sl[m].empty()) {
        launch_sl_group(m, sl[m].data(), (int)sl[m].size(), gst_);
        ++launches_;
      }
    if (!tr.empty()) {
      launch_trace_group(tr.data(), (int)tr.size(), gst_);
      ++launches_;
    }
    std::stable_sort(mh.begin(), mh.end(),
                     [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t i = 0; i < mh.size();) {
      size_t j = i;
      std::vector<MarchOpArgs> ops;
      while (j < mh.size() && mh[j].first == mh[i].first) ops.push_back(mh[j++].second);
      if (!launch_march_group(mh[i].first / 16, mh[i].first % 16, ops.data(), (int)ops.size(),
                              gst_))
        note(cudaErrorInvalidValue);
      ++launches_;
      i = j;
    }
    note(cudaGetLastError());
    note(cudaEventRecord(done_, gst_));
    for (cudaStream_t st : streams_) note(cudaStreamWaitEvent(st, done_, 0));
    ops_ += (long long)pending_.size();
    pending_.clear();
    streams_.clear();
    ++epoch_;
    cv_.notify_all();
  }

  std::mutex mu_, err_mu_;
  std::condition_variable cv_;
  int live_;
  const int wait_us_;
  uint64_t epoch_ = 0;
  std::vector<GroupOp> pending_;
  std::vector<cudaStream_t> streams_;
  cudaStream_t gst_;
  cudaEvent_t done_;
  cudaError_t err_ = cudaSuccess;
  long long ops_ = 0, launches_ = 0;
};

thread_local LaunchGroup* tl_group = nullptr;
static thread_local cudaEvent_t tl_group_event = nullptr;

void group_post(const GroupOp& op, cudaStream_t st) { tl_group->post(op, st, tl_group_event); }

}  // namespace claire

// Solves the pairs on their own streams, one host thread per pair (grouped:
// every pair, its SL steps, traces and FD8 marches combined by a LaunchGroup)
// or up to max_threads threads (ungrouped).
static claire_status solve_batch_impl(claire_ctx** ctxs, int npairs, const double* betas,
                                      int nlevels, float** v_inout, claire_stats* stats,
                                      int max_threads, bool grouped, int wait_us,
                                      long long* group_launches, long long* group_ops) {
  if (!ctxs || npairs < 1 || !v_inout || (betas && nlevels < 1)) return CLAIRE_EINVAL;
  for (int i = 0; i < npairs; ++i) {
    if (!ctxs[i] || !v_inout[i]) return CLAIRE_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], CLAIRE_EINVAL, "context given twice");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CLAIRE_ECUDA;
  // every pair runs on a stream of its own so that the pairs overlap on the GPU
  std::vector<cudaStream_t> saved(npairs);
  for (int i = 0; i < npairs; ++i) {
    claire_ctx* c = ctxs[i];
    saved[i] = c->st;
    if (c->st == nullptr) {
      if (c->own == nullptr)
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
      c->st = c->own;
      CUFFT_TRY(c, cufftSetStream(c->r2c, c->st));
      CUFFT_TRY(c, cufftSetStream(c->c2r, c->st));
      TRY(tl_set_streams(c));                      // the two-level plans follow
    }
  }
  std::vector<claire_status> res(npairs, CLAIRE_OK);
  const int nt = grouped ? npairs
                         : std::max(1, std::min(npairs, max_threads > 0 ? max_threads : npairs));
  // grouped: the group's stream and events (launches captured into a pair's
  // graphs stay in the graph; the rest is posted)
  cudaStream_t gst = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> evs(grouped ? nt : 0, nullptr);
  claire_status setup = CLAIRE_OK;
  if (grouped) {
    if (cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess)
      setup = CLAIRE_ECUDA;
    for (int t = 0; t < nt && setup == CLAIRE_OK; ++t)
      if (cudaEventCreateWithFlags(&evs[t], cudaEventDisableTiming) != cudaSuccess)
        setup = CLAIRE_ECUDA;
  }
  LaunchGroup group(nt, gst, done, wait_us);
  std::atomic<int> next{0};
  auto worker = [&](int t) {
    cudaSetDevice(dev);
    if (grouped) {
      tl_group = &group;
      tl_group_event = evs[t];
    }
    for (int i = next++; i < npairs; i = next++) {
      claire_ctx* c = ctxs[i];
      const double b = c->beta_v;
      res[i] = betas ? solve_levels(c, betas, nlevels, v_inout[i], v_inout[i],
                                    stats ? stats + i : nullptr)
                     : solve_levels(c, &b, 1, v_inout[i], v_inout[i],
                                    stats ? stats + i : nullptr);
    }
    if (grouped) {
      group.leave();
      tl_group = nullptr;
      tl_group_event = nullptr;
    }
  };
  if (setup == CLAIRE_OK) {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker, t);
    for (auto& t : pool) t.join();
  }
  if (grouped) {
    if (gst && cudaStreamSynchronize(gst) != cudaSuccess && setup == CLAIRE_OK)
      setup = CLAIRE_ECUDA;
    if (group.error() != cudaSuccess && setup == CLAIRE_OK) setup = CLAIRE_ECUDA;
    if (group_launches) *group_launches = group.launches();
    if (group_ops) *group_ops = group.ops();
    for (cudaEvent_t e : evs)
      if (e) cudaEventDestroy(e);
    if (done) cudaEventDestroy(done);
    if (gst) cudaStreamDestroy(gst);
  }
  for (int i = 0; i < npairs; ++i) {
    claire_ctx* c = ctxs[i];
    if (c->st != saved[i]) {
      cudaStreamSynchronize(c->st);
      c->st = saved[i];
      cufftSetStream(c->r2c, c->st);
      cufftSetStream(c->c2r, c->st);
      if (tl_set_streams(c) != CLAIRE_OK && res[i] == CLAIRE_OK) res[i] = CLAIRE_ECUDA;
    }
  }
  claire_status worst = setup;
  for (int i = 0; i < npairs; ++i)
    if (res[i] != CLAIRE_OK && res[i] != CLAIRE_ENOTCONV) worst = res[i];
  if (worst == CLAIRE_OK)
    for (int i = 0; i < npairs; ++i)
      if (res[i] != CLAIRE_OK) worst = res[i];
  return worst;
}

extern "C" {

claire_status claire_solve_batch(claire_ctx** ctxs, int npairs, const double* betas,
                                 int nlevels, float** v_inout, claire_stats* stats,
                                 int max_threads) {
  return solve_batch_impl(ctxs, npairs, betas, nlevels, v_inout, stats, max_threads, false, 0,
                          nullptr, nullptr);
}

claire_status claire_solve_batch_grouped(claire_ctx** ctxs, int npairs, const double* betas,
                                         int nlevels, float** v_inout, claire_stats* stats,
                                         int wait_us, long long* group_launches,
                                         long long* group_ops) {
  return solve_batch_impl(ctxs, npairs, betas, nlevels, v_inout, stats, 0, true, wait_us,
                          group_launches, group_ops);
}

claire_status claire_far_nodes(claire_ctx* c, long long* fwd, long long* bwd) {
  if (!c || !fwd || !bwd) return CLAIRE_EINVAL;
  ENTER(c);
  if (!c->have_eval) return fail(c, CLAIRE_EORDER, "far_nodes needs an evaluated velocity");
  long long* res[2] = {fwd, bwd};
  const float* d[2] = {c->df, c->db};
  for (int k = 0; k < 2; ++k) {
    unsigned long long n = 0;
    CUDA_TRY(c, cudaMemsetAsync(c->far, 0, sizeof n, c->st));
    launch_count_far(c->g, d[k], c->far, c->st);
    TRY(check_launch(c, "far nodes"));
    CUDA_TRY(c, cudaMemcpyAsync(&n, c->far, sizeof n, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    *res[k] = (long long)n;
  }
  return CLAIRE_OK;
}

claire_status claire_autotune(claire_ctx* c, int* sl_t1, int* march_t1) {
  if (!c) return CLAIRE_EINVAL;
  ENTER(c);
  if (!c->have_eval) TRY(evaluate(c));
  TRY(autotune(c));
  drop_graphs(c);                                  // captured with the previous shapes
  if (sl_t1) *sl_t1 = c->tune.sl_t1;
  if (march_t1) *march_t1 = c->tune.march_t1;
  return CLAIRE_OK;
}

claire_status claire_set_tuning(claire_ctx* c, int sl_gather, int sl_t1, int march_t1) {
  if (!c) return CLAIRE_EINVAL;
  ENTER(c);
  if (sl_gather != SL_GATHER_TMA && sl_gather != SL_GATHER_WINDOW &&
      sl_gather != SL_GATHER_CPASYNC)
    return fail(c, CLAIRE_EINVAL, "sl_gather must be 0, 1 or 2");
  if (sl_t1 != 4 && sl_t1 != 8 && sl_t1 != 16)
    return fail(c, CLAIRE_EINVAL, "sl_t1 must be 4, 8 or 16");
  if (march_t1 != 8 && march_t1 != 16 && march_t1 != 32 && march_t1 != 64)
    return fail(c, CLAIRE_EINVAL, "march_t1 must be 8, 16, 32 or 64");
  c->tune.sl_gather = sl_gather;
  c->tune.sl_t1 = sl_t1;
  c->tune.march_t1 = march_t1;
  c->tuned = true;                                 // options.autotune keeps these shapes
  drop_graphs(c);                                  // captured with the previous shapes
  return CLAIRE_OK;
}

claire_status claire_get_tuning(const claire_ctx* c, int* sl_gather, int* sl_t1,
                                int* march_t1) {
  if (!c) return CLAIRE_EINVAL;
  if (sl_gather) *sl_gather = c->tune.sl_gather;
  if (sl_t1) *sl_t1 = c->tune.sl_t1;
  if (march_t1) *march_t1 = c->tune.march_t1;
  return CLAIRE_OK;
}

claire_status claire_profile_reset(claire_ctx* c, int timing) {
  if (!c) return CLAIRE_EINVAL;
  ENTER(c);
  c->prof.reset(timing != 0);
  return CLAIRE_OK;
}

int claire_profile_read(claire_ctx* c, claire_kernel_stat* out, int max) {
  if (!c) return -1;
  if (c->prof.resolve() != cudaSuccess) return -1;
  int n = 0;
  for (int k = 0; k < K_COUNT && (out == nullptr || n < max); ++k, ++n) {
    if (!out) continue;
    out[n].name = kernel_kind_name(k);
    out[n].launches = c->prof.launches[k];
    out[n].timed = c->prof.timed[k];
    out[n].bytes = c->prof.bytes[k];
    out[n].ms = c->prof.ms[k];
    out[n].timed_bytes = c->prof.timed_bytes[k];
  }
  return out ? n : (int)K_COUNT;
}

}  // extern "C"
