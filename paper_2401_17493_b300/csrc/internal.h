// Internal declarations shared by the kernel launchers and the host solver.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cufft.h>
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace claire {

// ---- launch accounting and optional per-kernel event timing ---------------
// Every launcher below counts its launch and the algorithmic bytes it moves
// (each input field read once, each output written once) in the profiler of
// the calling context; with timing on it also brackets the launch with a pair
// of CUDA events on the launch stream.
enum KernelKind {
  K_TRACE, K_SL, K_ADJFAC, K_GRAD8, K_DIV8, K_SDOT, K_ACCUM, K_SPECTRAL, K_REDUCE, K_VECTOR,
  K_DETF, K_CUFFT, K_PRECOND, K_COUNT
};
const char* kernel_kind_name(int k);

struct Profiler {
  bool timing = false;
  long long launches[K_COUNT] = {};
  double bytes[K_COUNT] = {};
  double ms[K_COUNT] = {};
  long long timed[K_COUNT] = {};
  double timed_bytes[K_COUNT] = {};   // algorithmic bytes of the event-timed launches
  struct Pending { int kind; cudaEvent_t a, b; double bytes; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  void reset(bool timing_on);
  cudaEvent_t take();
  // waits for the recorded events and folds their times into ms[]
  cudaError_t resolve();
  void release();
};

// The profiler of the context whose API call is running on this thread.
extern thread_local Profiler* tl_prof;

// Tile shapes picked by the autotuner for one grid: the SL gather variant
// (0: 64 shared loads per node, the default; 1: register window along x1 with
// a deferred queue), the x1 depth of the SL brick (4, 8 or 16 nodes) and
// planes per CTA of the FD8 march (8, 16, 32 or 64).
// SL gather variants: the 64-tap gather from a brick staged by TMA tiled loads
// (default) or by the threads' 16-byte cp.async copies, or the register window.
enum SlGather { SL_GATHER_TMA = 0, SL_GATHER_WINDOW = 1, SL_GATHER_CPASYNC = 2 };
struct Tuning {
  int sl_gather = SL_GATHER_TMA;
  int sl_t1 = 8;
  int march_t1 = 32;
};
extern thread_local const Tuning* tl_tune;
int tuned_sl_t1();
bool tuned_sl_window();
bool tuned_sl_tma();
int tuned_march_t1();
// Threads whose bounded wait for a TMA-staged SL brick ran out since the last
// call (their outputs are left unwritten); reads and resets.  One counter for
// the FP32 kernels (kernels.cu), one for the FP16 ones (mixed.cu).
unsigned int take_brick_timeouts();
unsigned int take_brick_timeouts_h();
// TMA tensor map of ncomp stacked fields (FP32, or FP16 with half) whose box is
// one SL brick of depth t1; false where TMA's alignment rules do not hold.
bool encode_brick_map(CUtensorMap* m, const void* base, bool half, const Grid& g, int ncomp,
                      int t1);

struct ProfileRange {
  int kind;
  double bytes;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfileRange(int k, double bytes, cudaStream_t s);
  ~ProfileRange();
};

void launch_trace(const Grid& g, const float* v, float* df, float* db, float ht, cudaStream_t st);
// adds to *out the nodes whose departure points d leave the SL brick (global gather)
void launch_count_far(const Grid& g, const float* d, unsigned long long* out, cudaStream_t st);
void launch_sl(const Grid& g, const float* u, const float* d, const float* scale, float sigma,
               const float* aux, float beta, float* out, cudaStream_t st);
void launch_adjoint_factor(const Grid& g, const float* D, const float* db, float ht, float* c,
                           cudaStream_t st);
void launch_grad8(const Grid& g, const float* u, float* gu, cudaStream_t st);
void launch_div8(const Grid& g, const float* w, float* out, cudaStream_t st);
void launch_div8_prod(const Grid& g, const float* lam, const float* w, float* out,
                      cudaStream_t st);
void launch_affine(int64_t n, float a, const float* x, float b, float* out, cudaStream_t st);
void launch_ncc_final(int64_t n, const float* m1, const float* m, float* lt, const double* sx,
                      const double* sy, double a, double b, double c, double h3,
                      cudaStream_t st);
void launch_sdot_hist(const Grid& g, const float* mhist, int nt, const float* vt, float scale0,
                      float* shist, cudaStream_t st);
// With partial != NULL (nt in {1, 2, 4, 8} only, see march_supported) also
// writes march_blocks() per-block shares of <dotv, out>.
void launch_accum_hist(const Grid& g, const float* lhist, const float* mhist, int nt,
                       const float* base, float base_coef, float* out, cudaStream_t st,
                       const float* dotv = nullptr, double* partial = nullptr);
int march_blocks(const Grid& g);
int march_blocks_max(const Grid& g);        // blocks at the shallowest tunable depth
int default_march_t1(const Grid& g);        // default planes per CTA for this grid
bool march_supported(int nt);
// partial (optional): per-block shares of <in, out>; means (optional): the
// three component means of the input field.  spectral_blocks() blocks.
void launch_spectral(const Grid& g, cufftComplex* X, int op, float alpha, float gamma,
                     float beta_w, cudaStream_t st, double* partial = nullptr,
                     double* means = nullptr);
int spectral_blocks(const Grid& g);
int vector_blocks(int64_t n);
void launch_reduce_final(const double* partial, int nblocks, int mode, double* out,
                         cudaStream_t st);
void launch_pcg_update(int64_t n, const double* rz, const double* sHs, float* vt, float* r,
                       const float* s, const float* Hs, double* partial, int nblocks, int* flag,
                       cudaStream_t st);
void launch_s_update(int64_t N, const double* rz_new, const double* rz_old, const double* means,
                     int first, const float* z, const float* r, float* s, float* hs,
                     cudaStream_t st);
void launch_reduce(int64_t n, const float* a, const float* b, int mode, double* partial,
                   int nblocks, double* out, cudaStream_t st);
void launch_axpby(int64_t n, float a, const float* x, float b, float* y, cudaStream_t st);
void launch_lincomb(int64_t n, float a, const float* x, float b, const float* y, float* out,
                    cudaStream_t st);
void launch_detf(const Grid& g, const float* v, const float* df, int nt, float* F, float* Fn,
                 float* A, float* Ay, float* det, cudaStream_t st);

// ---- grouped launches of a batch (claire_solve_batch_grouped, group.cu) ----
// Each worker thread of a grouped batch drives one pair's solve.  Its FP32 SL
// steps, adjoint factors, traces and FD8 history marches are not launched on
// the pair's stream but posted to the batch's LaunchGroup: when every live
// worker has posted one, the group launches each kind once for all of them
// (a persistent kernel over the (pair, tile) items, kernels.cu) on its own
// stream, ordered after each pair's earlier work and before its later work by
// events.  The per-tile code is the single launch's, so the results are
// bitwise those of per-pair launches.
struct SlOpArgs {            // one k_sl launch (mode 0: SL step, 1: adjoint factor)
  Grid g;
  const float* u; const float* d; const float* scale; const float* aux;
  float* out;
  float sigma, beta, ht;
  int t1, tma;               // tile depth; TMA staging wanted (gather variant 0)
};
struct TraceOpArgs {         // one k_trace launch
  Grid g;
  const float* v; float* df; float* db;
  float ht;
  int t1, tma;
};
struct MarchOpArgs {         // one k_hist_march<mode, nf, float> launch
  Grid g;
  const float* mhist; const float* lhist; const float* vt; const double* vmax;
  const float* base; float* out; float* hout; const float* dotv; double* partial;
  float scale0, base_coef, umul;
  int mt1;
};
enum GroupKind { GOP_SL0 = 0, GOP_SL1 = 1, GOP_TRACE = 2, GOP_MARCH = 3 };
struct GroupOp {
  int kind;
  int mode, nf;              // GOP_MARCH: the march template
  SlOpArgs sl;
  TraceOpArgs tr;
  MarchOpArgs mh;
};
class LaunchGroup;
extern thread_local LaunchGroup* tl_group;
// Posts op for the calling worker (blocks until it has been launched; st's
// later work waits for it).
void group_post(const GroupOp& op, cudaStream_t st);
// Persistent grouped kernels over all ops' tiles (any count: launched in chunks).
void launch_sl_group(int mode, const SlOpArgs* ops, int n, cudaStream_t st);
void launch_trace_group(const TraceOpArgs* ops, int n, cudaStream_t st);
bool launch_march_group(int mode, int nf, const MarchOpArgs* ops, int n, cudaStream_t st);

// Mixed-precision (FP16 storage) launchers, see mixed.cu.
void launch_sl_h(const Grid& g, const __half* u, const float* d, const float* scale,
                 float sigma, const __half* aux, float beta, __half* out, cudaStream_t st);
bool launch_sdot_hist_h(const Grid& g, const __half* mhist, int nt, const float* vt,
                        float scale0, const double* vmax, __half* shist, cudaStream_t st);
bool launch_accum_hist_h(const Grid& g, const __half* lhist, const __half* mhist, int nt,
                         const double* vmax, float umul, const float* base, float base_coef,
                         float* out, const float* dotv, double* partial, cudaStream_t st);
void launch_axpy_h(int64_t n, float a, const float* x, float b, const __half* z, __half* y,
                   cudaStream_t st);
void launch_h2f(int64_t n, float a, const __half* x, float* y, cudaStream_t st);
void launch_sqdiff_h(int64_t n, const __half* m, float a, const float* m1, double* partial,
                     int nblocks, double* out, cudaStream_t st);

// Two-level preconditioner kernels (precond.cu).
void launch_tl_split(const Grid& gf, cufftComplex* X, cufftComplex* C, int ncomp, int symbol,
                     float alpha, float gamma, float scale, cudaStream_t st);
void launch_tl_merge(const Grid& gf, cufftComplex* X, const cufftComplex* C, cufftComplex* X2,
                     float alpha, float gamma, float sf, float sc, cudaStream_t st);
void launch_tl_outer(int64_t n, const float* gm, const float* q, float* w, cudaStream_t st);
void launch_tl_unscale_h(int64_t n, const __half* h, float inv, float* out, cudaStream_t st);
// Device-side control of the nested CG inside a graph with a conditional while node.
void launch_tl_cg_begin(cudaGraphConditionalHandle h, const double* rr0, const double* rtol,
                        double* stop2, double* count, int max_inner, cudaStream_t st);
void launch_tl_cg_control(cudaGraphConditionalHandle h, double* rr, const double* rr_new,
                          const double* pAp, const double* stop2, double* count, double* total,
                          int max_inner, cudaStream_t st);
void launch_set_scalar(double* p, double v, cudaStream_t st);
int tl_spec_blocks(const Grid& gc);
void launch_tl_spec_table(const Grid& gc, float alpha, float gamma, float2* fw, cudaStream_t st);
// Nested CG on coarse half spectra.  Each scalar (<b,b>, <p,Ap>, ||r||^2) is finished
// by the last block of its kernel; count points to a zeroed counter the kernel
// leaves at zero.
void launch_tl_spec_finish(const Grid& gc, const float2* fw, const cufftComplex* p,
                           const cufftComplex* y, cufftComplex* Ap, float scale, double* partial,
                           unsigned* count, double* pAp, cudaStream_t st);
void launch_tl_spec_step(const Grid& gc, const float2* fw, const double* rr, const double* pAp,
                         cufftComplex* x, cufftComplex* r, const cufftComplex* p,
                         const cufftComplex* Ap, double* partial, unsigned* count,
                         double* rr_new, cudaStream_t st);
void launch_tl_spec_init(const Grid& gc, const float2* fw, cufftComplex* b, cufftComplex* x,
                         cufftComplex* r, cufftComplex* p, double* partial, unsigned* count,
                         double* bb, cudaStream_t st);
void launch_tl_dir_scale(const Grid& gc, const float2* fw, const double* rr_new,
                         const double* rr_old, const cufftComplex* r, cufftComplex* p,
                         cufftComplex* cc, cudaStream_t st);

enum ReduceMode {
  RED_DOT = 0, RED_SQDIFF = 1, RED_ABSMAX = 2, RED_SQ = 3, RED_MAX = 4, RED_MIN = 5, RED_SUM = 6
};

}  // namespace claire
