// Two-level zero-velocity preconditioner (Sec. 2.5.6): the spectral kernels
// that split a residual into the part restricted to the grid of half the
// resolution and the high-frequency remainder, merge the coarse solution back,
// and the kernels of the nested CG, which runs on coarse spectra (the
// pointwise outer product is the only real-space step).
//
// Fine half spectra are [3][n1][n2][n3/2+1] (cuFFT R2C layout), coarse ones
// [3][n1/2][n2/2][n3/4+1].  A fine mode is "low" when |k_i| < n_i / 4 on every
// axis (representable on the coarse grid without its Nyquist mode); F_L keeps
// the low modes, F_H = I - F_L.  R^-1/2 has the symbol (alpha sigma(k))^-1/2
// with sigma = |k|^(2 gamma) and the zero symbol set to one.
#include "internal.h"
#include "reduce.cuh"

namespace claire {
namespace {

struct ModeIdx {
  int k1, k2, k3;
  bool low;
  int64_t ci;          // coarse half-spectrum index (valid when low)
};

// (i < 2^31: a half spectrum of a grid with 3 N < 2^31, so 32-bit index math)
__device__ __forceinline__ ModeIdx fine_mode(const Grid& g, int64_t i, int c1n, int c2n) {
  const unsigned nh = (unsigned)(g.n3 / 2 + 1), u = (unsigned)i;
  const unsigned q = u / nh;
  const int j3 = (int)(u - q * nh);
  const int j1 = (int)(q / (unsigned)g.n2);
  const int j2 = (int)(q - (unsigned)j1 * (unsigned)g.n2);
  ModeIdx m;
  m.k1 = j1 <= g.n1 / 2 ? j1 : j1 - g.n1;
  m.k2 = j2 <= g.n2 / 2 ? j2 : j2 - g.n2;
  m.k3 = j3;
  m.low = abs(m.k1) < g.n1 / 4 && abs(m.k2) < g.n2 / 4 && m.k3 < g.n3 / 4;
  const int c1 = m.k1 >= 0 ? m.k1 : m.k1 + c1n;
  const int c2 = m.k2 >= 0 ? m.k2 : m.k2 + c2n;
  const int ch = g.n3 / 4 + 1;                     // coarse half-spectrum length
  m.ci = ((int64_t)c1 * c2n + c2) * ch + m.k3;
  return m;
}

__device__ __forceinline__ float inv_sqrt_symbol(int k1, int k2, int k3, float alpha,
                                                 float gamma) {
  const float kap = (float)(k1 * k1 + k2 * k2 + k3 * k3);
  float sig = gamma == 1.0f ? kap : powf(kap, gamma);
  if (kap == 0.0f) sig = 1.0f;
  return rsqrtf(alpha * sig);
}

// Split (ncomp fields): with symbol, X <- R^-1/2 X on the high modes and 0 on
// the low ones, whose values R^-1/2 X * scale go to the coarse spectrum C;
// without symbol, X is left alone and C gets X * scale on the low modes.  C
// must be zeroed before (its coarse Nyquist modes are never written).
__global__ void k_tl_split(Grid g, cufftComplex* __restrict__ X, cufftComplex* __restrict__ C,
                           int ncomp, int symbol, float alpha, float gamma, float scale) {
  const int64_t Nh = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  const int64_t Ch = (int64_t)(g.n1 / 2) * (g.n2 / 2) * (g.n3 / 4 + 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nh) return;
  const ModeIdx m = fine_mode(g, i, g.n1 / 2, g.n2 / 2);
  const float f = symbol ? inv_sqrt_symbol(m.k1, m.k2, m.k3, alpha, gamma) : 1.0f;
  for (int a = 0; a < ncomp; ++a) {
    cufftComplex x = X[a * Nh + i];
    x.x *= f;
    x.y *= f;
    if (m.low) {
      C[a * Ch + m.ci] = make_cuComplex(x.x * scale, x.y * scale);
      if (symbol) x = make_cuComplex(0.f, 0.f);
    }
    if (symbol) X[a * Nh + i] = x;
  }
}

// Merge: U = low ? C * sc : X * sf (coarse solution prolonged, high part kept),
// X <- R^-1/2 U (the preconditioned residual z) and X2 <- alpha sigma(k) R^-1/2 U
// (alpha L z, zero mean).
__global__ void k_tl_merge(Grid g, cufftComplex* __restrict__ X, const cufftComplex* __restrict__ C,
                           cufftComplex* __restrict__ X2, float alpha, float gamma, float sf,
                           float sc) {
  const int64_t Nh = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  const int64_t Ch = (int64_t)(g.n1 / 2) * (g.n2 / 2) * (g.n3 / 4 + 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nh) return;
  const ModeIdx m = fine_mode(g, i, g.n1 / 2, g.n2 / 2);
  const float f = inv_sqrt_symbol(m.k1, m.k2, m.k3, alpha, gamma);
  const float kap = (float)(m.k1 * m.k1 + m.k2 * m.k2 + m.k3 * m.k3);
  const float sig = gamma == 1.0f ? kap : powf(kap, gamma);   // 0 at k = 0
  for (int a = 0; a < 3; ++a) {
    cufftComplex u;
    if (m.low) {
      const cufftComplex cv = C[a * Ch + m.ci];
      u = make_cuComplex(cv.x * sc, cv.y * sc);
    } else {
      const cufftComplex xv = X[a * Nh + i];
      u = make_cuComplex(xv.x * sf, xv.y * sf);
    }
    const cufftComplex z = make_cuComplex(u.x * f, u.y * f);
    X[a * Nh + i] = z;
    X2[a * Nh + i] = make_cuComplex(alpha * sig * z.x, alpha * sig * z.y);
  }
}

// w = gm (gm . q) pointwise (3 components, n nodes).
__global__ void k_tl_outer(int64_t n, const float* __restrict__ gm, const float* __restrict__ q,
                           float* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g0 = gm[i], g1 = gm[n + i], g2 = gm[2 * n + i];
    const float d = g0 * q[i] + g1 * q[n + i] + g2 * q[2 * n + i];
    w[i] = g0 * d;
    w[n + i] = g1 * d;
    w[2 * n + i] = g2 * d;
  }
}

// ---- nested CG in the coarse spectral domain.  Vectors are coarse half spectra
// [3][Ch] in the normalisation of cuFFT's unnormalised C2R (u = C2R(u^)), so the
// split kernel's output is the right-hand side and the merge kernel reads the
// solution directly.  Inner products are Parseval sums over the half spectrum:
// modes with k3 = 0 or k3 = n3/2 count once, the others twice (the common factor
// N_c drops out of every CG ratio).

// Per coarse mode: x = R^-1/2 symbol, y = Parseval weight (1 for k3 = 0 or
// k3 = n3/2, else 2).  Rebuilt whenever beta_v may have changed.
__global__ void k_tl_spec_table(int64_t Ch, int n1, int n2, int n3, float alpha, float gamma,
                                float2* __restrict__ fw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ch) return;
  const unsigned nh = (unsigned)(n3 / 2 + 1), u = (unsigned)i;
  const unsigned q = u / nh;
  const int j3 = (int)(u - q * nh);
  const int j1 = (int)(q / (unsigned)n2);
  const int j2 = (int)(q - (unsigned)j1 * (unsigned)n2);
  const int k1 = j1 <= n1 / 2 ? j1 : j1 - n1;
  const int k2 = j2 <= n2 / 2 ? j2 : j2 - n2;
  fw[i] = make_float2(inv_sqrt_symbol(k1, k2, j3, alpha, gamma),
                      (j3 == 0 || 2 * j3 == n3) ? 1.0f : 2.0f);
}

// The kernels below run a grid-stride loop over the Ch modes; each thread
// handles the three fields of a mode (one table read), and the partial sums go
// to partial[blockIdx.x].
#define CLAIRE_SPEC_LOOP                                                                  \
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < Ch;                \
       m += (int64_t)gridDim.x * blockDim.x)

// The block's share goes to partial[blockIdx.x]; the last block to finish (a ticket
// on *count) adds the shares in block order, writes *out and resets *count, so a
// CG scalar needs no separate final-reduction launch.  The shares are read past L1
// after the fences, and the order of the final sum is fixed.
__device__ __forceinline__ void spec_partial_final(double* partial, const KahanF& acc,
                                                   unsigned* count, double* out) {
  __shared__ bool last;
  const double b = block_sum(acc.value());
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += __ldcg(partial + i);
  v = block_sum(v);
  if (threadIdx.x == 0) {
    *out = v;
    *count = 0u;
  }
}

// Ap = p + scale R^-1/2 y (y = R2C of the pointwise product) and <p, Ap>.
__global__ void __launch_bounds__(256) k_tl_spec_finish(int64_t Ch, const float2* __restrict__ fw,
                                                        const cufftComplex* __restrict__ p,
                                                        const cufftComplex* __restrict__ y,
                                                        cufftComplex* __restrict__ Ap,
                                                        float scale,
                                                        double* __restrict__ partial,
                                                        unsigned* __restrict__ count,
                                                        double* __restrict__ pAp) {
  KahanF acc;
  CLAIRE_SPEC_LOOP {
    const float2 t = fw[m];
    const float f = scale * t.x;
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cufftComplex pv = p[c * Ch + m], yv = y[c * Ch + m];
      const cufftComplex a = make_cuComplex(fmaf(f, yv.x, pv.x), fmaf(f, yv.y, pv.y));
      Ap[c * Ch + m] = a;
      d = fmaf(pv.x, a.x, fmaf(pv.y, a.y, d));
    }
    acc.add(t.y * d);
  }
  spec_partial_final(partial, acc, count, pAp);
}

// CG step on spectra: a = rr / pAp (0 when pAp <= 0 or not finite), x += a p,
// r -= a Ap, and ||r||^2 into *rr_new.
__global__ void __launch_bounds__(256) k_tl_spec_step(int64_t Ch, const float2* __restrict__ fw,
                                                      const double* __restrict__ rr,
                                                      const double* __restrict__ pAp,
                                                      cufftComplex* __restrict__ x,
                                                      cufftComplex* __restrict__ r,
                                                      const cufftComplex* __restrict__ p,
                                                      const cufftComplex* __restrict__ Ap,
                                                      double* __restrict__ partial,
                                                      unsigned* __restrict__ count,
                                                      double* __restrict__ rr_new) {
  const double q = *pAp;
  const float a = (q > 0.0 && isfinite(q)) ? (float)(*rr / q) : 0.0f;
  KahanF acc;
  CLAIRE_SPEC_LOOP {
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = c * Ch + m;
      const cufftComplex pv = p[i], av = Ap[i];
      cufftComplex xv = x[i], rv = r[i];
      xv.x = fmaf(a, pv.x, xv.x); xv.y = fmaf(a, pv.y, xv.y);
      rv.x = fmaf(-a, av.x, rv.x); rv.y = fmaf(-a, av.y, rv.y);
      x[i] = xv;
      r[i] = rv;
      d = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, d));
    }
    acc.add(fw[m].y * d);
  }
  spec_partial_final(partial, acc, count, rr_new);
}

// x = 0, r = p = b, ||b||^2 into *bb, and b in place scaled to R^-1/2 b: the input
// of the first operator application.
__global__ void __launch_bounds__(256) k_tl_spec_init(int64_t Ch, const float2* __restrict__ fw,
                                                      cufftComplex* __restrict__ b,
                                                      cufftComplex* __restrict__ x,
                                                      cufftComplex* __restrict__ r,
                                                      cufftComplex* __restrict__ p,
                                                      double* __restrict__ partial,
                                                      unsigned* __restrict__ count,
                                                      double* __restrict__ bb) {
  KahanF acc;
  CLAIRE_SPEC_LOOP {
    const float2 t = fw[m];
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = c * Ch + m;
      const cufftComplex v = b[i];
      x[i] = make_cuComplex(0.f, 0.f);
      r[i] = v;
      p[i] = v;
      b[i] = make_cuComplex(t.x * v.x, t.x * v.y);
      d = fmaf(v.x, v.x, fmaf(v.y, v.y, d));
    }
    acc.add(t.y * d);
  }
  spec_partial_final(partial, acc, count, bb);
}

// p = r + (rr_new / rr_old) p, and R^-1/2 p into cc: the direction update fused
// with the scaling that starts the next operator application.
__global__ void k_tl_dir_scale(int64_t Ch, const float2* __restrict__ fw,
                               const double* __restrict__ rr_new,
                               const double* __restrict__ rr_old,
                               const cufftComplex* __restrict__ r, cufftComplex* __restrict__ p,
                               cufftComplex* __restrict__ cc) {
  const float bt = (float)(*rr_new / *rr_old);
  CLAIRE_SPEC_LOOP {
    const float f = fw[m].x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = c * Ch + m;
      const cufftComplex rv = r[i], pv = p[i];
      const cufftComplex q = make_cuComplex(fmaf(bt, pv.x, rv.x), fmaf(bt, pv.y, rv.y));
      p[i] = q;
      cc[i] = make_cuComplex(f * q.x, f * q.y);
    }
  }
}
#undef CLAIRE_SPEC_LOOP

// FP16 field (scaled by sig) -> FP32 field / sig.
__global__ void k_tl_unscale_h(int64_t n, const __half* __restrict__ h, float inv,
                               float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = inv * __half2float(h[i]);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void launch_tl_split(const Grid& gf, cufftComplex* X, cufftComplex* C, int ncomp, int symbol,
                     float alpha, float gamma, float scale, cudaStream_t st) {
  const int64_t Nh = (int64_t)gf.n1 * gf.n2 * (gf.n3 / 2 + 1);
  ProfileRange pr(K_PRECOND, (double)Nh * ncomp * (symbol ? 16 : 8) + (double)Nh * ncomp, st);
  k_tl_split<<<nblk(Nh), 256, 0, st>>>(gf, X, C, ncomp, symbol, alpha, gamma, scale);
}

void launch_tl_merge(const Grid& gf, cufftComplex* X, const cufftComplex* C, cufftComplex* X2,
                     float alpha, float gamma, float sf, float sc, cudaStream_t st) {
  const int64_t Nh = (int64_t)gf.n1 * gf.n2 * (gf.n3 / 2 + 1);
  ProfileRange pr(K_PRECOND, (double)Nh * 3 * 24, st);
  k_tl_merge<<<nblk(Nh), 256, 0, st>>>(gf, X, C, X2, alpha, gamma, sf, sc);
}

void launch_tl_outer(int64_t n, const float* gm, const float* q, float* w, cudaStream_t st) {
  ProfileRange pr(K_PRECOND, (double)n * 36, st);
  k_tl_outer<<<vector_blocks(n), 256, 0, st>>>(n, gm, q, w);
}


static int64_t coarse_half(const Grid& gc) { return (int64_t)gc.n1 * gc.n2 * (gc.n3 / 2 + 1); }
static unsigned spec_grid(const Grid& gc) { return (unsigned)vector_blocks(coarse_half(gc)); }
int tl_spec_blocks(const Grid& gc) { return vector_blocks(coarse_half(gc)); }

void launch_tl_spec_table(const Grid& gc, float alpha, float gamma, float2* fw, cudaStream_t st) {
  const int64_t Ch = coarse_half(gc);
  ProfileRange pr(K_PRECOND, (double)Ch * 8, st);
  k_tl_spec_table<<<nblk(Ch), 256, 0, st>>>(Ch, gc.n1, gc.n2, gc.n3, alpha, gamma, fw);
}

void launch_tl_spec_finish(const Grid& gc, const float2* fw, const cufftComplex* p,
                           const cufftComplex* y, cufftComplex* Ap, float scale, double* partial,
                           unsigned* count, double* pAp, cudaStream_t st) {
  const int64_t Ch = coarse_half(gc);
  ProfileRange pr(K_PRECOND, (double)Ch * 3 * 24, st);
  k_tl_spec_finish<<<spec_grid(gc), 256, 0, st>>>(Ch, fw, p, y, Ap, scale, partial, count, pAp);
}

void launch_tl_spec_step(const Grid& gc, const float2* fw, const double* rr, const double* pAp,
                         cufftComplex* x, cufftComplex* r, const cufftComplex* p,
                         const cufftComplex* Ap, double* partial, unsigned* count,
                         double* rr_new, cudaStream_t st) {
  const int64_t Ch = coarse_half(gc);
  ProfileRange pr(K_PRECOND, (double)Ch * 3 * 48, st);
  k_tl_spec_step<<<spec_grid(gc), 256, 0, st>>>(Ch, fw, rr, pAp, x, r, p, Ap, partial, count,
                                                 rr_new);
}

void launch_tl_spec_init(const Grid& gc, const float2* fw, cufftComplex* b, cufftComplex* x,
                         cufftComplex* r, cufftComplex* p, double* partial, unsigned* count,
                         double* bb, cudaStream_t st) {
  const int64_t Ch = coarse_half(gc);
  ProfileRange pr(K_PRECOND, (double)Ch * 3 * 40, st);
  k_tl_spec_init<<<spec_grid(gc), 256, 0, st>>>(Ch, fw, b, x, r, p, partial, count, bb);
}

void launch_tl_dir_scale(const Grid& gc, const float2* fw, const double* rr_new,
                         const double* rr_old, const cufftComplex* r, cufftComplex* p,
                         cufftComplex* cc, cudaStream_t st) {
  const int64_t Ch = coarse_half(gc);
  ProfileRange pr(K_PRECOND, (double)Ch * 3 * 32, st);
  k_tl_dir_scale<<<spec_grid(gc), 256, 0, st>>>(Ch, fw, rr_new, rr_old, r, p, cc);
}

// ---- nested CG driven on the device (a captured graph with a conditional while
// node): the same iteration and the same stopping decisions as the host loop of
// the preconditioner, taken by one thread from the FP64 slots.

// Before the loop: stop2 = rtol^2 <b, b>, iteration count 0, and whether to iterate.
__global__ void k_tl_cg_begin(cudaGraphConditionalHandle h, const double* __restrict__ rr0,
                              const double* __restrict__ rtol, double* __restrict__ stop2,
                              double* __restrict__ count, int max_inner) {
  const double r = *rr0, t = *rtol;
  const double s2 = t * t * r;
  *stop2 = s2;
  *count = 0.0;
  cudaGraphSetConditional(h, (max_inner > 0 && r > s2 && isfinite(r)) ? 1u : 0u);
}

// After an iteration (step, then direction): rr <- rr_new, count the iteration, and
// continue only after a positive-curvature step that left the residual above the
// tolerance, below the iteration cap.
__global__ void k_tl_cg_control(cudaGraphConditionalHandle h, double* __restrict__ rr,
                                const double* __restrict__ rr_new, const double* __restrict__ pAp,
                                const double* __restrict__ stop2, double* __restrict__ count,
                                double* __restrict__ total, int max_inner) {
  const double q = *pAp, rn = *rr_new;
  const double it = *count + 1.0;
  *count = it;
  *total += 1.0;
  *rr = rn;
  const bool go = q > 0.0 && isfinite(q) && rn > *stop2 && it < (double)max_inner;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_set_scalar(double* __restrict__ p, double v) { *p = v; }

void launch_tl_cg_begin(cudaGraphConditionalHandle h, const double* rr0, const double* rtol,
                        double* stop2, double* count, int max_inner, cudaStream_t st) {
  ProfileRange pr(K_PRECOND, 32.0, st);
  k_tl_cg_begin<<<1, 1, 0, st>>>(h, rr0, rtol, stop2, count, max_inner);
}

void launch_tl_cg_control(cudaGraphConditionalHandle h, double* rr, const double* rr_new,
                          const double* pAp, const double* stop2, double* count, double* total,
                          int max_inner, cudaStream_t st) {
  ProfileRange pr(K_PRECOND, 56.0, st);
  k_tl_cg_control<<<1, 1, 0, st>>>(h, rr, rr_new, pAp, stop2, count, total, max_inner);
}

void launch_set_scalar(double* p, double v, cudaStream_t st) {
  ProfileRange pr(K_VECTOR, 8.0, st);
  k_set_scalar<<<1, 1, 0, st>>>(p, v);
}

void launch_tl_unscale_h(int64_t n, const __half* h, float inv, float* out, cudaStream_t st) {
  ProfileRange pr(K_PRECOND, (double)n * 6, st);
  k_tl_unscale_h<<<vector_blocks(n), 256, 0, st>>>(n, h, inv, out);
}

}  // namespace claire
