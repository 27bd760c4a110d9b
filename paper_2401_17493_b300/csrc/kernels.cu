// Device kernels of the registration hot path and their host launchers.
//
//  k_trace            RK2 departure points, both directions      (Sec. 2.5.2)
//  k_sl               one SL step: out = s(x) gather(u, x + d) + beta aux(x)
//  k_adjoint_factor   c(x) of the RK2 adjoint step with f = lam div v
//  k_grad8 / k_div8   FD8 gradient / divergence                   (Sec. 2.5.3)
//  k_sdot_hist        s^j = grad8(m^j) . v~ for the whole state history
//  k_accum_hist       out = base_coef * base + sum_j w_j lam^j grad8(m^j)
//  k_spectral         diagonal Fourier multipliers between cuFFT R2C / C2R
//  k_reduce*          FP64 reductions (fixed block count, fixed order)
//  small vector kernels for PCG and the line search
//
// All grids are [n1][n2][n3] with n3 fastest; 3D kernels use 32 x 4 x 2
// thread blocks (x3 along threadIdx.x for coalescing, a compact 3D footprint
// for the L1 reuse of the 64-tap gathers).
#include <math_constants.h>

#include "internal.h"

namespace claire {

#define CLAIRE_KERNEL_INDEX                                               \
  const int i3 = blockIdx.x * blockDim.x + threadIdx.x;                   \
  const int i2 = blockIdx.y * blockDim.y + threadIdx.y;                   \
  const int i1 = blockIdx.z * blockDim.z + threadIdx.z;                   \
  if (i1 >= g.n1 || i2 >= g.n2 || i3 >= g.n3) return;                     \
  const int64_t idx = lin(g, i1, i2, i3);

static dim3 block3() { return dim3(32, 4, 2); }
static dim3 grid3(const Grid& g) {
  return dim3((g.n3 + 31) / 32, (g.n2 + 3) / 4, (g.n1 + 1) / 2);
}

// ---------------------------------------------------------------- trace

__global__ void __launch_bounds__(256) k_trace(Grid g, const float* __restrict__ v,
                                               float* __restrict__ df, float* __restrict__ db,
                                               float ht) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  const float u1 = v[idx] * g.inv_h1;       // velocity in grid units per unit time
  const float u2 = v[N + idx] * g.inv_h2;
  const float u3 = v[2 * N + idx] * g.inv_h3;
  const int s1 = g.n2 * g.n3;
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    float* out = dir == 0 ? df : db;
    if (out == nullptr) continue;
    // transport along +v (dir 0) or -v (dir 1): predictor y~ = x -+ h_t v(x)
    const float s = dir == 0 ? -ht : ht;
    Taps a, b, c;
    axis_taps(i1, s * u1, g.n1, s1, a);
    axis_taps(i2, s * u2, g.n2, g.n3, b);
    axis_taps(i3, s * u3, g.n3, 1, c);
    const float w1 = gather64(v, a, b, c) * g.inv_h1;
    const float w2 = gather64(v + N, a, b, c) * g.inv_h2;
    const float w3 = gather64(v + 2 * N, a, b, c) * g.inv_h3;
    // corrector y = x -+ (h_t / 2)(v(x) + v(y~)), stored as y - x in grid units
    out[idx] = 0.5f * s * (u1 + w1);
    out[N + idx] = 0.5f * s * (u2 + w2);
    out[2 * N + idx] = 0.5f * s * (u3 + w3);
  }
}

// ---------------------------------------------------------------- SL step

__global__ void __launch_bounds__(256) k_sl(Grid g, const float* __restrict__ u,
                                            const float* __restrict__ d,
                                            const float* __restrict__ scale, float sigma,
                                            const float* __restrict__ aux, float beta,
                                            float* __restrict__ out) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  Taps a, b, c;
  axis_taps(i1, d[idx], g.n1, g.n2 * g.n3, a);
  axis_taps(i2, d[N + idx], g.n2, g.n3, b);
  axis_taps(i3, d[2 * N + idx], g.n3, 1, c);
  float r = gather64(u, a, b, c);
  r *= scale ? scale[idx] : sigma;
  if (aux) r = fmaf(beta, aux[idx], r);
  out[idx] = r;
}

// c(x) = 1 + (h_t/2)(D(y) + D(x) + h_t D(x) D(y)): one RK2 step of
// d_t lam = lam D along -v collapses to lam^j(x) = c(x) lam^{j+1}(y).
__global__ void __launch_bounds__(256) k_adjoint_factor(Grid g, const float* __restrict__ D,
                                                        const float* __restrict__ db,
                                                        float ht, float* __restrict__ cf) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  Taps a, b, c;
  axis_taps(i1, db[idx], g.n1, g.n2 * g.n3, a);
  axis_taps(i2, db[N + idx], g.n2, g.n3, b);
  axis_taps(i3, db[2 * N + idx], g.n3, 1, c);
  const float Dy = gather64(D, a, b, c);
  const float Dx = D[idx];
  cf[idx] = 1.0f + 0.5f * ht * (Dy + Dx + ht * Dx * Dy);
}

// ---------------------------------------------------------------- FD8

__global__ void __launch_bounds__(256) k_grad8(Grid g, const float* __restrict__ u,
                                               float* __restrict__ gu) {
  CLAIRE_KERNEL_INDEX
  float gr[3];
  grad8_at(u, g, i1, i2, i3, gr);
  gu[idx] = gr[0];
  gu[g.N + idx] = gr[1];
  gu[2 * g.N + idx] = gr[2];
}

__device__ __forceinline__ float d8_axis(const float* __restrict__ u, const Grid& g, int i1,
                                         int i2, int i3, int axis) {
  float m[4], p[4];
  if (axis == 0) {
    const int64_t s1 = (int64_t)g.n2 * g.n3;
    const float* base = u + (int64_t)i2 * g.n3 + i3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m[k] = __ldg(base + wrap_near(i1 - 1 - k, g.n1) * s1);
      p[k] = __ldg(base + wrap_near(i1 + 1 + k, g.n1) * s1);
    }
    return fd8(m[3], m[2], m[1], m[0], p[0], p[1], p[2], p[3], g.inv_h1);
  } else if (axis == 1) {
    const float* base = u + (int64_t)i1 * g.n2 * g.n3 + i3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m[k] = __ldg(base + (int64_t)wrap_near(i2 - 1 - k, g.n2) * g.n3);
      p[k] = __ldg(base + (int64_t)wrap_near(i2 + 1 + k, g.n2) * g.n3);
    }
    return fd8(m[3], m[2], m[1], m[0], p[0], p[1], p[2], p[3], g.inv_h2);
  }
  const float* base = u + ((int64_t)i1 * g.n2 + i2) * g.n3;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    m[k] = __ldg(base + wrap_near(i3 - 1 - k, g.n3));
    p[k] = __ldg(base + wrap_near(i3 + 1 + k, g.n3));
  }
  return fd8(m[3], m[2], m[1], m[0], p[0], p[1], p[2], p[3], g.inv_h3);
}

__global__ void __launch_bounds__(256) k_div8(Grid g, const float* __restrict__ w,
                                              float* __restrict__ out) {
  CLAIRE_KERNEL_INDEX
  out[idx] = d8_axis(w, g, i1, i2, i3, 0) + d8_axis(w + g.N, g, i1, i2, i3, 1) +
             d8_axis(w + 2 * g.N, g, i1, i2, i3, 2);
}

// s^j = grad8(m^j) . vt for j = 0..nt (m^j = mhist + j N); s^0 is scaled by scale0.
__global__ void __launch_bounds__(256) k_sdot_hist(Grid g, const float* __restrict__ mhist,
                                                   int nt, const float* __restrict__ vt,
                                                   float scale0, float* __restrict__ shist) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  const float t1 = vt[idx], t2 = vt[N + idx], t3 = vt[2 * N + idx];
  for (int j = 0; j <= nt; ++j) {
    float gr[3];
    grad8_at(mhist + j * N, g, i1, i2, i3, gr);
    float s = gr[0] * t1;
    s = fmaf(gr[1], t2, s);
    s = fmaf(gr[2], t3, s);
    shist[j * N + idx] = j == 0 ? scale0 * s : s;
  }
}

// out = base_coef * base + sum_{j=0..nt} w_j lam^j grad8(m^j), trapezoid weights
// w_j = h_t (1/2, 1, ..., 1, 1/2)  (Sec. 2.5.1).  base may be NULL.
__global__ void __launch_bounds__(256) k_accum_hist(Grid g, const float* __restrict__ lhist,
                                                    const float* __restrict__ mhist, int nt,
                                                    const float* __restrict__ base,
                                                    float base_coef, float* __restrict__ out) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  const float ht = 1.0f / nt;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int j = 0; j <= nt; ++j) {
    float gr[3];
    grad8_at(mhist + j * N, g, i1, i2, i3, gr);
    const float wl = ((j == 0 || j == nt) ? 0.5f * ht : ht) * lhist[j * N + idx];
    acc0 = fmaf(wl, gr[0], acc0);
    acc1 = fmaf(wl, gr[1], acc1);
    acc2 = fmaf(wl, gr[2], acc2);
  }
  if (base) {
    acc0 = fmaf(base_coef, base[idx], acc0);
    acc1 = fmaf(base_coef, base[N + idx], acc1);
    acc2 = fmaf(base_coef, base[2 * N + idx], acc2);
  }
  out[idx] = acc0;
  out[N + idx] = acc1;
  out[2 * N + idx] = acc2;
}

// ---------------------------------------------------------------- spectral

// Half spectrum [n1][n2][n3/2+1] of 3 components (stride Nc).  Integer
// wavenumbers k_i in FFT order; scale folds in cuFFT's 1/N.
__global__ void k_spectral(int n1, int n2, int n3, int64_t Nc, cufftComplex* __restrict__ X,
                           int op, float alpha, float gamma, float beta_w, float scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nc) return;
  const int nh = n3 / 2 + 1;
  const int j3 = (int)(i % nh);
  const int j2 = (int)((i / nh) % n2);
  const int j1 = (int)(i / ((int64_t)nh * n2));
  const float k1 = (float)(j1 <= n1 / 2 ? j1 : j1 - n1);
  const float k2 = (float)(j2 <= n2 / 2 ? j2 : j2 - n2);
  const float k3 = (float)j3;
  const float kap = k1 * k1 + k2 * k2 + k3 * k3;
  cufftComplex x0 = X[i], x1 = X[Nc + i], x2 = X[2 * Nc + i];
  if (op == 0 || op == 1) {
    float sig = gamma == 1.0f ? kap : powf(kap, gamma);
    float f;
    if (op == 0) {
      f = sig * scale;                                  // L = (-Laplacian)^gamma
    } else {
      if (kap == 0.0f) sig = 1.0f;                      // zero symbol set to one
      f = scale / (alpha * sig);                        // (alpha L)^-1
    }
    x0.x *= f; x0.y *= f; x1.x *= f; x1.y *= f; x2.x *= f; x2.y *= f;
  } else {
    // P_par = k k^T / |k|^2 with Nyquist components of k zeroed (real result)
    const float q1 = (j1 == n1 / 2) ? 0.f : k1;
    const float q2 = (j2 == n2 / 2) ? 0.f : k2;
    const float q3 = (j3 == n3 / 2) ? 0.f : k3;
    const float qq = q1 * q1 + q2 * q2 + q3 * q3;
    float f = 0.0f;
    if (qq > 0.0f) {
      f = scale / qq;
      if (op == 3) {
        const float num = beta_w * (1.0f + kap);
        f *= num / (num + alpha * kap);
      }
    }
    const float re = (q1 * x0.x + q2 * x1.x + q3 * x2.x) * f;
    const float im = (q1 * x0.y + q2 * x1.y + q3 * x2.y) * f;
    x0.x = q1 * re; x0.y = q1 * im;
    x1.x = q2 * re; x1.y = q2 * im;
    x2.x = q3 * re; x2.y = q3 * im;
  }
  X[i] = x0; X[Nc + i] = x1; X[2 * Nc + i] = x2;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// max that keeps a NaN (fmax would drop it): the infinity norm must expose non-finite fields
__device__ __forceinline__ double nanmax(double a, double b) {
  return a != a ? a : (b != b ? b : fmax(a, b));
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double nanmin(double a, double b) {
  return a != a ? a : (b != b ? b : fmin(a, b));
}

// Reduction modes (ReduceMode): 0 sum a b, 1 sum (a - b)^2, 2 max |a|, 3 sum a^2,
// 4 max a, 5 min a, 6 sum a.  Max / min keep NaNs so non-finite fields show.
__device__ __forceinline__ bool red_is_max(int mode) { return mode == 2 || mode == 4; }
__device__ __forceinline__ double red_init(int mode) {
  return mode == 4 ? -CUDART_INF : (mode == 5 ? CUDART_INF : 0.0);
}
__device__ __forceinline__ double red_combine(int mode, double a, double b) {
  return red_is_max(mode) ? nanmax(a, b) : (mode == 5 ? nanmin(a, b) : a + b);
}
__device__ __forceinline__ double warp_red(int mode, double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = red_combine(mode, v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_red(int mode, double acc) {
  __shared__ double sh[32];
  acc = warp_red(mode, acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  double v = red_init(mode);
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : red_init(mode);
    v = warp_red(mode, v);
  }
  return v;
}

__global__ void __launch_bounds__(256) k_reduce(int64_t n, const float* __restrict__ a,
                                                const float* __restrict__ b, int mode,
                                                double* __restrict__ partial) {
  double acc = red_init(mode);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i];
    double t;
    switch (mode) {
      case 0: t = x * (double)b[i]; break;
      case 1: { const double d = x - (double)b[i]; t = d * d; } break;
      case 2: t = fabs(x); break;
      case 3: t = x * x; break;
      default: t = x;
    }
    acc = red_combine(mode, acc, t);
  }
  const double v = block_red(mode, acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

__global__ void k_reduce_final(const double* __restrict__ partial, int nb, int mode,
                               double* __restrict__ out) {
  double acc = red_init(mode);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc = red_combine(mode, acc, partial[i]);
  const double v = block_red(mode, acc);
  if (threadIdx.x == 0) *out = v;
}

// ---------------------------------------------------------------- vectors

__global__ void k_axpby(int64_t n, float a, const float* __restrict__ x, float b,
                        float* __restrict__ y) {   // y = a x + b y
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], b * y[i]);
}

__global__ void k_lincomb(int64_t n, float a, const float* __restrict__ x, float b,
                          const float* __restrict__ y, float* __restrict__ out) {  // out = a x + b y
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fmaf(a, x[i], b * y[i]);
}

// ---------------------------------------------------------------- det F1

// One RK2 SL step of d_t F = (grad v) F along +v (Appendix, eq. def-grad):
// f0 = A(y) F(y), F~ = F(y) + h_t f0, f1 = A(x) F~, F' = F(y) + (h_t/2)(f0 + f1).
// F, A, Ay hold 9 fields [3a + b][N]; det (optional) receives det F'.
__global__ void __launch_bounds__(256) k_detf_step(Grid g, const float* __restrict__ F,
                                                   const float* __restrict__ df,
                                                   const float* __restrict__ A,
                                                   const float* __restrict__ Ay, float ht,
                                                   float* __restrict__ Fn,
                                                   float* __restrict__ det) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  Taps a, b, c;
  axis_taps(i1, df[idx], g.n1, g.n2 * g.n3, a);
  axis_taps(i2, df[N + idx], g.n2, g.n3, b);
  axis_taps(i3, df[2 * N + idx], g.n3, 1, c);
  float Fy[9], Ax[9], Ayy[9], f0[9], Ft[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Fy[k] = gather64(F + k * N, a, b, c);
    Ax[k] = A[k * N + idx];
    Ayy[k] = Ay[k * N + idx];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) s = fmaf(Ayy[3 * r + k], Fy[3 * k + q], s);
      f0[3 * r + q] = s;
      Ft[3 * r + q] = fmaf(ht, s, Fy[3 * r + q]);
    }
  float Fo[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float f1 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) f1 = fmaf(Ax[3 * r + k], Ft[3 * k + q], f1);
      Fo[3 * r + q] = fmaf(0.5f * ht, f0[3 * r + q] + f1, Fy[3 * r + q]);
      Fn[(3 * r + q) * N + idx] = Fo[3 * r + q];
    }
  if (det) {
    det[idx] = Fo[0] * (Fo[4] * Fo[8] - Fo[5] * Fo[7]) - Fo[1] * (Fo[3] * Fo[8] - Fo[5] * Fo[6]) +
               Fo[2] * (Fo[3] * Fo[7] - Fo[4] * Fo[6]);
  }
}

// A[3a + b] = d_b v_a (FD8) and its values at the departure points y.
__global__ void __launch_bounds__(256) k_detf_init(Grid g, const float* __restrict__ v,
                                                   float* __restrict__ A,
                                                   float* __restrict__ F) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float gr[3];
    grad8_at(v + r * N, g, i1, i2, i3, gr);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A[(3 * r + q) * N + idx] = gr[q];
      F[(3 * r + q) * N + idx] = r == q ? 1.0f : 0.0f;
    }
  }
}

// ---------------------------------------------------------------- profiler

thread_local Profiler* tl_prof = nullptr;

const char* kernel_kind_name(int k) {
  static const char* names[K_COUNT] = {"trace", "sl_step", "adjoint_factor", "grad8", "div8",
                                       "sdot_hist", "accum_hist", "spectral_diag", "reduce",
                                       "vector", "detf", "cufft"};
  return (k >= 0 && k < K_COUNT) ? names[k] : "?";
}

void Profiler::reset(bool timing_on) {
  resolve();
  timing = timing_on;
  for (int k = 0; k < K_COUNT; ++k) {
    launches[k] = 0;
    bytes[k] = 0.0;
    ms[k] = 0.0;
    timed[k] = 0;
  }
}

cudaEvent_t Profiler::take() {
  if (pool.empty()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}

cudaError_t Profiler::resolve() {
  cudaError_t err = cudaSuccess;
  for (auto& p : pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e == cudaSuccess) {
      ms[p.kind] += t;
      timed[p.kind] += 1;
    } else if (err == cudaSuccess) {
      err = e;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  return err;
}

void Profiler::release() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

ProfileRange::ProfileRange(int k, double b, cudaStream_t s) : kind(k), st(s) {
  Profiler* p = tl_prof;
  if (!p) return;
  p->launches[k] += 1;
  p->bytes[k] += b;
  if (p->timing) {
    a = p->take();
    if (a) cudaEventRecord(a, s);
  }
}

ProfileRange::~ProfileRange() {
  Profiler* p = tl_prof;
  if (!p || !a) return;
  cudaEvent_t b = p->take();
  if (!b) return;
  cudaEventRecord(b, st);
  p->pending.push_back({kind, a, b});
  if (p->pending.size() > 8192) p->resolve();
}

// ---------------------------------------------------------------- launchers

static int g_num_sms = 0;
static int vec_blocks(int64_t n) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  int64_t want = (n + 255) / 256;
  int64_t cap = (int64_t)g_num_sms * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

void launch_trace(const Grid& g, const float* v, float* df, float* db, float ht,
                  cudaStream_t st) {
  ProfileRange pr(K_TRACE, (double)g.N * (12 + 12 * ((df != nullptr) + (db != nullptr))), st);
  k_trace<<<grid3(g), block3(), 0, st>>>(g, v, df, db, ht);
}
void launch_sl(const Grid& g, const float* u, const float* d, const float* scale, float sigma,
               const float* aux, float beta, float* out, cudaStream_t st) {
  ProfileRange pr(K_SL, (double)g.N * (20 + 4 * (scale != nullptr) + 4 * (aux != nullptr)), st);
  k_sl<<<grid3(g), block3(), 0, st>>>(g, u, d, scale, sigma, aux, beta, out);
}
void launch_adjoint_factor(const Grid& g, const float* D, const float* db, float ht, float* c,
                           cudaStream_t st) {
  ProfileRange pr(K_ADJFAC, (double)g.N * 20, st);
  k_adjoint_factor<<<grid3(g), block3(), 0, st>>>(g, D, db, ht, c);
}
void launch_grad8(const Grid& g, const float* u, float* gu, cudaStream_t st) {
  ProfileRange pr(K_GRAD8, (double)g.N * 16, st);
  k_grad8<<<grid3(g), block3(), 0, st>>>(g, u, gu);
}
void launch_div8(const Grid& g, const float* w, float* out, cudaStream_t st) {
  ProfileRange pr(K_DIV8, (double)g.N * 16, st);
  k_div8<<<grid3(g), block3(), 0, st>>>(g, w, out);
}
void launch_sdot_hist(const Grid& g, const float* mhist, int nt, const float* vt, float scale0,
                      float* shist, cudaStream_t st) {
  ProfileRange pr(K_SDOT, (double)g.N * (12 + 8 * (nt + 1)), st);
  k_sdot_hist<<<grid3(g), block3(), 0, st>>>(g, mhist, nt, vt, scale0, shist);
}
void launch_accum_hist(const Grid& g, const float* lhist, const float* mhist, int nt,
                       const float* base, float base_coef, float* out, cudaStream_t st) {
  ProfileRange pr(K_ACCUM, (double)g.N * (8 * (nt + 1) + 12 + 12 * (base != nullptr)), st);
  k_accum_hist<<<grid3(g), block3(), 0, st>>>(g, lhist, mhist, nt, base, base_coef, out);
}
void launch_spectral(const Grid& g, cufftComplex* X, int op, float alpha, float gamma,
                     float beta_w, cudaStream_t st) {
  const int64_t Nc = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  const float scale = (float)(1.0 / (double)g.N);
  ProfileRange pr(K_SPECTRAL, (double)Nc * 3 * 16, st);
  k_spectral<<<(unsigned)((Nc + 255) / 256), 256, 0, st>>>(g.n1, g.n2, g.n3, Nc, X, op, alpha,
                                                           gamma, beta_w, scale);
}
void launch_reduce(int64_t n, const float* a, const float* b, int mode, double* partial,
                   int nblocks, double* out, cudaStream_t st) {
  ProfileRange pr(K_REDUCE, (double)n * 4 * (b != nullptr ? 2 : 1), st);
  if (tl_prof) tl_prof->launches[K_REDUCE] += 1;    // two kernels per reduction
  k_reduce<<<nblocks, 256, 0, st>>>(n, a, b, mode, partial);
  k_reduce_final<<<1, 1024, 0, st>>>(partial, nblocks, mode, out);
}
void launch_axpby(int64_t n, float a, const float* x, float b, float* y, cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 12, st);
  k_axpby<<<vec_blocks(n), 256, 0, st>>>(n, a, x, b, y);
}
void launch_lincomb(int64_t n, float a, const float* x, float b, const float* y, float* out,
                    cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 12, st);
  k_lincomb<<<vec_blocks(n), 256, 0, st>>>(n, a, x, b, y, out);
}
void launch_detf(const Grid& g, const float* v, const float* df, int nt, float* F, float* Fn,
                 float* A, float* Ay, float* det, cudaStream_t st) {
  {
    ProfileRange pr(K_DETF, (double)g.N * (12 + 36 + 36), st);
    k_detf_init<<<grid3(g), block3(), 0, st>>>(g, v, A, F);
  }
  for (int k = 0; k < 9; ++k)
    launch_sl(g, A + k * g.N, df, nullptr, 1.0f, nullptr, 0.f, Ay + k * g.N, st);
  const float ht = 1.0f / nt;
  for (int j = 0; j < nt; ++j) {
    ProfileRange pr(K_DETF, (double)g.N * (12 + 36 * 4 + (j == nt - 1 ? 4 : 0)), st);
    k_detf_step<<<grid3(g), block3(), 0, st>>>(g, F, df, A, Ay, ht, Fn,
                                               j == nt - 1 ? det : nullptr);
    float* t = F;
    F = Fn;
    Fn = t;
  }
}

}  // namespace claire
