// Mixed-precision form: the gathered and stencilled fields (state, adjoint,
// incremental state / adjoint histories) are stored in FP16; interpolation
// weights, arithmetic, departure points and PCG vectors stay FP32, reductions
// FP64.  Stored fields carry power-of-two scales (exact in FP16) so that
// they stay inside the FP16 range: the images are scaled to max |m| in
// (1/2, 1], the incremental fields by 2^-ceil(log2 ||s||_inf) of the
// direction s.  Results are unscaled in FP32.
//
// Brick layout for FP16 (tricubic gather): every staged row of 40 halves is
// held twice as half2 words, copy A pairs (u0,u1),(u2,u3),... and copy B
// pairs (u1,u2),(u3,u4),..., so the four x3 taps u_c..u_{c+3} are always two
// aligned 32-bit shared loads (A when c is even, B when c is odd) instead of
// four.  Copy B starts 16 banks after copy A: neighbouring lanes (which have
// opposite parity) read disjoint banks.
#include <cuda_fp16.h>
#include <math_constants.h>

#include <mutex>

#include "internal.h"
#include "reduce.cuh"
#include "sl_brick.cuh"
#include "fd8_march.cuh"

namespace claire {

constexpr int HROW_W = 32;                         // words per row of a copy (20 used)
constexpr int HX3 = BX3;                           // 40 staged halves per row
// words of one copy at tile depth t1, the offset of copy B (16 banks after A)
// and the brick size: 6272 / 6288 / 12560 words at depth 8
__host__ __device__ inline int hcopy_w(int t1) { return brick_rows(t1) * HROW_W; }
__host__ __device__ inline int hb_off(int t1) { return hcopy_w(t1) + 16; }
__host__ __device__ inline int hbrick_w(int t1) { return hb_off(t1) + hcopy_w(t1); }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Stage an FP16 field over the tile plus halo into copy A, then derive copy B.
__device__ __forceinline__ void stage_brick_h(const __half* __restrict__ u, const Grid& g,
                                              int i1_0, int i2_0, int i3_0,
                                              uint32_t* __restrict__ s, int t1) {
  const int rows = brick_rows(t1), boff = hb_off(t1);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int x3s = i3_0 - HB3_LO;
  const bool vec = (g.n3 % 4 == 0) && x3s >= 0 && x3s + HX3 <= g.n3 &&
                   ((reinterpret_cast<uintptr_t>(u) & 7) == 0);
  __half* sh = reinterpret_cast<__half*>(s);
  if (vec) {
    constexpr int Q = HX3 / 4;                     // 8-byte chunks per row
    for (int item = tid; item < rows * Q; item += BRICK_THREADS) {
      const int row = item / Q, q = item - row * Q;
      const int r1 = row / BB2, r2 = row - r1 * BB2;
      const int g1 = wrap_any(i1_0 - HB_LO + r1, g.n1);
      const int g2 = wrap_any(i2_0 - HB_LO + r2, g.n2);
      const __half* src = u + ((int64_t)g1 * g.n2 + g2) * g.n3 + x3s + 4 * q;
      cp_async8(s + row * HROW_W + 2 * q, src);
    }
    cp_async_wait_all();
  } else {
    for (int item = tid; item < rows * HX3; item += BRICK_THREADS) {
      const int row = item / HX3, e = item - row * HX3;
      const int r1 = row / BB2, r2 = row - r1 * BB2;
      const int g1 = wrap_any(i1_0 - HB_LO + r1, g.n1);
      const int g2 = wrap_any(i2_0 - HB_LO + r2, g.n2);
      sh[row * 2 * HROW_W + e] =
          u[((int64_t)g1 * g.n2 + g2) * g.n3 + wrap_any(x3s + e, g.n3)];
    }
  }
  __syncthreads();
  // copy B: word w = (u_{2w+1}, u_{2w+2}) for w = 0..18
  for (int item = tid; item < rows * 19; item += BRICK_THREADS) {
    const int row = item / 19, w = item - row * 19;
    const uint32_t lo = s[row * HROW_W + w], hi = s[row * HROW_W + w + 1];
    s[boff + row * HROW_W + w] = __byte_perm(lo, hi, 0x5432);   // (lo.hi, hi.lo)
  }
}

__device__ __forceinline__ float2 unpack_h2(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

__device__ __forceinline__ float gather_brick_h(const uint32_t* __restrict__ s,
                                                const NodeTaps& t, int k, int ty, int lane,
                                                int boff) {
  const int c0 = lane + HB3_LO + t.p3 - 1;                     // first x3 tap, in halves
  const uint32_t* b = s + ((c0 & 1) ? boff : 0) +
                      ((k + HB_LO + t.p1 - 1) * BB2 + (ty + HB_LO + t.p2 - 1)) * HROW_W +
                      (c0 >> 1);
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float acc2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t* row = b + (i * BB2 + j) * HROW_W;
      const float2 p = unpack_h2(row[0]), q = unpack_h2(row[1]);
      float acc3 = t.w3[0] * p.x;
      acc3 = fmaf(t.w3[1], p.y, acc3);
      acc3 = fmaf(t.w3[2], q.x, acc3);
      acc3 = fmaf(t.w3[3], q.y, acc3);
      acc2 = fmaf(t.w2[j], acc3, acc2);
    }
    acc = fmaf(t.w1[i], acc2, acc);
  }
  return acc;
}

__device__ __forceinline__ float gather_global_h(const __half* __restrict__ u, const Grid& g,
                                                 const NodeTaps& t, int i1, int i2, int i3) {
  int o1[4], o2[4], o3[4];
  const int b1 = wrap_any(i1 + t.p1 - 1, g.n1);
  const int b2 = wrap_any(i2 + t.p2 - 1, g.n2);
  const int b3 = wrap_any(i3 + t.p3 - 1, g.n3);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    o1[k] = wrap_near(b1 + k, g.n1) * g.n2 * g.n3;
    o2[k] = wrap_near(b2 + k, g.n2) * g.n3;
    o3[k] = wrap_near(b3 + k, g.n3);
  }
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float acc2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __half* row = u + o1[i] + o2[j];
      float acc3 = t.w3[0] * __half2float(row[o3[0]]);
      acc3 = fmaf(t.w3[1], __half2float(row[o3[1]]), acc3);
      acc3 = fmaf(t.w3[2], __half2float(row[o3[2]]), acc3);
      acc3 = fmaf(t.w3[3], __half2float(row[o3[3]]), acc3);
      acc2 = fmaf(t.w2[j], acc3, acc2);
    }
    acc = fmaf(t.w1[i], acc2, acc);
  }
  return acc;
}

// out = (scale ? scale(x) : sigma) u(x + d) + beta aux(x), u / aux / out in FP16.
__global__ void __launch_bounds__(BRICK_THREADS) k_sl_h(Grid g, const __half* __restrict__ u,
                                                        const float* __restrict__ d,
                                                        const float* __restrict__ scale,
                                                        float sigma,
                                                        const __half* __restrict__ aux,
                                                        float beta, __half* __restrict__ out,
                                                        int t1) {
  extern __shared__ __align__(16) uint32_t smw[];
  const int i1_0 = blockIdx.z * t1, i2_0 = blockIdx.y * TB2, i3_0 = blockIdx.x * TB3;
  stage_brick_h(u, g, i1_0, i2_0, i3_0, smw, t1);
  const int boff = hb_off(t1);
  __syncthreads();
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  if (i2 >= g.n2 || i3 >= g.n3) return;
  const int64_t N = g.N;
  const int kmax = min(t1, g.n1 - i1_0);
#pragma unroll 2
  for (int k = 0; k < kmax; ++k) {
    const int i1 = i1_0 + k;
    const int64_t idx = lin(g, i1, i2, i3);
    NodeTaps t;
    node_taps(d[idx], d[N + idx], d[2 * N + idx], t);
    const float y = taps_in_brick(t) ? gather_brick_h(smw, t, k, ty, lane, boff)
                                     : gather_global_h(u, g, t, i1, i2, i3);
    float r = y * (scale ? scale[idx] : sigma);
    if (aux) r = fmaf(beta, __half2float(aux[idx]), r);
    out[idx] = __float2half_rn(r);
  }
}

// ------------------------------------------------------------------ FD8 march

// Stage an FP16 plane (tile + FD8 halo) into shared memory as FP32: the
// conversion happens once per staged element instead of once per stencil read.
__device__ __forceinline__ void stage_plane_h(const __half* __restrict__ u, const Grid& g, int i1,
                                              int i2_0, int i3_0, float* __restrict__ s) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const __half* plane = u + (int64_t)i1 * g.n2 * g.n3;
  const int x3s = i3_0 - 4;
  const bool vec = (g.n3 % 4 == 0) && x3s >= 0 && x3s + MP3 <= g.n3 &&
                   ((reinterpret_cast<uintptr_t>(u) & 7) == 0);
  if (vec) {
    constexpr int Q = MP3 / 4;
    for (int item = tid; item < MP2 * Q; item += 32 * MT2) {
      const int r2 = item / Q, q = item - r2 * Q;
      const __half* src = plane + (int64_t)wrap_any(i2_0 - 4 + r2, g.n2) * g.n3 + x3s + 4 * q;
      const uint2 raw = __ldg(reinterpret_cast<const uint2*>(src));
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
      *reinterpret_cast<float4*>(s + r2 * MP3 + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
    }
  } else {
    for (int item = tid; item < MP2 * MP3; item += 32 * MT2) {
      const int r2 = item / MP3, e = item - r2 * MP3;
      s[item] = __half2float(
          plane[(int64_t)wrap_any(i2_0 - 4 + r2, g.n2) * g.n3 + wrap_any(x3s + e, g.n3)]);
    }
  }
}

// All NF history planes at once: every thread first issues its loads for all
// fields (at most one 8-byte chunk per field with 256 threads), then converts
// and stores, so the loads of the NF planes are in flight together.
template <int NF>
__device__ __forceinline__ void stage_planes_h(const __half* __restrict__ mhist, int64_t N,
                                               const Grid& g, int i1, int i2_0, int i3_0,
                                               float (*sp)[MPLANE]) {
  constexpr int Q = MP3 / 4;
  static_assert(MP2 * Q <= 32 * MT2, "one chunk per thread and field");
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int x3s = i3_0 - 4;
  const bool vec = (g.n3 % 4 == 0) && x3s >= 0 && x3s + MP3 <= g.n3 &&
                   ((reinterpret_cast<uintptr_t>(mhist) & 7) == 0);
  if (!vec) {
#pragma unroll
    for (int f = 0; f < NF; ++f) stage_plane_h(mhist + f * N, g, i1, i2_0, i3_0, sp[f]);
    return;
  }
  if (tid >= MP2 * Q) return;
  const int r2 = tid / Q, q = tid - r2 * Q;
  const int64_t off = (int64_t)i1 * g.n2 * g.n3 +
                      (int64_t)wrap_any(i2_0 - 4 + r2, g.n2) * g.n3 + x3s + 4 * q;
  uint2 raw[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) raw[f] = __ldg(reinterpret_cast<const uint2*>(mhist + f * N + off));
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw[f].x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw[f].y));
    *reinterpret_cast<float4*>(sp[f] + r2 * MP3 + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// 2^-ceil(log2 x) for x > 0 (power-of-two scale that maps x into (1/2, 1]), 1 otherwise.
__device__ __forceinline__ float pow2_scale(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0f;
  int e;
  frexp(x, &e);                                    // x = m 2^e, m in [1/2, 1)
  e = e < -120 ? -120 : (e > 120 ? 120 : e);
  return ldexpf(1.0f, -e);
}

// MODE 0 (SDOT): s^j = (j == 0 ? scale0 : 1) * grad8(m^j) . (sig_s vt), FP16 out, where
//                sig_s = pow2_scale(*vmax) keeps the incremental fields in range.
// MODE 1 (ACCUM): out = base_coef * base + unscale * sum_j w_j lam^j grad8(m^j) (FP32),
//                unscale = umul / sig_s (sig_s = 1 when vmax == NULL); optional
//                partial <dotv, out>.
template <int MODE, int NF>
__global__ void __launch_bounds__(32 * MT2) k_hist_march_h(
    Grid g, const __half* __restrict__ mhist, const __half* __restrict__ lhist,
    const float* __restrict__ vt, float scale0, const double* __restrict__ vmax,
    const float* __restrict__ base, float base_coef, float umul, float* __restrict__ out,
    __half* __restrict__ hout, const float* __restrict__ dotv, double* __restrict__ partial,
    int mt1) {
  __shared__ __align__(16) float sp[NF][MPLANE];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i3_0 = blockIdx.x * MT3, i2_0 = blockIdx.y * MT2, i1_0 = blockIdx.z * mt1;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N;
  const int64_t s1 = (int64_t)g.n2 * g.n3;
  const int64_t col = active ? (int64_t)i2 * g.n3 + i3 : 0;
  const int nt = NF - 1;
  const float ht = 1.0f / (float)nt;
  const float sig = vmax ? pow2_scale(*vmax) : 1.0f;
  const float unscale = umul / sig;
  float q[NF][9];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      q[f][k] = active ? __half2float(mhist[f * N + wrap_any(i1_0 - 4 + k, g.n1) * s1 + col])
                       : 0.f;
  const int i1_end = min(i1_0 + mt1, g.n1);
  const int c = (ty + 4) * MP3 + lane + 4;
  KahanF dacc;
  for (int i1 = i1_0; i1 < i1_end; ++i1) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      q[f][8] = active ? __half2float(mhist[f * N + wrap_near(i1 + 4, g.n1) * s1 + col]) : 0.f;
    __syncthreads();
    stage_planes_h<NF>(mhist, N, g, i1, i2_0, i3_0, sp);
    __syncthreads();
    if (active) {
      const int64_t idx = (int64_t)i1 * s1 + col;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      if (MODE == 0) {
        t1 = sig * vt[idx]; t2 = sig * vt[N + idx]; t3 = sig * vt[2 * N + idx];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* p = sp[f];
        const float gx = fd8(q[f][0], q[f][1], q[f][2], q[f][3], q[f][5], q[f][6], q[f][7],
                             q[f][8], g.inv_h1);
        const float gy = fd8(p[c - 4 * MP3], p[c - 3 * MP3], p[c - 2 * MP3], p[c - MP3],
                             p[c + MP3], p[c + 2 * MP3], p[c + 3 * MP3], p[c + 4 * MP3],
                             g.inv_h2);
        const float gz = fd8(p[c - 4], p[c - 3], p[c - 2], p[c - 1], p[c + 1], p[c + 2],
                             p[c + 3], p[c + 4], g.inv_h3);
        if (MODE == 0) {
          float sd = gx * t1;
          sd = fmaf(gy, t2, sd);
          sd = fmaf(gz, t3, sd);
          hout[f * N + idx] = __float2half_rn(f == 0 ? scale0 * sd : sd);
        } else {
          const float wl = ((f == 0 || f == nt) ? 0.5f * ht : ht) *
                           __half2float(lhist[f * N + idx]);
          a0 = fmaf(wl, gx, a0);
          a1 = fmaf(wl, gy, a1);
          a2 = fmaf(wl, gz, a2);
        }
      }
      if (MODE == 1) {
        a0 *= unscale; a1 *= unscale; a2 *= unscale;
        if (base) {
          a0 = fmaf(base_coef, base[idx], a0);
          a1 = fmaf(base_coef, base[N + idx], a1);
          a2 = fmaf(base_coef, base[2 * N + idx], a2);
        }
        out[idx] = a0;
        out[N + idx] = a1;
        out[2 * N + idx] = a2;
        if (partial)
          dacc.add(dotv[idx] * a0 + dotv[N + idx] * a1 + dotv[2 * N + idx] * a2);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < 8; ++k) q[f][k] = q[f][k + 1];
  }
  if (MODE == 1 && partial) {
    const double b = block_sum(dacc.value());
    if (threadIdx.x == 0 && threadIdx.y == 0)
      partial[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
  }
}

// ------------------------------------------------------------------ small kernels

// y = half(a x + b z) (z optional, FP16) -- conversions and the final
// condition lam(1) = sig_m m1 - m(1) of the adjoint.
__global__ void k_axpy_h(int64_t n, float a, const float* __restrict__ x, float b,
                         const __half* __restrict__ z, __half* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float r = a * x[i];
    if (z) r = fmaf(b, __half2float(z[i]), r);
    y[i] = __float2half_rn(r);
  }
}

// partial sums of (a m(x) - m1(x))^2 with m in FP16 (objective's distance term).
__global__ void __launch_bounds__(256) k_sqdiff_h(int64_t n, const __half* __restrict__ m,
                                                  float a, const float* __restrict__ m1,
                                                  double* __restrict__ partial) {
  KahanF acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = a * __half2float(m[i]) - m1[i];
    acc.add(d * d);
  }
  const double b = block_sum(acc.value());
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// ------------------------------------------------------------------ launchers

void launch_sl_h(const Grid& g, const __half* u, const float* d, const float* scale,
                 float sigma, const __half* aux, float beta, __half* out, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_sl_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         hbrick_w(16) * (int)sizeof(uint32_t));
  });
  const int t1 = tuned_sl_t1();
  ProfileRange pr(K_SL, (double)g.N * (16 + 4 * (scale != nullptr) + 2 * (aux != nullptr)), st);
  k_sl_h<<<brick_grid(g, t1), dim3(32, TB2), hbrick_w(t1) * sizeof(uint32_t), st>>>(
      g, u, d, scale, sigma, aux, beta, out, t1);
}

template <int MODE>
static bool launch_march_h(const Grid& g, const __half* mhist, const __half* lhist,
                           const float* vt, float scale0, const double* vmax, const float* base,
                           float base_coef, float umul, float* out, __half* hout, int nt,
                           const float* dotv, double* partial, cudaStream_t st) {
  const int mt1 = tuned_march_t1();
  const dim3 grid = march_grid(g, mt1), block(32, MT2);
#define CLAIRE_MARCH_H(NF)                                                                   \
  k_hist_march_h<MODE, NF><<<grid, block, 0, st>>>(g, mhist, lhist, vt, scale0, vmax, base,  \
                                                   base_coef, umul, out, hout, dotv, partial, \
                                                   mt1)
  switch (nt) {
    case 1: CLAIRE_MARCH_H(2); return true;
    case 2: CLAIRE_MARCH_H(3); return true;
    case 4: CLAIRE_MARCH_H(5); return true;
    case 8: CLAIRE_MARCH_H(9); return true;
    default: return false;
  }
#undef CLAIRE_MARCH_H
}

bool launch_sdot_hist_h(const Grid& g, const __half* mhist, int nt, const float* vt,
                        float scale0, const double* vmax, __half* shist, cudaStream_t st) {
  ProfileRange pr(K_SDOT, (double)g.N * (12 + 4 * (nt + 1)), st);
  return launch_march_h<0>(g, mhist, nullptr, vt, scale0, vmax, nullptr, 0.f, 1.f, nullptr,
                           shist, nt, nullptr, nullptr, st);
}

bool launch_accum_hist_h(const Grid& g, const __half* lhist, const __half* mhist, int nt,
                         const double* vmax, float umul, const float* base, float base_coef,
                         float* out, const float* dotv, double* partial, cudaStream_t st) {
  ProfileRange pr(K_ACCUM, (double)g.N * (4 * (nt + 1) + 12 + 12 * (base != nullptr) +
                                          12 * (partial != nullptr)), st);
  return launch_march_h<1>(g, mhist, lhist, nullptr, 0.f, vmax, base, base_coef, umul, out,
                           nullptr, nt, dotv, partial, st);
}

void launch_axpy_h(int64_t n, float a, const float* x, float b, const __half* z, __half* y,
                   cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * (6 + 2 * (z != nullptr)), st);
  k_axpy_h<<<vector_blocks(n), 256, 0, st>>>(n, a, x, b, z, y);
}

void launch_sqdiff_h(int64_t n, const __half* m, float a, const float* m1, double* partial,
                     int nblocks, double* out, cudaStream_t st) {
  ProfileRange pr(K_REDUCE, (double)n * 6, st);
  k_sqdiff_h<<<nblocks, 256, 0, st>>>(n, m, a, m1, partial);
  launch_reduce_final(partial, nblocks, RED_SUM, out, st);
}

}  // namespace claire
