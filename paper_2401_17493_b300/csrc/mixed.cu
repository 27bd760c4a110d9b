// Mixed-precision form: the gathered and stencilled fields (state, adjoint,
// incremental state / adjoint histories) are stored in FP16; interpolation
// weights, arithmetic, departure points and PCG vectors stay FP32, reductions
// FP64.  Stored fields carry power-of-two scales (exact in FP16) so that
// they stay inside the FP16 range: the images are scaled to max |m| in
// (1/2, 1], the incremental fields by 2^-ceil(log2 ||s||_inf) of the
// direction s.  Results are unscaled in FP32.
//
// SL bricks of FP16 fields are converted to FP32 once while they are staged in
// shared memory (interior bricks land by one TMA box and are converted in place,
// sl_tma.cuh; the others are copied with cp.async), so the 64-tap gather is the
// FP32 one: the gather is shared-memory / issue bound, and converting each
// staged value once is cheaper than converting every tap.  (A layout holding each row twice as
// half2 pairs, halving the shared loads, was slower: every half still needs a
// conversion instruction in the gather.)  The FD8 history march is the same
// template as the FP32 form, instantiated for FP16 storage.
#include <cuda_fp16.h>
#include <math_constants.h>

#include <mutex>

#include "device_setup.h"
#include "internal.h"
#include "reduce.cuh"
#include "sl_brick.cuh"
#include "sl_tma.cuh"
#include "sl_window.cuh"
#include "fd8_march.cuh"

namespace claire {


// Stage an FP16 field over the tile plus halo into an FP32 brick with the
// layout of stage_brick (rows of BB3 = 64 floats): the conversion happens once
// per staged value, and the gather is then the FP32 64-tap gather.  The raw
// halves of a row are first copied asynchronously into the row's own padding
// (floats 40..59 of the 64: 80 bytes), then every thread converts the chunks it
// copied itself into floats 0..39, so no extra shared memory and no barrier
// between the two phases are needed.
__device__ __forceinline__ void stage_brick_h32(const __half* __restrict__ u, const Grid& g,
                                                int i1_0, int i2_0, int i3_0,
                                                float* __restrict__ s, int t1) {
  static_assert(BB3 - BX3 >= BX3 / 2, "raw FP16 row must fit in the row padding");
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int rows = brick_rows(t1);
  const int x3s = i3_0 - HB3_LO;
  // chunks of 4 halves never straddle the periodic wrap (x3s % 4 == 0)
  const bool vec = (g.n3 % 4 == 0) && ((reinterpret_cast<uintptr_t>(u) & 7) == 0);
  const bool near = brick_wrap_near(g, t1);
  if (vec) {
    constexpr int Q = BX3 / 4;                     // 4 halves (8 bytes) per chunk
    const int nitems = rows * Q;
    for (int item = tid; item < nitems; item += BRICK_THREADS) {
      const int row = item / Q, q = item - row * Q;
      const int r1 = row / BB2, r2 = row - r1 * BB2;
      const int g1 = wrap_sel(i1_0 - HB_LO + r1, g.n1, near);
      const int g2 = wrap_sel(i2_0 - HB_LO + r2, g.n2, near);
      cp_async8(s + row * BB3 + BX3 + 2 * q,
                u + ((int64_t)g1 * g.n2 + g2) * g.n3 + wrap_sel(x3s + 4 * q, g.n3, near));
    }
    cp_async_wait_all();
    for (int item = tid; item < nitems; item += BRICK_THREADS) {
      const int row = item / Q, q = item - row * Q;
      const uint2 raw = *reinterpret_cast<const uint2*>(s + row * BB3 + BX3 + 2 * q);
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
      *reinterpret_cast<float4*>(s + row * BB3 + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
    }
  } else {
    for (int item = tid; item < rows * BX3; item += BRICK_THREADS) {
      const int row = item / BX3, e = item - row * BX3;
      const int r1 = row / BB2, r2 = row - r1 * BB2;
      const int g1 = wrap_any(i1_0 - HB_LO + r1, g.n1);
      const int g2 = wrap_any(i2_0 - HB_LO + r2, g.n2);
      s[row * BB3 + e] =
          __half2float(u[((int64_t)g1 * g.n2 + g2) * g.n3 + wrap_any(x3s + e, g.n3)]);
    }
  }
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
// With tma != 0 the interior bricks land by TMA from umap (FP16 boxes).
__global__ void __launch_bounds__(BRICK_THREADS, 4) k_sl_h(Grid g, const __half* __restrict__ u,
                                                        const float* __restrict__ d,
                                                        const float* __restrict__ scale,
                                                        float sigma,
                                                        const __half* __restrict__ aux,
                                                        float beta, __half* __restrict__ out,
                                                        int t1,
                                                        const __grid_constant__ CUtensorMap umap,
                                                        int tma) {
  extern __shared__ __align__(128) float smf[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(smf) +
                                               brick_floats(t1) * sizeof(float) + 128);
  const int i1_0 = blockIdx.z * t1, i2_0 = blockIdx.y * TB2, i3_0 = blockIdx.x * TB3;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N, s1 = (int64_t)g.n2 * g.n3;
  const int64_t idx0 = active ? lin(g, i1_0, i2, i3) : 0;
  const bool use_tma = tma && brick_tma_ok(g, i1_0, i2_0, i3_0, t1);
  if (use_tma) {
    brick_mbar_init(mbar);
    __syncthreads();
    issue_brick_tma_h(&umap, 0, g, i1_0, i2_0, i3_0, smf, t1, mbar);
  }
  float dn[3];                                     // departure points, one node ahead
#pragma unroll
  for (int a = 0; a < 3; ++a) dn[a] = active ? d[a * N + idx0] : 0.f;
  bool ok = true;
  if (use_tma) {
    ok = wait_brick_tma(mbar, 0u);
    convert_brick_h(smf, t1);                      // ends with a barrier
  } else {
    stage_brick_h32(u, g, i1_0, i2_0, i3_0, smf, t1);
    __syncthreads();
  }
  if (!active || !ok) return;
  const int kmax = min(t1, g.n1 - i1_0);
#pragma unroll 2
  for (int k = 0; k < kmax; ++k) {
    const int i1 = i1_0 + k;
    const int64_t idx = idx0 + k * s1;
    // the epilogue operands are requested before the gather, which hides their latency
    const float sc = scale ? __ldg(scale + idx) : sigma;
    const float ax = aux ? __half2float(aux[idx]) : 0.0f;
    NodeTaps t;
    node_taps(dn[0], dn[1], dn[2], t);
    if (k + 1 < kmax) {
#pragma unroll
      for (int a = 0; a < 3; ++a) dn[a] = d[a * N + idx + s1];
    }
    const float y = taps_in_brick(t) ? gather_brick(smf, t, k, ty, lane)
                                     : gather_global_h(u, g, t, i1, i2, i3);
    float r = y * sc;
    if (aux) r = fmaf(beta, ax, r);
    out[idx] = __float2half_rn(r);
  }
}

// k_sl_h with the register-window gather (sl_window.cuh): the FP16 brick is
// converted to FP32 while it is staged, then the gather is the FP32 window
// march; the FP16 aux field is staged as a dense 16-bit tile.
__global__ void __launch_bounds__(WIN_THREADS, 2) k_slw_h(Grid g, const __half* __restrict__ u,
                                                      const float* __restrict__ d,
                                                      const float* __restrict__ scale,
                                                      float sigma,
                                                      const __half* __restrict__ aux,
                                                      float beta, __half* __restrict__ out,
                                                      int t1) {
  extern __shared__ __align__(16) float smf[];
  float* td = smf + brick_floats(t1);                      // [3][t1][TB2][TB3]
  float* tsc = td + 3 * tile_elems(t1);                    // scale tile (if any)
  __half* tax = reinterpret_cast<__half*>(tsc + (scale ? tile_elems(t1) : 0));
  int* queue = reinterpret_cast<int*>(tax + (aux ? tile_elems(t1) : 0));
  int* qcount = queue + tile_elems(t1);
  const int i1_0 = blockIdx.z * t1, i2_0 = blockIdx.y * TB2, i3_0 = blockIdx.x * TB3;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const bool active = i2_0 + ty < g.n2 && i3_0 + lane < g.n3;
  const int kmax = min(t1, g.n1 - i1_0);
  if (ty == 0 && lane == 0) *qcount = 0;
  stage_tile(d, g.N, 3, g, i1_0, i2_0, i3_0, t1, td);
  if (scale) stage_tile(scale, g.N, 1, g, i1_0, i2_0, i3_0, t1, tsc);
  if (aux) stage_tile(aux, g.N, 1, g, i1_0, i2_0, i3_0, t1, tax);
  stage_brick_h32(u, g, i1_0, i2_0, i3_0, smf, t1);
  cp_async_wait_all();              // the tiles' copies (the brick's scalar path issues none)
  __syncthreads();
  auto disp = [&](int k, int y, int l, float dd[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) dd[a] = td[tile_at(t1, a, k, y, l)];
  };
  auto epi = [&](int k, int y, int l, float val) {
    const int at = tile_at(t1, 0, k, y, l);
    float r = val * (scale ? tsc[at] : sigma);
    if (aux) r = fmaf(beta, __half2float(tax[at]), r);
    out[lin(g, i1_0 + k, i2_0 + y, i3_0 + l)] = __float2half_rn(r);
  };
  int r1 = 0, r2 = 0, r3 = 0;
  if (active) {
    float dr[3];
    disp(min(t1 / 2, kmax - 1), ty, lane, dr);
    window_reference(dr[0], dr[1], dr[2], r1, r2, r3);
  }
  window_march(smf, kmax, ty, lane, active, r1, r2, r3, disp, epi, queue, qcount);
  __syncthreads();
  window_deferred(smf, i1_0, i2_0, i3_0, *qcount, queue, disp, epi,
                  [&](const NodeTaps& t, int i1, int i2, int i3) {
                    return gather_global_h(u, g, t, i1, i2, i3);
                  });
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

// y = a float(x), x in FP16 (a stored field back to FP32, unscaled).
__global__ void k_h2f(int64_t n, float a, const __half* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * __half2float(x[i]);
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

unsigned int take_brick_timeouts_h() {
  unsigned int n = 0;
  const unsigned int zero = 0;
  if (cudaMemcpyFromSymbol(&n, g_brick_timeouts, sizeof n) != cudaSuccess ||
      cudaMemcpyToSymbol(g_brick_timeouts, &zero, sizeof zero) != cudaSuccess)
    return 0;
  return n;
}

void launch_sl_h(const Grid& g, const __half* u, const float* d, const float* scale,
                 float sigma, const __half* aux, float beta, __half* out, cudaStream_t st) {
  static std::once_flag once[kSetupDevices];
  once_per_device(once, [] {
    cudaFuncSetAttribute(k_sl_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)brick_h_smem_bytes(16));
    cudaFuncSetAttribute(k_slw_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         window_smem_bytes(16, 4, 1));
  });
  const int t1 = tuned_sl_t1();
  ProfileRange pr(K_SL, (double)g.N * (16 + 4 * (scale != nullptr) + 2 * (aux != nullptr)), st);
  if (tuned_sl_window())
    k_slw_h<<<brick_grid(g, t1), dim3(32, TB2),
              window_smem_bytes(t1, 3 + (scale != nullptr), aux != nullptr), st>>>(
        g, u, d, scale, sigma, aux, beta, out, t1);
  else {
    CUtensorMap m;
    const int tma = tuned_sl_tma() && encode_brick_map(&m, u, true, g, 1, t1);
    k_sl_h<<<brick_grid(g, t1), dim3(32, TB2), brick_h_smem_bytes(t1), st>>>(
        g, u, d, scale, sigma, aux, beta, out, t1, m, tma);
  }
}

template <int MODE>
static bool launch_march_h(const Grid& g, const __half* mhist, const __half* lhist,
                           const float* vt, float scale0, const double* vmax, const float* base,
                           float base_coef, float umul, float* out, __half* hout, int nt,
                           const float* dotv, double* partial, cudaStream_t st) {
  const int mt1 = tuned_march_t1();
  const dim3 grid = march_grid(g, mt1), block(32, MT2);
#define CLAIRE_MARCH_H(NF)                                                                 \
  k_hist_march<MODE, NF, __half><<<grid, block, 0, st>>>(g, mhist, lhist, vt, scale0, vmax, \
                                                         base, base_coef, umul, out, hout,   \
                                                         dotv, partial, mt1)
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

void launch_h2f(int64_t n, float a, const __half* x, float* y, cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 6, st);
  k_h2f<<<vector_blocks(n), 256, 0, st>>>(n, a, x, y);
}

void launch_sqdiff_h(int64_t n, const __half* m, float a, const float* m1, double* partial,
                     int nblocks, double* out, cudaStream_t st) {
  ProfileRange pr(K_REDUCE, (double)n * 6, st);
  k_sqdiff_h<<<nblocks, 256, 0, st>>>(n, m, a, m1, partial);
  launch_reduce_final(partial, nblocks, RED_SUM, out, st);
}

}  // namespace claire
