// Learned warm start: kernels of a small 3D U-Net that predicts a velocity from
// the (m0, m1) pair on a 64^3 grid, and the spectral resampling between the
// registration grid and the network grid.
//
// Activations are channels-last BF16 [V][C] (V = batch x D x H x W voxels,
// x-fastest spatial order as the registration fields), weights BF16
// [Cout][27][Cin], accumulation FP32.  Convolutions are 3x3x3 with periodic
// padding (the images live on a periodic grid) and run as implicit GEMMs on
// the tensor cores (mma.sync m16n8k16 BF16 -> FP32):
//   forward  Y[v][n]  = sum_{t, c} W[n][t][c] X[nbr_t(v)][c]          (M = V, N = Cout, K = 27 Cin)
//   dgrad    dX[v][c] = sum_{t, n} W[n][26 - t][c] dY[nbr_t(v)][n]   (forward with flipped weights)
//   wgrad    dW[n][t][c] = sum_v dY[v][n] X[nbr_t(v)][c]              (M = Cout, N = Cin, K = V)
#include <cuda_bf16.h>
#include <cufft.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/claire.h"
#include "reduce.cuh"

namespace claire {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct Vol {
  int B, D, H, W;
};

// Neighbour of voxel v at offset (dz, dy, dx) with periodic wrap inside its sample.
__device__ __forceinline__ int64_t nbr(const Vol& s, int64_t v, int dz, int dy, int dx) {
  int x = (int)(v % s.W);
  int64_t r = v / s.W;
  int y = (int)(r % s.H);
  r /= s.H;
  int z = (int)(r % s.D);
  const int64_t b = r / s.D;
  x += dx; x = x < 0 ? x + s.W : (x >= s.W ? x - s.W : x);
  y += dy; y = y < 0 ? y + s.H : (y >= s.H ? y - s.H : y);
  z += dz; z = z < 0 ? z + s.D : (z >= s.D ? z - s.D : z);
  return ((b * s.D + z) * s.H + y) * s.W + x;
}

// ------------------------------------------------------------------ forward / dgrad

// CTA: 4 warps x 16 voxels = 64 output voxels, NT output channels (blockIdx.y
// selects the channel tile).  K loop: 27 taps x Cin / 16 channel chunks.  A
// fragments come straight from the channels-last activations (a channel pair
// is one 32-bit word), B fragments from the weights (L1 / L2 resident).
template <int NT>
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ X, Vol s, int Cin,
                                                  const bf16* __restrict__ Wt,
                                                  const float* __restrict__ bias, int Cout,
                                                  int relu, bf16* __restrict__ Y,
                                                  float* __restrict__ Y32) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int64_t V = (int64_t)s.B * s.D * s.H * s.W;
  const int64_t m0 = (int64_t)blockIdx.x * 64 + warp * 16;
  const int n0 = blockIdx.y * NT;
  const int64_t r0 = m0 + g, r1 = m0 + g + 8;
  const int64_t v0 = r0 < V ? r0 : 0, v1 = r1 < V ? r1 : 0;
  float acc[NT / 8][4];
#pragma unroll
  for (int j = 0; j < NT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const int cw = Cin >> 1;                                     // 32-bit words per voxel
  for (int t = 0; t < 27; ++t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const uint32_t* xa = reinterpret_cast<const uint32_t*>(X) + nbr(s, v0, dz, dy, dx) * cw;
    const uint32_t* xb = reinterpret_cast<const uint32_t*>(X) + nbr(s, v1, dz, dy, dx) * cw;
    for (int c = 0; c < Cin; c += 16) {
      const int w = c >> 1;
      uint32_t a[4];
      a[0] = __ldg(xa + w + q);
      a[1] = __ldg(xb + w + q);
      a[2] = __ldg(xa + w + 4 + q);
      a[3] = __ldg(xb + w + 4 + q);
#pragma unroll
      for (int j = 0; j < NT / 8; ++j) {
        const uint32_t* wp =
            reinterpret_cast<const uint32_t*>(Wt + ((int64_t)(n0 + j * 8 + g) * 27 + t) * Cin);
        uint32_t b[2];
        b[0] = __ldg(wp + w + q);
        b[1] = __ldg(wp + w + 4 + q);
        mma16816(acc[j], a, b);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NT / 8; ++j) {
    const int n = n0 + j * 8 + 2 * q;
    const float b0 = bias ? bias[n] : 0.f, b1 = bias ? bias[n + 1] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = h ? r1 : r0;
      if (r >= V) continue;
      float y0 = acc[j][2 * h] + b0, y1 = acc[j][2 * h + 1] + b1;
      if (relu) {
        y0 = fmaxf(y0, 0.f);
        y1 = fmaxf(y1, 0.f);
      }
      if (Y)
        *reinterpret_cast<uint32_t*>(Y + r * Cout + n) =
            pack_bf16(__float2bfloat16_rn(y0), __float2bfloat16_rn(y1));
      if (Y32) {
        Y32[r * Cout + n] = y0;
        Y32[r * Cout + n + 1] = y1;
      }
    }
  }
}

// W' [Cin][27][Cout] = W [Cout][26 - t][Cin]: dgrad is the forward conv of dY with W'.
__global__ void k_flip_weights(const bf16* __restrict__ W, int Cout, int Cin,
                               bf16* __restrict__ Wf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)Cout * 27 * Cin;
  if (i >= n) return;
  const int c = (int)(i % Cin);
  const int t = (int)((i / Cin) % 27);
  const int o = (int)(i / ((int64_t)Cin * 27));
  Wf[((int64_t)c * 27 + (26 - t)) * Cout + o] = W[i];
}

// ------------------------------------------------------------------ wgrad

// dW[n][t][c] over a chunk of voxels (blockIdx.x) for channel tile n0..n0+15
// (blockIdx.z) and tap t (blockIdx.y); the 4 warps take interleaved 16-voxel
// slices, combine in shared memory and write one deterministic partial.
template <int CT>
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ X, Vol s, int Cin,
                                                    const bf16* __restrict__ dY, int Cout,
                                                    int64_t chunk, float* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int t = blockIdx.y, n0 = blockIdx.z * 16;
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int64_t V = (int64_t)s.B * s.D * s.H * s.W;
  const int64_t x_begin = (int64_t)blockIdx.x * chunk;
  const int64_t x_end = min(V, x_begin + chunk);
  float acc[CT / 8][4];
#pragma unroll
  for (int j = 0; j < CT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int64_t x0 = x_begin + warp * 16; x0 < x_end; x0 += 64) {
    int64_t xs[4] = {x0 + 2 * q, x0 + 2 * q + 1, x0 + 2 * q + 8, x0 + 2 * q + 9};
    bf16 ya[4], yb[4];                     // dY rows n0+g, n0+g+8 at the 4 voxels
    int64_t nb[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool ok = xs[e] < x_end;
      const int64_t xv = ok ? xs[e] : x_begin;
      ya[e] = ok ? dY[xv * Cout + n0 + g] : __float2bfloat16_rn(0.f);
      yb[e] = ok ? dY[xv * Cout + n0 + g + 8] : __float2bfloat16_rn(0.f);
      nb[e] = nbr(s, xv, dz, dy, dx) * Cin;
    }
    uint32_t a[4];
    a[0] = pack_bf16(ya[0], ya[1]);
    a[1] = pack_bf16(yb[0], yb[1]);
    a[2] = pack_bf16(ya[2], ya[3]);
    a[3] = pack_bf16(yb[2], yb[3]);
#pragma unroll
    for (int j = 0; j < CT / 8; ++j) {
      const int cc = j * 8 + g;
      uint32_t b[2];
      b[0] = pack_bf16(X[nb[0] + cc], X[nb[1] + cc]);
      b[1] = pack_bf16(X[nb[2] + cc], X[nb[3] + cc]);
      mma16816(acc[j], a, b);
    }
  }
  // combine the 4 warps: each owns a [16][CT] tile in C-fragment layout
  __shared__ float red[4][16 * CT];
#pragma unroll
  for (int j = 0; j < CT / 8; ++j) {
    const int col = j * 8 + 2 * q;
    red[warp][g * CT + col] = acc[j][0];
    red[warp][g * CT + col + 1] = acc[j][1];
    red[warp][(g + 8) * CT + col] = acc[j][2];
    red[warp][(g + 8) * CT + col + 1] = acc[j][3];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * CT; i += 128) {
    const float v = (red[0][i] + red[1][i]) + (red[2][i] + red[3][i]);
    const int n = n0 + i / CT, c = i % CT;
    if (c < Cin)
      part[(((int64_t)blockIdx.x * Cout + n) * 27 + t) * Cin + c] = v;
  }
}

__global__ void k_sum_partials(const float* __restrict__ part, int nsplit, int64_t n,
                               float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int k = 0; k < nsplit; ++k) acc += part[k * n + i];
  out[i] = acc;
}

// db[n] = sum_v dY[v][n] (deterministic two-level sum per channel)
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ dY, int64_t V, int C,
                                                   float* __restrict__ db) {
  const int n = blockIdx.x;
  KahanF acc;
  for (int64_t v = threadIdx.x; v < V; v += blockDim.x) acc.add(__bfloat162float(dY[v * C + n]));
  const double b = block_sum(acc.value());
  if (threadIdx.x == 0) db[n] = (float)b;
}

// ------------------------------------------------------------------ layer ops

__global__ void k_relu_bwd(int64_t n, const bf16* __restrict__ y, bf16* __restrict__ dy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16_rn(0.f);
}

// 2x2x2 average pooling forward (mode 0) / backward (mode 1), channels-last.
__global__ void k_pool2(Vol fine, int C, const bf16* __restrict__ in, bf16* __restrict__ out,
                        int mode) {
  const int D2 = fine.D / 2, H2 = fine.H / 2, W2 = fine.W / 2;
  const int64_t n = (int64_t)fine.B * D2 * H2 * W2 * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % C);
  int64_t r = i / C;
  const int x = (int)(r % W2); r /= W2;
  const int y = (int)(r % H2); r /= H2;
  const int z = (int)(r % D2);
  const int64_t b = r / D2;
  auto fidx = [&](int dz, int dy, int dx) {
    return ((((b * fine.D + 2 * z + dz) * fine.H + 2 * y + dy) * fine.W + 2 * x + dx) * C + c);
  };
  if (mode == 0) {
    float acc = 0.f;
    for (int k = 0; k < 8; ++k) acc += __bfloat162float(in[fidx(k >> 2, (k >> 1) & 1, k & 1)]);
    out[i] = __float2bfloat16_rn(0.125f * acc);
  } else {
    const bf16 gv = __float2bfloat16_rn(0.125f * __bfloat162float(in[i]));
    for (int k = 0; k < 8; ++k) out[fidx(k >> 2, (k >> 1) & 1, k & 1)] = gv;
  }
}

// Nearest 2x upsampling into channels [c_off, c_off + C) of a [V][Cdst] tensor
// (forward, mode 0), or its adjoint: sum of the 8 children (backward, mode 1).
__global__ void k_up2(Vol coarse, int C, const bf16* __restrict__ in, int Cdst, int c_off,
                      bf16* __restrict__ out, int mode) {
  const int64_t n = (int64_t)coarse.B * coarse.D * coarse.H * coarse.W * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % C);
  int64_t r = i / C;
  const int x = (int)(r % coarse.W); r /= coarse.W;
  const int y = (int)(r % coarse.H); r /= coarse.H;
  const int z = (int)(r % coarse.D);
  const int64_t b = r / coarse.D;
  const int D = 2 * coarse.D, H = 2 * coarse.H, W = 2 * coarse.W;
  auto fidx = [&](int k) {
    return ((((b * D + 2 * z + (k >> 2)) * H + 2 * y + ((k >> 1) & 1)) * W + 2 * x + (k & 1)) *
                Cdst + c_off + c);
  };
  if (mode == 0) {
    for (int k = 0; k < 8; ++k) out[fidx(k)] = in[i];
  } else {
    float acc = 0.f;
    for (int k = 0; k < 8; ++k) acc += __bfloat162float(in[fidx(k)]);
    out[i] = __float2bfloat16_rn(acc);
  }
}

// Copy channels [0, C) of a [V][C] tensor into channels [c_off, c_off + C) of a
// [V][Cdst] tensor (mode 0), or back out of it (mode 1).
__global__ void k_channel_copy(int64_t V, int C, const bf16* __restrict__ src, int Cdst,
                               int c_off, bf16* __restrict__ dst, int mode) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * C) return;
  const int64_t v = i / C;
  const int c = (int)(i % C);
  if (mode == 0) dst[v * Cdst + c_off + c] = src[i];
  else dst[i] = src[v * Cdst + c_off + c];
}

__global__ void k_add(int64_t n, const bf16* __restrict__ a, bf16* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(__bfloat162float(b[i]) + __bfloat162float(a[i]));
}

// Pack FP32 planar fields [nf][V] into channels-last BF16 [V][C] (channels >= nf zero).
__global__ void k_pack(int64_t V, int nf, const float* __restrict__ f, float scale, int C,
                       bf16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * C) return;
  const int64_t v = i / C;
  const int c = (int)(i % C);
  out[i] = __float2bfloat16_rn(c < nf ? scale * f[c * V + v] : 0.f);
}

// Loss 1/(3V) sum (scale y - target)^2 over the first 3 channels of an FP32
// [V][C] output, its gradient in BF16 [V][C] (zero in the padded channels),
// and the planar FP32 prediction [3][V].
__global__ void __launch_bounds__(256) k_mse(int64_t V, int C, const float* __restrict__ y,
                                             const float* __restrict__ target, float scale,
                                             bf16* __restrict__ dy, float* __restrict__ pred,
                                             double* __restrict__ partial) {
  KahanF acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / C;
    const int c = (int)(i % C);
    float grad = 0.f;
    if (c < 3) {
      const float p = scale * y[i];
      if (pred) pred[c * V + v] = p;
      if (target) {
        const float d = p - target[c * V + v];
        acc.add(d * d);
        grad = 2.f * d * scale / (3.f * (float)V);
      }
    }
    if (dy) dy[i] = __float2bfloat16_rn(grad);
  }
  const double b = block_sum(acc.value());
  if (threadIdx.x == 0 && partial) partial[blockIdx.x] = b;
}

// out = scale * sum of n doubles (one block, fixed order).
__global__ void __launch_bounds__(256) k_sum_double(const double* __restrict__ x, int n,
                                                    double scale, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
  const double b = block_sum(acc);
  if (threadIdx.x == 0) *out = scale * b;
}

// Adam on FP32 master weights, refreshing their BF16 copy.
__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ gr,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                       float b2, float eps, float c1, float c2, bf16* __restrict__ pb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (pb) pb[i] = __float2bfloat16_rn(pi);
}

// ------------------------------------------------------------------ spectral resample

// Half spectrum of an n-grid -> half spectrum of an m-grid: keep the modes with
// |k_i| < min(n_i, m_i) / 2 on every axis, zero the others (spectral
// restriction when m < n, zero-padding prolongation when m > n), scaled by
// 1/N_n (cuFFT's transforms are unnormalised).  blockIdx.y = component.
__global__ void k_resample_modes(int n1, int n2, int n3, const cufftComplex* __restrict__ src,
                                 int m1, int m2, int m3, cufftComplex* __restrict__ dst,
                                 float scale) {
  const int mh = m3 / 2 + 1, nh = n3 / 2 + 1;
  const int64_t total = (int64_t)m1 * m2 * mh;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  src += (int64_t)blockIdx.y * n1 * n2 * nh;
  dst += (int64_t)blockIdx.y * total;
  const int j3 = (int)(i % mh);
  const int j2 = (int)((i / mh) % m2);
  const int j1 = (int)(i / ((int64_t)mh * m2));
  const int k1 = j1 <= m1 / 2 ? j1 : j1 - m1;
  const int k2 = j2 <= m2 / 2 ? j2 : j2 - m2;
  const int k3 = j3;
  const int l1 = min(n1, m1) / 2, l2 = min(n2, m2) / 2, l3 = min(n3, m3) / 2;
  cufftComplex val = make_cuComplex(0.f, 0.f);
  if (abs(k1) < l1 && abs(k2) < l2 && k3 < l3) {
    const int s1 = k1 < 0 ? k1 + n1 : k1, s2 = k2 < 0 ? k2 + n2 : k2;
    val = src[((int64_t)s1 * n2 + s2) * nh + k3];
    val.x *= scale;
    val.y *= scale;
  }
  dst[i] = val;
}

// Batched cuFFT plans and spectral buffers of one resampling shape, kept for
// the process lifetime (per device, stream and shape): the warm start restricts
// and prolongs once per registration, and creating plans costs milliseconds.
struct ResamplePlan {
  int dev;
  cudaStream_t st;
  int n[3], m[3], ncomp;
  cufftHandle pf, pi;
  cufftComplex *a, *b;
};
std::mutex g_resample_mu;
std::vector<ResamplePlan> g_resample_plans;

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace claire

using namespace claire;

// ====================================================================== C ABI

extern "C" {

claire_status claire_conv3d_forward(const void* x, int B, int D, int H, int W, int cin,
                                    const void* w, const float* bias, int cout, int relu,
                                    void* y_bf16, float* y_f32, void* stream) {
  if (!x || !w || (!y_bf16 && !y_f32) || B < 1 || D < 1 || H < 1 || W < 1 || cin % 16 ||
      cout % 16 || cin < 16 || cout < 16)
    return CLAIRE_EINVAL;
  const Vol s{B, D, H, W};
  const int64_t V = (int64_t)B * D * H * W;
  const int nt = cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16);
  const dim3 grid(blocks(V, 64), cout / nt);
  cudaStream_t st = (cudaStream_t)stream;
  const bf16* X = (const bf16*)x;
  const bf16* Wt = (const bf16*)w;
  bf16* Y = (bf16*)y_bf16;
  if (nt == 64) k_conv_fwd<64><<<grid, 128, 0, st>>>(X, s, cin, Wt, bias, cout, relu, Y, y_f32);
  else if (nt == 32) k_conv_fwd<32><<<grid, 128, 0, st>>>(X, s, cin, Wt, bias, cout, relu, Y, y_f32);
  else k_conv_fwd<16><<<grid, 128, 0, st>>>(X, s, cin, Wt, bias, cout, relu, Y, y_f32);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_conv3d_flip_weights(const void* w, int cout, int cin, void* wf,
                                         void* stream) {
  if (!w || !wf || cout < 1 || cin < 1) return CLAIRE_EINVAL;
  const int64_t n = (int64_t)cout * 27 * cin;
  k_flip_weights<<<blocks(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)w, cout, cin,
                                                                (bf16*)wf);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_conv3d_wgrad(const void* x, int B, int D, int H, int W, int cin,
                                  const void* dy, int cout, float* partial, int nsplit,
                                  float* dw, void* stream) {
  if (!x || !dy || !partial || !dw || nsplit < 1 || cout % 16 || cout < 16 ||
      !(cin == 16 || cin == 32 || cin == 48 || cin == 64 || cin == 96 || cin == 128 ||
        cin == 192))
    return CLAIRE_EINVAL;
  const Vol s{B, D, H, W};
  const int64_t V = (int64_t)B * D * H * W;
  int64_t chunk = (V + nsplit - 1) / nsplit;
  chunk = ((chunk + 63) / 64) * 64;
  const int ns = (int)((V + chunk - 1) / chunk);
  const dim3 grid(ns, 27, cout / 16);
  cudaStream_t st = (cudaStream_t)stream;
  const bf16* X = (const bf16*)x;
  const bf16* dY = (const bf16*)dy;
  // the channel tile is exactly the input channel count
#define CLAIRE_WG(CT) k_conv_wgrad<CT><<<grid, 128, 0, st>>>(X, s, cin, dY, cout, chunk, partial)
  switch (cin) {
    case 16: CLAIRE_WG(16); break;
    case 32: CLAIRE_WG(32); break;
    case 48: CLAIRE_WG(48); break;
    case 64: CLAIRE_WG(64); break;
    case 96: CLAIRE_WG(96); break;
    case 128: CLAIRE_WG(128); break;
    default: CLAIRE_WG(192); break;
  }
#undef CLAIRE_WG
  const int64_t n = (int64_t)cout * 27 * cin;
  k_sum_partials<<<blocks(n), 256, 0, st>>>(partial, ns, n, dw);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_unet_op(int op, const void* a, void* b, long long V, int C, int Cdst,
                             int c_off, int B, int D, int H, int W, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const Vol s{B, D, H, W};
  switch (op) {
    case 0:  // relu backward: b (dy) *= (a (y) > 0)
      k_relu_bwd<<<blocks(V * C), 256, 0, st>>>(V * C, (const bf16*)a, (bf16*)b);
      break;
    case 1:  // pool forward (s = fine grid)
    case 2:  // pool backward
      k_pool2<<<blocks((int64_t)B * (D / 2) * (H / 2) * (W / 2) * C), 256, 0, st>>>(
          s, C, (const bf16*)a, (bf16*)b, op - 1);
      break;
    case 3:  // upsample forward (s = coarse grid) into channels [c_off, c_off + C) of Cdst
    case 4:  // upsample backward
      k_up2<<<blocks((int64_t)B * D * H * W * C), 256, 0, st>>>(s, C, (const bf16*)a, Cdst,
                                                               c_off, (bf16*)b, op - 3);
      break;
    case 5:  // channel copy in
    case 6:  // channel copy out
      k_channel_copy<<<blocks(V * C), 256, 0, st>>>(V, C, (const bf16*)a, Cdst, c_off,
                                                    (bf16*)b, op - 5);
      break;
    case 7:  // b += a
      k_add<<<blocks(V * C), 256, 0, st>>>(V * C, (const bf16*)a, (bf16*)b);
      break;
    default:
      return CLAIRE_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_unet_bias_grad(const void* dy, long long V, int C, float* db,
                                    void* stream) {
  k_bias_grad<<<C, 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, V, C, db);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_unet_pack(long long V, int nf, const float* f, float scale, int C,
                               void* out, void* stream) {
  if (nf > C) return CLAIRE_EINVAL;
  k_pack<<<blocks(V * C), 256, 0, (cudaStream_t)stream>>>(V, nf, f, scale, C, (bf16*)out);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_unet_mse(long long V, int C, const float* y, const float* target,
                              float scale, void* dy, float* pred, double* partial, int nblocks,
                              double* loss, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (target && (!partial || nblocks < 1)) return CLAIRE_EINVAL;
  k_mse<<<nblocks, 256, 0, st>>>(V, C, y, target, scale, (bf16*)dy, pred, partial);
  if (loss && partial && target) k_sum_double<<<1, 256, 0, st>>>(partial, nblocks, 1.0 / (3.0 * V), loss);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_unet_adam(long long n, float* p, const float* g, float* m, float* v,
                               float lr, float b1, float b2, float eps, int step, void* pb,
                               void* stream) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2,
                                                      (bf16*)pb);
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

claire_status claire_resample(int n1, int n2, int n3, const float* in, int m1, int m2, int m3,
                              float* out, int ncomp, void* stream) {
  if (!in || !out || ncomp < 1 || n1 < 2 || n2 < 2 || n3 < 2 || m1 < 2 || m2 < 2 || m3 < 2 ||
      n1 % 2 || n2 % 2 || n3 % 2 || m1 % 2 || m2 % 2 || m3 % 2)
    return CLAIRE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t Nn = (int64_t)n1 * n2 * n3, Nm = (int64_t)m1 * m2 * m3;
  const int64_t Cn = (int64_t)n1 * n2 * (n3 / 2 + 1), Cm = (int64_t)m1 * m2 * (m3 / 2 + 1);
  if (Nn > INT32_MAX || Nm > INT32_MAX || Cn * ncomp > INT32_MAX) return CLAIRE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CLAIRE_ECUDA;
  std::lock_guard<std::mutex> lock(g_resample_mu);
  ResamplePlan* plan = nullptr;
  for (auto& p : g_resample_plans)
    if (p.dev == dev && p.st == st && p.ncomp == ncomp && p.n[0] == n1 && p.n[1] == n2 &&
        p.n[2] == n3 && p.m[0] == m1 && p.m[1] == m2 && p.m[2] == m3)
      plan = &p;
  if (!plan) {
    ResamplePlan p{dev, st, {n1, n2, n3}, {m1, m2, m3}, ncomp, 0, 0, nullptr, nullptr};
    int nn[3] = {n1, n2, n3}, mm[3] = {m1, m2, m3};
    bool ok = cudaMalloc(&p.a, Cn * ncomp * sizeof(cufftComplex)) == cudaSuccess &&
              cudaMalloc(&p.b, Cm * ncomp * sizeof(cufftComplex)) == cudaSuccess;
    ok = ok &&
         cufftPlanMany(&p.pf, 3, nn, nullptr, 1, (int)Nn, nullptr, 1, (int)Cn, CUFFT_R2C,
                       ncomp) == CUFFT_SUCCESS &&
         cufftPlanMany(&p.pi, 3, mm, nullptr, 1, (int)Cm, nullptr, 1, (int)Nm, CUFFT_C2R,
                       ncomp) == CUFFT_SUCCESS &&
         cufftSetStream(p.pf, st) == CUFFT_SUCCESS && cufftSetStream(p.pi, st) == CUFFT_SUCCESS;
    if (!ok) {
      if (p.pf) cufftDestroy(p.pf);
      if (p.pi) cufftDestroy(p.pi);
      cudaFree(p.a);
      cudaFree(p.b);
      return CLAIRE_ENOMEM;
    }
    g_resample_plans.push_back(p);
    plan = &g_resample_plans.back();
  }
  if (cufftExecR2C(plan->pf, (cufftReal*)in, plan->a) != CUFFT_SUCCESS) return CLAIRE_ECUDA;
  k_resample_modes<<<dim3(blocks(Cm), ncomp), 256, 0, st>>>(n1, n2, n3, plan->a, m1, m2, m3,
                                                           plan->b, 1.0f / (float)Nn);
  if (cufftExecC2R(plan->pi, plan->b, (cufftReal*)out) != CUFFT_SUCCESS) return CLAIRE_ECUDA;
  return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
}

}  // extern "C"
