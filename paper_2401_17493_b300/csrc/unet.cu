// Learned warm start: kernels of a small 3D U-Net that predicts a velocity from
// the (m0, m1) pair on a 64^3 grid, and the spectral resampling between the
// registration grid and the network grid.
//
// Activations are channels-last BF16 [V][C] (V = batch x D x H x W voxels,
// x-fastest spatial order as the registration fields), weights BF16
// [Cout][27][Cin], accumulation FP32.  Convolutions are 3x3x3 with periodic
// padding (the images live on a periodic grid) and run as implicit GEMMs on
// the tensor cores (forward and data gradient: tcgen05 kind::f16 with the
// accumulator in TMEM; weight gradient: mma.sync m16n8k16 BF16 -> FP32):
//   forward  Y[v][n]  = sum_{t, c} W[n][t][c] X[nbr_t(v)][c]          (M = V, N = Cout, K = 27 Cin)
//   dgrad    dX[v][c] = sum_{t, n} W[n][26 - t][c] dY[nbr_t(v)][n]   (forward with flipped weights)
//   wgrad    dW[n][t][c] = sum_v dY[v][n] X[nbr_t(v)][c]              (M = Cout, N = Cin, K = V)
#include <cuda_bf16.h>
#include <cufft.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/claire.h"
#include "common.cuh"
#include "device_setup.h"
#include "reduce.cuh"
#include "tc_sm100.cuh"

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

// Voxel coordinates (batch, z, y, x) of a linear index (the volume of one call has
// fewer than 2^31 voxels, so 32-bit divisions suffice), computed once per voxel.
struct Vox {
  int b, z, y, x;
};
__device__ __forceinline__ Vox vox_of(const Vol& s, int v) {
  Vox o;
  o.x = v % s.W;
  int r = v / s.W;
  o.y = r % s.H;
  r /= s.H;
  o.z = r % s.D;
  o.b = r / s.D;
  return o;
}

// Neighbour at offset (dz, dy, dx) with periodic wrap inside its sample.
__device__ __forceinline__ int nbr_of(const Vol& s, const Vox& p, int dz, int dy, int dx) {
  int x = p.x + dx, y = p.y + dy, z = p.z + dz;
  x = x < 0 ? x + s.W : (x >= s.W ? x - s.W : x);
  y = y < 0 ? y + s.H : (y >= s.H ? y - s.H : y);
  z = z < 0 ? z + s.D : (z >= s.D ? z - s.D : z);
  return ((p.b * s.D + z) * s.H + y) * s.W + x;
}

// ------------------------------------------------------------------ forward / dgrad

// Implicit-GEMM convolution on the fifth-generation tensor cores (tcgen05):
// a CTA of 128 threads owns M = 128 consecutive output voxels and N output
// channels; the FP32 accumulator D[128][N] lives in TMEM.  The K loop runs over
// the 27 taps x Cin channels in stages of KC chunks of 16 channels of one tap
// (channel groups outer, taps inner, so the activation rows a CTA re-reads for
// the 27 taps stay in L1: the gathers use cp.async.ca):
// every thread gathers its own voxel's neighbour row (cp.async, 16 bytes at a
// time) and a share of the weight rows into shared memory in the no-swizzle
// K-major core-matrix layout, then one thread issues the stage's kind::f16
// MMAs (M = 128, N, K = 16 each) and commits them to the stage's mbarrier.
// Four stage buffers, gathers issued two stages ahead (cp.async groups): the
// gathers of stages i + 1 and i + 2 are in flight while stage i is waited for
// and multiplied, and a buffer is refilled only after the mbarrier reports the
// MMAs of its previous use done.  The epilogue reads the thread's TMEM lane (its
// voxel) 16 columns at a time, adds the bias, applies the ReLU and stores BF16
// and / or FP32.  Every wait is bounded; one that runs out ends the CTA's later
// waits and makes its outputs NaN instead of hanging.
constexpr int CONV_M = 128;
constexpr int CONV_S = 4;                         // stage buffers
constexpr int CONV_L = 2;                         // stages gathered ahead
constexpr uint32_t CONV_WAIT = 1u << 22;          // try_wait calls of <= 1 us each
constexpr int CONV_STAGE_BYTES = 24 * 1024;       // shared memory per stage

// Threads whose bounded tensor-core wait ran out since the last claire_wait_status
// (their outputs are NaN); read and reset by claire_wait_status.
__device__ unsigned int g_wait_timeouts = 0;
__device__ __forceinline__ void note_timeout(bool ok) {
  if (!ok) atomicAdd(&g_wait_timeouts, 1u);
}

template <int N, int KC>
struct ConvSmem {
  static constexpr int A = KC * CONV_M * 32;       // bytes of A per stage
  static constexpr int B = KC * N * 32;            // bytes of B per stage
  static constexpr int bytes = CONV_S * (A + B);
};

template <int N, int KC>
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ X, Vol s, int Cin,
                                                  const bf16* __restrict__ Wt,
                                                  const float* __restrict__ bias, int Cout,
                                                  int relu, bf16* __restrict__ Y,
                                                  float* __restrict__ Y32) {
  using SM = ConvSmem<N, KC>;
  constexpr uint32_t NCOL = N < 32 ? 32 : N;
  extern __shared__ __align__(128) uint8_t conv_smem[];
  __shared__ __align__(8) uint64_t mbar[CONV_S];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.y * N;
  const int64_t V = (int64_t)s.B * s.D * s.H * s.W;
  const int64_t v = (int64_t)blockIdx.x * CONV_M + tid;        // this thread's row / voxel
  const bool rv = v < V;
  const Vox p = vox_of(s, rv ? (int)v : 0);
  if (warp == 0) {
    tmem_alloc(&tmem_base, NCOL);
    tmem_relinquish();
  }
  if (tid == 0)
    for (int k = 0; k < CONV_S; ++k) mbar_init(&mbar[k], 1);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(CONV_M, N);
  const int chunks = Cin >> 4;                                 // 16-channel chunks per tap
  const int per_tap = (chunks + KC - 1) / KC;                  // stages per tap
  const int nstage = 27 * per_tap;
  // issue the gathers of stage i into its buffer (one cp.async group)
  auto gather = [&](int i) {
    if (i < nstage) {
      uint8_t* sa = conv_smem + (i % CONV_S) * (SM::A + SM::B);
      uint8_t* sb = sa + SM::A;
      const int t = i % 27, c_first = (i / 27) * KC;     // channel group outer, tap inner
      const int kc_n = min(KC, chunks - c_first);
      const bf16* xr =
          X + (int64_t)nbr_of(s, p, t / 9 - 1, (t / 3) % 3 - 1, t % 3 - 1) * Cin + c_first * 16;
      const int arow = (tid >> 3) * 128 + (tid & 7) * 16;
      for (int kc = 0; kc < kc_n; ++kc)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint8_t* dst = sa + kc * (CONV_M * 32) + h * (CONV_M * 16) + arow;
          if (rv) cp_async16_ca(dst, xr + kc * 16 + h * 8);
          else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
      for (int j = tid; j < kc_n * 2 * N; j += 128) {
        const int kc = j / (2 * N), r = j - kc * 2 * N;
        const int n = r >> 1, h = r & 1;
        cp_async16_ca(sb + kc * (N * 32) + h * (N * 16) + (n >> 3) * 128 + (n & 7) * 16,
                      Wt + ((int64_t)(n0 + n) * 27 + t) * Cin + (c_first + kc) * 16 + h * 8);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  bool ok = true;
  for (int i = 0; i < CONV_L; ++i) gather(i);
  for (int i = 0; i < nstage; ++i) {
    const int j = i + CONV_L;                                  // stage to gather now
    if (ok && j < nstage && j >= CONV_S)                       // its buffer's previous MMAs
      ok = mbar_wait(&mbar[j % CONV_S], ((j - CONV_S) / CONV_S) & 1, CONV_WAIT);
    gather(j);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(CONV_L) : "memory");   // stage i landed
    fence_proxy_async_smem();
    ok = __syncthreads_and(ok);          // a timed-out wait ends the waits of the whole CTA
    if (tid == 0) {
      tc_fence_after_sync();
      uint8_t* sa = conv_smem + (i % CONV_S) * (SM::A + SM::B);
      uint8_t* sb = sa + SM::A;
      const int kc_n = min(KC, chunks - (i / 27) * KC);
      for (int kc = 0; kc < kc_n; ++kc)
        umma_bf16(tmem, umma_smem_desc(sa + kc * (CONV_M * 32), CONV_M * 16, 128),
                  umma_smem_desc(sb + kc * (N * 32), N * 16, 128), idesc,
                  (i > 0 || kc > 0) ? 1u : 0u);
      umma_commit(&mbar[i % CONV_S]);
    }
  }
  ok &= mbar_wait(&mbar[(nstage - 1) % CONV_S], ((nstage - 1) / CONV_S) & 1, CONV_WAIT);
  note_timeout(ok);
  tc_fence_after_sync();
#pragma unroll 1
  for (int c = 0; c < N; c += 16) {
    float y[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, y);
    if (!rv) continue;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float t = y[e] + (bias ? bias[n0 + c + e] : 0.f);
      if (relu) t = fmaxf(t, 0.f);
      y[e] = ok ? t : __int_as_float(0x7fc00000);
    }
    if (Y) {
      uint32_t w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e)
        w[e] = pack_bf16(__float2bfloat16_rn(y[2 * e]), __float2bfloat16_rn(y[2 * e + 1]));
      uint4* dst = reinterpret_cast<uint4*>(Y + v * Cout + n0 + c);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    if (Y32) {
      float4* dst = reinterpret_cast<float4*>(Y32 + v * Cout + n0 + c);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        dst[e] = make_float4(y[4 * e], y[4 * e + 1], y[4 * e + 2], y[4 * e + 3]);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOL);
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
      nb[e] = (int64_t)nbr_of(s, vox_of(s, (int)xv), dz, dy, dx) * Cin;
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

// Weight gradient on the tensor cores (tcgen05) for volumes with W % 8 == 0,
// H % 16 == 0 and cin <= cout <= 128, one group of 16 input channels per blockIdx.y:
//   dW[co][t][ci] = sum_v dY[v][co] X[v + off(t)][ci]
// as D[co][(t, ci)] += A[co][v] B_t[ci][v] with M = 128 (co, rows >= Cout zero) and
// K = voxels.  A persistent CTA walks 8 x 16-voxel tiles of one (sample, z)
// (the tiles blockIdx.x, blockIdx.x + gridDim.x, ...), accumulating all 27 taps in
// 432 TMEM columns.  Per tile it stages A = dY transposed, [y][co][x] x 2 bytes
// (K-major: 8-voxel x runs are the 16-byte K rows), and the input neighbourhood
// transposed once per x shift, XT[dx][z'][y'][ci][x] (so every tap's B operand is
// 16-byte aligned).  The transposes run in registers on 8 x 8 blocks (movmatrix):
// a warp loads 8 voxels x 8 channels, 4 bytes a lane, and stores 8 channel rows of
// 8 voxels as one 128-byte run, so the staging stores meet no bank conflicts.  With
// an XT block pitch of 256 bytes the three y shifts of one (dz, dx) pair are
// consecutive 128-byte groups of B rows, so one MMA with N = 48 (dy, ci) covers
// them: one thread issues 9 x 8 MMAs (K = 16: two y rows each) per tile while the
// CTA stages the next tile into the other of two buffers.  TMEM column
// (dz 3 + dx) 48 + dy 16 + ci holds tap (dz, dy, dx).  The CTA's partial dW goes to
// part[blockIdx.x]; k_sum_partials adds them in order.  Every wait is bounded; a
// timed-out one makes the CTA's partial NaN.
// A: 16 y x (128 co x 8 x + 16 bytes) (the leading byte offset of A is the y pitch)
constexpr int WG_AP = 128 * 16 + 16;                      // 2064 bytes per y
constexpr int WG_XP = 16 * 16;                            // 256 bytes per (dx, z, y) block
constexpr int WG_A = 16 * WG_AP;
constexpr int WG_XT = 3 * 3 * 18 * WG_XP;                 // XT: 3 dx x 3 z x 18 y blocks
constexpr int WG_BUF = WG_A + WG_XT;                      // one tile's operands
// two buffers; more than half an SM's shared memory, so that one CTA (holding all 512
// TMEM columns) runs per SM
constexpr int WG_SMEM = 2 * WG_BUF;
static_assert(WG_SMEM > 114 * 1024 && WG_SMEM <= 227 * 1024, "weight-gradient buffers");
static_assert(WG_AP % 16 == 0 && WG_XP == 2 * 128 && WG_BUF % 16 == 0,
              "operand offsets in 16-byte units; XT blocks two 8-row groups apart");
// 512 threads: more global loads in flight while a tile is staged (transposed)
// than with 256
constexpr int WG_THREADS = 512;

// 8 x 8 transpose of 16-bit elements across a warp: lane l holds row l / 4,
// columns 2 (l % 4) and 2 (l % 4) + 1 of the source (low half first) and
// receives the same positions of the transpose.
__device__ __forceinline__ uint32_t movm_trans(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(d) : "r"(a));
  return d;
}

__global__ void __launch_bounds__(WG_THREADS) k_conv_wgrad_tc(const bf16* __restrict__ X, Vol s,
                                                              int Cin,
                                                              const bf16* __restrict__ dY,
                                                              int Cout,
                                                              float* __restrict__ part) {
  extern __shared__ __align__(128) uint8_t wg_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = blockIdx.y;                                  // input channels 16 g .. 16 g + 15
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  // rows co >= Cout of A (and the pitch padding) stay zero in both buffers
  for (int i = tid; i < WG_SMEM / 16; i += WG_THREADS)
    reinterpret_cast<uint4*>(wg_smem)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(CONV_M, 48);
  constexpr int NWARPS = WG_THREADS / 32;
  const int xb = s.W / 8, yb = s.H / 16;
  const int ntiles = s.B * s.D * yb * xb;
  const int xr = lane >> 2, cp = 2 * (lane & 3);             // a lane's place in an 8 x 8 block
  // the operands of tile q into buffer buf (warp-uniform loops: movmatrix)
  auto stage = [&](int q, int buf) {
    uint8_t* A = wg_smem + buf * WG_BUF;
    uint8_t* XT = A + WG_A;
    const int x0 = (q % xb) * 8;
    q /= xb;
    const int y0 = (q % yb) * 16;
    q /= yb;
    const int z = q % s.D, b = q / s.D;
    // A[y][co][x] = dY[(x0 + x, y0 + y)][co]: blocks of (8 x) x (8 co)
    const int na = 16 * (Cout / 8);
#pragma unroll 2
    for (int blk = warp; blk < na; blk += NWARPS) {
      const int y = blk & 15, c8 = blk >> 4;
      const int64_t v = ((int64_t)(b * s.D + z) * s.H + y0 + y) * s.W + x0 + xr;
      const uint32_t d = movm_trans(*reinterpret_cast<const uint32_t*>(dY + v * Cout + c8 * 8 + cp));
      *reinterpret_cast<uint32_t*>(A + y * WG_AP + (c8 * 8 + xr) * 16 + cp * 2) = d;
    }
    // XT[dxi][zp][yp][ci][x] = X[(x0 + x + dxi - 1, y0 + yp - 1, z + zp - 1)][16 g + ci]:
    // blocks of (8 x) x (8 ci), hh = which half of the 16 channels
#pragma unroll 4
    for (int blk2 = warp; blk2 < 2 * 3 * 3 * 18; blk2 += NWARPS) {
      const int hh = blk2 & 1, blk = blk2 >> 1;
      const int yp = blk % 18, zp = (blk / 18) % 3, dxi = blk / 54;
      int xx = x0 + xr + dxi - 1, yy = y0 + yp - 1, zz = z + zp - 1;
      xx = xx < 0 ? xx + s.W : (xx >= s.W ? xx - s.W : xx);
      yy = yy < 0 ? yy + s.H : (yy >= s.H ? yy - s.H : yy);
      zz = zz < 0 ? zz + s.D : (zz >= s.D ? zz - s.D : zz);
      const int64_t v = ((int64_t)(b * s.D + zz) * s.H + yy) * s.W + xx;
      const uint32_t d =
          movm_trans(*reinterpret_cast<const uint32_t*>(X + v * Cin + g * 16 + hh * 8 + cp));
      *reinterpret_cast<uint32_t*>(XT + blk * WG_XP + (hh * 8 + xr) * 16 + cp * 2) = d;
    }
    fence_proxy_async_smem();
  };
  bool ok = true;
  int it = 0;
  if ((int)blockIdx.x < ntiles) stage(blockIdx.x, 0);
  ok = __syncthreads_and(ok);
  for (int q0 = blockIdx.x; q0 < ntiles && ok; q0 += gridDim.x, ++it) {
    const int buf = it & 1;
    if (tid == 0) {
      tc_fence_after_sync();
      const uint8_t* A = wg_smem + buf * WG_BUF;
      const uint8_t* XT = A + WG_A;
      // the operands' descriptors advance from the buffer's first ones; B rows
      // (dy, ci): K halves WG_XP apart, 8-row groups 128 bytes apart
      const uint64_t dA = umma_smem_desc(A, WG_AP, 128), dX = umma_smem_desc(XT, WG_XP, 128);
      for (int dz = 0; dz < 3; ++dz)
        for (int dx = 0; dx < 3; ++dx) {
          const uint64_t dXt = umma_desc_advance(dX, ((dx * 3 + dz) * 18) * WG_XP);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            umma_bf16(tmem + (uint32_t)((dz * 3 + dx) * 48), umma_desc_advance(dA, j * 2 * WG_AP),
                      umma_desc_advance(dXt, 2 * j * WG_XP), idesc, (it > 0 || j > 0) ? 1u : 0u);
        }
      umma_commit(&mbar[buf]);
    }
    const int q1 = q0 + gridDim.x;
    if (q1 < ntiles) {
      // the other buffer was read by the MMAs of tile it - 1
      if (it >= 1) ok = mbar_wait(&mbar[buf ^ 1], ((it - 1) >> 1) & 1, CONV_WAIT);
      ok = __all_sync(0xffffffffu, ok);   // the staging's movmatrix needs whole warps
      if (ok) stage(q1, buf ^ 1);
    }
    ok = __syncthreads_and(ok);          // a timed-out wait ends the loop of the whole CTA
  }
  if (it > 0) ok &= mbar_wait(&mbar[(it - 1) & 1], ((it - 1) >> 1) & 1, CONV_WAIT);
  note_timeout(ok);
  tc_fence_after_sync();
  if (warp < 4) {                                            // TMEM lanes 0..127 = co
    const int co = warp * 32 + lane;
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
      const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
      float y[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((dz * 3 + dx) * 48 + dy * 16),
                y);
      if (co >= Cout) continue;
#pragma unroll
      for (int e = 0; e < 16; ++e)
        y[e] = !ok ? __int_as_float(0x7fc00000) : (it > 0 ? y[e] : 0.f);
      float4* dst = reinterpret_cast<float4*>(
          part + (((int64_t)blockIdx.x * Cout + co) * 27 + t) * Cin + g * 16);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        dst[e] = make_float4(y[4 * e], y[4 * e + 1], y[4 * e + 2], y[4 * e + 3]);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// Weight gradient on the tensor cores in the transposed orientation, for the
// layers the kernel above does not take (more input than output channels, or
// H % 16 != 0 such as the 8^3 bottleneck); needs W % 8 == 0 and H % 8 == 0:
//   D[ci][(t, co)] += A_t[ci][v] B[co][v]
// with M = 128 input channels (blockIdx.y / (cout / 16) selects the block of 128,
// rows >= cin unused), N = 16 output channels (blockIdx.y % (cout / 16)), K =
// voxels.  A persistent CTA walks 8 x 8-voxel tiles of one (sample, z) in three
// stages per tile, one per x shift dx: a stage holds the input neighbourhood of
// that shift transposed, XT[z'(3)][y'(10)][ci(128)][x(8)] (every tap's A operand
// starts on a 16-byte row), and dY of the tile transposed, [y(8)][co(16)][x(8)]
// (the B operand); one thread issues the 9 taps of the shift x 4 MMAs (K = 16:
// two y rows each) while the CTA stages the next stage into the other of two
// buffers.  All 27 taps accumulate in 432 TMEM columns.  The CTA's partial dW goes
// to part[blockIdx.x]; every wait is bounded (a timed-out one makes it NaN).
constexpr int WT_XP = 128 * 16 + 16;                      // 2064 bytes per (z', y') block
constexpr int WT_XT = 3 * 10 * WT_XP;                     // 61920
constexpr int WT_BP = 16 * 16 + 16;                       // 272 bytes per y row of B
constexpr int WT_B = 8 * WT_BP;                           // 2176
constexpr int WT_BUF = WT_XT + WT_B;                      // one stage's operands
constexpr int WT_SMEM = 2 * WT_BUF;
static_assert(WT_BUF % 16 == 0 && WT_XP % 16 == 0 && WT_BP % 16 == 0,
              "stage buffers and operand offsets on 16-byte boundaries");
static_assert(WT_SMEM > 114 * 1024 && WT_SMEM <= 227 * 1024, "one CTA per SM");
__global__ void __launch_bounds__(WG_THREADS) k_conv_wgrad_tc_t(const bf16* __restrict__ X,
                                                                Vol s, int Cin,
                                                                const bf16* __restrict__ dY,
                                                                int Cout,
                                                                float* __restrict__ part) {
  extern __shared__ __align__(128) uint8_t wt_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ncg = Cout / 16;
  const int g = blockIdx.y % ncg;                            // output channels 16 g ..
  const int m0 = (blockIdx.y / ncg) * 128;                   // input channels m0 ..
  const int cm = min(128, Cin - m0);                         // real rows of A
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  for (int i = tid; i < WT_SMEM / 16; i += WG_THREADS)
    reinterpret_cast<uint4*>(wt_smem)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(CONV_M, 16);
  const int xb = s.W / 8, yb = s.H / 8;
  const int ntiles = s.B * s.D * yb * xb;
  const int nloc = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / gridDim.x + 1 : 0;
  const int nst = 3 * nloc;                                  // stages: (local tile, dx)
  // the operands of stage st into buffer buf
  auto stage = [&](int st, int buf) {
    uint8_t* XT = wt_smem + buf * WT_BUF;
    uint8_t* Bo = XT + WT_XT;
    int q = (int)blockIdx.x + (st / 3) * (int)gridDim.x;
    const int dx = st % 3;
    const int x0 = (q % xb) * 8;
    q /= xb;
    const int y0 = (q % yb) * 8;
    q /= yb;
    const int z = q % s.D, b = q / s.D;
    // B[y][co][x] = dY[(x0 + x, y0 + y)][16 g + co]
    if (tid < 128) {
      const int v = tid & 63, c8 = tid >> 6;
      const int y = v >> 3, x = v & 7;
      const int64_t vv = ((int64_t)(b * s.D + z) * s.H + y0 + y) * s.W + x0 + x;
      const uint4 d = *reinterpret_cast<const uint4*>(dY + vv * Cout + g * 16 + c8 * 8);
      const uint16_t* h = reinterpret_cast<const uint16_t*>(&d);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        *reinterpret_cast<uint16_t*>(Bo + y * WT_BP + (c8 * 8 + e) * 16 + x * 2) = h[e];
    }
    // XT[zp][yp][ci][x] = X[(x0 + x + dx - 1, y0 + yp - 1, z + zp - 1)][m0 + ci]; a warp's
    // lanes take 8 x by 4 consecutive (zp, yp) blocks (block pitch 2064 bytes: the
    // four blocks start in different banks)
    const int nch = cm / 8;
#pragma unroll 4
    for (int i = tid; i < 256 * nch; i += WG_THREADS) {
      const int x = i & 7, c8 = (i >> 8);
      const int blk = ((i >> 5) & 7) * 4 + ((i >> 3) & 3);
      if (blk >= 30) continue;
      const int yp = blk % 10, zp = blk / 10;
      int xx = x0 + x + dx - 1, yy = y0 + yp - 1, zz = z + zp - 1;
      xx = xx < 0 ? xx + s.W : (xx >= s.W ? xx - s.W : xx);
      yy = yy < 0 ? yy + s.H : (yy >= s.H ? yy - s.H : yy);
      zz = zz < 0 ? zz + s.D : (zz >= s.D ? zz - s.D : zz);
      const int64_t vv = ((int64_t)(b * s.D + zz) * s.H + yy) * s.W + xx;
      const uint4 d = *reinterpret_cast<const uint4*>(X + vv * Cin + m0 + c8 * 8);
      const uint16_t* h = reinterpret_cast<const uint16_t*>(&d);
      uint8_t* row = XT + blk * WT_XP + c8 * 8 * 16 + x * 2;
#pragma unroll
      for (int e = 0; e < 8; ++e) *reinterpret_cast<uint16_t*>(row + e * 16) = h[e];
    }
    fence_proxy_async_smem();
  };
  bool ok = true;
  if (nst > 0) stage(0, 0);
  ok = __syncthreads_and(ok);
  int st = 0;
  for (; st < nst && ok; ++st) {
    const int buf = st & 1;
    if (tid == 0) {
      tc_fence_after_sync();
      const uint8_t* XT = wt_smem + buf * WT_BUF;
      const uint8_t* Bo = XT + WT_XT;
      const int dx = st % 3, lt = st / 3;
      // the operands' descriptors advance from the buffer's first ones
      const uint64_t dX = umma_smem_desc(XT, WT_XP, 128), dB = umma_smem_desc(Bo, WT_BP, 128);
      for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy) {
          const int t = dz * 9 + dy * 3 + dx;
          const uint64_t dXt = umma_desc_advance(dX, (dz * 10 + dy) * WT_XP);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            umma_bf16(tmem + (uint32_t)(t * 16), umma_desc_advance(dXt, 2 * j * WT_XP),
                      umma_desc_advance(dB, j * 2 * WT_BP), idesc, (lt > 0 || j > 0) ? 1u : 0u);
        }
      umma_commit(&mbar[buf]);
    }
    if (st + 1 < nst) {
      // the other buffer was read by the MMAs of stage st - 1
      if (st >= 1) ok = mbar_wait(&mbar[buf ^ 1], ((st - 1) >> 1) & 1, CONV_WAIT);
      if (ok) stage(st + 1, buf ^ 1);
    }
    ok = __syncthreads_and(ok);          // a timed-out wait ends the loop of the whole CTA
  }
  if (st > 0) ok &= mbar_wait(&mbar[(st - 1) & 1], ((st - 1) >> 1) & 1, CONV_WAIT);
  note_timeout(ok);
  tc_fence_after_sync();
  if (warp < 4) {                                            // TMEM lanes 0..127 = ci
    const int ci = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
      float y[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 16), y);
      if (ci >= Cin || warp * 32 + (tid & 31) >= cm) continue;
#pragma unroll
      for (int n = 0; n < 16; ++n)
        part[(((int64_t)blockIdx.x * Cout + g * 16 + n) * 27 + t) * Cin + ci] =
            !ok ? __int_as_float(0x7fc00000) : (st > 0 ? y[n] : 0.f);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

__global__ void k_sum_partials(const float* __restrict__ part, int nsplit, int64_t n,
                               float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int k = 0; k < nsplit; ++k) acc += part[k * n + i];
  out[i] = acc;
}

// Bias gradient db[c] = sum_v dY[v][c] in two deterministic stages.
// Stage 1: CTA b sums the voxels [b chunk, (b + 1) chunk) for every channel:
// thread t takes the channel pair (2 p, 2 p + 1), p = t % (C / 2), of every
// (256 / (C / 2))-th voxel from t / (C / 2) on (bf16x2 loads, a warp reads
// whole voxel rows), compensated FP32 per thread, then the threads of a pair
// are added in a fixed order in FP64 into part[b][c].
__global__ void __launch_bounds__(256) k_bias_grad_part(const bf16* __restrict__ dY, int64_t V,
                                                        int C, int64_t chunk,
                                                        double* __restrict__ part) {
  __shared__ double red[256][2];
  const int P = C >> 1, t = threadIdx.x;
  const int rows = 256 / P;
  const int p = t % P, r = t / P;
  const int64_t v0 = (int64_t)blockIdx.x * chunk;
  const int64_t v1 = v0 + chunk < V ? v0 + chunk : V;
  KahanF a0, a1;
  if (r < rows) {
#pragma unroll 4
    for (int64_t v = v0 + r; v < v1; v += rows) {
      const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162*>(dY + v * C + 2 * p);
      a0.add(__low2float(x));
      a1.add(__high2float(x));
    }
  }
  red[t][0] = a0.value();
  red[t][1] = a1.value();
  __syncthreads();
  if (t < P) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < rows; ++q) {
      s0 += red[q * P + t][0];
      s1 += red[q * P + t][1];
    }
    part[(int64_t)blockIdx.x * C + 2 * t] = s0;
    part[(int64_t)blockIdx.x * C + 2 * t + 1] = s1;
  }
}

// Stage 2: db[c] = sum over the CTAs of part[b][c], one warp per channel: lane l
// adds the CTAs l, l + 32, ... in order, then the lanes are combined by a
// shuffle tree (a fixed order, so the result is deterministic).
__global__ void __launch_bounds__(256) k_bias_grad_final(const double* __restrict__ part,
                                                         int nblocks, int C,
                                                         float* __restrict__ db) {
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= C) return;                                       // whole warps leave together
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * C + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) db[c] = (float)s;
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

// Halo-tile variant for volumes with W % 8 == 0 and H % 16 == 0: a CTA owns the
// 8 (x) x 16 (y) output voxels of one (sample, z) and stages their 10 x 18 x 3
// input neighbourhood once per group of G 16-channel chunks, in the K-major
// core-matrix layout [chunk][K half][z'][y'][x'] x 16 bytes.  The A operand of tap
// (dz, dy, dx) is then a descriptor into that tile: rows of an 8-voxel x run are
// 16 bytes apart, the 16 runs (y) HALO_TX * 16 bytes apart (the stride byte
// offset), the two K halves HALO_PLANE * 16 bytes apart (the leading byte
// offset), starting at the tile row of the tap's first input voxel.  Each input
// row is copied into shared memory once per CTA instead of 27 times.  With a
// single chunk group whose 27 taps of weights fit beside the tile (res), the
// weights are staged with it and one thread issues all 27 x G MMAs behind one
// barrier; otherwise they stream through four stage buffers, one tap (G MMAs) per
// stage, and the tile of the next group is staged once the MMAs of the previous
// one completed.  Output rows: r = 8 y + x, the thread of TMEM lane r writes voxel
// (x0 + r % 8, y0 + r / 8).
constexpr int HALO_TX = 10, HALO_TY = 18, HALO_TZ = 3;
constexpr int HALO_PLANE = HALO_TX * HALO_TY * HALO_TZ;   // 540 voxel rows
constexpr int HALO_RES_BYTES = 100 * 1024;                // tile + all weights, resident
template <int N, int G>
struct HaloSmem {
  static constexpr int A = G * 2 * HALO_PLANE * 16;       // the input tile of one group
  static constexpr int B = G * N * 32;                     // the weights of one tap
  static constexpr bool res_fits = A + 27 * B <= HALO_RES_BYTES;
  static constexpr int bytes = A + (res_fits ? 27 : CONV_S) * B;
};

template <int N, int G>
__global__ void __launch_bounds__(128) k_conv_fwd_halo(const bf16* __restrict__ X, Vol s,
                                                       int Cin, const bf16* __restrict__ Wt,
                                                       const float* __restrict__ bias,
                                                       int Cout, int relu,
                                                       bf16* __restrict__ Y,
                                                       float* __restrict__ Y32) {
  using SM = HaloSmem<N, G>;
  constexpr uint32_t NCOL = N < 32 ? 32 : N;
  extern __shared__ __align__(128) uint8_t conv_smem[];
  __shared__ __align__(8) uint64_t mbar[CONV_S];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.y * N;
  const int groups = Cin / (16 * G);
  const bool res = SM::res_fits && groups == 1;
  // CTA -> (sample, z, y block, x block)
  const int xb = s.W / 8, yb = s.H / 16;
  int q = blockIdx.x;
  const int x0 = (q % xb) * 8;
  q /= xb;
  const int y0 = (q % yb) * 16;
  q /= yb;
  const int z = q % s.D, b = q / s.D;
  uint8_t* tile = conv_smem;
  uint8_t* bbuf = conv_smem + SM::A;
  if (warp == 0) {
    tmem_alloc(&tmem_base, NCOL);
    tmem_relinquish();
  }
  if (tid == 0)
    for (int k = 0; k < CONV_S; ++k) mbar_init(&mbar[k], 1);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(CONV_M, N);
  // the input tile of chunk group g, periodic in x, y, z
  auto stage_tile = [&](int g) {
    for (int j = tid; j < HALO_PLANE * G * 2; j += 128) {
      const int vr = j % HALO_PLANE, ch = j / HALO_PLANE;    // ch = 2 chunk + K half
      const int xp = vr % HALO_TX, yp = (vr / HALO_TX) % HALO_TY,
                zp = vr / (HALO_TX * HALO_TY);
      int x = x0 - 1 + xp, y = y0 - 1 + yp, zz = z - 1 + zp;
      x = x < 0 ? x + s.W : (x >= s.W ? x - s.W : x);
      y = y < 0 ? y + s.H : (y >= s.H ? y - s.H : y);
      zz = zz < 0 ? zz + s.D : (zz >= s.D ? zz - s.D : zz);
      const int64_t src =
          ((int64_t)((b * s.D + zz) * s.H + y) * s.W + x) * Cin + g * G * 16 + ch * 8;
      cp_async16_ca(tile + (ch * HALO_PLANE + vr) * 16, X + src);
    }
  };
  // weights of tap t, chunk group g, into buffer dst
  auto stage_tap = [&](int t, int g, uint8_t* dst) {
    for (int j = tid; j < G * 2 * N; j += 128) {
      const int c = j / (2 * N), r = j - c * 2 * N;
      const int n = r >> 1, h = r & 1;
      cp_async16_ca(dst + c * (N * 32) + h * (N * 16) + (n >> 3) * 128 + (n & 7) * 16,
                    Wt + ((int64_t)(n0 + n) * 27 + t) * Cin + (g * G + c) * 16 + h * 8);
    }
  };
  // the G MMAs of tap t, B from buffer src; the first MMA of the call overwrites D
  // (descriptors advanced from the tile's and the buffer's first ones)
  auto mma_tap = [&](int t, const uint8_t* src, bool first) {
    const int tap = (t / 9) * (HALO_TX * HALO_TY) + ((t / 3) % 3) * HALO_TX + t % 3;
    const uint64_t dT = umma_smem_desc(tile, HALO_PLANE * 16, HALO_TX * 16);
    const uint64_t dS = umma_smem_desc(src, N * 16, 128);
#pragma unroll
    for (int c = 0; c < G; ++c)
      umma_bf16(tmem, umma_desc_advance(dT, (c * 2 * HALO_PLANE + tap) * 16),
                umma_desc_advance(dS, c * (N * 32)), idesc, (first && c == 0) ? 0u : 1u);
  };
  bool ok = true;
  int last = 0;                                                // index of the last commit
  if (res) {
    stage_tile(0);
    for (int t = 0; t < 27; ++t) stage_tap(t, 0, bbuf + t * SM::B);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      for (int t = 0; t < 27; ++t) mma_tap(t, bbuf + t * SM::B, t == 0);
      umma_commit(&mbar[0]);
    }
  } else {
    const int nstage = 27 * groups;                            // (group, tap), taps inner
    auto gather = [&](int i) {
      if (i < nstage) {
        if (i % 27 == 0) stage_tile(i / 27);                   // the group's first stage
        stage_tap(i % 27, i / 27, bbuf + (i % CONV_S) * SM::B);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int i = 0; i < nstage; ++i) {
      // a group's tile replaces the previous one once all its MMAs completed
      if (ok && i % 27 == 0 && i > 0)
        ok = mbar_wait(&mbar[(i - 1) % CONV_S], ((i - 1) / CONV_S) & 1, CONV_WAIT);
      if (i % 27 == 0) {
        ok = __syncthreads_and(ok);
        for (int k = 0; k < CONV_L; ++k) gather(i + k);
      }
      const int j = i + CONV_L;                                // stage to gather now
      if (ok && j < nstage && j % 27 >= CONV_L && j >= CONV_S)
        ok = mbar_wait(&mbar[j % CONV_S], ((j - CONV_S) / CONV_S) & 1, CONV_WAIT);
      if (j % 27 >= CONV_L) gather(j);                         // else: the next group's
      else asm volatile("cp.async.commit_group;\n" ::: "memory");   // first stages wait
      asm volatile("cp.async.wait_group %0;\n" ::"n"(CONV_L) : "memory");
      fence_proxy_async_smem();
      ok = __syncthreads_and(ok);        // a timed-out wait ends the waits of the whole CTA
      if (tid == 0) {
        tc_fence_after_sync();
        mma_tap(i % 27, bbuf + (i % CONV_S) * SM::B, i == 0);
        umma_commit(&mbar[i % CONV_S]);
      }
    }
    last = nstage - 1;
  }
  ok &= mbar_wait(&mbar[last % CONV_S], (last / CONV_S) & 1, CONV_WAIT);
  note_timeout(ok);
  tc_fence_after_sync();
  const int64_t v = ((int64_t)(b * s.D + z) * s.H + y0 + (tid >> 3)) * s.W + x0 + (tid & 7);
#pragma unroll 1
  for (int c = 0; c < N; c += 16) {
    float y[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, y);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float t = y[e] + (bias ? bias[n0 + c + e] : 0.f);
      if (relu) t = fmaxf(t, 0.f);
      y[e] = ok ? t : __int_as_float(0x7fc00000);
    }
    if (Y) {
      uint32_t w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e)
        w[e] = pack_bf16(__float2bfloat16_rn(y[2 * e]), __float2bfloat16_rn(y[2 * e + 1]));
      uint4* dst = reinterpret_cast<uint4*>(Y + v * Cout + n0 + c);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    if (Y32) {
      float4* dst = reinterpret_cast<float4*>(Y32 + v * Cout + n0 + c);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        dst[e] = make_float4(y[4 * e], y[4 * e + 1], y[4 * e + 2], y[4 * e + 3]);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOL);
}

template <int N, int G>
void launch_conv_fwd_halo_g(cudaStream_t st, const bf16* X, const Vol& s, int cin,
                            const bf16* Wt, const float* bias, int cout, int relu, bf16* Y,
                            float* Y32) {
  constexpr int bytes = HaloSmem<N, G>::bytes;
  static std::once_flag once[kSetupDevices];
  once_per_device(once, [] {
    cudaFuncSetAttribute(k_conv_fwd_halo<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
  });
  const dim3 grid(s.B * s.D * (s.H / 16) * (s.W / 8), cout / N);
  k_conv_fwd_halo<N, G><<<grid, 128, bytes, st>>>(X, s, cin, Wt, bias, cout, relu, Y, Y32);
}

// The halo-tile kernel where it applies (W % 8 == 0, H % 16 == 0); chunk groups of
// G = the largest of 4, 3, 2, 1 that divides the 16-channel chunks.
template <int N>
bool launch_conv_fwd_halo(cudaStream_t st, const bf16* X, const Vol& s, int cin,
                          const bf16* Wt, const float* bias, int cout, int relu, bf16* Y,
                          float* Y32) {
  if (s.W % 8 || s.H % 16) return false;
  const int chunks = cin / 16;
  if (chunks % 4 == 0) launch_conv_fwd_halo_g<N, 4>(st, X, s, cin, Wt, bias, cout, relu, Y, Y32);
  else if (chunks % 3 == 0) launch_conv_fwd_halo_g<N, 3>(st, X, s, cin, Wt, bias, cout, relu, Y, Y32);
  else if (chunks % 2 == 0) launch_conv_fwd_halo_g<N, 2>(st, X, s, cin, Wt, bias, cout, relu, Y, Y32);
  else launch_conv_fwd_halo_g<N, 1>(st, X, s, cin, Wt, bias, cout, relu, Y, Y32);
  return true;
}

template <int N, int KC>
void launch_conv_fwd_kc(dim3 grid, cudaStream_t st, const bf16* X, const Vol& s, int cin,
                        const bf16* Wt, const float* bias, int cout, int relu, bf16* Y,
                        float* Y32) {
  constexpr int bytes = ConvSmem<N, KC>::bytes;
  static std::once_flag once[kSetupDevices];
  once_per_device(once, [] {
    cudaFuncSetAttribute(k_conv_fwd<N, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
  k_conv_fwd<N, KC><<<grid, 128, bytes, st>>>(X, s, cin, Wt, bias, cout, relu, Y, Y32);
}

// K per stage: KC 16-channel chunks, as many as divide the tap's chunks while a
// stage stays within CONV_STAGE_BYTES of shared memory (four stage buffers).
// Measured at 64^3 x 4 samples: deeper stages win (48 -> 16: 613 / 671 / 723 us
// for KC = 3 / 2 / 1).
template <int N>
void launch_conv_fwd(dim3 grid, cudaStream_t st, const bf16* X, const Vol& s, int cin,
                     const bf16* Wt, const float* bias, int cout, int relu, bf16* Y, float* Y32) {
  if (launch_conv_fwd_halo<N>(st, X, s, cin, Wt, bias, cout, relu, Y, Y32)) return;
  const int chunks = cin / 16;
  const int kc_max = CONV_STAGE_BYTES / (CONV_M * 32 + N * 32);
  int kc = 1;
  for (int k = 4; k >= 1; --k)
    if (k <= kc_max && chunks % k == 0) {
      kc = k;
      break;
    }
  switch (kc) {
    case 4: launch_conv_fwd_kc<N, 4>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, Y32); break;
    case 3: launch_conv_fwd_kc<N, 3>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, Y32); break;
    case 2: launch_conv_fwd_kc<N, 2>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, Y32); break;
    default: launch_conv_fwd_kc<N, 1>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, Y32); break;
  }
}

// The failure path of the bounded tensor-core waits, run on purpose: one CTA polls
// phase 0 of an mbarrier at most max_polls times.  With arrive == 0 nothing
// arrives and every thread gives up (and counts the timeout); with arrive != 0
// thread 0 arrives first and every wait succeeds.  No copy or MMA is in flight,
// so giving up leaves nothing behind.  result = number of threads that gave up.
__device__ int g_selftest_result = 0;
__global__ void k_wait_selftest(uint32_t max_polls, int arrive) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int gave_up;
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    gave_up = 0;
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&mbar);
  const bool ok = mbar_wait(&mbar, 0, max_polls);
  note_timeout(ok);
  if (!ok) atomicAdd(&gave_up, 1);
  __syncthreads();
  if (threadIdx.x == 0) g_selftest_result = gave_up;
}

}  // namespace
// threads whose bounded wait for a TMA-staged SL brick ran out (kernels.cu, mixed.cu)
unsigned int take_brick_timeouts();
unsigned int take_brick_timeouts_h();
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
  if (V >= INT32_MAX) return CLAIRE_EINVAL;
  const int nt = cout % 128 == 0 ? 128 : (cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16));
  const dim3 grid(blocks(V, CONV_M), cout / nt);
  cudaStream_t st = (cudaStream_t)stream;
  const bf16* X = (const bf16*)x;
  const bf16* Wt = (const bf16*)w;
  bf16* Y = (bf16*)y_bf16;
  switch (nt) {
    case 128: launch_conv_fwd<128>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, y_f32); break;
    case 64: launch_conv_fwd<64>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, y_f32); break;
    case 32: launch_conv_fwd<32>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, y_f32); break;
    default: launch_conv_fwd<16>(grid, st, X, s, cin, Wt, bias, cout, relu, Y, y_f32); break;
  }
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
  if (V >= INT32_MAX) return CLAIRE_EINVAL;
  cudaStream_t st0 = (cudaStream_t)stream;
  if (W % 8 == 0 && H % 16 == 0 && cout <= 128 && cin <= cout) {
    // tensor-core path: one persistent CTA per SM (each holds all 512 TMEM columns).
    // Measured faster than the mma.sync kernel where cin <= cout (16 -> 16 at 64^3:
    // 500 vs 957 us); with more input than output channels the 128-row padding of
    // the output channels and one pass per 16 input channels make it slower.
    const int nsm = device_sm_count();
    if (nsm == 0) return CLAIRE_ECUDA;
    static std::once_flag once[kSetupDevices];
    once_per_device(once, [] {
      cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           WG_SMEM);
    });
    const int ntiles = B * D * (H / 16) * (W / 8);
    const int ncta = std::max(1, std::min(std::min(nsplit, nsm), ntiles));
    k_conv_wgrad_tc<<<dim3(ncta, cin / 16), WG_THREADS, WG_SMEM, st0>>>(
        (const bf16*)x, s, cin, (const bf16*)dy, cout, partial);
    const int64_t n = (int64_t)cout * 27 * cin;
    k_sum_partials<<<blocks(n), 256, 0, st0>>>(partial, ncta, n, dw);
    return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
  }
  if (W % 8 == 0 && H % 8 == 0 && (cout <= 32 || H % 16 != 0)) {
    // tensor-core path, transposed: input channels as the 128 MMA rows (one grid row
    // per block of 128 input channels and 16 output channels), one persistent CTA per SM.
    // Each grid row stages the input neighbourhood again, so with 64 or more output
    // channels on H % 16 == 0 grids (192 -> 64 at 16^3: 235 vs 194 us) mma.sync stays
    const int nsm_t = device_sm_count();
    if (nsm_t == 0) return CLAIRE_ECUDA;
    static std::once_flag once_t[kSetupDevices];
    once_per_device(once_t, [] {
      cudaFuncSetAttribute(k_conv_wgrad_tc_t, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           WT_SMEM);
    });
    const int ntiles = B * D * (H / 8) * (W / 8);
    const int ncta = std::max(1, std::min(std::min(nsplit, nsm_t), ntiles));
    const int nmt = (cin + 127) / 128;
    k_conv_wgrad_tc_t<<<dim3(ncta, nmt * (cout / 16)), WG_THREADS, WT_SMEM, st0>>>(
        (const bf16*)x, s, cin, (const bf16*)dy, cout, partial);
    const int64_t n = (int64_t)cout * 27 * cin;
    k_sum_partials<<<blocks(n), 256, 0, st0>>>(partial, ncta, n, dw);
    return cudaGetLastError() == cudaSuccess ? CLAIRE_OK : CLAIRE_ECUDA;
  }
  // mma.sync path: chunks of at least 4096 voxels (more splits only add partials to sum)
  const int64_t nsp = std::max<int64_t>(1, std::min<int64_t>(nsplit, V / 4096));
  int64_t chunk = (V + nsp - 1) / nsp;
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
                                    double* partial, int nblocks, void* stream) {
  if (!dy || !db || !partial || V < 1 || nblocks < 1 || C < 2 || C % 2 || C > 512 ||
      (reinterpret_cast<uintptr_t>(dy) & 3))
    return CLAIRE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t chunk = (V + nblocks - 1) / nblocks;
  const int nb = (int)((V + chunk - 1) / chunk);           // CTAs that own voxels
  k_bias_grad_part<<<nb, 256, 0, st>>>((const bf16*)dy, V, C, chunk, partial);
  k_bias_grad_final<<<(C + 7) / 8, 256, 0, st>>>(partial, nb, C, db);
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

claire_status claire_wait_status(int* timeouts) {
  if (cudaDeviceSynchronize() != cudaSuccess) return CLAIRE_ECUDA;
  unsigned int n = 0;
  const unsigned int zero = 0;
  if (cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof n) != cudaSuccess ||
      cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof zero) != cudaSuccess)
    return CLAIRE_ECUDA;
  n += take_brick_timeouts() + take_brick_timeouts_h();
  if (timeouts) *timeouts = (int)n;
  return n ? CLAIRE_ETIMEOUT : CLAIRE_OK;
}

claire_status claire_wait_selftest(int max_polls, int arrive, void* stream) {
  if (max_polls < 1 || max_polls > (1 << 20)) return CLAIRE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  k_wait_selftest<<<1, 32, 0, st>>>((uint32_t)max_polls, arrive);
  int gave_up = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyFromSymbolAsync(&gave_up, g_selftest_result, sizeof gave_up, 0,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CLAIRE_ECUDA;
  return gave_up ? CLAIRE_ETIMEOUT : CLAIRE_OK;
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
