// FD8 over the state history by marching along x1 (Sec. 2.5.3).
//
// A CTA owns an x2 x x3 tile of MT2 x 32 nodes and marches MT1 planes along
// x1.  For each of the NF = nt + 1 history fields it keeps, per thread, a
// 9-deep register queue of the field along x1 (the x1 derivative), and per
// plane it stages the tile plus a 4-node halo in x2 and x3 in shared memory
// (the x2 and x3 derivatives).  Each history value is read once from HBM for
// the queue; the plane halo is re-read from L2.
//
//   SDOT:  s^j = (j == 0 ? scale0 : 1) * grad8(m^j) . vt              j = 0..nt
//   ACCUM: out = base_coef * base + sum_j w_j lam^j grad8(m^j)        (trapezoid w_j)
//          and, when partial != NULL, this block's share of <dotv, out> in
//          partial[linear block id] (the PCG curvature <s, H s>).
// The trapezoid weight is applied as 0.5 * (ht * lam) at the end points.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "reduce.cuh"

namespace claire {

constexpr int MT2 = 8, MT3 = 32, MT1 = 32;          // tile x2, x3; planes per CTA without a context
constexpr int MP2 = MT2 + 8, MP3 = MT3 + 8;         // staged plane with the FD8 halo
constexpr int MPLANE = MP2 * MP3;                   // 640 floats

__host__ inline dim3 march_grid(const Grid& g, int mt1 = MT1) {
  return dim3((g.n3 + MT3 - 1) / MT3, (g.n2 + MT2 - 1) / MT2, (g.n1 + mt1 - 1) / mt1);
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
template <typename T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_f<__half>(float x) { return __float2half_rn(x); }

// 2^-ceil(log2 x) for x > 0 (power-of-two scale that maps x into (1/2, 1]), 1 otherwise.
__device__ __forceinline__ float pow2_scale(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0f;
  int e;
  frexp(x, &e);                                    // x = m 2^e, m in [1/2, 1)
  e = e < -120 ? -120 : (e > 120 ? 120 : e);
  return ldexpf(1.0f, -e);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {      // all but the newest group done
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Two FD8 first derivatives at once on packed FP32 pairs (fma.rn.f32x2): the same
// arithmetic as fd8() per component, the differences as fused multiply-adds by -1.
__device__ __forceinline__ float2 fd8_pair(float2 m4, float2 m3, float2 m2, float2 m1, float2 p1,
                                           float2 p2, float2 p3, float2 p4, float2 inv_h) {
  const float2 neg = make_float2(-1.0f, -1.0f);
  const float c1 = 672.0f / 840.0f, c2 = 168.0f / 840.0f, c3 = 32.0f / 840.0f,
              c4 = 3.0f / 840.0f;
  float2 r = __fmul2_rn(make_float2(c1, c1), __ffma2_rn(neg, m1, p1));
  r = __ffma2_rn(make_float2(-c2, -c2), __ffma2_rn(neg, m2, p2), r);
  r = __ffma2_rn(make_float2(c3, c3), __ffma2_rn(neg, m3, p3), r);
  r = __ffma2_rn(make_float2(-c4, -c4), __ffma2_rn(neg, m4, p4), r);
  return __fmul2_rn(r, inv_h);
}

// Staging of plane i1 (tile plus the 4-node halo in x2 and x3) in chunks of 4
// elements (16 bytes FP32, 8 bytes FP16).  The staged x3 window starts on a
// multiple of 4, so with n3 % 4 == 0 a chunk never straddles the periodic
// wrap, and the MP2 x MP3 / 4 = 160 chunks of a plane are at most one per
// thread: each thread computes its chunk's in-plane source offset once
// (plane_chunk) and per plane and field issues a single cp.async.
struct PlaneChunk {
  int src;   // in-plane element offset of the chunk, -1: this thread has none
  int dst;   // element offset in the staged plane
};
static_assert(MP2 * (MP3 / 4) <= 32 * MT2, "at most one plane chunk per thread");

__device__ __forceinline__ PlaneChunk plane_chunk(const Grid& g, int i2_0, int i3_0) {
  constexpr int Q = MP3 / 4;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  PlaneChunk c{-1, 0};
  if (tid < MP2 * Q) {
    const int r2 = tid / Q, q = tid - r2 * Q;
    c.src = wrap_any(i2_0 - 4 + r2, g.n2) * g.n3 + wrap_any(i3_0 - 4 + 4 * q, g.n3);
    c.dst = r2 * MP3 + 4 * q;
  }
  return c;
}

template <typename T>
__device__ __forceinline__ void stage_plane_async(const T* __restrict__ u, const Grid& g, int i1,
                                                  int i2_0, int i3_0, const PlaneChunk& ch,
                                                  bool vec, T* __restrict__ s) {
  const T* plane = u + (int64_t)i1 * g.n2 * g.n3;
  if (vec) {
    if (ch.src >= 0) {
      if (sizeof(T) == 4) cp_async16(s + ch.dst, plane + ch.src);
      else cp_async8(s + ch.dst, plane + ch.src);
    }
  } else {
    // n3 % 4 != 0: element copies (4-byte cp.async for FP32, plain loads for FP16)
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int item = tid; item < MP2 * MP3; item += 32 * MT2) {
      const int r2 = item / MP3, e = item - r2 * MP3;
      const T* src = plane + (int64_t)wrap_any(i2_0 - 4 + r2, g.n2) * g.n3 +
                     wrap_any(i3_0 - 4 + e, g.n3);
      if (sizeof(T) == 4) cp_async4(s + item, src);
      else s[item] = *src;
    }
  }
}

// MODE 0 (SDOT):  hout^j = (j == 0 ? scale0 : 1) * grad8(m^j) . (sig vt)
// MODE 1 (ACCUM): out = base_coef * base + (umul / sig) sum_j w_j lam^j grad8(m^j),
//                 and, when partial != NULL, this block's share of <dotv, out>.
// sig = pow2_scale(*vmax) when vmax != NULL (the FP16 form keeps the
// incremental fields in range with it), else 1; T = float or __half storage
// of the histories.  NF = nt + 1 history fields.
//
// Software pipeline: while plane i1 is computed, plane i1 + 1 is already being
// copied into the other shared-memory buffer (cp.async) and the per-node
// values of plane i1 + 1 (queue head, lam^j, vt, base, dotv) are already
// loading into registers, so each plane costs one barrier round instead of a
// global-memory round trip.
//
// march_tile does the work of the CTA at tile (bx, by, bz) of a launch with
// gx x gy tiles per x1 slab (the partial sum goes to partial[(bz gy + by) gx
// + bx]); sp / fp are the CTA's shared staging buffers (MarchSmem).  It ends
// with a barrier, so the buffers may be reused right after it.
template <int NF, typename T>
struct MarchSmem {
  // sp: staged planes as stored (double buffer).  FP16 planes are converted
  // into the FP32 plane fp by the threads that copied them, once per element,
  // so the 16 stencil reads per field and node need no conversion.
  static constexpr bool kHalf = sizeof(T) == 2;
  __align__(16) T sp[2][NF][MPLANE];
  __align__(16) float fp[kHalf ? NF : 1][kHalf ? MPLANE : 4];
};

template <int MODE, int NF, typename T>
__device__ __forceinline__ void march_tile(
    const Grid& g, const T* __restrict__ mhist, const T* __restrict__ lhist,
    const float* __restrict__ vt, float scale0, const double* __restrict__ vmax,
    const float* __restrict__ base, float base_coef, float umul, float* __restrict__ out,
    T* __restrict__ hout, const float* __restrict__ dotv, double* __restrict__ partial, int mt1,
    int bx, int by, int bz, int gx, int gy, MarchSmem<NF, T>& S) {
  constexpr bool kHalf = MarchSmem<NF, T>::kHalf;
  auto& sp = S.sp;
  auto& fp = S.fp;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i3_0 = bx * MT3, i2_0 = by * MT2, i1_0 = bz * mt1;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N;
  const int64_t s1 = (int64_t)g.n2 * g.n3;
  const int64_t col = active ? (int64_t)i2 * g.n3 + i3 : 0;   // (i2, i3) offset in a plane
  const int nt = NF - 1;
  const float ht = 1.0f / (float)nt;
  const float sig = vmax ? pow2_scale(*vmax) : 1.0f;
  const float unscale = umul / sig;
  const bool has_base = MODE == 1 && base != nullptr;
  const bool has_dot = MODE == 1 && partial != nullptr;
  // register queues q[f][k] = m^f(i1 - 4 + k), k = 0..8
  float q[NF][9];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      q[f][k] = active ? to_f(mhist[f * N + wrap_any(i1_0 - 4 + k, g.n1) * s1 + col]) : 0.f;
  const int i1_end = min(i1_0 + mt1, g.n1);
  // prefetched per-node values of the next plane
  T hn[NF], ln[NF];
  float xn[3];
  float dn[3];
  auto fetch = [&](int i1) {
    const int64_t idx = (int64_t)i1 * s1 + col;
#pragma unroll
    for (int f = 0; f < NF; ++f) hn[f] = mhist[f * N + wrap_near(i1 + 4, g.n1) * s1 + col];
    if (MODE == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) xn[a] = vt[a * N + idx];
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) ln[f] = lhist[f * N + idx];
      if (has_base) {
#pragma unroll
        for (int a = 0; a < 3; ++a) xn[a] = base[a * N + idx];
      }
      if (has_dot) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dn[a] = dotv[a * N + idx];
      }
    }
  };
  const PlaneChunk ch = plane_chunk(g, i2_0, i3_0);
  const bool vec = (g.n3 % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(mhist) & (4 * sizeof(T) - 1)) == 0);
#pragma unroll
  for (int f = 0; f < NF; ++f)
    stage_plane_async(mhist + f * N, g, i1_0, i2_0, i3_0, ch, vec, sp[0][f]);
  cp_async_commit();
  if (active) fetch(i1_0);
  KahanF dacc;
  const int c = (ty + 4) * MP3 + lane + 4;                     // node in the staged plane
  for (int i1 = i1_0; i1 < i1_end; ++i1) {
    const int cur = (i1 - i1_0) & 1;
    float lc[NF], xc[3], dc[3];
    if (active) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        q[f][8] = to_f(hn[f]);
        lc[f] = MODE == 1 ? ht * to_f(ln[f]) : 0.f;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        xc[a] = (MODE == 0 || has_base) ? xn[a] : 0.f;
        dc[a] = has_dot ? dn[a] : 0.f;
      }
    }
    if (i1 + 1 < i1_end) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        stage_plane_async(mhist + f * N, g, i1 + 1, i2_0, i3_0, ch, vec, sp[cur ^ 1][f]);
      if (active) fetch(i1 + 1);
    }
    cp_async_commit();
    cp_async_wait_prev();
    if constexpr (kHalf) {
      // convert the chunks (or elements) this thread staged itself
      if (vec) {
        if (ch.src >= 0) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const uint2 raw = *reinterpret_cast<const uint2*>(&sp[cur][f][ch.dst]);
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
            *reinterpret_cast<float4*>(&fp[f][ch.dst]) = make_float4(a.x, a.y, b.x, b.y);
          }
        }
      } else {
        const int tid = threadIdx.y * 32 + threadIdx.x;
        for (int item = tid; item < MPLANE; item += 32 * MT2)
#pragma unroll
          for (int f = 0; f < NF; ++f) fp[f][item] = to_f(sp[cur][f][item]);
      }
    }
    __syncthreads();                                           // plane i1 staged by all
    if (active) {
      const int64_t idx = (int64_t)i1 * s1 + col;
      float a0 = 0.f;
      float2 a12 = make_float2(0.f, 0.f);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* p;
        if constexpr (kHalf) p = fp[f];
        else p = sp[cur][f];
        const float gx = fd8(q[f][0], q[f][1], q[f][2], q[f][3], q[f][5], q[f][6], q[f][7],
                             q[f][8], g.inv_h1);
        // the x2 and x3 derivatives as one packed FP32 pair
        const float2 gyz = fd8_pair(
            make_float2(p[c - 4 * MP3], p[c - 4]), make_float2(p[c - 3 * MP3], p[c - 3]),
            make_float2(p[c - 2 * MP3], p[c - 2]), make_float2(p[c - MP3], p[c - 1]),
            make_float2(p[c + MP3], p[c + 1]), make_float2(p[c + 2 * MP3], p[c + 2]),
            make_float2(p[c + 3 * MP3], p[c + 3]), make_float2(p[c + 4 * MP3], p[c + 4]),
            make_float2(g.inv_h2, g.inv_h3));
        if (MODE == 0) {
          float sd = gx * (sig * xc[0]);
          sd = fmaf(gyz.x, sig * xc[1], sd);
          sd = fmaf(gyz.y, sig * xc[2], sd);
          hout[f * N + idx] = from_f<T>(f == 0 ? scale0 * sd : sd);
        } else {
          const float wl = (f == 0 || f == nt) ? 0.5f * lc[f] : lc[f];
          a0 = fmaf(wl, gx, a0);
          a12 = __ffma2_rn(make_float2(wl, wl), gyz, a12);
        }
      }
      if (MODE == 1) {
        float a1 = a12.x, a2 = a12.y;
        a0 *= unscale; a1 *= unscale; a2 *= unscale;
        if (has_base) {
          a0 = fmaf(base_coef, xc[0], a0);
          a1 = fmaf(base_coef, xc[1], a1);
          a2 = fmaf(base_coef, xc[2], a2);
        }
        out[idx] = a0;
        out[N + idx] = a1;
        out[2 * N + idx] = a2;
        if (has_dot) dacc.add(dc[0] * a0 + dc[1] * a1 + dc[2] * a2);
      }
    }
    // advance the queues
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < 8; ++k) q[f][k] = q[f][k + 1];
    __syncthreads();                                           // buffer cur consumed
  }
  if (has_dot) {
    const double b = block_sum(dacc.value());
    if (threadIdx.x == 0 && threadIdx.y == 0)
      partial[((int64_t)bz * gy + by) * gx + bx] = b;
  }
}

template <int MODE, int NF, typename T>
__global__ void __launch_bounds__(32 * MT2, NF <= 5 ? 2 : 1)
k_hist_march(Grid g, const T* __restrict__ mhist, const T* __restrict__ lhist,
             const float* __restrict__ vt, float scale0, const double* __restrict__ vmax,
             const float* __restrict__ base, float base_coef, float umul,
             float* __restrict__ out, T* __restrict__ hout, const float* __restrict__ dotv,
             double* __restrict__ partial, int mt1) {
  __shared__ MarchSmem<NF, T> S;
  march_tile<MODE, NF, T>(g, mhist, lhist, vt, scale0, vmax, base, base_coef, umul, out, hout,
                          dotv, partial, mt1, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x,
                          gridDim.y, S);
}

}  // namespace claire
