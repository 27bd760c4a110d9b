// Brick-staged tricubic gathers (Sec. 2.5.4) for the SL steps and the trace.
//
// A CTA owns a tile of TB1 x TB2 x TB3 arrival nodes (x1 x x2 x x3) and stages
// the source field over the tile plus a halo into shared memory with
// coalesced, periodic-wrapped loads (float4 along x3 when the row segment is
// aligned and does not wrap).  Each thread then evaluates the 64-tap
// interpolation of its TB1 nodes from shared memory.  A node whose taps leave
// the staged brick (|displacement| beyond the halo) takes the global-memory
// gather instead, so any displacement is handled exactly.
//
// Tap nodes of a node i with displacement d are i + floor(d) - 1 .. + 2, so
// the brick covers floor(d) in [-(H_lo - 1), H_hi - 2] on each axis.
#pragma once

#include "common.cuh"

namespace claire {

// tile: x1 (loop, depth t1 chosen at launch from {4, 8, 16} by the autotuner),
// x2 (threadIdx.y), x3 (lane)
constexpr int TB1 = 8, TB2 = 8, TB3 = 32;      // TB1: default depth
constexpr int HB_LO = 3, HB_HI = 3;            // x1 / x2 halo: floor(d) in [-2, 1]
constexpr int HB3_LO = 4, HB3_HI = 4;          // x3 halo (float4 aligned): floor(d) in [-3, 2]
constexpr int BB1 = TB1 + HB_LO + HB_HI;       // 14
constexpr int BB2 = TB2 + HB_LO + HB_HI;       // 14
constexpr int BX3 = TB3 + HB3_LO + HB3_HI;     // 40 staged floats per row
// Row pitch 64 floats: row and plane strides are multiples of the 32 banks, so
// lanes whose displacement floors put them in different rows or planes read
// disjoint banks (only an x3 span wider than 32 words can still conflict).
constexpr int BB3 = 64;
constexpr int BRICK_FLOATS = BB1 * BB2 * BB3;  // 12544 floats = 49 KiB at depth 8
__host__ __device__ inline int brick_rows(int t1) { return (t1 + HB_LO + HB_HI) * BB2; }
__host__ __device__ inline int brick_floats(int t1) { return brick_rows(t1) * BB3; }
constexpr int BRICK_THREADS = 32 * TB2;        // 256

__host__ inline dim3 brick_grid(const Grid& g, int t1 = TB1) {
  return dim3((g.n3 + TB3 - 1) / TB3, (g.n2 + TB2 - 1) / TB2, (g.n1 + t1 - 1) / t1);
}

// The staged coordinates lie in [-n, 2n) on every axis when the grid is at
// least one brick wide (n1 >= t1 + 6, n2 >= BB2, n3 >= BX3): one compare
// and add instead of an integer modulo per staged chunk.
__device__ __forceinline__ bool brick_wrap_near(const Grid& g, int t1) {
  return g.n1 >= t1 + HB_LO + HB_HI && g.n2 >= BB2 && g.n3 >= BX3;
}
__device__ __forceinline__ int wrap_sel(int i, int n, bool near) {
  return near ? wrap_near(i, n) : wrap_any(i, n);
}

// Stage field u over the tile of (i1_0, i2_0, i3_0) plus halo into
// s[t1 + 6][BB2][BB3] (t1 = tile depth along x1).
__device__ __forceinline__ void stage_brick(const float* __restrict__ u, const Grid& g, int i1_0,
                                            int i2_0, int i3_0, float* __restrict__ s,
                                            int t1 = TB1) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int x3s = i3_0 - HB3_LO;
  // x3s is a multiple of 4, so with n3 % 4 == 0 a 4-float chunk never
  // straddles the periodic wrap: edge tiles copy whole wrapped chunks too
  const bool vec = (g.n3 % 4 == 0) && ((reinterpret_cast<uintptr_t>(u) & 15) == 0);
  const bool near = brick_wrap_near(g, t1);
  constexpr int Q = BX3 / 4;                         // float4 per staged row
  const int nitems = brick_rows(t1) * Q;
  for (int item = tid; item < nitems; item += BRICK_THREADS) {
    const int row = item / Q, q = item - row * Q;
    const int r1 = row / BB2, r2 = row - r1 * BB2;
    const int g1 = wrap_sel(i1_0 - HB_LO + r1, g.n1, near);
    const int g2 = wrap_sel(i2_0 - HB_LO + r2, g.n2, near);
    const float* src = u + ((int64_t)g1 * g.n2 + g2) * g.n3;
    float* dst = s + row * BB3 + 4 * q;
    if (vec) {
      cp_async16(dst, src + wrap_sel(x3s + 4 * q, g.n3, near));
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) cp_async4(dst + e, src + wrap_any(x3s + 4 * q + e, g.n3));
    }
  }
  cp_async_wait_all();          // this thread's copies; the caller's barrier publishes them
}

// Per-node interpolation setup shared by the brick and the global paths.
struct NodeTaps {
  int p1, p2, p3;            // floor of the displacement
  float w1[4], w2[4], w3[4]; // Lagrange weights
};

__device__ __forceinline__ void node_taps(float d1, float d2, float d3, NodeTaps& t) {
  const float f1 = floorf(d1), f2 = floorf(d2), f3 = floorf(d3);
  t.p1 = (int)f1; t.p2 = (int)f2; t.p3 = (int)f3;
  lagrange4(d1 - f1, t.w1);
  lagrange4(d2 - f2, t.w2);
  lagrange4(d3 - f3, t.w3);
}

__device__ __forceinline__ bool taps_in_brick(const NodeTaps& t) {
  return t.p1 >= 1 - HB_LO && t.p1 <= HB_HI - 2 && t.p2 >= 1 - HB_LO && t.p2 <= HB_HI - 2 &&
         t.p3 >= 1 - HB3_LO && t.p3 <= HB3_HI - 2;
}

// 64-tap sum from the staged brick; (k, ty, lane) is the node's tile position.
// The contraction runs on packed FP32 pairs (fma.rn.f32x2 of the sm_100 family):
// rows j = 0, 1 and j = 2, 3 of each x1 plane share one instruction per x3 tap,
// the x2 weights are applied pairwise and the two halves are added at the end.
// Same FP32 arithmetic as the scalar form, half the FMA instructions, another
// summation order (a zero displacement still returns the node value exactly:
// its weights are (0, 1, 0, 0) on every axis).
__device__ __forceinline__ float gather_brick(const float* __restrict__ s, const NodeTaps& t, int k,
                                              int ty, int lane) {
  const float* b = s + ((k + HB_LO + t.p1 - 1) * BB2 + (ty + HB_LO + t.p2 - 1)) * BB3 +
                   (lane + HB3_LO + t.p3 - 1);
  const float2 w2a = make_float2(t.w2[0], t.w2[1]), w2b = make_float2(t.w2[2], t.w2[3]);
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float* p = b + i * BB2 * BB3;            // row (i, j = 0); rows j are BB3 apart
    float2 ra = make_float2(0.0f, 0.0f), rb = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float2 w = make_float2(t.w3[c], t.w3[c]);
      ra = __ffma2_rn(w, make_float2(p[c], p[BB3 + c]), ra);
      rb = __ffma2_rn(w, make_float2(p[2 * BB3 + c], p[3 * BB3 + c]), rb);
    }
    float2 a2 = __fmul2_rn(w2a, ra);
    a2 = __ffma2_rn(w2b, rb, a2);
    acc = __ffma2_rn(make_float2(t.w1[i], t.w1[i]), a2, acc);
  }
  return acc.x + acc.y;
}

// Same 64-tap sum from global memory with periodic wrap (any displacement).
__device__ __forceinline__ float gather_global(const float* __restrict__ u, const Grid& g,
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
      const float* row = u + o1[i] + o2[j];
      float acc3 = t.w3[0] * __ldg(row + o3[0]);
      acc3 = fmaf(t.w3[1], __ldg(row + o3[1]), acc3);
      acc3 = fmaf(t.w3[2], __ldg(row + o3[2]), acc3);
      acc3 = fmaf(t.w3[3], __ldg(row + o3[3]), acc3);
      acc2 = fmaf(t.w2[j], acc3, acc2);
    }
    acc = fmaf(t.w1[i], acc2, acc);
  }
  return acc;
}

}  // namespace claire
