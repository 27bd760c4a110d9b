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
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace claire {

constexpr int MT2 = 8, MT3 = 32, MT1 = 32;          // tile x2, x3; default planes per CTA
constexpr int MP2 = MT2 + 8, MP3 = MT3 + 8;         // staged plane with the FD8 halo
constexpr int MPLANE = MP2 * MP3;                   // 640 floats

__host__ inline dim3 march_grid(const Grid& g, int mt1 = MT1) {
  return dim3((g.n3 + MT3 - 1) / MT3, (g.n2 + MT2 - 1) / MT2, (g.n1 + mt1 - 1) / mt1);
}

__device__ __forceinline__ void stage_plane(const float* __restrict__ u, const Grid& g, int i1,
                                            int i2_0, int i3_0, float* __restrict__ s) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const float* plane = u + (int64_t)i1 * g.n2 * g.n3;
  const int x3s = i3_0 - 4;
  const bool vec = (g.n3 % 4 == 0) && x3s >= 0 && x3s + MP3 <= g.n3 &&
                   ((reinterpret_cast<uintptr_t>(u) & 15) == 0);
  constexpr int Q = MP3 / 4;
  for (int item = tid; item < MP2 * Q; item += 32 * MT2) {
    const int r2 = item / Q, q = item - r2 * Q;
    const float* src = plane + (int64_t)wrap_any(i2_0 - 4 + r2, g.n2) * g.n3;
    float* dst = s + r2 * MP3 + 4 * q;
    if (vec) {
      cp_async16(dst, src + x3s + 4 * q);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) cp_async4(dst + e, src + wrap_any(x3s + 4 * q + e, g.n3));
    }
  }
}

// MODE 0 = SDOT, MODE 1 = ACCUM; NF = nt + 1 history fields.
template <int MODE, int NF>
__global__ void __launch_bounds__(32 * MT2) k_hist_march(Grid g, const float* __restrict__ mhist,
                                                         const float* __restrict__ lhist,
                                                         const float* __restrict__ vt,
                                                         float scale0,
                                                         const float* __restrict__ base,
                                                         float base_coef,
                                                         float* __restrict__ out,
                                                         const float* __restrict__ dotv,
                                                         double* __restrict__ partial,
                                                         int mt1) {
  __shared__ __align__(16) float sp[NF][MPLANE];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i3_0 = blockIdx.x * MT3, i2_0 = blockIdx.y * MT2, i1_0 = blockIdx.z * mt1;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N;
  const int64_t s1 = (int64_t)g.n2 * g.n3;
  const int64_t col = active ? (int64_t)i2 * g.n3 + i3 : 0;   // (i2, i3) offset in a plane
  const int nt = NF - 1;
  const float ht = 1.0f / (float)nt;
  // register queues q[f][k] = m^f(i1 - 4 + k), k = 0..8
  float q[NF][9];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      q[f][k] = active ? __ldg(mhist + f * N + wrap_any(i1_0 - 4 + k, g.n1) * s1 + col) : 0.f;
  const int i1_end = min(i1_0 + mt1, g.n1);
  KahanF dacc;
  const int c = (ty + 4) * MP3 + lane + 4;                     // node in the staged plane
  for (int i1 = i1_0; i1 < i1_end; ++i1) {
    // queue head m(i1 + 4)
#pragma unroll
    for (int f = 0; f < NF; ++f)
      q[f][8] = active ? __ldg(mhist + f * N + wrap_near(i1 + 4, g.n1) * s1 + col) : 0.f;
    __syncthreads();                                           // previous plane consumed
#pragma unroll
    for (int f = 0; f < NF; ++f) stage_plane(mhist + f * N, g, i1, i2_0, i3_0, sp[f]);
    cp_async_wait_all();
    __syncthreads();
    if (active) {
      const int64_t idx = (int64_t)i1 * s1 + col;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      if (MODE == 0) {
        t1 = vt[idx]; t2 = vt[N + idx]; t3 = vt[2 * N + idx];
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
          out[f * N + idx] = f == 0 ? scale0 * sd : sd;
        } else {
          const float wl = ((f == 0 || f == nt) ? 0.5f * ht : ht) * lhist[f * N + idx];
          a0 = fmaf(wl, gx, a0);
          a1 = fmaf(wl, gy, a1);
          a2 = fmaf(wl, gz, a2);
        }
      }
      if (MODE == 1) {
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
    // advance the queues
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

}  // namespace claire
