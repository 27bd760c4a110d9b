// Shared device helpers: grid geometry, periodic wrap, cubic Lagrange weights
// and the FD8 first-derivative stencil.  Every kernel of the library includes
// this file; nothing here allocates or synchronises.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace claire {

// Periodic grid n1 x n2 x n3 on [-pi, pi)^3, x3 fastest (Sec. 2.5.1).
struct Grid {
  int n1, n2, n3;
  int64_t N;            // n1 * n2 * n3
  float inv_h1, inv_h2, inv_h3;   // 1 / h_i, h_i = 2 pi / n_i
  float h1, h2, h3;
};

__host__ __device__ inline int64_t lin(const Grid& g, int i1, int i2, int i3) {
  return ((int64_t)i1 * g.n2 + i2) * g.n3 + i3;
}

// i mod n for any int i (n > 0).
__device__ __forceinline__ int wrap_any(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// i mod n for i in [-n, 2n).
__device__ __forceinline__ int wrap_near(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Cubic Lagrange basis on the nodes {-1, 0, 1, 2} at offset t in [0, 1)
// (Sec. 2.5.4, p = 3): phi_k(t) = prod_{j != k} (t - j) / (k - j).
__device__ __forceinline__ void lagrange4(float t, float w[4]) {
  const float tp1 = t + 1.0f, tm1 = t - 1.0f, tm2 = t - 2.0f;
  const float a = t * tm1;           // t (t - 1)
  const float b = tp1 * tm2;         // (t + 1)(t - 2)
  w[0] = a * tm2 * (-1.0f / 6.0f);
  w[1] = b * tm1 * 0.5f;
  w[2] = b * t * -0.5f;
  w[3] = a * tp1 * (1.0f / 6.0f);
}

// Tap geometry along one axis for a displacement d (grid units) from node i:
// the four node indices (already multiplied by the axis stride) and weights.
struct Taps {
  int off[4];
  float w[4];
};

__device__ __forceinline__ void axis_taps(int i, float d, int n, int stride, Taps& t) {
  const float fl = floorf(d);
  const float frac = d - fl;                 // in [0, 1); computed from d, not x + d
  const int base = wrap_any(i + (int)fl - 1, n);
  lagrange4(frac, t.w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int j = base + k;
    j = j >= n ? j - n : j;
    t.off[k] = j * stride;
  }
}

// Tensor-product interpolation of one field given precomputed taps.
__device__ __forceinline__ float gather64(const float* __restrict__ u, const Taps& a,
                                          const Taps& b, const Taps& c) {
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float acc2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float* row = u + a.off[i] + b.off[j];
      float acc3 = c.w[0] * __ldg(row + c.off[0]);
      acc3 = fmaf(c.w[1], __ldg(row + c.off[1]), acc3);
      acc3 = fmaf(c.w[2], __ldg(row + c.off[2]), acc3);
      acc3 = fmaf(c.w[3], __ldg(row + c.off[3]), acc3);
      acc2 = fmaf(b.w[j], acc3, acc2);
    }
    acc = fmaf(a.w[i], acc2, acc);
  }
  return acc;
}

// FD8 first derivative from the 8 neighbours (Sec. 2.5.3):
// (672 (u1 - u_1) - 168 (u2 - u_2) + 32 (u3 - u_3) - 3 (u4 - u_4)) / (840 h).
__device__ __forceinline__ float fd8(float m4, float m3, float m2, float m1,
                                     float p1, float p2, float p3, float p4, float inv_h) {
  const float c1 = 672.0f / 840.0f, c2 = 168.0f / 840.0f, c3 = 32.0f / 840.0f,
              c4 = 3.0f / 840.0f;
  float r = c1 * (p1 - m1);
  r = fmaf(-c2, p2 - m2, r);
  r = fmaf(c3, p3 - m3, r);
  r = fmaf(-c4, p4 - m4, r);
  return r * inv_h;
}

// FD8 gradient of u at node (i1, i2, i3) read straight from global memory.
__device__ __forceinline__ void grad8_at(const float* __restrict__ u, const Grid& g, int i1,
                                         int i2, int i3, float out[3]) {
  const int64_t s1 = (int64_t)g.n2 * g.n3, s2 = g.n3;
  const float* base1 = u + (int64_t)i2 * s2 + i3;          // varies along axis 1
  const float* base2 = u + (int64_t)i1 * s1 + i3;          // along axis 2
  const float* base3 = u + (int64_t)i1 * s1 + (int64_t)i2 * s2;
  float a[8], b[8], c[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[3 - k] = __ldg(base1 + wrap_near(i1 - 1 - k, g.n1) * s1);
    a[4 + k] = __ldg(base1 + wrap_near(i1 + 1 + k, g.n1) * s1);
    b[3 - k] = __ldg(base2 + wrap_near(i2 - 1 - k, g.n2) * s2);
    b[4 + k] = __ldg(base2 + wrap_near(i2 + 1 + k, g.n2) * s2);
    c[3 - k] = __ldg(base3 + wrap_near(i3 - 1 - k, g.n3));
    c[4 + k] = __ldg(base3 + wrap_near(i3 + 1 + k, g.n3));
  }
  out[0] = fd8(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], g.inv_h1);
  out[1] = fd8(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], g.inv_h2);
  out[2] = fd8(c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], g.inv_h3);
}

// Asynchronous global -> shared copies (cp.async): all copies of a staging loop
// are in flight together instead of one load-store round trip per element.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace claire
