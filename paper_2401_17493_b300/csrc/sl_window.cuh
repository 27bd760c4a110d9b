// Tricubic gathers (Sec. 2.5.4) with a per-lane register window along x1.
//
// The brick-staged gather of sl_brick.cuh reads the 64 taps of every node from
// shared memory: 256 bytes per node through a 128 B/clk/SM pipe, which bounds
// an SL step well below the HBM roofline.  Consecutive nodes of one thread
// (x1 neighbours) whose displacement floors agree share 48 of their 64 taps
// (three of the four x1 planes of the 4 x 4 x 4 footprint).  Here every lane
// keeps the four planes of its footprint in registers and, per node, loads
// only the one new plane (16 taps):
//
//  * each lane fixes a reference floor (p1, p2, p3): that of the middle node
//    of its column of t1 nodes (clamped into the staged halo); its window
//    slides by one plane per node whatever the node's own floor is;
//  * a node whose floor equals the reference is contracted from the window
//    (same FP32 arithmetic in the same order as gather_brick, so the result
//    is bitwise the same as the brick gather);
//  * every other node is appended to a CTA-wide queue in shared memory and
//    gathered afterwards by all threads of the CTA with full warps
//    (gather_brick, or gather_global for taps outside the brick).  Predicated
//    per-lane reloads would cost the warp a full shared-memory wavefront per
//    load for a few lanes; the compacted queue keeps every warp full.
//
// The per-node operands (departure points, the epilogue's scale / aux fields)
// are staged as dense tiles [component][k][ty][lane] with cp.async together
// with the brick, so all of a CTA's global reads are in flight at once.
#pragma once

#include "sl_brick.cuh"

namespace claire {

constexpr int WIN_THREADS = BRICK_THREADS;     // 32 lanes (x3) x TB2 warps (x2)
__host__ __device__ inline int tile_elems(int t1) { return t1 * TB2 * TB3; }

// Shared-memory bytes of a windowed CTA: brick (FP32), ntiles dense FP32
// tiles, nhtiles dense 16-bit tiles, the deferred queue (one int per node of
// the tile) and two queue counters.
__host__ __device__ inline int window_smem_bytes(int t1, int ntiles, int nhtiles) {
  return brick_floats(t1) * 4 + ntiles * tile_elems(t1) * 4 + nhtiles * tile_elems(t1) * 2 +
         tile_elems(t1) * 4 + 16;
}

// Stage ncomp components (component stride cstride elements) of a dense
// per-node field over the tile's nodes into s[c][k][ty][lane], no halo and no
// wrap.  Nodes outside the grid are not copied (never read).  T = float or a
// 16-bit type; rows of 32 elements are copied as 16-byte chunks when the row
// start is 16-byte aligned.
template <typename T>
__device__ __forceinline__ void stage_tile(const T* __restrict__ src, int64_t cstride, int ncomp,
                                           const Grid& g, int i1_0, int i2_0, int i3_0, int t1,
                                           T* __restrict__ s) {
  constexpr int EPC = 16 / sizeof(T);            // elements per 16-byte chunk
  constexpr int CPR = TB3 / EPC;                 // chunks per 32-node row
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int rows = ncomp * t1 * TB2;
  const bool vec = (g.n3 % EPC == 0) && (cstride % EPC == 0) &&
                   ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  if (vec) {
    for (int item = tid; item < rows * CPR; item += WIN_THREADS) {
      const int row = item / CPR, q = item - row * CPR;
      const int c = row / (t1 * TB2), r = row - c * (t1 * TB2);
      const int k = r / TB2, y = r - k * TB2;
      const int i1 = i1_0 + k, i2 = i2_0 + y, i3 = i3_0 + q * EPC;
      if (i1 < g.n1 && i2 < g.n2 && i3 < g.n3)
        cp_async16(s + row * TB3 + q * EPC, src + c * cstride + lin(g, i1, i2, i3));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  } else {
    for (int item = tid; item < rows * TB3; item += WIN_THREADS) {
      const int row = item / TB3, l = item - row * TB3;
      const int c = row / (t1 * TB2), r = row - c * (t1 * TB2);
      const int k = r / TB2, y = r - k * TB2;
      const int i1 = i1_0 + k, i2 = i2_0 + y, i3 = i3_0 + l;
      if (i1 < g.n1 && i2 < g.n2 && i3 < g.n3) s[row * TB3 + l] = src[c * cstride + lin(g, i1, i2, i3)];
    }
  }
}

// Index of node (k, ty, lane) of component c in a staged dense tile.
__device__ __forceinline__ int tile_at(int t1, int c, int k, int ty, int lane) {
  return ((c * t1 + k) * TB2 + ty) * TB3 + lane;
}

// Reference floor of a lane: the floor of the displacement d (grid units),
// or (0, 0, 0) when the taps of that floor would leave the staged brick.
__device__ __forceinline__ void window_reference(float d1, float d2, float d3, int& r1, int& r2,
                                                 int& r3) {
  r1 = (int)floorf(d1);
  r2 = (int)floorf(d2);
  r3 = (int)floorf(d3);
  const bool in = r1 >= 1 - HB_LO && r1 <= HB_HI - 2 && r2 >= 1 - HB_LO && r2 <= HB_HI - 2 &&
                  r3 >= 1 - HB3_LO && r3 <= HB3_HI - 2;
  if (!in) r1 = r2 = r3 = 0;
}

// One x1 plane of a lane's footprint (4 rows x 4 columns) as two float2
// columns per x3 tap: rows (0, 1) and rows (2, 3), the operand pairs of the
// packed contraction.
struct WinPlane {
  float2 a[4], b[4];
};

__device__ __forceinline__ void window_load(WinPlane& w, const float* __restrict__ p) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    w.a[c] = make_float2(p[c], p[BB3 + c]);
    w.b[c] = make_float2(p[2 * BB3 + c], p[3 * BB3 + c]);
  }
}

// Partial sums of one window plane for node taps t: the x3 contraction of
// rows (0, 1) and (2, 3), then the x2 weights, in gather_brick's order.
__device__ __forceinline__ float2 window_plane_sum(const WinPlane& q, const NodeTaps& t) {
  float2 ra = make_float2(0.0f, 0.0f), rb = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float2 w = make_float2(t.w3[c], t.w3[c]);
    ra = __ffma2_rn(w, q.a[c], ra);
    rb = __ffma2_rn(w, q.b[c], rb);
  }
  const float2 a2 = __fmul2_rn(make_float2(t.w2[0], t.w2[1]), ra);
  return __ffma2_rn(make_float2(t.w2[2], t.w2[3]), rb, a2);
}

// Append every lane's queued nodes (bit k of `mask`: node k of the lane's
// column, k < kmax <= 16) to the CTA queue as codes k << 8 | ty << 5 | lane,
// ordered by node row k and then by lane (consecutive queue entries then sit
// in different lanes, so the deferred gather's warps hit fewer shared-memory
// banks twice than with each lane's nodes stored together); one shared-memory
// atomic per warp.  Every lane of the warp must call it.
__device__ __forceinline__ void window_enqueue(unsigned mask, int kmax, int ty, int lane,
                                               int* __restrict__ queue, int* __restrict__ qcount) {
  const unsigned below = (1u << lane) - 1u;
  int total = 0;
  for (int k = 0; k < kmax; ++k) total += __popc(__ballot_sync(0xffffffffu, (mask >> k) & 1u));
  if (total == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(qcount, total);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int k = 0; k < kmax; ++k) {
    const unsigned m = __ballot_sync(0xffffffffu, (mask >> k) & 1u);
    if ((mask >> k) & 1u) queue[base + __popc(m & below)] = (k << 8) | (ty << 5) | lane;
    base += __popc(m);
  }
}

// March of one lane over its column of kmax (<= t1 <= 16) nodes in the staged
// brick s.  disp(k, ty, lane, d[3]) gives a node's displacement in grid units;
// epi(k, ty, lane, value) consumes its interpolated value.  (r1, r2, r3) is
// the lane's reference floor.  Nodes with another floor go to the queue.  The
// new plane of node k + 1 is requested as soon as node k's first plane has
// been contracted (its slot is free then), so its latency overlaps the rest of
// node k.  Must be called by every thread of the CTA (inactive lanes pass
// active = false: they load planes inside the brick but neither store nor
// enqueue).
template <class Disp, class Epi>
__device__ __forceinline__ void window_march(const float* __restrict__ s, int kmax, int ty,
                                             int lane, bool active, int r1, int r2, int r3,
                                             Disp&& disp, Epi&& epi, int* __restrict__ queue,
                                             int* __restrict__ qcount) {
  constexpr int PL = BB2 * BB3;
  const float* base =
      s + ((HB_LO + r1 - 1) * BB2 + ty + HB_LO + r2 - 1) * BB3 + lane + HB3_LO + r3 - 1;
  WinPlane w0, w1, w2, w3;                      // slot (k + i) & 3 holds plane i of node k
  window_load(w0, base);
  window_load(w1, base + PL);
  window_load(w2, base + 2 * PL);
  window_load(w3, base + 3 * PL);
  unsigned slow = 0u;
#define CLAIRE_WIN_STEP(KK, Q0, Q1, Q2, Q3)                                       \
  {                                                                              \
    const int k = k0 + (KK);                                                     \
    if (k < kmax) {                                                              \
      float d[3];                                                                \
      disp(k, ty, lane, d);                                                      \
      NodeTaps t;                                                                \
      node_taps(d[0], d[1], d[2], t);                                            \
      float2 acc = __ffma2_rn(make_float2(t.w1[0], t.w1[0]), window_plane_sum(Q0, t), \
                              make_float2(0.0f, 0.0f));                          \
      if (k + 1 < kmax) window_load(Q0, base + (k + 4) * PL);                    \
      acc = __ffma2_rn(make_float2(t.w1[1], t.w1[1]), window_plane_sum(Q1, t), acc); \
      acc = __ffma2_rn(make_float2(t.w1[2], t.w1[2]), window_plane_sum(Q2, t), acc); \
      acc = __ffma2_rn(make_float2(t.w1[3], t.w1[3]), window_plane_sum(Q3, t), acc); \
      const bool same = t.p1 == r1 && t.p2 == r2 && t.p3 == r3;                  \
      if (active && same) epi(k, ty, lane, acc.x + acc.y);                       \
      if (active && !same) slow |= 1u << k;                                      \
    }                                                                            \
  }
#pragma unroll 1
  for (int k0 = 0; k0 < kmax; k0 += 4) {
    CLAIRE_WIN_STEP(0, w0, w1, w2, w3)
    CLAIRE_WIN_STEP(1, w1, w2, w3, w0)
    CLAIRE_WIN_STEP(2, w2, w3, w0, w1)
    CLAIRE_WIN_STEP(3, w3, w0, w1, w2)
  }
#undef CLAIRE_WIN_STEP
  window_enqueue(slow, kmax, ty, lane, queue, qcount);
}

// Gather the queued nodes with all threads of the CTA (call after a barrier
// that follows window_march).  far(t, i1, i2, i3) gathers a node whose taps
// leave the brick from the field in global memory.
template <class Disp, class Epi, class Far>
__device__ __forceinline__ void window_deferred(const float* __restrict__ s, int i1_0, int i2_0,
                                                int i3_0, int nq, const int* __restrict__ queue,
                                                Disp&& disp, Epi&& epi, Far&& far) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int q = tid; q < nq; q += WIN_THREADS) {
    const int code = queue[q];
    const int k = code >> 8, y = (code >> 5) & (TB2 - 1), l = code & 31;
    float d[3];
    disp(k, y, l, d);
    NodeTaps t;
    node_taps(d[0], d[1], d[2], t);
    const float val = taps_in_brick(t) ? gather_brick(s, t, k, y, l)
                                       : far(t, i1_0 + k, i2_0 + y, i3_0 + l);
    epi(k, y, l, val);
  }
}

}  // namespace claire
