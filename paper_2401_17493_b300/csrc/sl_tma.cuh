// TMA staging of the SL bricks (Sec. 2.5.4 gathers): tile predicate, mbarrier
// set-up, the tiled loads and the bounded waits, shared by the FP32 kernels
// (kernels.cu) and the FP16-storage kernels (mixed.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "sl_brick.cuh"
#include "tc_sm100.cuh"

namespace claire {

// The SL bricks of k_sl and k_trace are staged by the tensor-memory accelerator
// where the brick lies inside the grid: the source field is a 3D tensor map
// (n3, n2, ncomp n1) and the whole brick is one box of BB3 x BB2 x (t1 + 6)
// FP32 values (x3 x x2 x x1) at (i3_0 - 4, i2_0 - 3, c n1 + i1_0 - 3), written
// densely into shared memory: rows of BB3 = 64 floats, the layout of
// stage_brick, of which the gather reads the first BX3 = 40 (values beyond n3
// in the padding are filled with zeros and never read).  One request per brick,
// issued by one thread.  Bricks that wrap around the periodic grid (the tiles
// at the ends of each axis, or grids narrower than a brick) are staged by the
// threads' cp.async copies instead.  The load completes on an mbarrier.  The
// wait is bounded: a thread whose wait runs out counts it in g_brick_timeouts
// (read by claire_wait_status), waits once more (bounded) for the copy in
// flight and leaves its outputs unwritten.
constexpr uint32_t BRICK_WAIT = 1u << 20;       // try_wait calls of <= 1 us each

// Threads whose brick wait ran out (one counter per translation unit; each
// unit's host code reads and resets its own).
static __device__ unsigned int g_brick_timeouts = 0;

// True when the tile's brick lies inside the grid on every axis: x3 range
// [i3_0 - 4, i3_0 + 36), x2 range [i2_0 - 3, i2_0 + 11), x1 range
// [i1_0 - 3, i1_0 + t1 + 3).
__device__ __forceinline__ bool brick_tma_ok(const Grid& g, int i1_0, int i2_0, int i3_0,
                                             int t1) {
  return i3_0 - HB3_LO >= 0 && i3_0 - HB3_LO + BX3 <= g.n3 && i2_0 - HB_LO >= 0 &&
         i2_0 + TB2 + HB_HI <= g.n2 && i1_0 - HB_LO >= 0 && i1_0 + t1 + HB_HI <= g.n1;
}

// mbarrier of the brick loads (one arrival per phase) set up by thread 0; the
// caller's barrier publishes it before the first load.
__device__ __forceinline__ void brick_mbar_init(uint64_t* mbar) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
}

// Thread 0 issues the TMA load of component c's brick into s; it completes on
// the mbarrier's current phase.  The mbarrier must be set up and published, and
// the shared brick no longer in use (a barrier since its last reads).
__device__ __forceinline__ void issue_brick_tma(const CUtensorMap* map, int c, const Grid& g,
                                                int i1_0, int i2_0, int i3_0,
                                                float* __restrict__ s, int t1, uint64_t* mbar) {
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  fence_proxy_async_smem();                     // earlier generic accesses of the brick first
  mbar_arrive_expect_tx(mbar, (uint32_t)brick_floats(t1) * (uint32_t)sizeof(float));
  tma_load_3d(s, map, i3_0 - HB3_LO, i2_0 - HB_LO, c * g.n1 + i1_0 - HB_LO, mbar);
}

// Bounded wait for the brick loads of phase `parity`; false if it ran out (counted).
__device__ __forceinline__ bool wait_brick_tma(uint64_t* mbar, uint32_t parity) {
  if (mbar_wait(mbar, parity, BRICK_WAIT)) return true;
  atomicAdd(&g_brick_timeouts, 1u);
  (void)mbar_wait(mbar, parity, BRICK_WAIT);    // the copies in flight, again bounded
  return false;
}

// ---- FP16 bricks (mixed form) ----------------------------------------------
//
// The source field is FP16; the gather reads the FP32 brick of stage_brick's
// layout.  A TMA box of 128 x 14 x (t1 + 6) halves starting at x3 = i3_0 - 8
// (a box's x start must be a multiple of 16 bytes: 8 halves) lands densely
// 128 bytes into the brick, row r at byte 128 + 256 r, so the 40 halves the
// brick row needs (x3 = i3_0 - 4 ..) sit at bytes 136 + 256 r .. 216 + 256 r.
// They are converted in place into the FP32 row r (bytes 256 r .. 256 r + 160):
// the only overlap is inside a row (FP32 values 34..39 over halves 0..11), and
// each row is converted by ten lanes of one warp that all load before any
// stores (__syncwarp).  The box's other halves fall on padding or on the
// not yet converted start of the next row; 128 bytes past the brick hold the
// last row's tail.
constexpr int BRICK_H_BOX = 128;                 // halves per box row (256 bytes)
__host__ __device__ inline size_t brick_h_smem_bytes(int t1) {
  return (size_t)brick_floats(t1) * sizeof(float) + 128 + 16;   // + tail, mbarrier
}

// Thread 0 issues the FP16 brick load (component c of a stacked map).
__device__ __forceinline__ void issue_brick_tma_h(const CUtensorMap* map, int c, const Grid& g,
                                                  int i1_0, int i2_0, int i3_0,
                                                  float* __restrict__ s, int t1,
                                                  uint64_t* mbar) {
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(mbar, (uint32_t)(brick_rows(t1) * BRICK_H_BOX * sizeof(__half)));
  tma_load_3d(reinterpret_cast<char*>(s) + 128, map, i3_0 - HB3_LO - 4, i2_0 - HB_LO,
              c * g.n1 + i1_0 - HB_LO, mbar);
}

// In-place conversion of the landed halves into the FP32 brick; ends with a
// barrier that publishes the brick.
__device__ __forceinline__ void convert_brick_h(float* __restrict__ s, int t1) {
  constexpr int Q = BX3 / 4;                     // 10 chunks of 4 values per row
  const int rows = brick_rows(t1);
  const int lane = threadIdx.x, w = threadIdx.y;
  const int sub = lane / Q, q = lane - sub * Q;  // 3 rows per warp and pass
  const char* raw = reinterpret_cast<const char*>(s) + 128 + 8;
  for (int base = 0; base < rows; base += 3 * (BRICK_THREADS / 32)) {
    const int row = base + 3 * w + sub;
    const bool on = lane < 3 * Q && row < rows;
    uint2 h = make_uint2(0u, 0u);
    if (on) h = *reinterpret_cast<const uint2*>(raw + 256 * row + 8 * q);
    __syncwarp();                                // the row's halves read before it is written
    if (on) {
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&h.y));
      *reinterpret_cast<float4*>(s + row * BB3 + 4 * q) = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncwarp();
  }
  __syncthreads();
}

}  // namespace claire
