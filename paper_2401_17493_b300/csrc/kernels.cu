// Device kernels of the registration hot path and their host launchers.
//
//  k_trace            RK2 departure points, both directions      (Sec. 2.5.2)
//  k_sl               one SL step: out = s(x) gather(u, x + d) + beta aux(x)
//  k_adjoint_factor   c(x) of the RK2 adjoint step with f = lam div v
//  k_grad8 / k_div8_march  FD8 gradient / divergence              (Sec. 2.5.3)
//  k_sdot_hist        s^j = grad8(m^j) . v~ for the whole state history
//  k_accum_hist       out = base_coef * base + sum_j w_j lam^j grad8(m^j)
//  k_spectral         diagonal Fourier multipliers between cuFFT R2C / C2R
//  k_reduce*          FP64 reductions (fixed block count, fixed order)
//  small vector kernels for PCG and the line search
//
// All grids are [n1][n2][n3] with n3 fastest; 3D kernels use 32 x 4 x 2
// thread blocks (x3 along threadIdx.x for coalescing, a compact 3D footprint
// for the L1 reuse of the 64-tap gathers).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math_constants.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "device_setup.h"
#include "internal.h"
#include "reduce.cuh"
#include "sl_brick.cuh"
#include "sl_window.cuh"
#include "fd8_march.cuh"
#include "tc_sm100.cuh"
#include "sl_tma.cuh"

namespace claire {

#define CLAIRE_KERNEL_INDEX                                               \
  const int i3 = blockIdx.x * blockDim.x + threadIdx.x;                   \
  const int i2 = blockIdx.y * blockDim.y + threadIdx.y;                   \
  const int i1 = blockIdx.z * blockDim.z + threadIdx.z;                   \
  if (i1 >= g.n1 || i2 >= g.n2 || i3 >= g.n3) return;                     \
  const int64_t idx = lin(g, i1, i2, i3);

static dim3 block3() { return dim3(32, 4, 2); }
static dim3 grid3(const Grid& g) {
  return dim3((g.n3 + 31) / 32, (g.n2 + 3) / 4, (g.n1 + 1) / 2);
}

// ---------------------------------------------------------------- trace

// RK2 departure points of both directions (Sec. 2.5.2) for the tile (bx, by, bz)
// of nodes.  The velocity components are staged one at a time into one brick,
// which serves both directions; the predictor y~ = x -+ h_t v(x) is
// interpolated from it, and the corrector y = x -+ (h_t / 2)(v(x) + v(y~)) is
// stored as y - x in grid units.  With use_tma the bricks come from vmap (v as
// an n3 x n2 x 3 n1 tensor: the components stacked along x1) and the loads
// complete on phases parity, parity ^ 1, parity of the mbarrier (set up and
// published by the caller, like a barrier since the brick's last use).
__device__ __forceinline__ void trace_tile(const Grid& g, const float* __restrict__ v,
                                           float* __restrict__ df, float* __restrict__ db,
                                           float ht, int t1, const CUtensorMap* vmap,
                                           bool use_tma, int bx, int by, int bz,
                                           float* __restrict__ sm, uint64_t* mbar,
                                           uint32_t parity) {
  const int i1_0 = bz * t1, i2_0 = by * TB2, i3_0 = bx * TB3;
  const int64_t N = g.N, s1 = (int64_t)g.n2 * g.n3;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int kmax = min(t1, g.n1 - i1_0);
  const int64_t idx0 = active ? lin(g, i1_0, i2, i3) : 0;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    if (c > 0) __syncthreads();                  // previous brick consumed
    if (use_tma) issue_brick_tma(vmap, c, g, i1_0, i2_0, i3_0, sm, t1, mbar);
    // v(x) of the first node is loaded while the brick is being staged
    float v0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v0[a] = active ? v[a * N + idx0] : 0.f;
    bool ok = true;
    if (use_tma) {
      ok = wait_brick_tma(mbar, parity ^ (uint32_t)(c & 1));
    } else {
      stage_brick(v + c * N, g, i1_0, i2_0, i3_0, sm, t1);
      __syncthreads();
    }
    if (!active || !ok) continue;
    const float ihc = c == 0 ? g.inv_h1 : (c == 1 ? g.inv_h2 : g.inv_h3);
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      float* out = dir == 0 ? df : db;
      if (out == nullptr) continue;
      const float sg = dir == 0 ? -ht : ht;      // transport along +v / -v
      // v(x) of the next node is loaded one node ahead
      float vn[3] = {v0[0], v0[1], v0[2]};
#pragma unroll 2
      for (int k = 0; k < kmax; ++k) {
        const int64_t idx = idx0 + k * s1;
        const float u1 = vn[0] * g.inv_h1, u2 = vn[1] * g.inv_h2,
                    u3 = vn[2] * g.inv_h3;             // v(x), grid units per unit time
        if (k + 1 < kmax) {
#pragma unroll
          for (int a = 0; a < 3; ++a) vn[a] = v[a * N + idx + s1];
        }
        NodeTaps t;
        node_taps(sg * u1, sg * u2, sg * u3, t);
        const float w = taps_in_brick(t) ? gather_brick(sm, t, k, ty, lane)
                                         : gather_global(v + c * N, g, t, i1_0 + k, i2, i3);
        const float uc = c == 0 ? u1 : (c == 1 ? u2 : u3);
        out[c * N + idx] = 0.5f * sg * (uc + w * ihc);
      }
    }
  }
}

// One CTA per tile.  With tma != 0 the interior bricks are staged by TMA.
__global__ void __launch_bounds__(BRICK_THREADS) k_trace(Grid g, const float* __restrict__ v,
                                                         float* __restrict__ df,
                                                         float* __restrict__ db, float ht,
                                                         int t1,
                                                         const __grid_constant__ CUtensorMap vmap,
                                                         int tma) {
  extern __shared__ __align__(128) float smb[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smb + brick_floats(t1));
  const bool use_tma =
      tma && brick_tma_ok(g, blockIdx.z * t1, blockIdx.y * TB2, blockIdx.x * TB3, t1);
  if (use_tma) {
    brick_mbar_init(mbar);
    __syncthreads();
  }
  trace_tile(g, v, df, db, ht, t1, &vmap, use_tma, blockIdx.x, blockIdx.y, blockIdx.z, smb, mbar,
             0u);
}

// ---------------------------------------------------------------- SL step

// MODE 0: out = (scale ? scale(x) : sigma) u(x + d) + beta aux(x)    (SL steps)
// MODE 1: out = 1 + (h_t/2)(u(y) + u(x) + h_t u(x) u(y)), u = div v: the factor
//         c(x) with which one RK2 step of d_t lam = lam div v along -v becomes
//         lam^j(x) = c(x) lam^{j+1}(y).
// For the tile (bx, by, bz); with use_tma the brick comes from umap and the load
// completes on phase `parity` of the mbarrier (set up and published by the
// caller, like a barrier since the brick's last use).
template <int MODE>
__device__ __forceinline__ void sl_tile(const Grid& g, const float* __restrict__ u,
                                        const float* __restrict__ d,
                                        const float* __restrict__ scale, float sigma,
                                        const float* __restrict__ aux, float beta, float ht,
                                        float* __restrict__ out, int t1, const CUtensorMap* umap,
                                        bool use_tma, int bx, int by, int bz,
                                        float* __restrict__ sm, uint64_t* mbar,
                                        uint32_t parity) {
  const int i1_0 = bz * t1, i2_0 = by * TB2, i3_0 = bx * TB3;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N, s1 = (int64_t)g.n2 * g.n3;
  const int64_t idx0 = active ? lin(g, i1_0, i2, i3) : 0;
  if (use_tma) issue_brick_tma(umap, 0, g, i1_0, i2_0, i3_0, sm, t1, mbar);
  // departure points of the next node are loaded one node ahead (the first
  // ones while the brick is being staged)
  float dn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dn[a] = active ? d[a * N + idx0] : 0.f;
  bool ok = true;
  if (use_tma) {
    ok = wait_brick_tma(mbar, parity);
  } else {
    stage_brick(u, g, i1_0, i2_0, i3_0, sm, t1);
    __syncthreads();
  }
  if (!active || !ok) return;
  const int ctr = (HB_LO * BB2 + ty + HB_LO) * BB3 + lane + HB3_LO;
  const int kmax = min(t1, g.n1 - i1_0);
#pragma unroll 2
  for (int k = 0; k < kmax; ++k) {
    const int i1 = i1_0 + k;
    const int64_t idx = idx0 + k * s1;
    // the epilogue operands are requested before the gather, which hides their latency
    const float sc = MODE == 0 && scale ? __ldg(scale + idx) : sigma;
    const float ax = MODE == 0 && aux ? __ldg(aux + idx) : 0.0f;
    NodeTaps t;
    node_taps(dn[0], dn[1], dn[2], t);
    if (k + 1 < kmax) {
#pragma unroll
      for (int a = 0; a < 3; ++a) dn[a] = d[a * N + idx + s1];
    }
    const float y = taps_in_brick(t) ? gather_brick(sm, t, k, ty, lane)
                                     : gather_global(u, g, t, i1, i2, i3);
    float r;
    if (MODE == 1) {
      const float x = sm[ctr + k * BB2 * BB3];
      r = 1.0f + 0.5f * ht * (y + x + ht * x * y);
    } else {
      r = y * sc;
      if (aux) r = fmaf(beta, ax, r);
    }
    out[idx] = r;
  }
}

// One CTA per tile.  With tma != 0 the interior bricks are staged by TMA.
template <int MODE>
__global__ void __launch_bounds__(BRICK_THREADS, 4) k_sl(Grid g, const float* __restrict__ u,
                                                      const float* __restrict__ d,
                                                      const float* __restrict__ scale,
                                                      float sigma,
                                                      const float* __restrict__ aux, float beta,
                                                      float ht, float* __restrict__ out,
                                                      int t1,
                                                      const __grid_constant__ CUtensorMap umap,
                                                      int tma) {
  extern __shared__ __align__(128) float smb[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smb + brick_floats(t1));
  const bool use_tma =
      tma && brick_tma_ok(g, blockIdx.z * t1, blockIdx.y * TB2, blockIdx.x * TB3, t1);
  if (use_tma) {
    brick_mbar_init(mbar);
    __syncthreads();
  }
  sl_tile<MODE>(g, u, d, scale, sigma, aux, beta, ht, out, t1, &umap, use_tma, blockIdx.x,
                blockIdx.y, blockIdx.z, smb, mbar, 0u);
}

// ------------------------------------------------------- grouped launches

// Persistent kernels of a grouped batch: one launch covers the tiles of up to
// GROUP_MAX ops (pairs).  The work queue is the concatenation of the ops'
// tiles (op o owns items first[o] .. first[o + 1] - 1, in the tile order of its
// single launch); CTA b takes items b, b + gridDim.x, ...  Each item is the
// tile function of the single launch, so every tile computes what that launch
// computes.  Parameters, TMA descriptors included, travel by value in the
// launch (__grid_constant__).
constexpr int GROUP_MAX = 32;

struct SlGroupOp {
  Grid g;
  const float* u; const float* d; const float* scale; const float* aux;
  float* out;
  float sigma, beta, ht;
  int t1, tma, tx, ty;              // tiles along x3, x2
};
struct alignas(64) SlGroup {
  CUtensorMap map[GROUP_MAX];
  SlGroupOp op[GROUP_MAX];
  int first[GROUP_MAX + 1];
  int nops, t1max;
};
struct TraceGroupOp {
  Grid g;
  const float* v; float* df; float* db;
  float ht;
  int t1, tma, tx, ty;
};
struct alignas(64) TraceGroup {
  CUtensorMap map[GROUP_MAX];
  TraceGroupOp op[GROUP_MAX];
  int first[GROUP_MAX + 1];
  int nops, t1max;
};
struct MarchGroup {
  MarchOpArgs op[GROUP_MAX];
  int tx[GROUP_MAX], ty[GROUP_MAX];
  int first[GROUP_MAX + 1];
  int nops;
};

// The op owning `item`: the largest o with first[o] <= item.
__device__ __forceinline__ int group_op_of(const int* first, int nops, int item) {
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int MODE>
__global__ void __launch_bounds__(BRICK_THREADS, 4) k_sl_group(const __grid_constant__ SlGroup G) {
  extern __shared__ __align__(128) float smb[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smb + brick_floats(G.t1max));
  brick_mbar_init(mbar);
  __syncthreads();
  uint32_t parity = 0;
  const int total = G.first[G.nops];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int o = group_op_of(G.first, G.nops, item);
    const SlGroupOp& op = G.op[o];
    const int tile = item - G.first[o], r = tile / op.tx;
    const int bx = tile - r * op.tx, bz = r / op.ty, by = r - bz * op.ty;
    const bool use_tma = op.tma && brick_tma_ok(op.g, bz * op.t1, by * TB2, bx * TB3, op.t1);
    sl_tile<MODE>(op.g, op.u, op.d, op.scale, op.sigma, op.aux, op.beta, op.ht, op.out, op.t1,
                  &G.map[o], use_tma, bx, by, bz, smb, mbar, parity);
    parity ^= use_tma ? 1u : 0u;
    __syncthreads();                              // brick consumed before the next item
  }
}

__global__ void __launch_bounds__(BRICK_THREADS) k_trace_group(const __grid_constant__ TraceGroup G) {
  extern __shared__ __align__(128) float smb[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smb + brick_floats(G.t1max));
  brick_mbar_init(mbar);
  __syncthreads();
  uint32_t parity = 0;
  const int total = G.first[G.nops];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int o = group_op_of(G.first, G.nops, item);
    const TraceGroupOp& op = G.op[o];
    const int tile = item - G.first[o], r = tile / op.tx;
    const int bx = tile - r * op.tx, bz = r / op.ty, by = r - bz * op.ty;
    const bool use_tma = op.tma && brick_tma_ok(op.g, bz * op.t1, by * TB2, bx * TB3, op.t1);
    trace_tile(op.g, op.v, op.df, op.db, op.ht, op.t1, &G.map[o], use_tma, bx, by, bz, smb,
               mbar, parity);
    parity ^= use_tma ? 1u : 0u;                  // three phases: p, p ^ 1, p
    __syncthreads();                              // brick consumed before the next item
  }
}

template <int MODE, int NF>
__global__ void __launch_bounds__(32 * MT2, NF <= 5 ? 2 : 1)
k_march_group(const __grid_constant__ MarchGroup G) {
  __shared__ MarchSmem<NF, float> S;
  const int total = G.first[G.nops];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int o = group_op_of(G.first, G.nops, item);
    const MarchOpArgs& op = G.op[o];
    const int tx = G.tx[o], ty = G.ty[o];
    const int tile = item - G.first[o], r = tile / tx;
    const int bx = tile - r * tx, bz = r / ty, by = r - bz * ty;
    march_tile<MODE, NF, float>(op.g, op.mhist, op.lhist, op.vt, op.scale0, op.vmax, op.base,
                                op.base_coef, op.umul, op.out, op.hout, op.dotv, op.partial,
                                op.mt1, bx, by, bz, tx, ty, S);
  }
}

// ------------------------------------------------- SL step, x1 register window

// The same SL step as k_sl with the register-window gather of sl_window.cuh:
// the departure points and the epilogue operands of the tile are staged as
// dense tiles beside the brick; each lane contracts the nodes that share its
// reference floor from four x1 planes held in registers (one new plane of 16
// shared loads per node instead of 64) and the rest are gathered from the
// brick by the whole CTA afterwards.  Bitwise the same results as k_sl.
template <int MODE>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_slw(Grid g, const float* __restrict__ u,
                                                    const float* __restrict__ d,
                                                    const float* __restrict__ scale,
                                                    float sigma,
                                                    const float* __restrict__ aux, float beta,
                                                    float ht, float* __restrict__ out,
                                                    int t1) {
  extern __shared__ __align__(16) float sm[];
  float* td = sm + brick_floats(t1);                       // [3][t1][TB2][TB3]
  float* tsc = td + 3 * tile_elems(t1);                    // scale tile (if any)
  float* tax = tsc + (scale ? tile_elems(t1) : 0);         // aux tile (if any)
  int* queue = reinterpret_cast<int*>(tax + (aux ? tile_elems(t1) : 0));
  int* qcount = queue + tile_elems(t1);
  const int i1_0 = blockIdx.z * t1, i2_0 = blockIdx.y * TB2, i3_0 = blockIdx.x * TB3;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const bool active = i2_0 + ty < g.n2 && i3_0 + lane < g.n3;
  const int kmax = min(t1, g.n1 - i1_0);
  if (ty == 0 && lane == 0) *qcount = 0;
  stage_tile(d, g.N, 3, g, i1_0, i2_0, i3_0, t1, td);
  if (MODE == 0 && scale) stage_tile(scale, g.N, 1, g, i1_0, i2_0, i3_0, t1, tsc);
  if (MODE == 0 && aux) stage_tile(aux, g.N, 1, g, i1_0, i2_0, i3_0, t1, tax);
  stage_brick(u, g, i1_0, i2_0, i3_0, sm, t1);
  __syncthreads();
  auto disp = [&](int k, int y, int l, float dd[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) dd[a] = td[tile_at(t1, a, k, y, l)];
  };
  auto epi = [&](int k, int y, int l, float val) {
    const int at = tile_at(t1, 0, k, y, l);
    float r;
    if (MODE == 1) {
      const float x = sm[((k + HB_LO) * BB2 + y + HB_LO) * BB3 + l + HB3_LO];
      r = 1.0f + 0.5f * ht * (val + x + ht * x * val);
    } else {
      r = val * (scale ? tsc[at] : sigma);
      if (aux) r = fmaf(beta, tax[at], r);
    }
    out[lin(g, i1_0 + k, i2_0 + y, i3_0 + l)] = r;
  };
  int r1 = 0, r2 = 0, r3 = 0;
  if (active) {
    float dr[3];
    disp(min(t1 / 2, kmax - 1), ty, lane, dr);
    window_reference(dr[0], dr[1], dr[2], r1, r2, r3);
  }
  window_march(sm, kmax, ty, lane, active, r1, r2, r3, disp, epi, queue, qcount);
  __syncthreads();
  window_deferred(sm, i1_0, i2_0, i3_0, *qcount, queue, disp, epi,
                  [&](const NodeTaps& t, int i1, int i2, int i3) {
                    return gather_global(u, g, t, i1, i2, i3);
                  });
}

// RK2 departure points of both directions (Sec. 2.5.2), register-window form
// of k_trace: v of the tile is staged once as a dense tile; each velocity
// component is staged once as a brick and gathered for both directions.
__global__ void __launch_bounds__(WIN_THREADS, 2) k_tracew(Grid g, const float* __restrict__ v,
                                                       float* __restrict__ df,
                                                       float* __restrict__ db, float ht,
                                                       int t1) {
  extern __shared__ __align__(16) float sm[];
  float* tv = sm + brick_floats(t1);                       // [3][t1][TB2][TB3]
  int* queue = reinterpret_cast<int*>(tv + 3 * tile_elems(t1));
  int* qcount = queue + tile_elems(t1);                    // two counters, by pass parity
  const int i1_0 = blockIdx.z * t1, i2_0 = blockIdx.y * TB2, i3_0 = blockIdx.x * TB3;
  const int64_t N = g.N;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const bool active = i2_0 + ty < g.n2 && i3_0 + lane < g.n3;
  const int kmax = min(t1, g.n1 - i1_0);
  if (ty == 0 && lane == 0) qcount[0] = qcount[1] = 0;
  stage_tile(v, N, 3, g, i1_0, i2_0, i3_0, t1, tv);
  const float ih[3] = {g.inv_h1, g.inv_h2, g.inv_h3};
  int pass = 0;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    if (c > 0) __syncthreads();                  // previous brick consumed
    stage_brick(v + c * N, g, i1_0, i2_0, i3_0, sm, t1);
    __syncthreads();
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      float* out = dir == 0 ? df : db;
      if (out == nullptr) continue;
      const float sg = dir == 0 ? -ht : ht;      // transport along +v / -v
      int* qc = qcount + (pass & 1);
      auto disp = [&](int k, int y, int l, float dd[3]) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dd[a] = sg * (tv[tile_at(t1, a, k, y, l)] * ih[a]);
      };
      const float ihc = c == 0 ? g.inv_h1 : (c == 1 ? g.inv_h2 : g.inv_h3);
      auto epi = [&](int k, int y, int l, float w) {
        const float uc = tv[tile_at(t1, c, k, y, l)] * ihc;
        out[c * N + lin(g, i1_0 + k, i2_0 + y, i3_0 + l)] = 0.5f * sg * (uc + w * ihc);
      };
      int r1 = 0, r2 = 0, r3 = 0;
      if (active) {
        float dr[3];
        disp(min(t1 / 2, kmax - 1), ty, lane, dr);
        window_reference(dr[0], dr[1], dr[2], r1, r2, r3);
      }
      window_march(sm, kmax, ty, lane, active, r1, r2, r3, disp, epi, queue, qc);
      __syncthreads();
      const int nq = *qc;
      if (ty == 0 && lane == 0) qcount[(pass + 1) & 1] = 0;   // the next pass's counter
      window_deferred(sm, i1_0, i2_0, i3_0, nq, queue, disp, epi,
                      [&](const NodeTaps& t, int i1, int i2, int i3) {
                        return gather_global(v + c * N, g, t, i1, i2, i3);
                      });
      __syncthreads();                           // queue consumed before the next pass
      ++pass;
    }
  }
}

// Nodes whose departure point d (grid units) puts a tap outside the staged brick,
// i.e. the nodes an SL step with these departure points interpolates with the
// global-memory gather (the predicate of k_sl); block counts added into *out.
__global__ void __launch_bounds__(256) k_count_far(int64_t N, const float* __restrict__ d,
                                                   unsigned long long* __restrict__ out) {
  unsigned cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    NodeTaps t;
    node_taps(d[i], d[N + i], d[2 * N + i], t);
    cnt += !taps_in_brick(t);
  }
  __shared__ unsigned warp_cnt[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < 8; ++w) b += warp_cnt[w];
    if (b) atomicAdd(out, b);
  }
}

// ---------------------------------------------------------------- FD8

__global__ void __launch_bounds__(256) k_grad8(Grid g, const float* __restrict__ u,
                                               float* __restrict__ gu) {
  CLAIRE_KERNEL_INDEX
  float gr[3];
  grad8_at(u, g, i1, i2, i3, gr);
  gu[idx] = gr[0];
  gu[g.N + idx] = gr[1];
  gu[2 * g.N + idx] = gr[2];
}

// FD8 derivative along `axis` of the product lam * u at node (i1, i2, i3).
__device__ __forceinline__ float d8_axis_prod(const float* __restrict__ lam,
                                              const float* __restrict__ u, const Grid& g, int i1,
                                              int i2, int i3, int axis) {
  int64_t base, stride;
  int i, n;
  float ih;
  if (axis == 0) {
    base = (int64_t)i2 * g.n3 + i3; stride = (int64_t)g.n2 * g.n3; i = i1; n = g.n1; ih = g.inv_h1;
  } else if (axis == 1) {
    base = (int64_t)i1 * g.n2 * g.n3 + i3; stride = g.n3; i = i2; n = g.n2; ih = g.inv_h2;
  } else {
    base = ((int64_t)i1 * g.n2 + i2) * g.n3; stride = 1; i = i3; n = g.n3; ih = g.inv_h3;
  }
  float m[4], p[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t a = base + wrap_near(i - 1 - k, n) * stride;
    const int64_t b = base + wrap_near(i + 1 + k, n) * stride;
    m[k] = __ldg(lam + a) * __ldg(u + a);
    p[k] = __ldg(lam + b) * __ldg(u + b);
  }
  return fd8(m[3], m[2], m[1], m[0], p[0], p[1], p[2], p[3], ih);
}

// q = div8(lam w): the full-Newton source of the incremental adjoint (eq. incadj).
__global__ void __launch_bounds__(256) k_div8_prod(Grid g, const float* __restrict__ lam,
                                                   const float* __restrict__ w,
                                                   float* __restrict__ out) {
  CLAIRE_KERNEL_INDEX
  out[idx] = d8_axis_prod(lam, w, g, i1, i2, i3, 0) +
             d8_axis_prod(lam, w + g.N, g, i1, i2, i3, 1) +
             d8_axis_prod(lam, w + 2 * g.N, g, i1, i2, i3, 2);
}


// div8(w) marching along x1 (the layout of the FD8 history kernels): a CTA owns
// an MT2 x MT3 (x2 x x3) tile and mt1 planes.  w1 goes through a 9-deep
// register queue (the x1 derivative: each value read once), the planes of w2
// and w3 with their 4-node halo are copied with cp.async into shared memory one
// plane ahead (the x2 and x3 derivatives).  Per node: fd8() along each axis,
// summed x1 + x2 + x3, with the x1 neighbours taken from registers instead of
// eight plane reads per node.
__global__ void __launch_bounds__(32 * MT2) k_div8_march(Grid g, const float* __restrict__ w,
                                                         float* __restrict__ out, int mt1) {
  __shared__ __align__(16) float sp[2][2][MPLANE];           // [buffer][w2, w3]
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i3_0 = blockIdx.x * MT3, i2_0 = blockIdx.y * MT2, i1_0 = blockIdx.z * mt1;
  const int i2 = i2_0 + ty, i3 = i3_0 + lane;
  const bool active = i2 < g.n2 && i3 < g.n3;
  const int64_t N = g.N, s1 = (int64_t)g.n2 * g.n3;
  const int64_t col = active ? (int64_t)i2 * g.n3 + i3 : 0;
  const float* w1 = w;
  const float* w2 = w + N;
  const float* w3 = w + 2 * N;
  float q[9];                                                  // w1(i1 - 4 + k)
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = active ? w1[wrap_any(i1_0 - 4 + k, g.n1) * s1 + col] : 0.f;
  const int i1_end = min(i1_0 + mt1, g.n1);
  const PlaneChunk ch = plane_chunk(g, i2_0, i3_0);
  const bool vec = (g.n3 % 4 == 0) && ((reinterpret_cast<uintptr_t>(w) & 15) == 0);
  stage_plane_async(w2, g, i1_0, i2_0, i3_0, ch, vec, sp[0][0]);
  stage_plane_async(w3, g, i1_0, i2_0, i3_0, ch, vec, sp[0][1]);
  cp_async_commit();
  float hn = active ? w1[wrap_near(i1_0 + 4, g.n1) * s1 + col] : 0.f;
  const int c = (ty + 4) * MP3 + lane + 4;                     // node in the staged plane
  for (int i1 = i1_0; i1 < i1_end; ++i1) {
    const int cur = (i1 - i1_0) & 1;
    q[8] = hn;
    if (i1 + 1 < i1_end) {
      stage_plane_async(w2, g, i1 + 1, i2_0, i3_0, ch, vec, sp[cur ^ 1][0]);
      stage_plane_async(w3, g, i1 + 1, i2_0, i3_0, ch, vec, sp[cur ^ 1][1]);
      if (active) hn = w1[wrap_near(i1 + 5, g.n1) * s1 + col];
    }
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();                                           // plane i1 staged by all
    if (active) {
      const float* p2 = sp[cur][0];
      const float* p3 = sp[cur][1];
      const float gx = fd8(q[0], q[1], q[2], q[3], q[5], q[6], q[7], q[8], g.inv_h1);
      const float gy = fd8(p2[c - 4 * MP3], p2[c - 3 * MP3], p2[c - 2 * MP3], p2[c - MP3],
                           p2[c + MP3], p2[c + 2 * MP3], p2[c + 3 * MP3], p2[c + 4 * MP3],
                           g.inv_h2);
      const float gz = fd8(p3[c - 4], p3[c - 3], p3[c - 2], p3[c - 1], p3[c + 1], p3[c + 2],
                           p3[c + 3], p3[c + 4], g.inv_h3);
      out[(int64_t)i1 * s1 + col] = gx + gy + gz;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    __syncthreads();                                           // buffer cur consumed
  }
}

// s^j = grad8(m^j) . vt for j = 0..nt (m^j = mhist + j N); s^0 is scaled by scale0.
__global__ void __launch_bounds__(256) k_sdot_hist(Grid g, const float* __restrict__ mhist,
                                                   int nt, const float* __restrict__ vt,
                                                   float scale0, float* __restrict__ shist) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  const float t1 = vt[idx], t2 = vt[N + idx], t3 = vt[2 * N + idx];
  for (int j = 0; j <= nt; ++j) {
    float gr[3];
    grad8_at(mhist + j * N, g, i1, i2, i3, gr);
    float s = gr[0] * t1;
    s = fmaf(gr[1], t2, s);
    s = fmaf(gr[2], t3, s);
    shist[j * N + idx] = j == 0 ? scale0 * s : s;
  }
}

// out = base_coef * base + sum_{j=0..nt} w_j lam^j grad8(m^j), trapezoid weights
// w_j = h_t (1/2, 1, ..., 1, 1/2)  (Sec. 2.5.1).  base may be NULL.
__global__ void __launch_bounds__(256) k_accum_hist(Grid g, const float* __restrict__ lhist,
                                                    const float* __restrict__ mhist, int nt,
                                                    const float* __restrict__ base,
                                                    float base_coef, float* __restrict__ out) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  const float ht = 1.0f / nt;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int j = 0; j <= nt; ++j) {
    float gr[3];
    grad8_at(mhist + j * N, g, i1, i2, i3, gr);
    const float wl = ((j == 0 || j == nt) ? 0.5f * ht : ht) * lhist[j * N + idx];
    acc0 = fmaf(wl, gr[0], acc0);
    acc1 = fmaf(wl, gr[1], acc1);
    acc2 = fmaf(wl, gr[2], acc2);
  }
  if (base) {
    acc0 = fmaf(base_coef, base[idx], acc0);
    acc1 = fmaf(base_coef, base[N + idx], acc1);
    acc2 = fmaf(base_coef, base[2 * N + idx], acc2);
  }
  out[idx] = acc0;
  out[N + idx] = acc1;
  out[2 * N + idx] = acc2;
}

// ---------------------------------------------------------------- spectral

// Half spectrum [n1][n2][n3/2+1] of 3 components (stride Nc).  Integer
// wavenumbers k_i in FFT order; scale folds in cuFFT's 1/N.
// Optional fused outputs: partial[blockIdx.x] = this block's share of the real
// inner product <in, out> by Parseval over the half spectrum (weight 2 for the
// modes whose conjugates are not stored); means[0..2] = the k = 0 coefficient
// of each component / N, i.e. the component means of the input field.
__global__ void __launch_bounds__(256) k_spectral(int n1, int n2, int n3, int64_t Nc,
                                                  cufftComplex* __restrict__ X, int op,
                                                  float alpha, float gamma, float beta_w,
                                                  float scale, double* __restrict__ partial,
                                                  double* __restrict__ means) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dot = 0.0;
  if (i < Nc) {
    // Nc < 2^31 (3 N < 2^31): 32-bit index math
    const unsigned nh = (unsigned)(n3 / 2 + 1), u = (unsigned)i;
    const unsigned q = u / nh;
    const int j3 = (int)(u - q * nh);
    const int j1 = (int)(q / (unsigned)n2);
    const int j2 = (int)(q - (unsigned)j1 * (unsigned)n2);
    const float k1 = (float)(j1 <= n1 / 2 ? j1 : j1 - n1);
    const float k2 = (float)(j2 <= n2 / 2 ? j2 : j2 - n2);
    const float k3 = (float)j3;
    const float kap = k1 * k1 + k2 * k2 + k3 * k3;
    const cufftComplex x0 = X[i], x1 = X[Nc + i], x2 = X[2 * Nc + i];
    cufftComplex y0, y1, y2;
    if (op == 0 || op == 1 || op == 4) {
      float sig = gamma == 1.0f ? kap : powf(kap, gamma);
      float f;
      if (op == 0) {
        f = sig * scale;                                  // L = (-Laplacian)^gamma
      } else {
        if (kap == 0.0f) sig = 1.0f;                      // zero symbol set to one
        f = op == 1 ? scale / (alpha * sig)               // (alpha L)^-1
                    : scale * rsqrtf(alpha * sig);        // (alpha L)^-1/2
      }
      y0 = make_cuComplex(x0.x * f, x0.y * f);
      y1 = make_cuComplex(x1.x * f, x1.y * f);
      y2 = make_cuComplex(x2.x * f, x2.y * f);
    } else {
      // P_par = k k^T / |k|^2 with Nyquist components of k zeroed (real result)
      const float q1 = (j1 == n1 / 2) ? 0.f : k1;
      const float q2 = (j2 == n2 / 2) ? 0.f : k2;
      const float q3 = (j3 == n3 / 2) ? 0.f : k3;
      const float qq = q1 * q1 + q2 * q2 + q3 * q3;
      float f = 0.0f;
      if (qq > 0.0f) {
        f = scale / qq;
        if (op == 3) {
          const float num = beta_w * (1.0f + kap);
          f *= num / (num + alpha * kap);
        }
      }
      const float re = (q1 * x0.x + q2 * x1.x + q3 * x2.x) * f;
      const float im = (q1 * x0.y + q2 * x1.y + q3 * x2.y) * f;
      y0 = make_cuComplex(q1 * re, q1 * im);
      y1 = make_cuComplex(q2 * re, q2 * im);
      y2 = make_cuComplex(q3 * re, q3 * im);
    }
    if (partial) {
      const float w = (j3 == 0 || 2 * j3 == n3) ? 1.0f : 2.0f;
      dot = (double)(w * (x0.x * y0.x + x0.y * y0.y + x1.x * y1.x + x1.y * y1.y +
                          x2.x * y2.x + x2.y * y2.y));
    }
    if (means && i == 0) {
      means[0] = (double)x0.x * (double)scale;
      means[1] = (double)x1.x * (double)scale;
      means[2] = (double)x2.x * (double)scale;
    }
    X[i] = y0; X[Nc + i] = y1; X[2 * Nc + i] = y2;
  }
  if (partial) {
    const double b = block_sum(dot);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
  }
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Each thread folds 4 elements (one float4 per operand) in FP32, then adds the
// chunk to an FP64 accumulator: FP64 work is 1/4 per element (B300's FP64 rate
// is low) while the rounding stays at FP32 level per chunk of 4.
__device__ __forceinline__ float red_term(int mode, float x, float y) {
  switch (mode) {
    case 0: return x * y;
    case 1: { const float d = x - y; return d * d; }
    case 2: return fabsf(x);
    case 3: return x * x;
    default: return x;
  }
}

__device__ __forceinline__ float red_chunk(int mode, float a, float b, float c, float d) {
  if (mode == 2 || mode == 4) return fmaxf(fmaxf(a, b), fmaxf(c, d));
  if (mode == 5) return fminf(fminf(a, b), fminf(c, d));
  return (a + b) + (c + d);
}

__global__ void __launch_bounds__(256) k_reduce(int64_t n, const float* __restrict__ a,
                                                const float* __restrict__ b, int mode,
                                                double* __restrict__ partial) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  const int64_t n4 = vec ? n / 4 : 0;
  const bool extremum = mode == 2 || mode == 4 || mode == 5;
  // max / min are exact in FP32; NaNs are tracked separately (fmaxf drops them)
  float ext = mode == 5 ? CUDART_INF_F : (mode == 4 ? -CUDART_INF_F : 0.0f);
  bool nan = false;
  KahanF sum;
  // unrolled so that several 16-byte loads per thread are in flight (the compensated
  // sum stays one sequential chain, in the same order)
#pragma unroll 4
  for (int64_t i = t0; i < n4; i += stride) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a) + i);
    const float4 y = b ? __ldg(reinterpret_cast<const float4*>(b) + i) : x;
    const float c = red_chunk(mode, red_term(mode, x.x, y.x), red_term(mode, x.y, y.y),
                              red_term(mode, x.z, y.z), red_term(mode, x.w, y.w));
    if (extremum) {
      nan |= (x.x != x.x) | (x.y != x.y) | (x.z != x.z) | (x.w != x.w);
      ext = mode == 5 ? fminf(ext, c) : fmaxf(ext, c);
    } else {
      sum.add(c);
    }
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    const float x = a[i], y = b ? b[i] : x;
    const float c = red_term(mode, x, y);
    if (extremum) {
      nan |= (x != x);
      ext = mode == 5 ? fminf(ext, c) : fmaxf(ext, c);
    } else {
      sum.add(c);
    }
  }
  double acc = extremum ? (nan ? CUDART_NAN : (double)ext) : sum.value();
  const double v = block_red(mode, acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// ---------------------------------------------------------------- PCG vectors

// Algorithm 2 update with device-side scalars: kappa = <r,z> / <s,Hs>;
// vt += kappa s, r -= kappa Hs, partial ||r||^2.  <s, Hs> <= 0 (negative
// curvature, Sec. 2.5.5) or a non-finite scalar leaves vt and r untouched and
// raises *flag.
__global__ void __launch_bounds__(256) k_pcg_update(int64_t n4, const double* __restrict__ rz,
                                                    const double* __restrict__ sHs,
                                                    float4* __restrict__ vt,
                                                    float4* __restrict__ r,
                                                    const float4* __restrict__ s,
                                                    const float4* __restrict__ Hs,
                                                    double* __restrict__ partial,
                                                    int* __restrict__ flag) {
  const double q = *sHs, p = *rz;
  const bool ok = q > 0.0 && isfinite(q) && isfinite(p);
  const float kappa = ok ? (float)(p / q) : 0.0f;
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) *flag = 1;
  KahanF acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 rv = r[i];
    if (ok) {
      const float4 sv = s[i], hv = Hs[i];
      float4 v = vt[i];
      v.x = fmaf(kappa, sv.x, v.x); v.y = fmaf(kappa, sv.y, v.y);
      v.z = fmaf(kappa, sv.z, v.z); v.w = fmaf(kappa, sv.w, v.w);
      vt[i] = v;
      rv.x = fmaf(-kappa, hv.x, rv.x); rv.y = fmaf(-kappa, hv.y, rv.y);
      rv.z = fmaf(-kappa, hv.z, rv.z); rv.w = fmaf(-kappa, hv.w, rv.w);
      r[i] = rv;
    }
    acc.add((rv.x * rv.x + rv.y * rv.y) + (rv.z * rv.z + rv.w * rv.w));
  }
  const double b = block_sum(acc.value());
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// mu = rz_new / rz_old (0 on the first iteration): s = z + mu s and the
// regularisation part of H s by recurrence, hs = (r - mean(r)) + mu hs, since
// beta_v L z = r - mean(r) for z = (beta_v L)^-1 r with the zero symbol set to one.
__global__ void __launch_bounds__(256) k_s_update(int64_t n4, int64_t N4,
                                                  const double* __restrict__ rz_new,
                                                  const double* __restrict__ rz_old,
                                                  const double* __restrict__ means, int first,
                                                  const float4* __restrict__ z,
                                                  const float4* __restrict__ r,
                                                  float4* __restrict__ s,
                                                  float4* __restrict__ hs) {
  const float mu = first ? 0.0f : (float)(*rz_new / *rz_old);
  const float m[3] = {(float)means[0], (float)means[1], (float)means[2]};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float mc = m[i / N4];
    const float4 zv = z[i], rv = r[i];
    float4 sv = first ? make_float4(0.f, 0.f, 0.f, 0.f) : s[i];
    float4 hv = first ? make_float4(0.f, 0.f, 0.f, 0.f) : hs[i];
    sv.x = fmaf(mu, sv.x, zv.x); sv.y = fmaf(mu, sv.y, zv.y);
    sv.z = fmaf(mu, sv.z, zv.z); sv.w = fmaf(mu, sv.w, zv.w);
    hv.x = fmaf(mu, hv.x, rv.x - mc); hv.y = fmaf(mu, hv.y, rv.y - mc);
    hv.z = fmaf(mu, hv.z, rv.z - mc); hv.w = fmaf(mu, hv.w, rv.w - mc);
    s[i] = sv;
    hs[i] = hv;
  }
}

__global__ void k_reduce_final(const double* __restrict__ partial, int nb, int mode,
                               double* __restrict__ out) {
  double acc = red_init(mode);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc = red_combine(mode, acc, partial[i]);
  const double v = block_red(mode, acc);
  if (threadIdx.x == 0) *out = v;
}

// ---------------------------------------------------------------- vectors

__global__ void k_axpby(int64_t n, float a, const float* __restrict__ x, float b,
                        float* __restrict__ y) {   // y = a x + b y
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], b * y[i]);
}

// NCC final condition of the incremental adjoint (Appendix): on entry lt = -m~(1),
// sx = sum m1 lt and sy = sum m(1) lt (device FP64); with the L2 inner products
// a = <m1, m(1)>, b = ||m1||^2, c = ||m(1)||^2 (h3 = cell volume):
//   lt = (2/b)(q1 m1 + q2 m(1) - q3 m~(1)),  al = <m1, m~>, ga = <m(1), m~>,
//   q1 = al/c - 2 a ga/c^2,  q2 = 4 a^2 ga/c^3 - 2 a al/c^2,  q3 = a^2/c^2.
__global__ void k_ncc_final(int64_t n, const float* __restrict__ m1, const float* __restrict__ m,
                            float* __restrict__ lt, const double* __restrict__ sx,
                            const double* __restrict__ sy, double a, double b, double c,
                            double h3) {
  const double al = -h3 * *sx, ga = -h3 * *sy;
  const float q1 = (float)(al / c - 2.0 * a * ga / (c * c));
  const float q2 = (float)(4.0 * a * a * ga / (c * c * c) - 2.0 * a * al / (c * c));
  const float q3 = (float)(a * a / (c * c));
  const float f = (float)(2.0 / b);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float mt = -lt[i];
    lt[i] = f * (fmaf(q1, m1[i], q2 * m[i]) - q3 * mt);
  }
}

__global__ void k_affine(int64_t n, float a, const float* __restrict__ x, float b,
                         float* __restrict__ out) {                               // out = a x + b
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fmaf(a, x[i], b);
}

__global__ void k_lincomb(int64_t n, float a, const float* __restrict__ x, float b,
                          const float* __restrict__ y, float* __restrict__ out) {  // out = a x + b y
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fmaf(a, x[i], b * y[i]);
}

// ---------------------------------------------------------------- det F1

// One RK2 SL step of d_t F = (grad v) F along +v (Appendix, eq. def-grad):
// f0 = A(y) F(y), F~ = F(y) + h_t f0, f1 = A(x) F~, F' = F(y) + (h_t/2)(f0 + f1).
// F, A, Ay hold 9 fields [3a + b][N]; det (optional) receives det F'.
__global__ void __launch_bounds__(256) k_detf_step(Grid g, const float* __restrict__ F,
                                                   const float* __restrict__ df,
                                                   const float* __restrict__ A,
                                                   const float* __restrict__ Ay, float ht,
                                                   float* __restrict__ Fn,
                                                   float* __restrict__ det) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
  Taps a, b, c;
  axis_taps(i1, df[idx], g.n1, g.n2 * g.n3, a);
  axis_taps(i2, df[N + idx], g.n2, g.n3, b);
  axis_taps(i3, df[2 * N + idx], g.n3, 1, c);
  float Fy[9], Ax[9], Ayy[9], f0[9], Ft[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Fy[k] = gather64(F + k * N, a, b, c);
    Ax[k] = A[k * N + idx];
    Ayy[k] = Ay[k * N + idx];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) s = fmaf(Ayy[3 * r + k], Fy[3 * k + q], s);
      f0[3 * r + q] = s;
      Ft[3 * r + q] = fmaf(ht, s, Fy[3 * r + q]);
    }
  float Fo[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float f1 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) f1 = fmaf(Ax[3 * r + k], Ft[3 * k + q], f1);
      Fo[3 * r + q] = fmaf(0.5f * ht, f0[3 * r + q] + f1, Fy[3 * r + q]);
      Fn[(3 * r + q) * N + idx] = Fo[3 * r + q];
    }
  if (det) {
    det[idx] = Fo[0] * (Fo[4] * Fo[8] - Fo[5] * Fo[7]) - Fo[1] * (Fo[3] * Fo[8] - Fo[5] * Fo[6]) +
               Fo[2] * (Fo[3] * Fo[7] - Fo[4] * Fo[6]);
  }
}

// A[3a + b] = d_b v_a (FD8) and its values at the departure points y.
__global__ void __launch_bounds__(256) k_detf_init(Grid g, const float* __restrict__ v,
                                                   float* __restrict__ A,
                                                   float* __restrict__ F) {
  CLAIRE_KERNEL_INDEX
  const int64_t N = g.N;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float gr[3];
    grad8_at(v + r * N, g, i1, i2, i3, gr);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A[(3 * r + q) * N + idx] = gr[q];
      F[(3 * r + q) * N + idx] = r == q ? 1.0f : 0.0f;
    }
  }
}

// ---------------------------------------------------------------- profiler

thread_local Profiler* tl_prof = nullptr;

const char* kernel_kind_name(int k) {
  static const char* names[K_COUNT] = {"trace", "sl_step", "adjoint_factor", "grad8", "div8",
                                       "sdot_hist", "accum_hist", "spectral_diag", "reduce",
                                       "vector", "detf", "cufft", "precond"};
  return (k >= 0 && k < K_COUNT) ? names[k] : "?";
}

void Profiler::reset(bool timing_on) {
  resolve();
  timing = timing_on;
  for (int k = 0; k < K_COUNT; ++k) {
    launches[k] = 0;
    bytes[k] = 0.0;
    ms[k] = 0.0;
    timed[k] = 0;
    timed_bytes[k] = 0.0;
  }
}

cudaEvent_t Profiler::take() {
  if (pool.empty()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}

cudaError_t Profiler::resolve() {
  cudaError_t err = cudaSuccess;
  for (auto& p : pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e == cudaSuccess) {
      ms[p.kind] += t;
      timed[p.kind] += 1;
      timed_bytes[p.kind] += p.bytes;
    } else if (err == cudaSuccess) {
      err = e;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  return err;
}

void Profiler::release() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

ProfileRange::ProfileRange(int k, double b, cudaStream_t s) : kind(k), bytes(b), st(s) {
  Profiler* p = tl_prof;
  if (!p) return;
  p->launches[k] += 1;
  p->bytes[k] += b;
  if (p->timing) {
    a = p->take();
    if (a) cudaEventRecord(a, s);
  }
}

ProfileRange::~ProfileRange() {
  Profiler* p = tl_prof;
  if (!p || !a) return;
  cudaEvent_t b = p->take();
  if (!b) return;
  cudaEventRecord(b, st);
  p->pending.push_back({kind, a, b, bytes});
  if (p->pending.size() > 8192) p->resolve();
}

// ---------------------------------------------------------------- launchers

static int vec_blocks(int64_t n) {
  int sms = device_sm_count();
  if (sms <= 0) sms = 148;
  int64_t want = (n + 255) / 256;
  int64_t cap = (int64_t)sms * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// True while st is being captured into a CUDA graph: captured launches stay
// per pair (they replay inside the pair's graph), everything else of a grouped
// batch is posted to its LaunchGroup.
static bool posts_to_group(cudaStream_t st) {
  if (!tl_group) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

thread_local const Tuning* tl_tune = nullptr;
static int tuned_sl_gather() { return tl_tune ? tl_tune->sl_gather : SL_GATHER_TMA; }
int tuned_sl_t1() { return tl_tune ? tl_tune->sl_t1 : TB1; }
bool tuned_sl_window() { return tuned_sl_gather() == SL_GATHER_WINDOW; }
bool tuned_sl_tma() { return tuned_sl_gather() == SL_GATHER_TMA; }
int tuned_march_t1() { return tl_tune ? tl_tune->march_t1 : MT1; }

unsigned int take_brick_timeouts() {
  unsigned int n = 0;
  const unsigned int zero = 0;
  if (cudaMemcpyFromSymbol(&n, g_brick_timeouts, sizeof n) != cudaSuccess ||
      cudaMemcpyToSymbol(g_brick_timeouts, &zero, sizeof zero) != cudaSuccess)
    return 0;
  return n;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of ncomp consecutive fields of the grid starting at base (FP32, or
// FP16 with half = true), as one n3 x n2 x (ncomp n1) tensor; box = one brick of
// depth t1: BB3 x BB2 x (t1 + 6) FP32 values, or BRICK_H_BOX x BB2 x (t1 + 6)
// halves.  Returns false (the caller stages with cp.async) unless the fields
// meet TMA's rules: base 16-byte aligned, the row pitch a multiple of 16 bytes
// (n3 % 4 == 0 for FP32, n3 % 8 == 0 for FP16), and the grid at least one brick
// wide on every axis.
bool encode_brick_map(CUtensorMap* m, const void* base, bool half, const Grid& g, int ncomp,
                      int t1) {
  std::memset(m, 0, sizeof *m);
  const auto enc = tensor_map_encoder();
  const int esize = half ? 2 : 4;
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (g.n3 * esize) % 16 != 0 ||
      g.n3 < BX3 || g.n2 < BB2 || g.n1 < t1 + HB_LO + HB_HI)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.n3, (cuuint64_t)g.n2, (cuuint64_t)ncomp * g.n1};
  const cuuint64_t strides[2] = {(cuuint64_t)g.n3 * esize, (cuuint64_t)g.n2 * g.n3 * esize};
  const cuuint32_t box[3] = {(cuuint32_t)(half ? BRICK_H_BOX : BB3), (cuuint32_t)BB2,
                             (cuuint32_t)(t1 + HB_LO + HB_HI)};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(m, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
static bool brick_map(const float* base, const Grid& g, int ncomp, int t1, CUtensorMap* m) {
  return encode_brick_map(m, base, false, g, ncomp, t1);
}

// dynamic shared memory of k_sl / k_trace: the brick and its mbarrier
static size_t brick_smem_bytes(int t1) {
  return (size_t)brick_floats(t1) * sizeof(float) + 16;
}

static void brick_attributes() {
  static std::once_flag once[kSetupDevices];
  once_per_device(once, [] {
    const int mx = (int)brick_smem_bytes(16);
    cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_sl<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_sl<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_sl_group<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_sl_group<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_trace_group, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    const int mw = window_smem_bytes(16, 5, 0);
    cudaFuncSetAttribute(k_tracew, cudaFuncAttributeMaxDynamicSharedMemorySize, mw);
    cudaFuncSetAttribute(k_slw<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mw);
    cudaFuncSetAttribute(k_slw<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mw);
  });
}
void launch_trace(const Grid& g, const float* v, float* df, float* db, float ht,
                  cudaStream_t st) {
  brick_attributes();
  const int t1 = tuned_sl_t1();
  if (!tuned_sl_window() && posts_to_group(st)) {
    GroupOp op{};
    op.kind = GOP_TRACE;
    op.tr = TraceOpArgs{g, v, df, db, ht, t1, tuned_sl_tma() ? 1 : 0};
    group_post(op, st);
    return;
  }
  ProfileRange pr(K_TRACE, (double)g.N * (12 + 12 * ((df != nullptr) + (db != nullptr))), st);
  if (tuned_sl_window()) {
    k_tracew<<<brick_grid(g, t1), dim3(32, TB2), window_smem_bytes(t1, 3, 0), st>>>(
        g, v, df, db, ht, t1);
  } else {
    CUtensorMap m;
    const int tma = tuned_sl_tma() && brick_map(v, g, 3, t1, &m);
    k_trace<<<brick_grid(g, t1), dim3(32, TB2), brick_smem_bytes(t1), st>>>(g, v, df, db, ht,
                                                                            t1, m, tma);
  }
}
void launch_sl(const Grid& g, const float* u, const float* d, const float* scale, float sigma,
               const float* aux, float beta, float* out, cudaStream_t st) {
  if (!tuned_sl_window() && posts_to_group(st)) {
    GroupOp op{};
    op.kind = GOP_SL0;
    op.sl = SlOpArgs{g, u, d, scale, aux, out, sigma, beta, 0.f, tuned_sl_t1(),
                     tuned_sl_tma() ? 1 : 0};
    group_post(op, st);
    return;
  }
  ProfileRange pr(K_SL, (double)g.N * (20 + 4 * (scale != nullptr) + 4 * (aux != nullptr)), st);
  brick_attributes();
  const int t1 = tuned_sl_t1();
  if (tuned_sl_window()) {
    k_slw<0><<<brick_grid(g, t1), dim3(32, TB2),
               window_smem_bytes(t1, 3 + (scale != nullptr) + (aux != nullptr), 0), st>>>(
        g, u, d, scale, sigma, aux, beta, 0.f, out, t1);
  } else {
    CUtensorMap m;
    const int tma = tuned_sl_tma() && brick_map(u, g, 1, t1, &m);
    k_sl<0><<<brick_grid(g, t1), dim3(32, TB2), brick_smem_bytes(t1), st>>>(
        g, u, d, scale, sigma, aux, beta, 0.f, out, t1, m, tma);
  }
}
void launch_adjoint_factor(const Grid& g, const float* D, const float* db, float ht, float* c,
                           cudaStream_t st) {
  if (!tuned_sl_window() && posts_to_group(st)) {
    GroupOp op{};
    op.kind = GOP_SL1;
    op.sl = SlOpArgs{g, D, db, nullptr, nullptr, c, 1.f, 0.f, ht, tuned_sl_t1(),
                     tuned_sl_tma() ? 1 : 0};
    group_post(op, st);
    return;
  }
  ProfileRange pr(K_ADJFAC, (double)g.N * 20, st);
  brick_attributes();
  const int t1 = tuned_sl_t1();
  if (tuned_sl_window()) {
    k_slw<1><<<brick_grid(g, t1), dim3(32, TB2), window_smem_bytes(t1, 3, 0), st>>>(
        g, D, db, nullptr, 1.f, nullptr, 0.f, ht, c, t1);
  } else {
    CUtensorMap m;
    const int tma = tuned_sl_tma() && brick_map(D, g, 1, t1, &m);
    k_sl<1><<<brick_grid(g, t1), dim3(32, TB2), brick_smem_bytes(t1), st>>>(
        g, D, db, nullptr, 1.f, nullptr, 0.f, ht, c, t1, m, tma);
  }
}
// Grid of a persistent grouped launch: every SM filled with as many CTAs as fit
// (at most one per item).
template <typename K>
static int group_blocks(K kernel, int threads, size_t smem, int total) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  int sms = device_sm_count();
  if (sms <= 0) sms = 148;
  return std::max(1, std::min(total, sms * per_sm));
}

void launch_sl_group(int mode, const SlOpArgs* ops, int n, cudaStream_t st) {
  brick_attributes();
  for (int base = 0; base < n; base += GROUP_MAX) {
    SlGroup G;
    std::memset(&G, 0, sizeof G);
    G.nops = std::min(GROUP_MAX, n - base);
    int total = 0;
    for (int o = 0; o < G.nops; ++o) {
      const SlOpArgs& a = ops[base + o];
      SlGroupOp& q = G.op[o];
      q.g = a.g; q.u = a.u; q.d = a.d; q.scale = a.scale; q.aux = a.aux; q.out = a.out;
      q.sigma = a.sigma; q.beta = a.beta; q.ht = a.ht; q.t1 = a.t1;
      q.tma = a.tma && brick_map(a.u, a.g, 1, a.t1, &G.map[o]);
      const dim3 b = brick_grid(a.g, a.t1);
      q.tx = (int)b.x; q.ty = (int)b.y;
      G.first[o] = total;
      total += (int)(b.x * b.y * b.z);
      G.t1max = std::max(G.t1max, a.t1);
    }
    G.first[G.nops] = total;
    const size_t smem = brick_smem_bytes(G.t1max);
    if (mode == 0)
      k_sl_group<0><<<group_blocks(k_sl_group<0>, BRICK_THREADS, smem, total),
                      dim3(32, TB2), smem, st>>>(G);
    else
      k_sl_group<1><<<group_blocks(k_sl_group<1>, BRICK_THREADS, smem, total),
                      dim3(32, TB2), smem, st>>>(G);
  }
}

void launch_trace_group(const TraceOpArgs* ops, int n, cudaStream_t st) {
  brick_attributes();
  for (int base = 0; base < n; base += GROUP_MAX) {
    TraceGroup G;
    std::memset(&G, 0, sizeof G);
    G.nops = std::min(GROUP_MAX, n - base);
    int total = 0;
    for (int o = 0; o < G.nops; ++o) {
      const TraceOpArgs& a = ops[base + o];
      TraceGroupOp& q = G.op[o];
      q.g = a.g; q.v = a.v; q.df = a.df; q.db = a.db; q.ht = a.ht; q.t1 = a.t1;
      q.tma = a.tma && brick_map(a.v, a.g, 3, a.t1, &G.map[o]);
      const dim3 b = brick_grid(a.g, a.t1);
      q.tx = (int)b.x; q.ty = (int)b.y;
      G.first[o] = total;
      total += (int)(b.x * b.y * b.z);
      G.t1max = std::max(G.t1max, a.t1);
    }
    G.first[G.nops] = total;
    const size_t smem = brick_smem_bytes(G.t1max);
    k_trace_group<<<group_blocks(k_trace_group, BRICK_THREADS, smem, total), dim3(32, TB2),
                    smem, st>>>(G);
  }
}

bool launch_march_group(int mode, int nf, const MarchOpArgs* ops, int n, cudaStream_t st) {
  for (int base = 0; base < n; base += GROUP_MAX) {
    MarchGroup G;
    std::memset(&G, 0, sizeof G);
    G.nops = std::min(GROUP_MAX, n - base);
    int total = 0;
    for (int o = 0; o < G.nops; ++o) {
      G.op[o] = ops[base + o];
      const dim3 b = march_grid(G.op[o].g, G.op[o].mt1);
      G.tx[o] = (int)b.x; G.ty[o] = (int)b.y;
      G.first[o] = total;
      total += (int)(b.x * b.y * b.z);
    }
    G.first[G.nops] = total;
#define CLAIRE_MARCH_GROUP(M, NF)                                                        \
  k_march_group<M, NF><<<group_blocks(k_march_group<M, NF>, 32 * MT2, 0, total),           \
                         dim3(32, MT2), 0, st>>>(G)
    switch (mode * 16 + nf) {
      case 2: CLAIRE_MARCH_GROUP(0, 2); break;
      case 3: CLAIRE_MARCH_GROUP(0, 3); break;
      case 5: CLAIRE_MARCH_GROUP(0, 5); break;
      case 9: CLAIRE_MARCH_GROUP(0, 9); break;
      case 18: CLAIRE_MARCH_GROUP(1, 2); break;
      case 19: CLAIRE_MARCH_GROUP(1, 3); break;
      case 21: CLAIRE_MARCH_GROUP(1, 5); break;
      case 25: CLAIRE_MARCH_GROUP(1, 9); break;
      default: return false;
    }
#undef CLAIRE_MARCH_GROUP
  }
  return true;
}

void launch_count_far(const Grid& g, const float* d, unsigned long long* out,
                      cudaStream_t st) {
  k_count_far<<<vec_blocks(g.N), 256, 0, st>>>(g.N, d, out);
}
void launch_grad8(const Grid& g, const float* u, float* gu, cudaStream_t st) {
  ProfileRange pr(K_GRAD8, (double)g.N * 16, st);
  k_grad8<<<grid3(g), block3(), 0, st>>>(g, u, gu);
}
void launch_div8_prod(const Grid& g, const float* lam, const float* w, float* out,
                      cudaStream_t st) {
  ProfileRange pr(K_DIV8, (double)g.N * 20, st);
  k_div8_prod<<<grid3(g), block3(), 0, st>>>(g, lam, w, out);
}
void launch_ncc_final(int64_t n, const float* m1, const float* m, float* lt, const double* sx,
                      const double* sy, double a, double b, double c, double h3,
                      cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 16, st);
  k_ncc_final<<<vec_blocks(n), 256, 0, st>>>(n, m1, m, lt, sx, sy, a, b, c, h3);
}
void launch_affine(int64_t n, float a, const float* x, float b, float* out, cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 8, st);
  k_affine<<<vec_blocks(n), 256, 0, st>>>(n, a, x, b, out);
}
void launch_div8(const Grid& g, const float* w, float* out, cudaStream_t st) {
  ProfileRange pr(K_DIV8, (double)g.N * 16, st);
  k_div8_march<<<march_grid(g, MT1), dim3(32, MT2), 0, st>>>(g, w, out, MT1);
}
// History FD8 kernels: the marching version for nt in {1, 2, 4, 8}, the
// per-node global-memory version for any other nt.
template <int MODE>
static bool launch_march(const Grid& g, const float* mhist, const float* lhist, const float* vt,
                         float scale0, const float* base, float base_coef, float* out, int nt,
                         cudaStream_t st, const float* dotv = nullptr,
                         double* partial = nullptr) {
  const int mt1 = tuned_march_t1();
  if (march_supported(nt) && posts_to_group(st)) {
    GroupOp op{};
    op.kind = GOP_MARCH;
    op.mode = MODE;
    op.nf = nt + 1;
    op.mh = MarchOpArgs{g, mhist, lhist, vt, nullptr, base, out, out, dotv, partial,
                        scale0, base_coef, 1.f, mt1};
    group_post(op, st);
    return true;
  }
  const dim3 grid = march_grid(g, mt1), block(32, MT2);
#define CLAIRE_MARCH(NF)                                                                    \
  k_hist_march<MODE, NF, float><<<grid, block, 0, st>>>(g, mhist, lhist, vt, scale0, nullptr, \
                                                        base, base_coef, 1.f, out, out, dotv,  \
                                                        partial, mt1)
  switch (nt) {
    case 1: CLAIRE_MARCH(2); return true;
    case 2: CLAIRE_MARCH(3); return true;
    case 4: CLAIRE_MARCH(5); return true;
    case 8: CLAIRE_MARCH(9); return true;
    default: return false;
  }
#undef CLAIRE_MARCH
}

int march_blocks(const Grid& g) {
  const dim3 m = march_grid(g, tuned_march_t1());
  return (int)(m.x * m.y * m.z);
}
int march_blocks_max(const Grid& g) {                 // at the shallowest depth, 8 planes
  const dim3 m = march_grid(g, 8);
  return (int)(m.x * m.y * m.z);
}
// 64 planes per CTA (fewer queue refills: each CTA re-reads 8 planes of every
// history field to fill its queues) where that still leaves at least four CTAs
// per multiprocessor, else 32.
int default_march_t1(const Grid& g) {
  int sms = device_sm_count();
  if (sms <= 0) sms = 148;
  const dim3 m = march_grid(g, 64);
  return (int64_t)m.x * m.y * m.z >= 4LL * sms ? 64 : 32;
}
bool march_supported(int nt) { return nt == 1 || nt == 2 || nt == 4 || nt == 8; }

void launch_sdot_hist(const Grid& g, const float* mhist, int nt, const float* vt, float scale0,
                      float* shist, cudaStream_t st) {
  ProfileRange pr(K_SDOT, (double)g.N * (12 + 8 * (nt + 1)), st);
  if (!launch_march<0>(g, mhist, nullptr, vt, scale0, nullptr, 0.f, shist, nt, st))
    k_sdot_hist<<<grid3(g), block3(), 0, st>>>(g, mhist, nt, vt, scale0, shist);
}
void launch_accum_hist(const Grid& g, const float* lhist, const float* mhist, int nt,
                       const float* base, float base_coef, float* out, cudaStream_t st,
                       const float* dotv, double* partial) {
  ProfileRange pr(K_ACCUM, (double)g.N * (8 * (nt + 1) + 12 + 12 * (base != nullptr) +
                                          12 * (partial != nullptr)), st);
  if (!launch_march<1>(g, mhist, lhist, nullptr, 0.f, base, base_coef, out, nt, st, dotv,
                       partial))
    k_accum_hist<<<grid3(g), block3(), 0, st>>>(g, lhist, mhist, nt, base, base_coef, out);
}
int spectral_blocks(const Grid& g) {
  const int64_t Nc = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  return (int)((Nc + 255) / 256);
}
void launch_spectral(const Grid& g, cufftComplex* X, int op, float alpha, float gamma,
                     float beta_w, cudaStream_t st, double* partial, double* means) {
  const int64_t Nc = (int64_t)g.n1 * g.n2 * (g.n3 / 2 + 1);
  const float scale = (float)(1.0 / (double)g.N);
  ProfileRange pr(K_SPECTRAL, (double)Nc * 3 * 16, st);
  k_spectral<<<spectral_blocks(g), 256, 0, st>>>(g.n1, g.n2, g.n3, Nc, X, op, alpha, gamma,
                                                 beta_w, scale, partial, means);
}
int vector_blocks(int64_t n) { return vec_blocks(n); }
void launch_reduce_final(const double* partial, int nblocks, int mode, double* out,
                         cudaStream_t st) {
  ProfileRange pr(K_REDUCE, (double)nblocks * 8, st);
  k_reduce_final<<<1, 1024, 0, st>>>(partial, nblocks, mode, out);
}
void launch_pcg_update(int64_t n, const double* rz, const double* sHs, float* vt, float* r,
                       const float* s, const float* Hs, double* partial, int nblocks, int* flag,
                       cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 24, st);
  k_pcg_update<<<nblocks, 256, 0, st>>>(n / 4, rz, sHs, (float4*)vt, (float4*)r,
                                        (const float4*)s, (const float4*)Hs, partial, flag);
}
void launch_s_update(int64_t N, const double* rz_new, const double* rz_old, const double* means,
                     int first, const float* z, const float* r, float* s, float* hs,
                     cudaStream_t st) {
  const int64_t n = 3 * N;
  ProfileRange pr(K_VECTOR, (double)n * (first ? 16 : 24), st);
  k_s_update<<<vec_blocks(n / 4), 256, 0, st>>>(n / 4, N / 4, rz_new, rz_old, means, first,
                                                 (const float4*)z, (const float4*)r,
                                                 (float4*)s, (float4*)hs);
}
void launch_reduce(int64_t n, const float* a, const float* b, int mode, double* partial,
                   int nblocks, double* out, cudaStream_t st) {
  ProfileRange pr(K_REDUCE, (double)n * 4 * (b != nullptr ? 2 : 1), st);
  if (tl_prof) tl_prof->launches[K_REDUCE] += 1;    // two kernels per reduction
  k_reduce<<<nblocks, 256, 0, st>>>(n, a, b, mode, partial);
  k_reduce_final<<<1, 1024, 0, st>>>(partial, nblocks, mode, out);
}
void launch_axpby(int64_t n, float a, const float* x, float b, float* y, cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 12, st);
  k_axpby<<<vec_blocks(n), 256, 0, st>>>(n, a, x, b, y);
}
void launch_lincomb(int64_t n, float a, const float* x, float b, const float* y, float* out,
                    cudaStream_t st) {
  ProfileRange pr(K_VECTOR, (double)n * 12, st);
  k_lincomb<<<vec_blocks(n), 256, 0, st>>>(n, a, x, b, y, out);
}
void launch_detf(const Grid& g, const float* v, const float* df, int nt, float* F, float* Fn,
                 float* A, float* Ay, float* det, cudaStream_t st) {
  {
    ProfileRange pr(K_DETF, (double)g.N * (12 + 36 + 36), st);
    k_detf_init<<<grid3(g), block3(), 0, st>>>(g, v, A, F);
  }
  for (int k = 0; k < 9; ++k)
    launch_sl(g, A + k * g.N, df, nullptr, 1.0f, nullptr, 0.f, Ay + k * g.N, st);  // A(y)
  const float ht = 1.0f / nt;
  for (int j = 0; j < nt; ++j) {
    ProfileRange pr(K_DETF, (double)g.N * (12 + 36 * 4 + (j == nt - 1 ? 4 : 0)), st);
    k_detf_step<<<grid3(g), block3(), 0, st>>>(g, F, df, A, Ay, ht, Fn,
                                               j == nt - 1 ? det : nullptr);
    float* t = F;
    F = Fn;
    Fn = t;
  }
}

}  // namespace claire
