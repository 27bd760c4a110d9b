// claire_transport_noalloc: the state transport m(1) for callers that cannot
// allocate device memory.
//
// Every other entry point works through a context whose workspace comes from
// cudaMalloc.  Some callers cannot allow that: processes whose device memory is
// reserved up front by another allocator (a framework's caching allocator or a
// fixed memory pool sized to the GPU), where an extra driver allocation fails or
// fragments the pool, and callers that must not pay the device-wide
// synchronisation a cudaMalloc / cudaFree may imply.  This entry point takes
// the inputs and the output from the caller and keeps its only scratch (the
// departure displacements and one intermediate field) in the file-scope device
// array below, which every GPU that loads the library holds until the process
// exits.  It allocates nothing: no cudaMalloc, no cudaFree, no allocating
// library call.
#include <mutex>

#include <cstdio>
#include <cstring>

#include "../../include/claire.h"
#include "internal.h"

using namespace claire;

namespace {

// 4 floats per voxel: departure displacements [3][N] and one intermediate field [N].
constexpr long long kFloatsPerVoxel = 4;
static __device__ __align__(256) float g_noalloc_scratch[kFloatsPerVoxel * CLAIRE_NOALLOC_MAX_VOXELS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};   // set once a lookup on that device succeeded

void set_error(char* err, size_t len, const char* fmt, long long a = 0, long long b = 0) {
  if (err && len > 0) snprintf(err, len, fmt, a, b);
}

// True when p is device memory of device dev (not host, managed or another GPU's memory).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();                   // clear the error state of the failed query
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" claire_status claire_transport_noalloc(int nx, int ny, int nz, int nt, const float* v,
                                                  const float* m0, float* m1_out, void* stream,
                                                  char* err, size_t err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (!v || !m0 || !m1_out) {
    set_error(err, err_len, "claire_transport_noalloc: NULL pointer argument");
    return CLAIRE_EINVAL;
  }
  if (nx < 16 || ny < 16 || nz < 16 || nx % 2 || ny % 2 || nz % 2 || nt < 1 || nt > 256) {
    set_error(err, err_len,
              "claire_transport_noalloc: sizes must be even and >= 16 and 1 <= nt <= 256");
    return CLAIRE_EINVAL;
  }
  const long long N = (long long)nx * ny * nz;
  if (N > CLAIRE_NOALLOC_MAX_VOXELS) {
    set_error(err, err_len,
              "claire_transport_noalloc: grid of %lld voxels exceeds the static scratch limit of "
              "%lld voxels (CLAIRE_NOALLOC_MAX_VOXELS); use claire_create + claire_transport",
              N, (long long)CLAIRE_NOALLOC_MAX_VOXELS);
    return CLAIRE_EINVAL;
  }
  const size_t fb = (size_t)N * sizeof(float);
  if (overlaps(m1_out, fb, m0, fb) || overlaps(m1_out, fb, v, 3 * fb)) {
    set_error(err, err_len, "claire_transport_noalloc: m1_out overlaps m0 or v");
    return CLAIRE_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(err, err_len, "claire_transport_noalloc: cudaGetDevice failed or device >= 64");
    return CLAIRE_ECUDA;
  }
  // The kernels run on the current device: every array must live there.
  if (!on_device(v, dev) || !on_device(m0, dev) || !on_device(m1_out, dev)) {
    set_error(err, err_len,
              "claire_transport_noalloc: v, m0 and m1_out must be device memory of the current "
              "device (%lld)", dev);
    return CLAIRE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    if (e != cudaSuccess) cudaGetLastError();
    set_error(err, err_len,
              "claire_transport_noalloc: the call synchronises its stream before returning, "
              "which a capturing stream does not allow");
    return CLAIRE_EINVAL;
  }
  // Set-up per device, with that device current: the host-side name of the
  // array is not a device address, so look the address up and cache it.  Only
  // a successful lookup is cached; a failed one is retried on the next call.
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        if (err && err_len > 0)
          snprintf(err, err_len, "claire_transport_noalloc: cudaGetSymbolAddress failed: %s",
                   cudaGetErrorString(e));
        return CLAIRE_ECUDA;
      }
      g_scratch_ptr[dev] = (float*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  float* d = scratch;                     // [3][N] displacements, fully rewritten below
  float* tmp = d + 3 * N;                 // [N] intermediate state, fully rewritten below

  Grid g{};
  g.n1 = nx; g.n2 = ny; g.n3 = nz;
  g.N = N;
  const double tp = 2.0 * M_PI;
  g.h1 = (float)(tp / nx); g.h2 = (float)(tp / ny); g.h3 = (float)(tp / nz);
  g.inv_h1 = (float)(nx / tp); g.inv_h2 = (float)(ny / tp); g.inv_h3 = (float)(nz / tp);
  const float ht = 1.0f / (float)nt;

  // Same kernels as claire_transport: RK2 departure points along +v, then nt
  // homogeneous SL steps.  Step j writes m1_out when nt-1-j is even, else the
  // scratch field, so the last step lands in m1_out and no step reads its output.
  launch_trace(g, v, d, nullptr, ht, st);
  const float* src = m0;
  for (int j = 0; j < nt; ++j) {
    float* dst = ((nt - 1 - j) % 2 == 0) ? m1_out : tmp;
    launch_sl(g, src, d, nullptr, 1.0f, nullptr, 0.0f, dst, st);
    src = dst;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (err && err_len > 0)
      snprintf(err, err_len, "claire_transport_noalloc: %s", cudaGetErrorString(e));
    return CLAIRE_ECUDA;
  }
  return CLAIRE_OK;
}
