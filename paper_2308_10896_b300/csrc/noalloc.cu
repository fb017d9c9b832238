// Allocation-free variant of the moment filter (dsm_filter_moments_noalloc).
//
// Some callers cannot allocate device memory while they run: a real-time render
// loop that works inside a fixed, preallocated memory budget, or a host
// application that owns the device memory pool and lets no other allocator
// touch the device.  dsm_filter_moments may grow its context's scratch with
// cudaMalloc; this entry point never allocates.  The caller passes the input
// and output maps.  Radii up to 15 run as one tiled kernel that needs no
// intermediate map.  Radii 16 to 32 run as two 1-D passes whose intermediate,
// row-filtered map lives in a static device array that is part of the loaded
// library, so no call ever reaches cudaMalloc or cudaFree.
#include <cmath>
#include <mutex>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {
namespace {

constexpr int kNoAllocMaxTexels = 1024 * 1024;   // largest map: 1024 x 1024 texels (8 MiB of float2)

// Intermediate of the separable filter (x pass -> y pass).  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) float2 g_filter_scratch[kNoAllocMaxTexels];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device (host code only
// sees a host-side stand-in for the symbol).  Looked up once per device, on
// that device's first call, and cached: after cudaDeviceReset (or any other
// teardown of the device's primary context) the cached address is stale, so
// the library must not be used on that device again in this process.
cudaError_t scratch_for_current_device(float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dsm

extern "C" dsm_status dsm_filter_moments_noalloc(const float* in, float* out, int32_t res, float sigma,
                                                 int32_t radius, int32_t kind, int32_t boundary, void* stream) {
  using namespace dsm;
  if (!in || !out || res < 1 || !filter_args_ok(sigma, radius, kind, boundary)) return DSM_ERR_INVALID_ARG;
  if ((long long)res * res > kNoAllocMaxTexels) return DSM_ERR_CAPACITY;   // beyond the static array
  float2* tmp = nullptr;
  if (scratch_for_current_device(&tmp) != cudaSuccess) return DSM_ERR_CUDA;
  // Radii up to 15 take the tiled kernel and never touch `tmp`.  For larger
  // radii the x pass overwrites every texel of the intermediate before the y
  // pass reads it, so nothing in the shared array has to be cleared between
  // calls.  No status word is passed, so the TMA-staged kernel (which reports
  // timeouts through one) is not used here.
  FilterArgs fa;
  make_filter_args(sigma, radius, kind, boundary, &fa);
  launch_filter(reinterpret_cast<const float2*>(in), tmp, reinterpret_cast<float2*>(out), res, fa,
                (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? DSM_OK : DSM_ERR_CUDA;
}
