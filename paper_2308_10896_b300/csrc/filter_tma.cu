// Separable moment filter m = G g (Eqs. moment1/moment2) and its adjoint G^T
// with the input tiles staged by the tensor memory accelerator.
//
// A persistent CTA walks its share of the 32 x 32 output tiles.  While it
// filters one tile from shared memory, the TMA (cp.async.bulk.tensor, one
// elected thread, completion counted on an mbarrier) already brings the next
// tile's input into the other of two staging buffers, so the loads of the
// whole kernel stay in flight back to back instead of being issued and waited
// for tile by tile.  The staged input is the tile with an r-texel halo, loaded
// as 16-texel-wide boxes with the 128-byte swizzle (16-byte chunk index XOR
// the row index within each 1024-byte group of eight 128-byte rows), so the
// x pass, whose lanes read one column across many rows, spreads its reads over
// the banks.  The arithmetic is that of filter_tile_kernel: x pass then y
// pass, taps in the same order, the same fold terms, so the results are
// bit-identical.
//
// Boundary handling: the TMA fills texels outside the map with zeros, which is
// the zero boundary and the adjoint's rule; for the clamp boundary the halo of
// a border tile is rewritten from the edge texels in shared memory.  The
// antialiased patch of the forward pass (texels listed by the antialiasing)
// is substituted from the listed-flag tile, which the TMA stages beside the
// input.  Every wait on an mbarrier is bounded: past the limit the CTA records
// a timeout in the device status word (dsm_sync reports it) and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <algorithm>
#include <cstdint>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace dsm {
namespace {

constexpr int kFT = 32;        // output tile side
constexpr int kXRun = 8;       // x-pass outputs per thread
constexpr int kYRun = 4;       // y-pass outputs per thread
constexpr int kTmaRmax = 8;    // largest radius staged by the TMA (shared memory)

template <int kR>
struct TmaGeom {
  static constexpr int S = kFT + 2 * kR;       // staged rows, and staged columns the filter reads
  static constexpr int SH = kR & 1;            // columns start one early for odd r (x must be even)
  static constexpr int W = S + SH;             // staged columns
  static constexpr int NB = (W + 15) / 16;     // boxes of 16 texels (128 bytes) per staged row
  static constexpr int BOX = ((S * 128 + 1023) / 1024) * 1024;   // bytes per box, 1024-aligned
  static constexpr int BUF = NB * BOX;         // one staging buffer
  static constexpr int HW = (W + 30) / 16 * 16;   // listed-flag box width in bytes (16-aligned start)
  static constexpr int HBOX = ((HW * S + 1023) / 1024) * 1024;
  static constexpr int PM = kFT + 1;           // x-pass output row stride (odd)
  static constexpr int MID = S * PM * 8;
  static constexpr size_t smem = 1024 + 2 * (size_t)BUF + 2 * (size_t)HBOX + MID + 16;
};

// Byte offset of staged texel (column c, row s) in a staging buffer: box c / 16,
// row s of 128 bytes, 16-byte chunk (c % 16) / 2 XOR (s % 8).
template <int kR>
__device__ __forceinline__ int swz(int c, int s) {
  const int xi = c & 15;
  return (c >> 4) * TmaGeom<kR>::BOX + s * 128 + ((((xi >> 1) ^ (s & 7)) << 4) | ((xi & 1) << 3));
}

__device__ __forceinline__ void fma2(float2& acc, float w, float2 v) {
  acc.x = fmaf(w, v.x, acc.x);
  acc.y = fmaf(w, v.y, acc.y);
}

// Run of kN outputs from the kN + 2 kR inputs ld(0), ld(1), ...: the sums and
// fold terms of filter_tile_kernel's tap_run, in the same order.
template <int kR, int kN, bool kFold, class Ld>
__device__ __forceinline__ void tap_run_ld(const Ld& ld, const FilterArgs& fa, int nfold, int first, int last,
                                           float2 (&acc)[kN]) {
#pragma unroll
  for (int u = 0; u < kN; ++u) acc[u] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < kN + 2 * kR; ++m) {
    const float2 v = ld(m);
#pragma unroll
    for (int u = 0; u < kN; ++u) {
      const int t = m - u;
      if (t >= 0 && t <= 2 * kR) fma2(acc[u], fa.w[t], v);
    }
  }
  if (kFold) {
    if (first >= 0) {
#pragma unroll
      for (int u = 0; u < kN; ++u)
        if (u == first)
#pragma unroll
          for (int q = 0; q < kR; ++q)
            if (q < nfold) fma2(acc[u], fa.fold[q], ld(u + kR + q));
    }
    if (last >= 0) {
#pragma unroll
      for (int u = 0; u < kN; ++u)
        if (u == last)
#pragma unroll
          for (int q = 0; q < kR; ++q)
            if (q < nfold) fma2(acc[u], fa.fold[q], ld(u + kR - q));
    }
  }
}

template <int kR, bool kAdjoint>
__global__ void __launch_bounds__(256) filter_tma_kernel(const __grid_constant__ CUtensorMap map_in,
                                                         const __grid_constant__ CUtensorMap map_flag,
                                                         float2* __restrict__ out, int R, FilterArgs fa,
                                                         FilterExtras ex, int has_flags, DevStatus* status) {
  using G = TmaGeom<kR>;
  constexpr int S = G::S, SH = G::SH, PM = G::PM;
  extern __shared__ unsigned char smraw[];
  // the swizzled boxes need 1024-byte alignment in the shared window (1 KB of slack is allocated)
  const uint32_t raw_off = smem_addr(smraw);
  unsigned char* const base = smraw + (((raw_off + 1023u) & ~1023u) - raw_off);
  unsigned char* const buf0 = base;
  unsigned char* const hb0 = base + 2 * G::BUF;
  float2* const mid = reinterpret_cast<float2*>(base + 2 * G::BUF + 2 * G::HBOX);
  uint64_t* const bar = reinterpret_cast<uint64_t*>(base + 2 * G::BUF + 2 * G::HBOX + G::MID);
  const int tid = threadIdx.x;
  const int tiles_x = (R + kFT - 1) / kFT, n_tiles = tiles_x * tiles_x;
  const bool clamp = !kAdjoint && fa.boundary == 0;
  const uint32_t tx_bytes = (uint32_t)(G::NB * S * 128 + (has_flags ? G::HW * S : 0));
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: the loads of tile t into staging buffer b
  auto issue = [&](int t, int b) {
    const int xs = (t % tiles_x) * kFT - kR - SH, ys = (t / tiles_x) * kFT - kR;
    mbar_expect_tx(&bar[b], tx_bytes);
#pragma unroll
    for (int k = 0; k < G::NB; ++k) tma_load_2d(buf0 + b * G::BUF + k * G::BOX, &map_in, xs + 16 * k, ys, &bar[b]);
    if (has_flags) tma_load_2d(hb0 + b * G::HBOX, &map_flag, xs & ~15, ys, &bar[b]);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < n_tiles) issue(t, 0);
  uint32_t parity = 0;   // bit b: phase of buffer b's barrier to wait for
  for (int it = 0; t < n_tiles; ++it, t += gridDim.x) {
    const int b = it & 1;
    if (tid == 0 && t + (int)gridDim.x < n_tiles) issue(t + gridDim.x, b ^ 1);
    const int ox = (t % tiles_x) * kFT, oy = (t / tiles_x) * kFT;
    // the adjoint's fold reads f at this thread's outputs: in flight during the wait
    float fpre[kYRun];
    if (kAdjoint) {
      const int col = tid % kFT, r0 = (tid / kFT) * kYRun;
#pragma unroll
      for (int u = 0; u < kYRun; ++u) {
        const int gy = oy + r0 + u, gx = ox + col;
        fpre[u] = (ex.gf && gx < R && gy < R) ? ex.fmap[(size_t)gy * R + gx].x : 0.f;
      }
    }
    const bool landed = mbar_wait_bounded(&bar[b], (parity >> b) & 1u);
    parity ^= 1u << b;
    if (!__syncthreads_and(landed)) {
      // give up: record the timeout, let the copies in flight finish (bounded) and leave
      if (tid == 0 && status) atomicExch(&status->timeout, 1);
      mbar_wait_bounded(&bar[b ^ 1], (parity >> (b ^ 1)) & 1u);
      return;
    }
    unsigned char* const buf = buf0 + b * G::BUF;
    auto at = [&](int c, int s) { return reinterpret_cast<float2*>(buf + swz<kR>(c + SH, s)); };
    if (!kAdjoint) {
      bool wrote = false;
      if (has_flags) {
        // the antialiased values of the listed texels replace (f, f^2)
        const unsigned char* hb = hb0 + b * G::HBOX;
        const int hx = (ox - kR - SH) & ~15;
        for (int k = tid; k < S * S; k += 256) {
          const int s = k / S, c = k - s * S;
          const int gx = ox - kR + c, gy = oy - kR + s;
          if (gx < 0 || gy < 0 || gx >= R || gy >= R) continue;
          if (hb[s * G::HW + (gx - hx)]) *at(c, s) = ex.patch[(size_t)gy * R + gx];
        }
        wrote = true;
      }
      if (clamp && (ox < kR || oy < kR || ox + kFT + kR > R || oy + kFT + kR > R)) {
        __syncthreads();   // substituted edge texels first
        for (int k = tid; k < S * S; k += 256) {
          const int s = k / S, c = k - s * S;
          const int gx = ox - kR + c, gy = oy - kR + s;
          if (gx >= 0 && gy >= 0 && gx < R && gy < R) continue;
          const int cx = min(max(gx, 0), R - 1), cy = min(max(gy, 0), R - 1);
          *at(c, s) = *at(cx - (ox - kR), cy - (oy - kR));
        }
        wrote = true;
      }
      // generic-proxy writes into the buffer come before the next bulk copy into it
      if (wrote) fence_proxy_async();
      __syncthreads();
    }
    // x pass over the S staged rows: thread -> (row, run of kXRun columns)
    const int nfold = min(kR, R);
    constexpr int kXItems = S * (kFT / kXRun);
    for (int k = tid; k < kXItems; k += 256) {
      const int row = k % S, c0 = (k / S) * kXRun;
      float2 acc[kXRun];
      const auto ld = [&](int m) { return *at(c0 + m, row); };
      if (kAdjoint && fa.boundary == 0) {
        const int first = (ox + c0 == 0) ? 0 : -1;
        const int last = (R - 1 - ox - c0 >= 0 && R - 1 - ox - c0 < kXRun) ? R - 1 - ox - c0 : -1;
        tap_run_ld<kR, kXRun, true>(ld, fa, nfold, first, last, acc);
      } else {
        tap_run_ld<kR, kXRun, false>(ld, fa, 0, -1, -1, acc);
      }
#pragma unroll
      for (int u = 0; u < kXRun; ++u) mid[row * PM + c0 + u] = acc[u];
    }
    __syncthreads();
    // y pass: thread -> (column, run of kYRun rows), 32 x 32 outputs
    {
      const int col = tid % kFT, r0 = (tid / kFT) * kYRun;
      float2 acc[kYRun];
      const auto ld = [&](int m) { return mid[(r0 + m) * PM + col]; };
      if (kAdjoint && fa.boundary == 0) {
        const int first = (oy + r0 == 0) ? 0 : -1;
        const int last = (R - 1 - oy - r0 >= 0 && R - 1 - oy - r0 < kYRun) ? R - 1 - oy - r0 : -1;
        tap_run_ld<kR, kYRun, true>(ld, fa, nfold, first, last, acc);
      } else {
        tap_run_ld<kR, kYRun, false>(ld, fa, 0, -1, -1, acc);
      }
      const int gx = ox + col;
      if (gx < R) {
#pragma unroll
        for (int u = 0; u < kYRun; ++u) {
          const int gy = oy + r0 + u;
          if (gy < R) {
            const size_t q = (size_t)gy * R + gx;
            out[q] = acc[u];
            if (kAdjoint && ex.gf) ex.gf[q] = moment_fold(acc[u], fpre[u], ex.ec);
          }
        }
      }
    }
    __syncthreads();   // the staging buffer and mid are free again
  }
}

template <int kR, bool kAdjoint>
bool launch_tma_r(const float2* in, float2* out, int R, const FilterArgs& fa, const FilterExtras& ex,
                  DevStatus* status, cudaStream_t st) {
  using G = TmaGeom<kR>;
  const bool flags = !kAdjoint && ex.hflag != nullptr;
  alignas(64) CUtensorMap map_in, map_flag;
  if (!encode_map(&map_in, in, CU_TENSOR_MAP_DATA_TYPE_UINT64, 8, R, R, 16, G::S, CU_TENSOR_MAP_SWIZZLE_128B))
    return false;
  if (flags) {
    if (!encode_map(&map_flag, ex.hflag, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, R, R, G::HW, G::S,
                    CU_TENSOR_MAP_SWIZZLE_NONE))
      return false;
  } else {
    map_flag = map_in;   // not read
  }
  static int per_sm = 0;   // resident CTAs per SM of this instance (queried once)
  static int n_sm = 0;
  if (per_sm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(filter_tma_kernel<kR, kAdjoint>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G::smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_tma_kernel<kR, kAdjoint>, 256, G::smem) !=
            cudaSuccess ||
        per_sm < 1) {
      per_sm = 0;
      return false;
    }
  }
  const int tiles = ((R + kFT - 1) / kFT) * ((R + kFT - 1) / kFT);
  const int grid = std::min(tiles, n_sm * per_sm);
  count_launches(1);
  filter_tma_kernel<kR, kAdjoint><<<grid, 256, G::smem, st>>>(map_in, map_flag, out, R, fa, ex, flags ? 1 : 0,
                                                                status);
  return true;
}

template <int kR, bool kAdjoint>
bool launch_tma_dispatch(const float2* in, float2* out, int R, const FilterArgs& fa, const FilterExtras& ex,
                         DevStatus* status, cudaStream_t st) {
  if (fa.r != kR) {
    if constexpr (kR < kTmaRmax) return launch_tma_dispatch<kR + 1, kAdjoint>(in, out, R, fa, ex, status, st);
    else return false;
  }
  return launch_tma_r<kR, kAdjoint>(in, out, R, fa, ex, status, st);
}

// Probe of the bounded wait: one CTA waits on an mbarrier whose phase
// completes only when `arrive` is set; otherwise the wait gives up after
// `limit` polls and records a timeout in the status word.
__global__ void bounded_wait_probe_kernel(DevStatus* status, int arrive, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
  bool done = false;
  for (long long it = 0; it < limit && !done; ++it) done = mbar_try_wait(&bar, 0);
  if (!__syncthreads_and(done) && threadIdx.x == 0) atomicExch(&status->timeout, 1);
}

}  // namespace

void launch_bounded_wait_probe(DevStatus* status, bool arrive, cudaStream_t st) {
  count_launches(1);
  bounded_wait_probe_kernel<<<1, 32, 0, st>>>(status, arrive ? 1 : 0, 4096);
}

bool launch_filter_tma(bool adjoint, const float2* in, float2* out, int R, const FilterArgs& fa,
                       const FilterExtras& ex, DevStatus* status, cudaStream_t st) {
  // tensor-map rules: 16-byte aligned bases, row strides a multiple of 16 bytes
  if (!status || fa.shape != 0 || fa.r < 1 || fa.r > kTmaRmax || R % 16 != 0 || R < kFT) return false;
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (ex.hflag && (reinterpret_cast<uintptr_t>(ex.hflag) & 15)))
    return false;
  return adjoint ? launch_tma_dispatch<1, true>(in, out, R, fa, ex, status, st)
                 : launch_tma_dispatch<1, false>(in, out, R, fa, ex, status, st);
}

}  // namespace dsm
