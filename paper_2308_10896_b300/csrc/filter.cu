// Separable moment filter m = G g (Eqs. moment1/moment2) and its adjoint
// G^T (Sec. 4: dm/dTheta = G grad f~).  G filters along x, then along y.
#include <algorithm>
#include <cmath>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {

bool filter_args_ok(float sigma, int radius, int kind, int boundary) {
  if ((kind != 0 && kind != 1) || (boundary != 0 && boundary != 1) || radius > 32) return false;
  const bool sigma_ok = std::isfinite(sigma) && sigma > 0.f;
  // the Gaussian's weights divide by sigma^2; without a radius, r = ceil(2 sigma)
  if (kind == 0 && !sigma_ok) return false;
  if (radius <= 0 && !sigma_ok) return false;
  return true;
}

void make_filter_args(double sigma, int radius, int kind, int boundary, FilterArgs* fa) {
  // the clamp to 32 taps happens in double, before the conversion to int
  const int r = radius > 0 ? std::min(radius, 32) : (int)std::min(std::ceil(2.0 * sigma), 32.0);
  fa->r = r;
  fa->boundary = boundary;
  fa->shape = 0;
  double w[65], s = 0.0;
  for (int k = -r; k <= r; ++k) {
    w[k + r] = (kind == 1) ? 1.0 : std::exp(-(double)k * k / (2.0 * sigma * sigma));
    s += w[k + r];
  }
  for (int k = 0; k < 2 * r + 1; ++k) fa->w[k] = (float)(w[k] / s);
  for (int k = 2 * r + 1; k < 65; ++k) fa->w[k] = 0.f;
  // fold[i] = sum_{k > i} w_k: weight of the taps that leave the map by more than i texels
  for (int i = 0; i < 33; ++i) {
    double f = 0.0;
    for (int k = i + 1; k <= r; ++k) f += w[k + r] / s;
    fa->fold[i] = (float)f;
  }
}

// One 1-D pass along x (kAxisY = false) or y.  kAdjoint applies the transpose:
// the same symmetric taps on in-range texels plus, for the clamp boundary, the
// folded weight of the taps that the forward pass clamped onto the edge texel.
template <bool kAxisY, bool kAdjoint>
__global__ void filter_pass_kernel(const float2* __restrict__ in, float2* __restrict__ out, int R, FilterArgs fa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= R || j >= R) return;
  const int pos = kAxisY ? j : i;
  const size_t stride = kAxisY ? (size_t)R : 1;
  const size_t base = (size_t)j * R + i - (size_t)pos * stride;
  const int r = fa.r;
  const bool clamp = fa.boundary == 0;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = -r; k <= r; ++k) {
    int q = pos + k;
    if (q < 0 || q >= R) {
      if (kAdjoint || !clamp) continue;
      q = q < 0 ? 0 : R - 1;
    }
    const float2 v = in[base + (size_t)q * stride];
    const float w = fa.w[k + r];
    acc.x = fmaf(w, v.x, acc.x);
    acc.y = fmaf(w, v.y, acc.y);
  }
  if (kAdjoint && clamp) {
    if (pos == 0) {
      for (int q = 0; q < r && q < R; ++q) {
        const float2 v = in[base + (size_t)q * stride];
        acc.x = fmaf(fa.fold[q], v.x, acc.x);
        acc.y = fmaf(fa.fold[q], v.y, acc.y);
      }
    }
    if (pos == R - 1) {
      for (int q = 0; q < r && q < R; ++q) {
        const float2 v = in[base + (size_t)(R - 1 - q) * stride];
        acc.x = fmaf(fa.fold[q], v.x, acc.x);
        acc.y = fmaf(fa.fold[q], v.y, acc.y);
      }
    }
  }
  out[(size_t)j * R + i] = acc;
}

// Both passes of G (or of G^T) in one kernel, for radii up to kFRmax (the
// radius is a template parameter, so every tap and weight index is fixed at
// compile time).  A CTA owns a 32 x 32 output tile:
//   1. the input tile with an r-texel halo, S x S texels (S = 32 + 2r), is
//      staged in shared memory, clamped (G, clamp boundary) or zero-filled;
//   2. the x pass runs over all S rows and the tile's 32 columns: each thread
//      produces a run of 8 outputs of one row from 8 + 2r staged texels, so a
//      texel is read once per run instead of once per tap;
//   3. the y pass: each thread produces a run of 4 outputs of one column and
//      writes them with coalesced stores.
// G = Gy Gx and the transpose G^T = Gx^T Gy^T: the two 1-D factors act on
// different axes and commute, so G^T also runs x first.  With symmetric taps a
// 1-D transpose is the same tap sum over zero-filled texels, plus, for the
// clamp boundary, the folded weight of the taps that the forward filter
// clamped onto texel 0 or R-1.  Row strides in shared memory are odd (in
// float2), so threads that own different rows hit different banks.
constexpr int kFT = 32;      // output tile side
constexpr int kFRmax = 15;   // largest radius handled by the tiled kernel (48 KB of shared memory)
constexpr int kXRun = 8;     // x-pass outputs per thread
constexpr int kYRun = 4;     // y-pass outputs per thread

__device__ __forceinline__ void fma2(float2& acc, float w, float2 v) {
  acc.x = fmaf(w, v.x, acc.x);
  acc.y = fmaf(w, v.y, acc.y);
}

template <int kR>
struct TileGeom {
  static constexpr int S = kFT + 2 * kR;      // staged side
  static constexpr int P = S | 1;             // input row stride (odd)
  static constexpr int PM = kFT + 1;          // x-pass output row stride (odd)
  static constexpr size_t smem = (size_t)(S * P + S * PM) * sizeof(float2);
};

// Run of kN outputs from kN + 2 kR consecutive texels at src[0], src[step], ...:
// out_u = sum_t w_t x_{u + kR + t}; with kFold, the fold terms of the output
// that sits on texel 0 (first) or R-1 (last) of the map, q < nfold.
template <int kR, int kN, bool kFold>
__device__ __forceinline__ void tap_run(const float2* src, int step, const FilterArgs& fa, int nfold, int first,
                                        int last, float2 (&acc)[kN]) {
#pragma unroll
  for (int u = 0; u < kN; ++u) acc[u] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < kN + 2 * kR; ++m) {
    const float2 v = src[m * step];
#pragma unroll
    for (int u = 0; u < kN; ++u) {
      const int t = m - u;
      if (t >= 0 && t <= 2 * kR) fma2(acc[u], fa.w[t], v);
    }
  }
  if (kFold) {
    // first: output u0 = first sits on texel 0 and collects fold_q x_q (q < r);
    // last: output u1 = last sits on texel R-1 and collects fold_q x_{R-1-q}
    if (first >= 0) {
#pragma unroll
      for (int u = 0; u < kN; ++u)
        if (u == first)
#pragma unroll
          for (int q = 0; q < kR; ++q)
            if (q < nfold) fma2(acc[u], fa.fold[q], src[(u + kR + q) * step]);
    }
    if (last >= 0) {
#pragma unroll
      for (int u = 0; u < kN; ++u)
        if (u == last)
#pragma unroll
          for (int q = 0; q < kR; ++q)
            if (q < nfold) fma2(acc[u], fa.fold[q], src[(u + kR - q) * step]);
    }
  }
}


template <int kR, bool kAdjoint>
__global__ void __launch_bounds__(256) filter_tile_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                          int R, FilterArgs fa, FilterExtras ex) {
  using G = TileGeom<kR>;
  constexpr int S = G::S, P = G::P, PM = G::PM;
  extern __shared__ float2 sm[];
  float2* tin = sm;            // S rows x S texels, stride P
  float2* mid = sm + S * P;    // S rows x kFT texels, stride PM
  const int ox = blockIdx.x * kFT, oy = blockIdx.y * kFT;
  const int tid = threadIdx.x;
  const bool clamp = fa.boundary == 0;
  // the adjoint's fold reads f at this thread's outputs: loaded first, so the
  // loads are in flight during the staging and both passes
  float fpre[kYRun];
  if (kAdjoint) {
    const int col = tid % kFT, r0 = (tid / kFT) * kYRun;
#pragma unroll
    for (int u = 0; u < kYRun; ++u) {
      const int gy = oy + r0 + u, gx = ox + col;
      fpre[u] = (ex.gf && gx < R && gy < R) ? ex.fmap[(size_t)gy * R + gx].x : 0.f;
    }
  }
  // 1. stage the input: every load of the thread is issued before the first
  // shared-memory store
  constexpr int kStage = (S * S + 255) / 256;
  float2 v[kStage];
#pragma unroll
  for (int it = 0; it < kStage; ++it) {
    const int k = tid + 256 * it;
    const int row = k / S, col = k - row * S;
    int gy = oy - kR + row, gx = ox - kR + col;
    v[it] = make_float2(0.f, 0.f);
    bool load = k < S * S;
    if (!kAdjoint && clamp) {
      gy = min(max(gy, 0), R - 1);
      gx = min(max(gx, 0), R - 1);
    } else {
      load = load && gy >= 0 && gy < R && gx >= 0 && gx < R;
    }
    if (load) {
      const size_t q = (size_t)gy * R + gx;
      v[it] = in[q];
      if (!kAdjoint && ex.hflag && ex.hflag[q]) v[it] = ex.patch[q];
    }
  }
#pragma unroll
  for (int it = 0; it < kStage; ++it) {
    const int k = tid + 256 * it;
    if (k < S * S) {
      const int row = k / S, col = k - row * S;
      tin[row * P + col] = v[it];
    }
  }
  __syncthreads();
  const bool fold = kAdjoint && clamp;
  const int nfold = min(kR, R);   // fold terms q < min(r, R)
  // 2. x pass over S rows: thread -> (row, run of kXRun columns)
  constexpr int kXItems = S * (kFT / kXRun);
  for (int k = tid; k < kXItems; k += 256) {
    const int row = k % S, c0 = (k / S) * kXRun;
    float2 acc[kXRun];
    if (fold) {
      const int first = (ox + c0 == 0) ? 0 : -1;
      const int last = (R - 1 - ox - c0 >= 0 && R - 1 - ox - c0 < kXRun) ? R - 1 - ox - c0 : -1;
      tap_run<kR, kXRun, true>(tin + row * P + c0, 1, fa, nfold, first, last, acc);
    } else {
      tap_run<kR, kXRun, false>(tin + row * P + c0, 1, fa, 0, -1, -1, acc);
    }
#pragma unroll
    for (int u = 0; u < kXRun; ++u) mid[row * PM + c0 + u] = acc[u];
  }
  __syncthreads();
  // 3. y pass: thread -> (column, run of kYRun rows), 32 x 32 outputs
  {
    const int col = tid % kFT, r0 = (tid / kFT) * kYRun;
    float2 acc[kYRun];
    if (fold) {
      const int first = (oy + r0 == 0) ? 0 : -1;
      const int last = (R - 1 - oy - r0 >= 0 && R - 1 - oy - r0 < kYRun) ? R - 1 - oy - r0 : -1;
      tap_run<kR, kYRun, true>(mid + r0 * PM + col, PM, fa, nfold, first, last, acc);
    } else {
      tap_run<kR, kYRun, false>(mid + r0 * PM + col, PM, fa, 0, -1, -1, acc);
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
}

// The extras on the two-pass path (radius above the tiled kernel's limit).
__global__ void compose_kernel(const float2* __restrict__ fmap, const uint8_t* __restrict__ hflag,
                               const float2* __restrict__ patch, float2* __restrict__ out, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = hflag[p] ? patch[p] : fmap[p];
}
__global__ void fold_kernel(const float2* __restrict__ fmap, const float2* __restrict__ g, float* __restrict__ gf,
                            int n, float ec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) gf[p] = moment_fold(g[p], fmap[p].x, ec);
}
static_assert(kFT * kFT == 256 * kYRun, "one y-pass run per thread");
static_assert(TileGeom<kFRmax>::S * (kFT / kXRun) <= 256, "one x-pass pass over the threads for every radius");
// the largest tile fits the default 48 KB of dynamic shared memory per block
static_assert(TileGeom<kFRmax>::smem <= 48 * 1024, "filter tile");

template <int kR>
static bool launch_tiled_r(bool adjoint, const float2* in, float2* out, int R, const FilterArgs& fa,
                           const FilterExtras& ex, cudaStream_t st) {
  if (fa.r != kR) {
    if constexpr (kR < kFRmax) return launch_tiled_r<kR + 1>(adjoint, in, out, R, fa, ex, st);
    else return false;
  }
  dim3 g((R + kFT - 1) / kFT, (R + kFT - 1) / kFT);
  count_launches(1);
  if (adjoint) filter_tile_kernel<kR, true><<<g, 256, TileGeom<kR>::smem, st>>>(in, out, R, fa, ex);
  else filter_tile_kernel<kR, false><<<g, 256, TileGeom<kR>::smem, st>>>(in, out, R, fa, ex);
  return true;
}

void launch_compose(const float2* fmap, const uint8_t* hflag, const float2* patch, float2* out, int n,
                    cudaStream_t st) {
  count_launches(1);
  compose_kernel<<<(n + 255) / 256, 256, 0, st>>>(fmap, hflag, patch, out, n);
}

void launch_filter(const float2* in, float2* tmp, float2* out, int R, const FilterArgs& fa, cudaStream_t st,
                   const uint8_t* hflag, const float2* patch, DevStatus* status) {
  const FilterExtras ex{hflag, patch, nullptr, nullptr, 0.f};
  // the TMA path stages whole tiles; the listed texels' substitution would then
  // wait on a patch load per tile, which costs more than the plain loads that
  // fetch the patch beside the tile, so it takes only the plain filter
  if (fa.shape == 0 && !hflag && launch_filter_tma(false, in, out, R, fa, ex, status, st)) return;
  if (fa.shape != 1 && launch_tiled_r<1>(false, in, out, R, fa, ex, st)) return;
  dim3 b(32, 8), g((R + 31) / 32, (R + 7) / 8);
  if (hflag) {
    // the substituted input is composed into `out` first (the passes read it back)
    const int n = R * R;
    count_launches(1);
    compose_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, hflag, patch, out, n);
    in = out;
  }
  count_launches(1);
  filter_pass_kernel<false, false><<<g, b, 0, st>>>(in, tmp, R, fa);
  count_launches(1);
  filter_pass_kernel<true, false><<<g, b, 0, st>>>(tmp, out, R, fa);
}

void launch_filter_adjoint(const float2* gout, float2* tmp, float2* gin, int R, const FilterArgs& fa,
                           cudaStream_t st, const float2* fmap, float* gf, float ec, DevStatus* status) {
  const FilterExtras ex{nullptr, nullptr, fmap, gf, ec};
  if (fa.shape == 0 && launch_filter_tma(true, gout, gin, R, fa, ex, status, st)) return;
  if (fa.shape != 1 && launch_tiled_r<1>(true, gout, gin, R, fa, ex, st)) return;
  dim3 b(32, 8), g((R + 31) / 32, (R + 7) / 8);
  count_launches(1);
  filter_pass_kernel<true, true><<<g, b, 0, st>>>(gout, tmp, R, fa);
  count_launches(1);
  filter_pass_kernel<false, true><<<g, b, 0, st>>>(tmp, gin, R, fa);
  if (gf) {
    const int n = R * R;
    count_launches(1);
    fold_kernel<<<(n + 255) / 256, 256, 0, st>>>(fmap, gin, gf, n, ec);
  }
}

}  // namespace dsm
