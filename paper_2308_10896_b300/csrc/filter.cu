// Separable moment filter m = G g (Eqs. moment1/moment2) and its adjoint
// G^T (Sec. 4: dm/dTheta = G grad f~).  G filters along x, then along y.
#include <cmath>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {

void make_filter_args(double sigma, int radius, int kind, int boundary, FilterArgs* fa) {
  int r = radius > 0 ? radius : (int)std::ceil(2.0 * sigma);
  if (r > 32) r = 32;
  fa->r = r;
  fa->boundary = boundary;
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

void launch_filter(const float2* in, float2* tmp, float2* out, int R, const FilterArgs& fa, cudaStream_t st) {
  dim3 b(32, 8), g((R + 31) / 32, (R + 7) / 8);
  count_launches(1);
  filter_pass_kernel<false, false><<<g, b, 0, st>>>(in, tmp, R, fa);
  count_launches(1);
  filter_pass_kernel<true, false><<<g, b, 0, st>>>(tmp, out, R, fa);
}

void launch_filter_adjoint(const float2* gout, float2* tmp, float2* gin, int R, const FilterArgs& fa,
                           cudaStream_t st) {
  dim3 b(32, 8), g((R + 31) / 32, (R + 7) / 8);
  count_launches(1);
  filter_pass_kernel<true, true><<<g, b, 0, st>>>(gout, tmp, R, fa);
  count_launches(1);
  filter_pass_kernel<false, true><<<g, b, 0, st>>>(tmp, gin, R, fa);
}

}  // namespace dsm
