// Adam update for the vertex optimisation of the reconstruction workload
// (Kingma & Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015,
// Algorithm 1): first and second moment estimates of the gradient, bias
// correction, then the step lr * m^ / (sqrt(v^) + eps), all in place.
#include <cmath>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {
namespace {

// Grid-stride loop over the parameters; c1 = 1 - beta1^t and c2 = 1 - beta2^t
// come from the host.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace
}  // namespace dsm

extern "C" dsm_status dsm_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int32_t step,
                                    float lr, float beta1, float beta2, float eps, void* stream) {
  if (n < 0 || step < 1 || (n > 0 && (!params || !grads || !m || !v)) || !(lr >= 0.f) || !(beta1 >= 0.f) ||
      !(beta1 < 1.f) || !(beta2 >= 0.f) || !(beta2 < 1.f) || !(eps > 0.f))
    return DSM_ERR_INVALID_ARG;
  if (n == 0) return DSM_OK;
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 8);
  dsm::count_launches(1);
  dsm::adam_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, lr, beta1, beta2, eps, c1,
                                                                  c2);
  return cudaGetLastError() == cudaSuccess ? DSM_OK : DSM_ERR_CUDA;
}
