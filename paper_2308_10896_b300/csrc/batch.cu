// Batched frames: n independent scenes advanced by one call per step
// (forward, L2 loss, backward of every scene).  Each scene keeps its own
// context (its scratch and saved state) and runs on its own stream, its views
// on the context's own streams forked from it; the scenes overlap one another
// and so do the views within each scene.  The first
// step with a given set of buffers runs eagerly, which sizes every context,
// and then records the same step into one CUDA graph; later steps with the
// same buffers replay the graph with a single launch.
#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <vector>
#include "dsm.h"
#include "kernels.h"

namespace dsm {
dsm_status tuning_search(dsm_tuning* cur, float* cur_ms,
                         const std::function<dsm_status(const dsm_tuning&, float*)>& measure);
}

struct dsm_batch {
  int n = 0;
  std::vector<dsm_ctx*> ctx;
  std::vector<cudaStream_t> ss;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t sig = 0;
  unsigned long long kernels_per_step = 0;
  std::string err = "ok";
};

namespace {

uint64_t mix_bytes(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// Everything a recorded step bakes in: buffers, sizes, host-side light and
// camera descriptions, parameters.
uint64_t step_signature(const dsm_batch_item* items, int n, const dsm_params* params) {
  uint64_t h = 1469598103934665603ull;
  h = mix_bytes(h, &n, sizeof(n));
  h = mix_bytes(h, params, sizeof(dsm_params));
  for (int i = 0; i < n; ++i) {
    const dsm_batch_item& it = items[i];
    h = mix_bytes(h, &it, sizeof(dsm_batch_item));
    if (it.lights && it.n_lights > 0) h = mix_bytes(h, it.lights, sizeof(dsm_light) * (size_t)it.n_lights);
  }
  return h;
}

dsm_status batch_fail(dsm_batch* b, dsm_status s, const std::string& m) {
  b->err = m;
  return s;
}

// Enqueue one step of every scene on the scene streams, forked from and joined
// back into `origin`.
dsm_status issue_step(dsm_batch* b, const dsm_batch_item* items, int n, const dsm_params* params,
                      cudaStream_t origin) {
  if (cudaEventRecord(b->ev_fork, origin) != cudaSuccess) return DSM_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    const dsm_batch_item& it = items[i];
    cudaStream_t s = b->ss[i];
    if (cudaStreamWaitEvent(s, b->ev_fork, 0) != cudaSuccess) return DSM_ERR_CUDA;
    dsm_params p = *params;
    p.stream = s;
    // the step's inputs from pinned host memory (copies inside the recorded step)
    const struct { const void* src; const void* dst; size_t bytes; } up[3] = {
        {it.host_verts, it.mesh.verts, sizeof(float) * 3 * (size_t)std::max(it.mesh.n_verts, 0)},
        {it.host_light_params, it.light_params, sizeof(float) * 6 * (size_t)std::max(it.n_lights, 0)},
        {it.host_albedo, it.mesh.albedo, sizeof(float) * 3 * (size_t)std::max(it.mesh.n_materials, 0)}};
    for (const auto& u : up)
      if (u.src && u.dst && u.bytes &&
          cudaMemcpyAsync(const_cast<void*>(u.dst), u.src, u.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return batch_fail(b, DSM_ERR_CUDA, "input upload of scene " + std::to_string(i));
    dsm_status st =
        dsm_render(b->ctx[i], &it.mesh, it.lights, it.light_params, it.n_lights, &it.camera, &p, it.image);
    if (st != DSM_OK) return batch_fail(b, st, std::string("scene ") + std::to_string(i) + ": " +
                                                   dsm_last_error(b->ctx[i]));
    // the loss and the backward in one (dL/dimage is formed where it is read)
    st = dsm_render_backward_l2(b->ctx[i], it.image, it.target, it.loss, it.dL_dverts, it.dL_dlight, it.dL_dalbedo);
    if (st != DSM_OK) return batch_fail(b, st, std::string("scene ") + std::to_string(i) + ": " +
                                                   dsm_last_error(b->ctx[i]));
    if (it.host_loss && cudaMemcpyAsync(it.host_loss, it.loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return batch_fail(b, DSM_ERR_CUDA, "loss download of scene " + std::to_string(i));
    if (cudaEventRecord(b->ev_join[i], s) != cudaSuccess) return DSM_ERR_CUDA;
    if (cudaStreamWaitEvent(origin, b->ev_join[i], 0) != cudaSuccess) return DSM_ERR_CUDA;
  }
  return DSM_OK;
}

}  // namespace

extern "C" {

dsm_status dsm_batch_create(dsm_batch** out, int32_t n) {
  if (!out || n < 1) return DSM_ERR_INVALID_ARG;
  *out = nullptr;
  dsm_batch* b = new dsm_batch();
  b->n = n;
  b->ctx.assign(n, nullptr);
  b->ss.assign(n, nullptr);
  b->ev_join.assign(n, nullptr);
  dsm_status st = DSM_OK;
  for (int i = 0; i < n && st == DSM_OK; ++i) {
    st = dsm_create(&b->ctx[i]);
    if (st == DSM_OK && cudaStreamCreateWithFlags(&b->ss[i], cudaStreamNonBlocking) != cudaSuccess)
      st = DSM_ERR_CUDA;
    if (st == DSM_OK && cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
      st = DSM_ERR_CUDA;
  }
  if (st == DSM_OK && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    st = DSM_ERR_CUDA;
  if (st != DSM_OK) {
    dsm_batch_destroy(b);
    return st;
  }
  *out = b;
  return DSM_OK;
}

void dsm_batch_destroy(dsm_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int i = 0; i < b->n; ++i) {
    if (b->ctx[i]) dsm_destroy(b->ctx[i]);
    if (b->ss[i]) cudaStreamDestroy(b->ss[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
}

dsm_ctx* dsm_batch_context(dsm_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->ctx[i];
}

dsm_status dsm_batch_step(dsm_batch* b, const dsm_batch_item* items, int32_t n, const dsm_params* params) {
  if (!b || !items || !params || n < 1 || n > b->n) return DSM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!items[i].image || !items[i].target || !items[i].loss)
      return batch_fail(b, DSM_ERR_INVALID_ARG, "scene " + std::to_string(i) + ": null image/target/loss buffer");
  cudaStream_t origin = (cudaStream_t)params->stream;
  const uint64_t sig = step_signature(items, n, params);
  if (b->exec && b->sig != 0 && sig == b->sig) {
    if (cudaGraphLaunch(b->exec, origin) != cudaSuccess) return batch_fail(b, DSM_ERR_CUDA, "graph launch");
    return DSM_OK;
  }
  // eager step: sizes every context (host synchronisations happen here only)
  dsm_status st = issue_step(b, items, n, params, origin);
  if (st != DSM_OK) return st;
  if (cudaStreamSynchronize(origin) != cudaSuccess) return batch_fail(b, DSM_ERR_CUDA, "eager step");
  for (int i = 0; i < n; ++i) {
    st = dsm_sync(b->ctx[i]);
    if (st != DSM_OK) return batch_fail(b, st, std::string("scene ") + std::to_string(i) + ": " +
                                                   dsm_last_error(b->ctx[i]));
  }
  // record the same step into a graph for the next calls
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const unsigned long long k0 = dsm_kernel_launches();
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return batch_fail(b, DSM_ERR_CUDA, "begin capture (the batch needs a stream other than the legacy default)");
  st = issue_step(b, items, n, params, origin);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
  if (st != DSM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess || !graph) return batch_fail(b, DSM_ERR_CUDA, "end capture");
  // node priorities: kernels keep the priority of the stream they were recorded on
  const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    b->exec = nullptr;
    return batch_fail(b, DSM_ERR_CUDA, "graph instantiate");
  }
  b->kernels_per_step = dsm_kernel_launches() - k0;
  b->sig = sig;
  return DSM_OK;
}

dsm_status dsm_batch_autotune(dsm_batch* b, const dsm_batch_item* items, int32_t n, const dsm_params* params,
                              int32_t reps) {
  if (!b || !items || !params || n < 1 || n > b->n) return DSM_ERR_INVALID_ARG;
  if (reps < 1 || reps > 100) return batch_fail(b, DSM_ERR_INVALID_ARG, "reps out of range");
  cudaStream_t origin = (cudaStream_t)params->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return batch_fail(b, DSM_ERR_CUDA, "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return batch_fail(b, DSM_ERR_CUDA, "event");
  }
  auto set_all = [&](const dsm_tuning& t) -> dsm_status {
    for (int i = 0; i < n; ++i) {
      const dsm_status st = dsm_set_tuning(b->ctx[i], &t);
      if (st != DSM_OK) return batch_fail(b, st, "tuning");
    }
    b->sig = 0;   // the next step records a new graph
    return DSM_OK;
  };
  // whole batched steps with shapes t: the eager step that records the graph
  // and one replay untimed, then `reps` timed replays
  auto measure = [&](const dsm_tuning& t, float* ms) -> dsm_status {
    dsm_status st = set_all(t);
    for (int k = 0; k < 2 && st == DSM_OK; ++k) st = dsm_batch_step(b, items, n, params);
    if (st == DSM_OK) st = dsm_batch_sync(b);
    if (st != DSM_OK) return st;
    if (cudaEventRecord(e0, origin) != cudaSuccess) return batch_fail(b, DSM_ERR_CUDA, "event record");
    for (int k = 0; k < reps && st == DSM_OK; ++k) st = dsm_batch_step(b, items, n, params);
    if (st != DSM_OK) return st;
    if (cudaEventRecord(e1, origin) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return batch_fail(b, DSM_ERR_CUDA, "event wait");
    st = dsm_batch_sync(b);
    if (st != DSM_OK) return st;
    float total = 0.f;
    if (cudaEventElapsedTime(&total, e0, e1) != cudaSuccess) return batch_fail(b, DSM_ERR_CUDA, "event time");
    *ms = total / reps;
    return DSM_OK;
  };
  dsm_tuning cur{};
  dsm_get_tuning(b->ctx[0], &cur);
  float cur_ms = 0.f;
  dsm_status st = measure(cur, &cur_ms);
  if (st == DSM_OK) st = dsm::tuning_search(&cur, &cur_ms, measure);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DSM_OK) return st;
  return set_all(cur);
}

dsm_status dsm_batch_sync(dsm_batch* b) {
  if (!b) return DSM_ERR_INVALID_ARG;
  for (int i = 0; i < b->n; ++i) {
    const dsm_status st = dsm_sync(b->ctx[i]);
    if (st != DSM_OK) return batch_fail(b, st, std::string("scene ") + std::to_string(i) + ": " +
                                                   dsm_last_error(b->ctx[i]));
  }
  return DSM_OK;
}

uint64_t dsm_batch_kernels_per_step(dsm_batch* b) { return b ? b->kernels_per_step : 0; }

const char* dsm_batch_last_error(dsm_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
