// C-ABI entry points: context, scratch management and the orchestration of the
// forward (Alg. 1 per light, Alg. 2 + Lambert per camera pixel) and backward
// passes.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>
#include <functional>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {
std::atomic<unsigned long long> g_kernel_launches{0};

static const char* const kStageNames[] = {
    "setup", "bin_fill", "raster", "sm_antialias", "filter", "shade", "final_antialias",
    "bwd_clear", "bwd_final_antialias", "bwd_shade", "bwd_shade_scatter", "bwd_filter", "bwd_sm_antialias",
    "bwd_sm_interp", "bwd_vertex", "bwd_recompute"};
constexpr int kStages = (int)(sizeof(kStageNames) / sizeof(kStageNames[0]));
enum Stage { ST_SETUP, ST_BIN_FILL, ST_RASTER, ST_SM_AA, ST_FILTER, ST_SHADE, ST_FINAL_AA,
             ST_BWD_CLEAR, ST_BWD_FINAL_AA, ST_BWD_SHADE, ST_BWD_SHADE_SCATTER, ST_BWD_FILTER, ST_BWD_SM_AA,
             ST_BWD_SM_INTERP, ST_BWD_VERTEX, ST_BWD_RECOMPUTE };

void build_adjacency(const int32_t* tris, int T, std::vector<int32_t>& adj);
void build_vertex_faces(const int32_t* tris, int T, int V, std::vector<int32_t>& off, std::vector<int32_t>& lst);

// Device buffer that only grows.
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

inline size_t sil_bytes(size_t T) { return (T + 15) / 16 * 16; }

struct ViewBufs {
  int W = 0, H = 0, tilesX = 0, tilesY = 0;
  Buf clip, snap, depth, setup, orient, sil, count, offset, list, gbuf, gclip;
  Buf big_index, big_tri, big_acc;
  Buf aa_list, aa_ctr, hflag;   // antialiasing work list, its counter, per-pixel "listed" flag
  Buf rim;                      // the raster tiles' rims for the detection's seam pass
  Buf color, gcolor, pgrad;     // camera views: colour before the final antialiasing, its adjoint, pixel gradients
  int list_cap = 0;
  BinShape bs{kTileLog2Default, kBigTilesDefault};
  // raster work units and the key slots of tiles split over several units
  Buf units, tile_done, skey;
  int units_cap = 0, slot_cap = 0;
  AAWork aa_work() { return AAWork{aa_list.as<int>(), aa_ctr.as<int>()}; }
  // the clip buffer holds V clip coordinates, then V float-float screen positions
  float4* scr(int V) { return clip.as<float4>() + std::max(V, 1); }
  // the sil buffer holds T silhouette masks, then (16-byte aligned) the packed flags
  uint32_t* silbits(int T) { return reinterpret_cast<uint32_t*>(sil.as<uint8_t>() + sil_bytes(std::max(T, 1))); }
  RimBufs rim_bufs() {
    const size_t keys = (size_t)tilesX * tilesY * 4 * (1 << bs.tile_log2);
    return RimBufs{rim.as<unsigned long long>(), reinterpret_cast<unsigned*>(rim.as<unsigned long long>() + keys)};
  }
  RasterUnits raster_units() {
    return RasterUnits{units.as<int4>(), units_cap, slot_cap, tile_done.as<int>(),
                       skey.as<unsigned long long>()};
  }
};

struct LightBufs {
  Buf fmap, ftilde, tmp, mom, gm, gft;
  FilterArgs fa;
  int res = 0;
};

}  // namespace dsm

using namespace dsm;

struct dsm_ctx {
  int device = 0;
  std::string err = "ok";
  int topo_T = -1, topo_V = -1;
  Buf adj, vf_off, vf_list;
  ViewBufs view[kMaxViews];
  LightBufs light[kMaxLightViews];
  Buf lights_dev, viewM, viewMlo, status, vnormal, vnlen, gnormal, gpos, gN, gface, gQ, gdirect, red;
  Buf scratch_dverts, scratch_dlight, scratch_dalbedo, filter_tmp, stats;
  DevStatus* hstatus = nullptr;
  // state of the last forward
  bool have_fwd = false;
  // the forward already zeroed every light's dL/dm accumulator and (stored
  // mode) the backward's internal accumulators, beside the light views'
  // chains; the first backward after it need not
  bool gm_zeroed = false;
  bool acc_zeroed = false;
  dsm_mesh mesh{};
  dsm_light lights[DSM_MAX_LIGHTS]{};   // the caller's lights
  int n_user = 0;                        // their number
  // light views: one per directional or spot light, six (cube faces) per point light
  int view_user[kMaxLightViews]{};       // caller's light of each light view
  int view_face[kMaxLightViews]{};       // its cube face, or -1
  int L = 0, C = 0;                      // light views, cameras
  dsm_camera cams[DSM_MAX_CAMERAS]{};
  dsm_params params{};
  // raster tile sides, big-triangle threshold and filter shape (dsm_autotune)
  dsm_tuning tuning{1 << kTileLog2Default, 1 << kTileLog2Default, kBigTilesDefault, 0};
  // recompute_in_backward: the views share two buffer sets (one for the
  // lights, one for the cameras) and the backward rebuilds what it reads
  bool recompute = false;
  // diagnostic gradient masks (dsm_set_grad_mask)
  int grad_mask = 0;
  cudaStream_t stream = nullptr;
  uint64_t sized_sig = 0;
  // internal streams: one per view (lights, then cameras), fork/join events
  cudaStream_t vs[kMaxViews] = {};
  // per camera: the final antialiasing adjoint and the shading adjoint of its
  // listed pixels, beside the shading adjoint's grid pass; at the device's
  // highest stream priority, so that the listed pixels' pass takes SMs as the
  // grid pass's CTAs retire instead of waiting for all of them
  cudaStream_t cside[DSM_MAX_CAMERAS] = {};
  cudaEvent_t ev_cside[DSM_MAX_CAMERAS] = {}, ev_cside_done[DSM_MAX_CAMERAS] = {};
  cudaStream_t aux = nullptr;            // side stream of the backward's output clear
  cudaEvent_t ev_aux = nullptr, ev_aux_done = nullptr;
  bool aux_pending = false;              // the shading adjoints wait for ev_aux_done
  cudaEvent_t ev_fork = nullptr, ev_bfork = nullptr, ev_sil = nullptr, ev_join[kMaxViews] = {};
  // per-stage timing (stage_override >= 0 books every stage under that one)
  bool prof = false;
  int stage_override = -1;
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> free_events;
};

namespace {

dsm_status fail(dsm_ctx* c, dsm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

dsm_status cuda_fail(dsm_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, DSM_ERR_OOM, m);
  return fail(c, DSM_ERR_CUDA, m);
}

#define DSM_CHECK(call)                                         \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call);  \
  } while (0)

// One launch that zeroes several buffers: segment blockIdx.y, 16-byte stores
// over its aligned body, 4-byte stores for an unaligned head and the tail.
constexpr int kMaxClear = 96;
struct ClearList {
  float* p[kMaxClear];
  long long n[kMaxClear];     // floats
  int count;
};

__global__ void clear_kernel(ClearList c) {
  const int s = blockIdx.y;
  if (s >= c.count) return;
  float* p = c.p[s];
  const long long n = c.n[s];
  const long long head = min(n, (long long)(((16 - ((uintptr_t)p & 15)) & 15) / 4));
  const long long body = (n - head) / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 < head) p[t0] = 0.f;
  float4* q = reinterpret_cast<float4*>(p + head);
  for (long long k = t0; k < body; k += stride) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long tail0 = head + 4 * body;
  if (t0 < n - tail0) p[tail0 + t0] = 0.f;
}

struct Clearer {
  ClearList list{};
  long long largest = 0;
  void add(void* p, size_t bytes) {
    if (!p || bytes == 0) return;
    list.p[list.count] = static_cast<float*>(p);
    list.n[list.count] = (long long)(bytes / 4);
    largest = std::max(largest, (long long)(bytes / 4));
    ++list.count;
  }
  void launch(cudaStream_t st) {
    if (!list.count) return;
    const long long per = 256LL * 4;
    const int gx = (int)std::min<long long>((largest + per - 1) / per, 1184);
    count_launches(1);
    clear_kernel<<<dim3(std::max(gx, 1), list.count), 256, 0, st>>>(list);
  }
};

cudaEvent_t take_event(dsm_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Event pair around one stage of one call (no-op unless profiling is on).
struct StageTimer {
  dsm_ctx* c;
  cudaStream_t st;
  int stage;
  cudaEvent_t a = nullptr;
  StageTimer(dsm_ctx* c_, int stage_, cudaStream_t st_)
      : c(c_), st(st_), stage(c_->stage_override >= 0 ? c_->stage_override : stage_) {
    if (c->prof && (a = take_event(c))) cudaEventRecord(a, st);
  }
  void stop() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (b) {
      cudaEventRecord(b, st);
      c->recs.push_back({stage, a, b});
    } else {
      c->free_events.push_back(a);
    }
    a = nullptr;
  }
  ~StageTimer() { stop(); }
};

cudaError_t ensure_streams(dsm_ctx* c) {
  if (c->ev_fork) return cudaSuccess;
  cudaError_t e;
  for (auto& v : c->vs)
    if ((e = cudaStreamCreateWithFlags(&v, cudaStreamNonBlocking)) != cudaSuccess) return e;
  int least = 0, greatest = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return e;
  for (int k = 0; k < DSM_MAX_CAMERAS; ++k) {
    if ((e = cudaStreamCreateWithPriority(&c->cside[k], cudaStreamNonBlocking, greatest)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&c->ev_cside[k], cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&c->ev_cside_done[k], cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  if ((e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&c->ev_bfork, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&c->ev_sil, cudaEventDisableTiming)) != cudaSuccess) return e;
  for (auto& ev : c->ev_join)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  // (the clear of the caller's outputs: a short launch that the shading adjoint waits for)
  if ((e = cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, greatest)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&c->ev_aux_done, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Stream of view w: its own stream, or the caller's while stage profiling is
// on (profiling serialises the views so that each stage's events bracket only
// its own kernels).
cudaStream_t view_stream(const dsm_ctx* c, int w, cudaStream_t st) {
  return c->prof ? st : c->vs[w];
}

// The streams of views [w0, w1) wait for the work enqueued so far on st.
cudaError_t fork_views(dsm_ctx* c, cudaStream_t st, cudaEvent_t ev, int w0, int w1) {
  if (c->prof || w1 <= w0) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev, st);
  for (int w = w0; w < w1 && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(c->vs[w], ev, 0);
  return e;
}

// st waits for the work enqueued so far on the streams of views [w0, w1).
cudaError_t join_views(dsm_ctx* c, cudaStream_t st, int w0, int w1) {
  if (c->prof) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int w = w0; w < w1 && e == cudaSuccess; ++w) {
    e = cudaEventRecord(c->ev_join[w], c->vs[w]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_join[w], 0);
  }
  return e;
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

namespace dsm {
// Coordinate search over the kernel shapes: from *cur (timed as *cur_ms by
// the caller), each knob in turn -- light tile, camera tile, bin depth from
// {4, 16, 64}, filter shape -- is set to each of its other values and kept
// when `measure` reports a step at least 2 % faster.
dsm_status tuning_search(dsm_tuning* cur, float* cur_ms,
                         const std::function<dsm_status(const dsm_tuning&, float*)>& measure) {
  const int32_t tiles[2] = {16, 32}, bins[3] = {4, 16, 64}, shapes[3] = {0, 1, 2};
  for (int knob = 0; knob < 4; ++knob) {
    const int32_t* vals = knob < 2 ? tiles : (knob == 2 ? bins : shapes);
    const int nv = knob >= 2 ? 3 : 2;
    const dsm_tuning base = *cur;
    for (int k = 0; k < nv; ++k) {
      dsm_tuning cand = base;
      int32_t* field = knob == 0 ? &cand.light_tile
                     : knob == 1 ? &cand.camera_tile
                     : knob == 2 ? &cand.big_tiles : &cand.filter_shape;
      if (*field == vals[k]) continue;
      *field = vals[k];
      float ms = 0.f;
      const dsm_status s = measure(cand, &ms);
      if (s != DSM_OK) return s;
      if (ms < 0.98f * *cur_ms) {
        *cur = cand;
        *cur_ms = ms;
      }
    }
  }
  return DSM_OK;
}
}  // namespace dsm

extern "C" {

dsm_status dsm_create(dsm_ctx** out) {
  if (!out) return DSM_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return DSM_ERR_CUDA;
  dsm_ctx* ctx = new dsm_ctx();
  ctx->device = dev;
  e = cudaMallocHost(&ctx->hstatus, sizeof(DevStatus));
  if (e != cudaSuccess) { delete ctx; return DSM_ERR_CUDA; }
  memset(ctx->hstatus, 0, sizeof(DevStatus));
  e = ctx->status.ensure(sizeof(DevStatus));
  if (e != cudaSuccess) { cudaFreeHost(ctx->hstatus); delete ctx; return DSM_ERR_OOM; }
  e = cudaMemset(ctx->status.p, 0, sizeof(DevStatus));
  if (e != cudaSuccess) { cudaFreeHost(ctx->hstatus); delete ctx; return DSM_ERR_CUDA; }
  *out = ctx;
  return DSM_OK;
}

void dsm_destroy(dsm_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  Buf* bufs[] = {&ctx->adj, &ctx->vf_off, &ctx->vf_list, &ctx->lights_dev, &ctx->viewM, &ctx->viewMlo, &ctx->status,
                 &ctx->vnormal, &ctx->vnlen, &ctx->gnormal, &ctx->gpos, &ctx->gN, &ctx->gface, &ctx->gQ, &ctx->gdirect,
                 &ctx->scratch_dverts, &ctx->scratch_dlight, &ctx->scratch_dalbedo, &ctx->filter_tmp, &ctx->red, &ctx->stats};
  for (Buf* b : bufs) b->release();
  for (auto& v : ctx->view) {
    Buf* vb[] = {&v.clip, &v.snap, &v.depth, &v.setup, &v.orient, &v.sil, &v.count, &v.offset, &v.list,
                 &v.gbuf, &v.gclip, &v.big_index, &v.big_tri, &v.big_acc, &v.aa_list, &v.aa_ctr,
                 &v.hflag, &v.rim, &v.color, &v.gcolor, &v.pgrad, &v.units, &v.tile_done, &v.skey};
    for (Buf* b : vb) b->release();
  }
  for (auto& l : ctx->light) {
    Buf* lb[] = {&l.fmap, &l.ftilde, &l.tmp, &l.mom, &l.gm, &l.gft};
    for (Buf* b : lb) b->release();
  }
  if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto v : ctx->vs) if (v) cudaStreamDestroy(v);
  for (int k = 0; k < DSM_MAX_CAMERAS; ++k) {
    if (ctx->cside[k]) cudaStreamDestroy(ctx->cside[k]);
    if (ctx->ev_cside[k]) cudaEventDestroy(ctx->ev_cside[k]);
    if (ctx->ev_cside_done[k]) cudaEventDestroy(ctx->ev_cside_done[k]);
  }
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->ev_aux) cudaEventDestroy(ctx->ev_aux);
  if (ctx->ev_aux_done) cudaEventDestroy(ctx->ev_aux_done);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_bfork) cudaEventDestroy(ctx->ev_bfork);
  if (ctx->ev_sil) cudaEventDestroy(ctx->ev_sil);
  for (auto e : ctx->ev_join) if (e) cudaEventDestroy(e);
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  delete ctx;
}

const char* dsm_last_error(dsm_ctx* ctx) {
  static thread_local std::string copy;
  copy = ctx ? ctx->err : std::string("null context");
  return copy.c_str();
}

dsm_status dsm_set_topology(dsm_ctx* ctx, const int32_t* tris, int32_t n_tris, int32_t n_verts) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (n_tris < 0 || n_verts < 0 || (n_tris > 0 && !tris))
    return fail(ctx, DSM_ERR_INVALID_ARG, "bad topology arguments");
  std::vector<int32_t> h((size_t)n_tris * 3);
  if (n_tris) DSM_CHECK(cudaMemcpy(h.data(), tris, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int32_t v : h)
    if (v < 0 || v >= n_verts) return fail(ctx, DSM_ERR_INVALID_ARG, "triangle index out of range");
  std::vector<int32_t> adj, off, lst;
  build_adjacency(h.data(), n_tris, adj);
  build_vertex_faces(h.data(), n_tris, n_verts, off, lst);
  DSM_CHECK(ctx->adj.ensure(std::max<size_t>(adj.size(), 1) * 4));
  DSM_CHECK(ctx->vf_off.ensure(off.size() * 4));
  DSM_CHECK(ctx->vf_list.ensure(std::max<size_t>(lst.size(), 1) * 4));
  if (!adj.empty()) DSM_CHECK(cudaMemcpy(ctx->adj.p, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice));
  DSM_CHECK(cudaMemcpy(ctx->vf_off.p, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
  if (!lst.empty()) DSM_CHECK(cudaMemcpy(ctx->vf_list.p, lst.data(), lst.size() * 4, cudaMemcpyHostToDevice));
  ctx->topo_T = n_tris;
  ctx->topo_V = n_verts;
  ctx->have_fwd = false;
  ctx->sized_sig = 0;
  return DSM_OK;
}

static dsm_status check_args(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights,
                             const float* light_params, int32_t n_lights, const dsm_camera* cams, int32_t n_cams,
                             const dsm_params* params, float* const* images) {
  if (!mesh || !cams || !params || !images) return fail(ctx, DSM_ERR_INVALID_ARG, "null argument");
  if (n_lights < 0 || n_lights > DSM_MAX_LIGHTS) return fail(ctx, DSM_ERR_INVALID_ARG, "n_lights out of range");
  if (n_cams < 1 || n_cams > DSM_MAX_CAMERAS) return fail(ctx, DSM_ERR_INVALID_ARG, "n_cameras out of range");
  if (n_lights > 0 && (!lights || !light_params)) return fail(ctx, DSM_ERR_INVALID_ARG, "null light arrays");
  if (mesh->n_verts < 0 || mesh->n_tris < 0) return fail(ctx, DSM_ERR_INVALID_ARG, "negative mesh size");
  if ((mesh->n_verts > 0 && !mesh->verts) || (mesh->n_tris > 0 && !mesh->tris))
    return fail(ctx, DSM_ERR_INVALID_ARG, "null mesh arrays");
  if (mesh->n_materials < 1 || !mesh->albedo) return fail(ctx, DSM_ERR_INVALID_ARG, "no albedo table");
  if (mesh->n_tris != ctx->topo_T || mesh->n_verts != ctx->topo_V)
    return fail(ctx, DSM_ERR_NO_TOPOLOGY, "dsm_set_topology was not called for this mesh size");
  for (int c = 0; c < n_cams; ++c) {
    if (!images[c]) return fail(ctx, DSM_ERR_INVALID_ARG, "null image");
    const dsm_camera& cam = cams[c];
    if (cam.width < 1 || cam.height < 1 || cam.width > 16384 || cam.height > 16384)
      return fail(ctx, DSM_ERR_INVALID_ARG, "camera size out of range");
  }
  int views = 0;
  for (int l = 0; l < n_lights; ++l) {
    const dsm_light& L = lights[l];
    if (L.type != 0 && L.type != 1 && L.type != 2) return fail(ctx, DSM_ERR_INVALID_ARG, "unknown light type");
    views += L.type == 2 ? 6 : 1;
    if (views > DSM_MAX_LIGHT_VIEWS) return fail(ctx, DSM_ERR_INVALID_ARG, "more than 24 shadow-map views");
    if (L.res < 1 || L.res > 16384) return fail(ctx, DSM_ERR_INVALID_ARG, "shadow-map size out of range");
    if (!(L.far_plane > L.near_plane)) return fail(ctx, DSM_ERR_INVALID_ARG, "far must exceed near");
    if (L.type != 0 && !(L.near_plane > 0.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "perspective near must be > 0");
    if (L.type == 0 && !(L.ortho_half > 0.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "ortho_half must be positive");
    if (L.type == 1 && !(L.fov_y_deg > 0.f && L.fov_y_deg < 180.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "bad fov");
  }
  if (params->filter_kind != 0 && params->filter_kind != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "filter_kind");
  if (params->filter_boundary != 0 && params->filter_boundary != 1)
    return fail(ctx, DSM_ERR_INVALID_ARG, "filter_boundary");
  for (int l = 0; l < n_lights; ++l)
    if (!filter_args_ok(lights[l].sigma, lights[l].radius, params->filter_kind, params->filter_boundary))
      return fail(ctx, DSM_ERR_INVALID_ARG,
                  "light filter: radius above 32, or no finite sigma > 0 where the filter needs one");
  if (params->recompute_in_backward != 0 && params->recompute_in_backward != 1)
    return fail(ctx, DSM_ERR_INVALID_ARG, "recompute_in_backward");
  if (!(params->min_variance >= 0.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "min_variance");
  if (params->moments != 0 && params->moments != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "moments");
  if (params->moments == 1 && !(params->exponent > 0.f && params->exponent <= 40.f))
    return fail(ctx, DSM_ERR_INVALID_ARG, "exponent of the exponential moments outside (0, 40]");
  return DSM_OK;
}

// Raster work units for the view's tiles and list capacity.  The per-tile
// counters and the key slots start at zero and every frame leaves them so;
// they are zeroed here when (re)allocated, never while a frame is recorded.
static dsm_status ensure_units(dsm_ctx* ctx, ViewBufs& v, bool reset = false) {
  const size_t tiles = (size_t)v.tilesX * v.tilesY;
  v.units_cap = (int)(tiles + (size_t)v.list_cap / kRasterBatch + 1);
  v.slot_cap = v.list_cap / (kRasterBatch + 1) + 1;
  DSM_CHECK(v.units.ensure((size_t)v.units_cap * sizeof(int4)));
  const size_t done_cap = v.tile_done.cap, key_cap = v.skey.cap;
  DSM_CHECK(v.tile_done.ensure(tiles * 4));
  DSM_CHECK(v.skey.ensure((size_t)v.slot_cap * 1024 * sizeof(unsigned long long)));
  if (reset || v.tile_done.cap != done_cap) DSM_CHECK(cudaMemset(v.tile_done.p, 0, v.tile_done.cap));
  if (reset || v.skey.cap != key_cap) DSM_CHECK(cudaMemset(v.skey.p, 0, v.skey.cap));
  return DSM_OK;
}

static dsm_status ensure_view(dsm_ctx* ctx, ViewBufs& v, int W, int H, int V, int T, bool is_light) {
  v.W = W;
  v.H = H;
  const int side = is_light ? ctx->tuning.light_tile : ctx->tuning.camera_tile;
  v.bs.tile_log2 = side == 16 ? 4 : 5;
  v.bs.big_tiles = ctx->tuning.big_tiles;
  const int tile = 1 << v.bs.tile_log2;
  v.tilesX = (W + tile - 1) / tile;
  v.tilesY = (H + tile - 1) / tile;
  const size_t tiles = (size_t)v.tilesX * v.tilesY;
  const size_t Vn = std::max(V, 1), Tn = std::max(T, 1);
  DSM_CHECK(v.clip.ensure(2 * Vn * sizeof(float4)));   // clip, then the float-float screen positions
  DSM_CHECK(v.snap.ensure(Vn * sizeof(VertSnap)));
  DSM_CHECK(v.setup.ensure(Tn * sizeof(TriSetup)));
  DSM_CHECK(v.orient.ensure(Tn));
  DSM_CHECK(v.sil.ensure(sil_bytes(Tn) + 4 * ((Tn + 31) / 32)));   // masks, then the packed flags
  DSM_CHECK(v.count.ensure(tiles * 4));
  DSM_CHECK(v.offset.ensure(2 * tiles * 4));
  DSM_CHECK(v.gbuf.ensure((size_t)W * H * sizeof(float4)));
  DSM_CHECK(v.gclip.ensure(Vn * sizeof(float4)));
  DSM_CHECK(v.big_index.ensure(Tn * 4));
  DSM_CHECK(v.big_tri.ensure(kMaxBig * 4));
  DSM_CHECK(v.big_acc.ensure((size_t)kMaxBig * kBigSlots * (is_light ? kBigStrideSm : kBigStrideCam) * 4));
  if (is_light) {
    DSM_CHECK(v.depth.ensure(Vn * 4));
  } else {
    DSM_CHECK(v.color.ensure((size_t)W * H * sizeof(float4)));
  }
  DSM_CHECK(v.aa_list.ensure((size_t)W * H * 4));
  DSM_CHECK(v.aa_ctr.ensure(sizeof(int)));
  DSM_CHECK(v.hflag.ensure((size_t)W * H));
  DSM_CHECK(v.rim.ensure(tiles * (4 * (size_t)tile * 8 + 4 * 4)));
  if (v.list_cap == 0) {
    const size_t cap = 2 * Tn + 2 * tiles + 1024;
    DSM_CHECK(v.list.ensure(cap * 4));
    v.list_cap = (int)cap;
  }
  return ensure_units(ctx, v);
}

namespace {

// Camera buffer set under recomputation (view[0] is the light set).
constexpr int kCamSlot = kMaxLightViews;

// Buffers of view w (lights 0..L-1, then cameras L..L+C-1).  Under
// recomputation every light view uses view[0] and every camera view
// view[kCamSlot], one after the other.
ViewBufs& vbuf(dsm_ctx* ctx, int w) {
  if (!ctx->recompute) return ctx->view[w];
  return ctx->view[w < ctx->L ? 0 : kCamSlot];
}

// Working maps of light l (f, the antialiased patch, filter scratch, dL/df~):
// shared by all lights under recomputation.  The moments and their adjoint
// stay per light (every camera reads all of them).
LightBufs& lwork(dsm_ctx* ctx, int l) { return ctx->recompute ? ctx->light[0] : ctx->light[l]; }

bool view_is_light(const dsm_ctx* ctx, int w) { return w < ctx->L; }

// Sizes the buffer set of view w for that view (buffers only grow).
dsm_status prepare_view(dsm_ctx* ctx, int w) {
  const int L = ctx->L;
  const bool light = view_is_light(ctx, w);
  const int W = light ? ctx->lights[ctx->view_user[w]].res : ctx->cams[w - L].width;
  const int H = light ? ctx->lights[ctx->view_user[w]].res : ctx->cams[w - L].height;
  return ensure_view(ctx, vbuf(ctx, w), W, H, ctx->mesh.n_verts, ctx->mesh.n_tris, light);
}

dsm_status prepare_light(dsm_ctx* ctx, int l) {
  const dsm_light& Lu = ctx->lights[ctx->view_user[l]];
  const int R = Lu.res;
  const size_t R2 = (size_t)R * R * sizeof(float2);
  LightBufs& wk = lwork(ctx, l);
  DSM_CHECK(wk.fmap.ensure(R2));
  DSM_CHECK(wk.ftilde.ensure(R2));
  DSM_CHECK(wk.tmp.ensure(R2));
  LightBufs& lb = ctx->light[l];
  DSM_CHECK(lb.mom.ensure(R2));
  DSM_CHECK(lb.gm.ensure(R2));
  lb.res = R;
  make_filter_args(Lu.sigma, Lu.radius, ctx->params.filter_kind, ctx->params.filter_boundary, &lb.fa);
  lb.fa.shape = ctx->tuning.filter_shape;
  return DSM_OK;
}

dsm_status grow_list(dsm_ctx* ctx, ViewBufs& v, long long need) {
  if (need <= v.list_cap) return DSM_OK;
  const long long cap = need + need / 2 + 1024;
  if (cap > 0x7fffffffLL) return fail(ctx, DSM_ERR_CAPACITY, "tile list above 2^31 entries");
  DSM_CHECK(v.list.ensure((size_t)cap * 4));
  v.list_cap = (int)cap;
  // (a frame that overflowed the old list may have left tiles unmerged)
  return ensure_units(ctx, v, true);
}

// Exponent of the moments' warp (0: variance shadow maps).
float warp_exponent(const dsm_ctx* ctx) { return ctx->params.moments == 1 ? ctx->params.exponent : 0.f; }

AAArgs aa_args(const dsm_ctx* ctx, ViewBufs& v) {
  return AAArgs{v.gbuf.as<float4>(), v.W, v.H, ctx->mesh.tris, v.sil.as<uint8_t>(), v.snap.as<VertSnap>(),
                v.clip.as<float4>(), v.scr(ctx->mesh.n_verts)};
}

// Transform, triangle setup and silhouettes of views [w0, w0 + n) in one fused
// pass, which also empties their tile counters and antialiasing lists.
ViewSetupArgs view_setup_args(dsm_ctx* ctx, int w0, int n) {
  ViewSetupArgs va{};
  va.n = n;
  va.view0 = w0;
  for (int k = 0; k < n; ++k) {
    const int w = w0 + k;
    ViewBufs& v = vbuf(ctx, w);
    va.W[k] = v.W; va.H[k] = v.H; va.tiles[k] = v.tilesX * v.tilesY;
    va.clip[k] = v.clip.as<float4>();
    va.scr[k] = v.scr(ctx->mesh.n_verts);
    va.snap[k] = v.snap.as<VertSnap>();
    va.depth[k] = view_is_light(ctx, w) ? v.depth.as<float>() : nullptr;
    va.setup[k] = v.setup.as<TriSetup>();
    va.orient[k] = v.orient.as<int8_t>();
    va.sil[k] = v.sil.as<uint8_t>();
    va.silbits[k] = v.silbits(ctx->mesh.n_tris);
    va.count[k] = v.count.as<int>();
    va.aa_count[k] = v.aa_ctr.as<int>();
    va.tilesX[k] = v.tilesX;
    va.bs[k] = v.bs;
    va.big_index[k] = v.big_index.as<int>();
    va.big_tri[k] = v.big_tri.as<int>();
  }
  return va;
}

void setup_views(dsm_ctx* ctx, int w0, int n, cudaStream_t st, bool silhouettes = true) {
  const dsm_mesh& m = ctx->mesh;
  launch_setup_all(m.verts, m.n_verts, m.tris, m.n_tris, ctx->adj.as<int>(), ctx->viewM.as<float>() + 20 * w0,
                   ctx->viewMlo.as<float>() + 16 * w0,
                   view_setup_args(ctx, w0, n), ctx->status.as<DevStatus>(), silhouettes, st);
}

void silhouette_views(dsm_ctx* ctx, int w0, int n, cudaStream_t st) {
  launch_silhouettes_all(ctx->adj.as<int>(), ctx->mesh.n_tris, view_setup_args(ctx, w0, n), st);
}

// List segments of view w's tiles; with `write`, also its big triangles' list
// entries and the raster work units.
void alloc_view(dsm_ctx* ctx, int w, bool write, cudaStream_t st) {
  ViewBufs& v = vbuf(ctx, w);
  StageTimer t(ctx, ST_SETUP, st);
  launch_alloc_units(v.count.as<int>(), v.tilesX * v.tilesY, v.offset.as<int>(), ctx->status.as<DevStatus>(), w,
                     v.setup.as<TriSetup>(), v.big_tri.as<int>(), v.tilesX, v.bs.tile_log2, v.list.as<int>(),
                     v.list_cap, v.raster_units(), write, st);
}

// First frame of a scene size: the list capacities from the segments' totals
// (one host read), then the segments again with the list entries and units.
// The views' streams have been joined into st.
dsm_status size_lists(dsm_ctx* ctx, int w0, int n, cudaStream_t st) {
  DSM_CHECK(cudaMemcpyAsync(ctx->hstatus, ctx->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  DSM_CHECK(cudaStreamSynchronize(st));
  DevStatus* ds = ctx->status.as<DevStatus>();
  for (int w = w0; w < w0 + n; ++w) {
    dsm_status s = grow_list(ctx, vbuf(ctx, w), ctx->hstatus->needed_pairs[w]);
    if (s != DSM_OK) return s;
    DSM_CHECK(cudaMemsetAsync(&ds->needed_pairs[w], 0, sizeof(int), st));
    alloc_view(ctx, w, true, st);
  }
  return DSM_OK;
}

// Whether view w antialiases: a light view its shadow map, a camera its image.
bool view_aa(const dsm_ctx* ctx, int w) {
  return view_is_light(ctx, w) ? ctx->params.aa_shadow != 0 : ctx->params.aa_final != 0;
}

// Bin fill and raster of view w (a light view also writes f, f^2), with the
// antialiasing detection when the view antialiases (its silhouettes must be
// complete on st).
void raster_view(dsm_ctx* ctx, int w, cudaStream_t st) {
  ViewBufs& v = vbuf(ctx, w);
  const bool light = view_is_light(ctx, w);
  const bool aa = view_aa(ctx, w);
  DevStatus* ds = ctx->status.as<DevStatus>();
  {
    StageTimer t(ctx, ST_BIN_FILL, st);
    launch_bin_fill(v.setup.as<TriSetup>(), ctx->mesh.n_tris, v.tilesX, v.bs, v.count.as<int>(), v.offset.as<int>(),
                    v.list.as<int>(), v.list_cap, ds, v.big_index.as<int>(), st);
  }
  StageTimer t(ctx, ST_RASTER, st);
  launch_raster(v.setup.as<TriSetup>(), v.list.as<int>(), v.tilesX, v.bs.tile_log2, v.W, v.H, v.clip.as<float4>(),
                v.scr(ctx->mesh.n_verts), ctx->mesh.tris, v.gbuf.as<float4>(),
                light ? v.depth.as<float>() : nullptr, light ? lwork(ctx, w).fmap.as<float2>() : nullptr,
                warp_exponent(ctx), v.raster_units(), ds, w, v.silbits(ctx->mesh.n_tris), aa ? v.hflag.as<uint8_t>() : nullptr,
                v.aa_work(), v.rim_bufs(), st);
  if (aa)
    launch_aa_seam(aa_args(ctx, v), v.tilesX, v.tilesY, v.bs.tile_log2, v.rim_bufs(), v.silbits(ctx->mesh.n_tris),
                   v.hflag.as<uint8_t>(), v.aa_work(), st);
}

// Alg. 1 after the raster: antialiasing of f, f^2 at the listed texels, then
// the moment filter (f~ = f except at the listed texels, whose values the list
// pass left in ftilde).
void light_maps(dsm_ctx* ctx, int l, cudaStream_t st) {
  ViewBufs& v = vbuf(ctx, l);
  LightBufs& wk = lwork(ctx, l);
  LightBufs& lb = ctx->light[l];
  const bool aa = ctx->params.aa_shadow != 0;
  {
    StageTimer t(ctx, ST_SM_AA, st);
    if (aa) launch_aa_forward2_list(aa_args(ctx, v), wk.fmap.as<float2>(), wk.ftilde.as<float2>(), v.aa_work(), st);
  }
  StageTimer t(ctx, ST_FILTER, st);
  launch_filter(wk.fmap.as<float2>(), wk.tmp.as<float2>(), lb.mom.as<float2>(), v.W, lb.fa, st,
                aa ? v.hflag.as<uint8_t>() : nullptr, wk.ftilde.as<float2>(), ctx->status.as<DevStatus>());
}

ShadeArgs shade_args(dsm_ctx* ctx, int c) {
  ViewBufs& cv = vbuf(ctx, ctx->L + c);
  const dsm_mesh& m = ctx->mesh;
  ShadeArgs sa{};
  sa.gbuf = cv.gbuf.as<float4>();
  sa.W = cv.W; sa.H = cv.H;
  sa.verts = m.verts; sa.tris = m.tris; sa.tri_mat = m.tri_material;
  sa.albedo = m.albedo; sa.n_mat = m.n_materials;
  sa.vnormal = ctx->vnormal.as<float>();
  sa.cam_clip = cv.clip.as<float4>();
  sa.cam_scr = cv.scr(m.n_verts);
  sa.lights = ctx->lights_dev.as<LightDev>(); sa.L = ctx->L;
  for (int l = 0; l < ctx->L; ++l) { sa.mom[l] = ctx->light[l].mom.as<float2>(); sa.res[l] = ctx->light[l].res; }
  sa.min_variance = ctx->params.min_variance;
  sa.ec = warp_exponent(ctx);
  return sa;
}

// Block-sum slots: dQ (20 per light view), direct terms (3), albedo (3 per
// material, when their block sums fit shared memory), the squared error (1).
int n_mat_red_of(const dsm_ctx* ctx) { return ctx->mesh.n_materials <= kMaxSharedMat ? ctx->mesh.n_materials : 0; }
int loss_index_of(const dsm_ctx* ctx) { return 23 * ctx->L + 3 * n_mat_red_of(ctx); }
int red_stride_of(const dsm_ctx* ctx) { return loss_index_of(ctx) + 1; }

ShadeGradArgs grad_args(dsm_ctx* ctx, int c, const ImageGrad& gimage, float* dalbedo, int red_stride) {
  ViewBufs& cv = vbuf(ctx, ctx->L + c);
  ShadeGradArgs ga{};
  ga.gcolor = cv.gcolor.as<float4>();
  ga.gimage = gimage;
  ga.hflag = ctx->params.aa_final ? cv.hflag.as<uint8_t>() : nullptr;
  ga.loss_index = gimage.g ? -1 : loss_index_of(ctx);
  ga.gpos = ctx->gpos.as<float4>();
  ga.gnormal = ctx->gnormal.as<float4>();
  ga.gclip = cv.gclip.as<float4>();
  ga.dalbedo = dalbedo;
  for (int l = 0; l < ctx->L; ++l) ga.gm[l] = ctx->light[l].gm.as<float2>();
  ga.red = ctx->red.as<double>();
  ga.red_stride = red_stride;
  ga.big = cv.big_index.as<int>();
  ga.big_acc = cv.big_acc.as<float>();
  ga.pgrad = cv.pgrad.as<float4>();
  return ga;
}

// Camera c: Alg. 2 x Lambert into its colour buffer and (with an image) into
// the image at the pixels the final antialiasing leaves as they are, then the
// antialiased values of the listed pixels.
dsm_status camera_colour(dsm_ctx* ctx, int c, float* image, cudaStream_t st) {
  ViewBufs& cv = vbuf(ctx, ctx->L + c);
  const bool aa = ctx->params.aa_final != 0;
  {
    StageTimer t(ctx, ST_SHADE, st);
    launch_shade(shade_args(ctx, c), cv.color.as<float4>(), reinterpret_cast<float4*>(image),
                 aa ? cv.hflag.as<uint8_t>() : nullptr, st);
  }
  if (!image || !aa) return DSM_OK;
  StageTimer t(ctx, ST_FINAL_AA, st);
  launch_aa_forward4_list(aa_args(ctx, cv), cv.color.as<float4>(), reinterpret_cast<float4*>(image), cv.aa_work(), st);
  return DSM_OK;
}

// Camera c, backward: final antialiasing adjoint, then the shading adjoint
// (dL/dm into every light's gm, per-pixel gradients for the scatter).
dsm_status camera_backward(dsm_ctx* ctx, int c, const ImageGrad& gimage, float* dalbedo, int red_stride,
                           cudaStream_t st) {
  ViewBufs& cv = vbuf(ctx, ctx->L + c);
  const ShadeArgs sa = shade_args(ctx, c);
  const ShadeGradArgs ga = grad_args(ctx, c, gimage, dalbedo, red_stride);
  // the listed pixels on the camera's side stream: dL/dcolour (the
  // antialiasing adjoint), then their shading adjoint; beside it the grid
  // pass, which reads dL/dimage
  cudaStream_t side = st;
  if (ctx->params.aa_final && !ctx->prof) {
    DSM_CHECK(ensure_streams(ctx));
    side = ctx->cside[c];
    DSM_CHECK(cudaEventRecord(ctx->ev_cside[c], st));
    DSM_CHECK(cudaStreamWaitEvent(side, ctx->ev_cside[c], 0));
  }
  if (ctx->params.aa_final) {
    StageTimer t(ctx, ST_BWD_FINAL_AA, side);
    launch_aa_backward4_list(aa_args(ctx, cv), cv.color.as<float4>(), gimage, cv.gcolor.as<float4>(),
                             cv.gclip.as<float4>(), cv.aa_work(), side);
  }
  if (ctx->aux_pending) {   // outputs cleared
    DSM_CHECK(cudaStreamWaitEvent(st, ctx->ev_aux_done, 0));
    if (side != st) DSM_CHECK(cudaStreamWaitEvent(side, ctx->ev_aux_done, 0));
  }
  {
    StageTimer t(ctx, ST_BWD_SHADE, st);
    launch_shade_backward(sa, ga, st);
  }
  if (ctx->params.aa_final) {
    StageTimer t(ctx, ST_BWD_SHADE, side);
    launch_shade_backward_listed(sa, ga, cv.aa_work(), side);
  }
  if (side != st) {
    DSM_CHECK(cudaEventRecord(ctx->ev_cside_done[c], side));
    DSM_CHECK(cudaStreamWaitEvent(st, ctx->ev_cside_done[c], 0));
  }
  return DSM_OK;
}

// Camera c, backward: the per-pixel gradients scattered to the triangle corners.
void camera_scatter(dsm_ctx* ctx, int c, float* dalbedo, int red_stride, cudaStream_t st) {
  StageTimer t(ctx, ST_BWD_SHADE_SCATTER, st);
  const ShadeArgs sa = shade_args(ctx, c);
  const ShadeGradArgs ga = grad_args(ctx, c, ImageGrad{}, dalbedo, red_stride);
  launch_shade_scatter(sa, ga, st);
  launch_shade_big_resolve(sa, ga, vbuf(ctx, ctx->L + c).big_tri.as<int>(), ctx->status.as<DevStatus>(), ctx->L + c,
                           st);
}

// Light l, backward: G^T (filter adjoint, folded through f^2 = f f), the
// antialiasing adjoint at the listed texels, the interpolation adjoint.
void light_backward(dsm_ctx* ctx, int l, cudaStream_t st) {
  ViewBufs& v = vbuf(ctx, l);
  LightBufs& wk = lwork(ctx, l);
  LightBufs& lb = ctx->light[l];
  const AAArgs aa = aa_args(ctx, v);
  {
    StageTimer t(ctx, ST_BWD_FILTER, st);
    launch_filter_adjoint(lb.gm.as<float2>(), wk.tmp.as<float2>(), wk.gft.as<float2>(), v.W, lb.fa, st,
                          wk.fmap.as<float2>(), wk.tmp.as<float>(), warp_exponent(ctx), ctx->status.as<DevStatus>());
  }
  // the band is the antialiasing detection's flag map, so it exists only with
  // the shadow maps' antialiasing on
  if ((ctx->grad_mask & DSM_GRAD_MASK_SM_BAND) && ctx->params.aa_shadow)
    launch_sm_band_mask(v.hflag.as<uint8_t>(), v.W * v.H, wk.gft.as<float2>(), wk.tmp.as<float>(), st);
  {
    StageTimer t(ctx, ST_BWD_SM_AA, st);
    if (ctx->params.aa_shadow)
      launch_sm_aa_adjoint_list(aa, wk.fmap.as<float2>(), wk.gft.as<float2>(), v.gclip.as<float4>(),
                                wk.tmp.as<float>(), warp_exponent(ctx), v.aa_work(), st);
  }
  StageTimer t(ctx, ST_BWD_SM_INTERP, st);
  BigArgs big{v.big_index.as<int>(), v.big_tri.as<int>(), v.big_acc.as<float>(), ctx->status.as<DevStatus>(), l};
  launch_sm_interp_adjoint(aa, wk.tmp.as<float>(), v.depth.as<float>(), v.gclip.as<float4>(), big, st);
}

// dL/dv += M^T dL/dclip over views [w0, w0 + n), and dQ of the lights among them.
void vertex_backward_views(dsm_ctx* ctx, int w0, int n, float* dverts, int red_stride, cudaStream_t st) {
  VertGradPtrs gp{};
  for (int k = 0; k < n; ++k) gp.gclip[k] = vbuf(ctx, w0 + k).gclip.as<float4>();
  const int n_lights = std::max(0, std::min(n, ctx->L - w0));
  double* red = ctx->red.as<double>() + (n_lights > 0 ? 20 * w0 : 0);
  launch_vertex_backward(ctx->mesh.verts, ctx->mesh.n_verts, ctx->viewM.as<float>() + 20 * w0, n, n_lights, gp,
                         dverts, red, red_stride, st);
}

// Under recomputation: view w through its shared buffer set (setup, binning,
// raster with the antialiasing detection); `maps` also rebuilds a light's
// filtered moments.
dsm_status rebuild_view(dsm_ctx* ctx, int w, bool sizing, bool maps, cudaStream_t st) {
  dsm_status s = prepare_view(ctx, w);
  if (s != DSM_OK) return s;
  {
    StageTimer t(ctx, ST_SETUP, st);
    setup_views(ctx, w, 1, st);
  }
  alloc_view(ctx, w, !sizing, st);
  if (sizing) {
    s = size_lists(ctx, w, 1, st);
    if (s != DSM_OK) return s;
  }
  raster_view(ctx, w, st);
  if (maps && view_is_light(ctx, w)) light_maps(ctx, w, st);
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

// The backward's internal accumulators (the cameras' vertex-normal and
// vertex-position gradients as float4 per vertex, so that the scatter adds each
// with one 16-byte atomic; light-matrix block sums; and per view the clip
// gradients and big-triangle slots), sized for the current frame.
dsm_status ensure_backward_accumulators(dsm_ctx* ctx) {
  const int V = ctx->mesh.n_verts;
  DSM_CHECK(ctx->gnormal.ensure(sizeof(float4) * std::max(V, 1)));
  DSM_CHECK(ctx->gpos.ensure(sizeof(float4) * std::max(V, 1)));
  DSM_CHECK(ctx->gQ.ensure(sizeof(double) * 20 * kMaxLightViews));
  DSM_CHECK(ctx->gdirect.ensure(sizeof(double) * 3 * kMaxLightViews));
  DSM_CHECK(ctx->red.ensure(sizeof(double) * kRedSlots * std::max(red_stride_of(ctx), 1)));
  return DSM_OK;
}
void add_backward_accumulators(dsm_ctx* ctx, Clearer& cl) {
  const int V = ctx->mesh.n_verts;
  cl.add(ctx->gnormal.p, sizeof(float4) * V);
  cl.add(ctx->gpos.p, sizeof(float4) * V);
  cl.add(ctx->gQ.p, sizeof(double) * 20 * kMaxLightViews);
  cl.add(ctx->gdirect.p, sizeof(double) * 3 * kMaxLightViews);
  cl.add(ctx->red.p, sizeof(double) * kRedSlots * red_stride_of(ctx));
  if (!ctx->recompute)
    for (int w = 0; w < ctx->L + ctx->C; ++w) {
      ViewBufs& v = vbuf(ctx, w);
      cl.add(v.gclip.p, sizeof(float4) * V);
      cl.add(v.big_acc.p, (size_t)kMaxBig * kBigSlots * (view_is_light(ctx, w) ? kBigStrideSm : kBigStrideCam) * 4);
    }
}

}  // namespace

dsm_status dsm_render_cameras(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights, const float* light_params,
                              int32_t n_lights, const dsm_camera* cams, int32_t n_cams, const dsm_params* params,
                              float* const* images) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  dsm_status s = check_args(ctx, mesh, lights, light_params, n_lights, cams, n_cams, params, images);
  if (s != DSM_OK) return s;
  ctx->have_fwd = false;
  ctx->gm_zeroed = false;
  ctx->acc_zeroed = false;
  cudaStream_t st = (cudaStream_t)params->stream;
  ctx->mesh = *mesh;
  int L = 0;
  for (int u = 0; u < n_lights; ++u) {
    ctx->lights[u] = lights[u];
    const int faces = lights[u].type == 2 ? 6 : 1;
    for (int f = 0; f < faces; ++f, ++L) {
      ctx->view_user[L] = u;
      ctx->view_face[L] = lights[u].type == 2 ? f : -1;
    }
  }
  ctx->n_user = n_lights;
  const int V = mesh->n_verts, T = mesh->n_tris, C = n_cams, NV = L + C;
  for (int c = 0; c < C; ++c) ctx->cams[c] = cams[c];
  ctx->L = L;
  ctx->C = C;
  ctx->params = *params;
  ctx->stream = st;
  ctx->recompute = params->recompute_in_backward != 0;

  // ---- buffers (all growth happens here, before any launch of this frame)
  uint64_t sig = mix(mix(mix(mix(mix(1, V), T), L), C), ctx->recompute ? 1 : 0);
  sig = mix(mix(mix(sig, ctx->tuning.light_tile), ctx->tuning.camera_tile), ctx->tuning.big_tiles);
  for (int c = 0; c < C; ++c) sig = mix(mix(sig, cams[c].width), cams[c].height);
  for (int u = 0; u < n_lights; ++u) sig = mix(mix(sig, lights[u].res), lights[u].type);
  const bool sizing = ctx->sized_sig != sig;
  for (int w = 0; w < NV; ++w) {
    s = prepare_view(ctx, w);
    if (s != DSM_OK) return s;
  }
  for (int l = 0; l < L; ++l) {
    s = prepare_light(ctx, l);
    if (s != DSM_OK) return s;
  }
  s = ensure_backward_accumulators(ctx);
  if (s != DSM_OK) return s;
  DSM_CHECK(ctx->lights_dev.ensure(sizeof(LightDev) * kMaxLightViews));
  DSM_CHECK(ctx->viewM.ensure(sizeof(float) * 20 * kMaxViews));
  if (!ctx->viewMlo.p) {
    // light views' clip-row residuals (written by the light setup); camera views' stay zero
    DSM_CHECK(ctx->viewMlo.ensure(sizeof(float) * 16 * kMaxViews));
    DSM_CHECK(cudaMemset(ctx->viewMlo.p, 0, sizeof(float) * 16 * kMaxViews));
  }
  DSM_CHECK(ctx->vnormal.ensure(sizeof(float) * 3 * std::max(V, 1)));
  DSM_CHECK(ctx->vnlen.ensure(sizeof(float) * std::max(V, 1)));

  // ---- light cameras and the camera matrices
  LightSetupArgs la{};
  la.n = L;
  for (int l = 0; l < L; ++l) {
    const dsm_light& Lh = lights[ctx->view_user[l]];
    LightConst& c = la.c[l];
    // a cube face is a perspective view with a 90 degree field of view (c = 1)
    c.type = Lh.type == 0 ? 0 : 1;
    c.res = Lh.res;
    c.user = ctx->view_user[l];
    c.face = ctx->view_face[l];
    c.dist = Lh.dist;
    c.ortho_half = Lh.ortho_half;
    c.near_plane = Lh.near_plane;
    c.far_plane = Lh.far_plane;
    c.persp_c = Lh.type == 2 ? 1.0 : Lh.type == 1 ? 1.0 / std::tan((double)Lh.fov_y_deg * M_PI / 360.0) : 0.0;
    c.intensity[0] = Lh.intensity[0]; c.intensity[1] = Lh.intensity[1]; c.intensity[2] = Lh.intensity[2];
  }
  float* viewM = ctx->viewM.as<float>();
  StageTimer t_setup(ctx, ST_SETUP, st);
  CamMats cm{};
  for (int c = 0; c < C; ++c)
    for (int k = 0; k < 16; ++k) cm.v[20 * c + k] = cams[c].clip[k];
  const VertNormalArgs vna{mesh->verts, V, mesh->tris, ctx->vf_off.as<int>(), ctx->vf_list.as<int>(),
                           ctx->vnormal.as<float>(), ctx->vnlen.as<float>()};
  launch_light_setup(light_params, la, ctx->lights_dev.as<LightDev>(), viewM, ctx->viewMlo.as<float>(), cm, C, vna,
                     st);

  if (ctx->recompute) {
    // ---- one view at a time through the shared buffer sets
    t_setup.stop();
    for (int w = 0; w < NV; ++w) {
      s = rebuild_view(ctx, w, sizing, true, st);
      if (s != DSM_OK) return s;
      if (w >= L) {
        s = camera_colour(ctx, w - L, images[w - L], st);
        if (s != DSM_OK) return s;
      }
    }
  } else {
    // every view at once: transform, triangle setup with the binning's count
    // pass (the silhouettes follow beside the segments: only the antialiasing
    // reads them)
    setup_views(ctx, 0, NV, st, false);
    t_setup.stop();
    // ---- per view on its own stream: list segments and work units (the views are independent until shading)
    DSM_CHECK(ensure_streams(ctx));
    DSM_CHECK(fork_views(ctx, st, ctx->ev_fork, 0, NV));
    for (int w = 0; w < NV; ++w) alloc_view(ctx, w, !sizing, view_stream(ctx, w, st));
    {
      StageTimer ts(ctx, ST_SETUP, st);
      silhouette_views(ctx, 0, NV, st);
    }
    DSM_CHECK(cudaEventRecord(ctx->ev_sil, st));
    DSM_CHECK(cudaGetLastError());
    if (sizing) {
      // first frame of this scene size: read the pair counts once and size the lists
      DSM_CHECK(join_views(ctx, st, 0, NV));
      s = size_lists(ctx, 0, NV, st);
      if (s != DSM_OK) return s;
      DSM_CHECK(fork_views(ctx, st, ctx->ev_fork, 0, NV));
    }
    // ---- per view: bin fill, raster with the antialiasing detection (which
    // reads the silhouettes); per light: Alg. 1 (f, f^2 -> antialias -> filter)
    for (int w = 0; w < NV; ++w) {
      cudaStream_t vst = view_stream(ctx, w, st);
      if (vst != st) DSM_CHECK(cudaStreamWaitEvent(vst, ctx->ev_sil, 0));
      raster_view(ctx, w, vst);
      if (w < L) light_maps(ctx, w, vst);
    }
    // the lights' dL/dm accumulators and the backward's other internal
    // accumulators start the first backward empty; zeroed on the render
    // stream, which holds the (shorter) camera raster, so the clears run
    // beside the lights' antialiasing and filter
    for (int l = 0; l < L; ++l) {
      const LightBufs& lb = ctx->light[l];
      DSM_CHECK(cudaMemsetAsync(lb.gm.p, 0, (size_t)lb.res * lb.res * sizeof(float2), st));
    }
    {
      Clearer cl;
      add_backward_accumulators(ctx, cl);
      cl.launch(st);
      ctx->acc_zeroed = true;
    }
    DSM_CHECK(join_views(ctx, st, 0, NV));
    DSM_CHECK(cudaGetLastError());
    // ---- cameras: shade (Alg. 2 x Lambert) and the final antialiasing, each on its stream
    if (C > 1) DSM_CHECK(fork_views(ctx, st, ctx->ev_fork, L, NV));
    for (int c = 0; c < C; ++c) {
      s = camera_colour(ctx, c, images[c], C > 1 ? view_stream(ctx, L + c, st) : st);
      if (s != DSM_OK) return s;
    }
    if (C > 1) DSM_CHECK(join_views(ctx, st, L, NV));
  }
  DSM_CHECK(cudaGetLastError());
  ctx->gm_zeroed = !ctx->recompute;
  ctx->acc_zeroed = ctx->acc_zeroed && !ctx->recompute;
  ctx->sized_sig = sig;
  ctx->have_fwd = true;
  return DSM_OK;
}

dsm_status dsm_render(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights, const float* light_params,
                      int32_t n_lights, const dsm_camera* cam, const dsm_params* params, float* image) {
  return dsm_render_cameras(ctx, mesh, lights, light_params, n_lights, cam, 1, params, &image);
}

namespace {

// The backward of the last forward from dL/dimage of every camera, or (l2:
// one camera) from the mean squared error of its image against a target,
// whose value goes to *l2_loss.
struct L2Target {
  const float* image;
  const float* target;
  float* loss;
};

dsm_status backward_impl(dsm_ctx* ctx, const float* const* dL_dimages, const L2Target* l2, float* dL_dverts,
                         float* dL_dlight, float* dL_dalbedo) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (!ctx->have_fwd) return fail(ctx, DSM_ERR_NO_FORWARD, "backward without a forward");
  if (l2) {
    if (ctx->C != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "last forward had several cameras");
    if (!l2->image || !l2->target || !l2->loss) return fail(ctx, DSM_ERR_INVALID_ARG, "null image, target or loss");
  } else {
    if (!dL_dimages) return fail(ctx, DSM_ERR_INVALID_ARG, "null dL_dimages");
    for (int c = 0; c < ctx->C; ++c)
      if (!dL_dimages[c]) return fail(ctx, DSM_ERR_INVALID_ARG, "null dL_dimage");
  }
  auto image_grad = [&](int c) {
    if (!l2) return ImageGrad{reinterpret_cast<const float4*>(dL_dimages[c]), nullptr, nullptr, 0.f};
    const int64_t n = (int64_t)ctx->cams[c].width * ctx->cams[c].height * 4;
    return ImageGrad{nullptr, reinterpret_cast<const float4*>(l2->image), reinterpret_cast<const float4*>(l2->target),
                     2.0f / (float)n};
  };
  cudaStream_t st = ctx->stream;
  const dsm_mesh& mesh = ctx->mesh;
  const int V = mesh.n_verts, T = mesh.n_tris, L = ctx->L, C = ctx->C, NV = L + C;
  if (!dL_dverts) {
    DSM_CHECK(ctx->scratch_dverts.ensure(sizeof(float) * 3 * std::max(V, 1)));
    dL_dverts = ctx->scratch_dverts.as<float>();
  }
  if (!dL_dlight) {
    DSM_CHECK(ctx->scratch_dlight.ensure(sizeof(float) * 6 * DSM_MAX_LIGHTS));
    dL_dlight = ctx->scratch_dlight.as<float>();
  }
  if (!dL_dalbedo) {
    DSM_CHECK(ctx->scratch_dalbedo.ensure(sizeof(float) * 3 * mesh.n_materials));
    dL_dalbedo = ctx->scratch_dalbedo.as<float>();
  }
  for (int c = 0; c < C; ++c) {
    ViewBufs& cv = vbuf(ctx, L + c);
    const size_t px = (size_t)ctx->cams[c].width * ctx->cams[c].height;
    DSM_CHECK(cv.gcolor.ensure(px * sizeof(float4)));
    DSM_CHECK(cv.pgrad.ensure(px * 2 * sizeof(float4)));
  }
  dsm_status sa = ensure_backward_accumulators(ctx);
  if (sa != DSM_OK) return sa;
  DSM_CHECK(ctx->gN.ensure(sizeof(float) * 3 * std::max(V, 1)));
  DSM_CHECK(ctx->gface.ensure(sizeof(float) * 3 * std::max(T, 1)));
  const int n_mat_red = n_mat_red_of(ctx);
  const int red_stride = red_stride_of(ctx);
  for (int l = 0; l < L; ++l) {
    const size_t R2 = (size_t)ctx->light[l].res * ctx->light[l].res * sizeof(float2);
    DSM_CHECK(ctx->light[l].gm.ensure(R2));
    DSM_CHECK(lwork(ctx, l).gft.ensure(R2));
  }
  auto clear_view = [&](Clearer& cl, int w) {
    ViewBufs& v = vbuf(ctx, w);
    cl.add(v.gclip.p, sizeof(float4) * V);
    cl.add(v.big_acc.p, (size_t)kMaxBig * kBigSlots * (view_is_light(ctx, w) ? kBigStrideSm : kBigStrideCam) * 4);
  };
  // ---- clear accumulators and outputs.  After a stored forward the internal
  // accumulators are already zero and only the caller's outputs are cleared,
  // on a side stream beside the final antialiasing adjoint (the first writer
  // of dL/dalbedo is the shading adjoint, which waits for it).
  const bool side = ctx->acc_zeroed && ctx->gm_zeroed && !ctx->prof;
  ctx->aux_pending = false;
  DSM_CHECK(ensure_streams(ctx));
  {
    StageTimer t(ctx, ST_BWD_CLEAR, st);
    Clearer cl;
    cl.add(dL_dverts, sizeof(float) * 3 * V);
    if (ctx->n_user) cl.add(dL_dlight, sizeof(float) * 6 * ctx->n_user);
    cl.add(dL_dalbedo, sizeof(float) * 3 * mesh.n_materials);
    if (!ctx->acc_zeroed) add_backward_accumulators(ctx, cl);
    if (!ctx->gm_zeroed)
      for (int l = 0; l < L; ++l)
        cl.add(ctx->light[l].gm.p, (size_t)ctx->light[l].res * ctx->light[l].res * sizeof(float2));
    ctx->gm_zeroed = false;   // this backward accumulates into them
    ctx->acc_zeroed = false;
    static_assert(8 + kMaxLightViews + 2 * kMaxViews <= kMaxClear, "clear list");
    if (side) {
      DSM_CHECK(cudaEventRecord(ctx->ev_aux, st));
      DSM_CHECK(cudaStreamWaitEvent(ctx->aux, ctx->ev_aux, 0));
      cl.launch(ctx->aux);
      DSM_CHECK(cudaEventRecord(ctx->ev_aux_done, ctx->aux));
      ctx->aux_pending = true;
    } else {
      cl.launch(st);
    }
  }
  DSM_CHECK(cudaGetLastError());

  // ---- normals: dL/dn of the cameras' pixels onto the vertices, with the
  // cameras' position gradients.  Its inputs come from the cameras' adjoints;
  // it adds to dverts with plain read-modify-writes, so it runs on st after
  // the camera scatters and before the vertex gather.
  auto normals = [&]() {
    StageTimer t(ctx, ST_BWD_VERTEX, st);
    launch_normals_backward(mesh.verts, V, mesh.tris, T, ctx->vf_off.as<int>(), ctx->vf_list.as<int>(),
                            ctx->vnormal.as<float>(), ctx->vnlen.as<float>(), ctx->gnormal.as<float4>(),
                            ctx->gpos.as<float4>(), ctx->gN.as<float>(), ctx->gface.as<float>(), dL_dverts, st);
  };
  if (ctx->recompute) {
    // ---- the filtered moment maps again (every camera's shading adjoint reads all of them)
    ctx->stage_override = ST_BWD_RECOMPUTE;
    for (int l = 0; l < L; ++l) {
      dsm_status s = rebuild_view(ctx, l, false, true, st);
      if (s != DSM_OK) { ctx->stage_override = -1; return s; }
    }
    ctx->stage_override = -1;
    // ---- per camera: G-buffer and colour again, then its adjoints and its share of dL/dv
    for (int c = 0; c < C; ++c) {
      ctx->stage_override = ST_BWD_RECOMPUTE;
      dsm_status s = rebuild_view(ctx, L + c, false, false, st);
      if (s == DSM_OK) s = camera_colour(ctx, c, nullptr, st);
      ctx->stage_override = -1;
      if (s != DSM_OK) return s;
      {
        StageTimer t(ctx, ST_BWD_CLEAR, st);
        Clearer cl;
        clear_view(cl, L + c);
        cl.launch(st);
      }
      s = camera_backward(ctx, c, image_grad(c), dL_dalbedo, red_stride, st);
      if (s != DSM_OK) return s;
      camera_scatter(ctx, c, dL_dalbedo, red_stride, st);
      StageTimer t(ctx, ST_BWD_VERTEX, st);
      vertex_backward_views(ctx, L + c, 1, dL_dverts, red_stride, st);
    }
    // ---- per light: G-buffer, f and the antialiasing list again, then its adjoints
    for (int l = 0; l < L; ++l) {
      ctx->stage_override = ST_BWD_RECOMPUTE;
      dsm_status s = rebuild_view(ctx, l, false, false, st);
      ctx->stage_override = -1;
      if (s != DSM_OK) return s;
      {
        StageTimer t(ctx, ST_BWD_CLEAR, st);
        Clearer cl;
        clear_view(cl, l);
        cl.launch(st);
      }
      light_backward(ctx, l, st);
      StageTimer t(ctx, ST_BWD_VERTEX, st);
      vertex_backward_views(ctx, l, 1, dL_dverts, red_stride, st);
    }
    normals();
  } else {
    // ---- per camera: final antialiasing adjoint and the shading adjoint
    DSM_CHECK(ensure_streams(ctx));
    if (C > 1) DSM_CHECK(fork_views(ctx, st, ctx->ev_bfork, L, NV));
    for (int c = 0; c < C; ++c) {
      dsm_status s = camera_backward(ctx, c, image_grad(c), dL_dalbedo, red_stride,
                                     C > 1 ? view_stream(ctx, L + c, st) : st);
      if (s != DSM_OK) return s;
    }
    if (C > 1) DSM_CHECK(join_views(ctx, st, L, NV));   // gm is complete
    // ---- per light on its own stream: G^T, antialiasing adjoint, interpolation
    // adjoint (they write only that light's buffers), beside the camera scatters
    DSM_CHECK(fork_views(ctx, st, ctx->ev_bfork, 0, L));
    for (int l = 0; l < L; ++l) light_backward(ctx, l, view_stream(ctx, l, st));
    for (int c = 0; c < C; ++c)
      camera_scatter(ctx, c, dL_dalbedo, red_stride, C > 1 ? view_stream(ctx, L + c, st) : st);
    if (C > 1) DSM_CHECK(join_views(ctx, st, L, NV));
    normals();   // beside the light views' adjoints
    DSM_CHECK(join_views(ctx, st, 0, L));
    StageTimer t(ctx, ST_BWD_VERTEX, st);
    vertex_backward_views(ctx, 0, NV, dL_dverts, red_stride, st);
  }
  // ---- the light matrices' and direct terms' block sums (the vertex gather
  // adds the light views' share), then the lights' parameters
  {
    StageTimer t(ctx, ST_BWD_VERTEX, st);
    launch_light_sums(ctx->red.as<double>(), red_stride, L, n_mat_red, ctx->lights_dev.as<LightDev>(), ctx->n_user,
                      ctx->gQ.as<double>(), ctx->gdirect.as<double>(), dL_dalbedo, dL_dlight, l2 ? l2->loss : nullptr,
                      (int64_t)ctx->cams[0].width * ctx->cams[0].height * 4, st);
  }
  if (ctx->aux_pending) {
    // the side stream's clear has been waited for by every shading adjoint;
    // join it to st as well so that the call's work ends on st
    DSM_CHECK(cudaStreamWaitEvent(st, ctx->ev_aux_done, 0));
    ctx->aux_pending = false;
  }
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

}  // namespace

dsm_status dsm_render_cameras_backward(dsm_ctx* ctx, const float* const* dL_dimages, float* dL_dverts,
                                       float* dL_dlight, float* dL_dalbedo) {
  return backward_impl(ctx, dL_dimages, nullptr, dL_dverts, dL_dlight, dL_dalbedo);
}

dsm_status dsm_render_backward(dsm_ctx* ctx, const float* dL_dimage, float* dL_dverts, float* dL_dlight,
                               float* dL_dalbedo) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (ctx->have_fwd && ctx->C != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "last forward had several cameras");
  return dsm_render_cameras_backward(ctx, &dL_dimage, dL_dverts, dL_dlight, dL_dalbedo);
}

dsm_status dsm_render_backward_l2(dsm_ctx* ctx, const float* image, const float* target, float* loss,
                                  float* dL_dverts, float* dL_dlight, float* dL_dalbedo) {
  const L2Target l2{image, target, loss};
  return backward_impl(ctx, nullptr, &l2, dL_dverts, dL_dlight, dL_dalbedo);
}

dsm_status dsm_set_grad_mask(dsm_ctx* ctx, int32_t flags) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (flags & ~DSM_GRAD_MASK_SM_BAND) return fail(ctx, DSM_ERR_INVALID_ARG, "unknown gradient mask flag");
  ctx->grad_mask = flags;
  return DSM_OK;
}

static bool tuning_ok(const dsm_tuning& t) {
  return (t.light_tile == 16 || t.light_tile == 32) && (t.camera_tile == 16 || t.camera_tile == 32) &&
         t.big_tiles >= 2 && t.big_tiles <= 4096 && t.filter_shape >= 0 && t.filter_shape <= 2;
}

dsm_status dsm_set_tuning(dsm_ctx* ctx, const dsm_tuning* tuning) {
  if (!ctx || !tuning) return DSM_ERR_INVALID_ARG;
  if (!tuning_ok(*tuning)) return fail(ctx, DSM_ERR_INVALID_ARG, "tuning value out of range");
  ctx->tuning = *tuning;
  ctx->have_fwd = false;
  return DSM_OK;
}

dsm_status dsm_get_tuning(dsm_ctx* ctx, dsm_tuning* tuning) {
  if (!ctx || !tuning) return DSM_ERR_INVALID_ARG;
  *tuning = ctx->tuning;
  return DSM_OK;
}

dsm_status dsm_autotune(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights, const float* light_params,
                        int32_t n_lights, const dsm_camera* cams, int32_t n_cams, const dsm_params* params,
                        float* const* images, int32_t reps, dsm_tuning* best, float* best_ms) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (reps < 1 || reps > 100) return fail(ctx, DSM_ERR_INVALID_ARG, "reps out of range");
  dsm_status s = check_args(ctx, mesh, lights, light_params, n_lights, cams, n_cams, params, images);
  if (s != DSM_OK) return s;
  cudaStream_t st = (cudaStream_t)params->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DSM_CHECK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, DSM_ERR_CUDA, "event");
  }
  const float* const* gimg = const_cast<const float* const*>(images);
  auto step = [&]() -> dsm_status {
    dsm_status r = dsm_render_cameras(ctx, mesh, lights, light_params, n_lights, cams, n_cams, params, images);
    if (r == DSM_OK) r = dsm_render_cameras_backward(ctx, gimg, nullptr, nullptr, nullptr);
    return r;
  };
  // time per step of shapes t (one untimed step first: it sizes the lists)
  auto measure = [&](const dsm_tuning& t, float* ms) -> dsm_status {
    ctx->tuning = t;
    dsm_status r = step();
    if (r == DSM_OK) r = dsm_sync(ctx);
    if (r != DSM_OK) return r;
    if (cudaEventRecord(e0, st) != cudaSuccess) return fail(ctx, DSM_ERR_CUDA, "event record");
    for (int k = 0; k < reps && r == DSM_OK; ++k) r = step();
    if (r != DSM_OK) return r;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return fail(ctx, DSM_ERR_CUDA, "event wait");
    r = dsm_sync(ctx);
    if (r != DSM_OK) return r;
    float total = 0.f;
    if (cudaEventElapsedTime(&total, e0, e1) != cudaSuccess) return fail(ctx, DSM_ERR_CUDA, "event time");
    *ms = total / reps;
    return DSM_OK;
  };
  dsm_tuning cur = ctx->tuning;
  float cur_ms = 0.f;
  s = measure(cur, &cur_ms);
  if (s == DSM_OK) s = dsm::tuning_search(&cur, &cur_ms, measure);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tuning = cur;
  ctx->have_fwd = false;
  if (s != DSM_OK) return s;
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return DSM_OK;
}

dsm_status dsm_l2_loss_grad(const float* image, const float* target, int64_t n, float* loss, float* dL_dimage,
                            void* stream) {
  if (n < 0 || !loss || (n > 0 && (!image || !target || !dL_dimage))) return DSM_ERR_INVALID_ARG;
  launch_l2(image, target, n, loss, dL_dimage, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? DSM_OK : DSM_ERR_CUDA;
}

dsm_status dsm_filter_moments(dsm_ctx* ctx, const float* in, float* out, int32_t res, float sigma, int32_t radius,
                              int32_t kind, int32_t boundary, void* stream) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (!in || !out || res < 1 || res > 16384 || !filter_args_ok(sigma, radius, kind, boundary))
    return fail(ctx, DSM_ERR_INVALID_ARG, "bad filter arguments");
  DSM_CHECK(ctx->filter_tmp.ensure((size_t)res * res * sizeof(float2)));
  FilterArgs fa;
  make_filter_args(sigma, radius, kind, boundary, &fa);
  fa.shape = ctx->tuning.filter_shape;
  launch_filter(reinterpret_cast<const float2*>(in), ctx->filter_tmp.as<float2>(), reinterpret_cast<float2*>(out), res,
                fa, (cudaStream_t)stream, nullptr, nullptr, ctx->status.as<DevStatus>());
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

dsm_status dsm_filter_moments_adjoint(dsm_ctx* ctx, const float* gout, float* gin, int32_t res, float sigma,
                                      int32_t radius, int32_t kind, int32_t boundary, void* stream) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (!gout || !gin || res < 1 || res > 16384 || !filter_args_ok(sigma, radius, kind, boundary))
    return fail(ctx, DSM_ERR_INVALID_ARG, "bad filter arguments");
  DSM_CHECK(ctx->filter_tmp.ensure((size_t)res * res * sizeof(float2)));
  FilterArgs fa;
  make_filter_args(sigma, radius, kind, boundary, &fa);
  fa.shape = ctx->tuning.filter_shape;
  launch_filter_adjoint(reinterpret_cast<const float2*>(gout), ctx->filter_tmp.as<float2>(),
                        reinterpret_cast<float2*>(gin), res, fa, (cudaStream_t)stream, nullptr, nullptr, 0.f,
                        ctx->status.as<DevStatus>());
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

dsm_status dsm_sync(dsm_ctx* ctx) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  DSM_CHECK(cudaMemcpyAsync(ctx->hstatus, ctx->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, ctx->stream));
  DSM_CHECK(cudaStreamSynchronize(ctx->stream));
  DSM_CHECK(cudaGetLastError());
  if (ctx->hstatus->capacity_overflow) {
    DSM_CHECK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int) * 2, ctx->stream));
    ctx->sized_sig = 0;
    return fail(ctx, DSM_ERR_CAPACITY, "tile list overflow: render again");
  }
  if (ctx->hstatus->timeout) {
    DSM_CHECK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int) * 2, ctx->stream));
    return fail(ctx, DSM_ERR_TIMEOUT, "device wait timed out");
  }
  return DSM_OK;
}

dsm_status dsm_bounded_wait_probe(dsm_ctx* ctx, int32_t arrive) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  launch_bounded_wait_probe(ctx->status.as<DevStatus>(), arrive != 0, ctx->stream);
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

dsm_status dsm_profile_enable(dsm_ctx* ctx, int32_t enable) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  ctx->prof = enable != 0;
  return DSM_OK;
}

int32_t dsm_profile_stage_count(void) { return kStages; }

const char* dsm_profile_stage_name(int32_t stage) {
  return (stage >= 0 && stage < kStages) ? kStageNames[stage] : nullptr;
}

dsm_status dsm_profile_read(dsm_ctx* ctx, double* ms, int64_t* calls, int32_t n) {
  if (!ctx || n < 0 || (n > 0 && (!ms || !calls))) return DSM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) { ms[i] = 0.0; calls[i] = 0; }
  for (auto& r : ctx->recs) {
    DSM_CHECK(cudaEventSynchronize(r.b));
    float t = 0.f;
    DSM_CHECK(cudaEventElapsedTime(&t, r.a, r.b));
    if (r.stage < n) { ms[r.stage] += t; calls[r.stage] += 1; }
    ctx->free_events.push_back(r.a);
    ctx->free_events.push_back(r.b);
  }
  ctx->recs.clear();
  return DSM_OK;
}

uint64_t dsm_kernel_launches(void) { return (uint64_t)g_kernel_launches.load(); }

dsm_status dsm_debug_copy(dsm_ctx* ctx, int32_t what, int32_t index, void* dst, size_t bytes) {
  if (!ctx || !dst) return DSM_ERR_INVALID_ARG;
  const int L = ctx->L, V = ctx->mesh.n_verts;
  if (ctx->recompute && what != 3 && what != 5 && what != 7)
    return fail(ctx, DSM_ERR_INVALID_ARG, "per-view buffers are not kept under recomputation");
  const void* src = nullptr;
  size_t size = 0;
  const bool light_ok = index >= 0 && index < L;
  const bool view_ok = index >= 0 && index < L + ctx->C;
  const bool cam_ok = index >= 0 && index < ctx->C;
  const size_t R2 = light_ok ? (size_t)ctx->light[index].res * ctx->light[index].res * 8 : 0;
  auto view_px = [&](int w) { return (size_t)ctx->view[w].W * ctx->view[w].H; };
  auto cam_px = [&](int c) { return (size_t)ctx->cams[c].width * ctx->cams[c].height; };
  switch (what) {
    case 0: if (view_ok) { src = ctx->view[index].gbuf.p; size = view_px(index) * 16; } break;
    case 1: if (light_ok) { src = ctx->light[index].fmap.p; size = R2; } break;
    case 2: if (light_ok) { src = ctx->light[index].ftilde.p; size = R2; } break;
    case 3: if (light_ok) { src = ctx->light[index].mom.p; size = R2; } break;
    case 4: if (cam_ok) { src = ctx->view[L + index].color.p; size = cam_px(index) * 16; } break;
    case 5: src = ctx->viewM.p; size = (size_t)L * 20 * 4; break;
    case 6: if (view_ok) { src = ctx->view[index].snap.p; size = (size_t)V * 16; } break;
    case 7: if (light_ok) { src = ctx->light[index].gm.p; size = R2; } break;
    case 8: if (view_ok) { src = ctx->view[index].gclip.p; size = (size_t)V * 16; } break;
    case 9: if (light_ok) { src = ctx->light[index].gft.p; size = R2; } break;
    case 10: if (cam_ok) { src = ctx->view[L + index].gcolor.p; size = cam_px(index) * 16; } break;
    case 11:
    case 12: {
      // shading-stage probe: camera index (11), or camera index / 64 and
      // light view index % 64 (12)
      const int c = what == 11 ? index : (index >= 0 ? index / 64 : -1);
      const int l = what == 11 ? -1 : (index >= 0 ? index % 64 : -1);
      if (c < 0 || c >= ctx->C || (what == 12 && l >= L)) break;
      if (bytes != cam_px(c) * 32) return fail(ctx, DSM_ERR_INVALID_ARG, "debug buffer size mismatch");
      launch_shade_probe(shade_args(ctx, c), l, static_cast<float4*>(dst), ctx->stream);
      DSM_CHECK(cudaGetLastError());
      DSM_CHECK(cudaStreamSynchronize(ctx->stream));
      return DSM_OK;
    }
    default: break;
  }
  if (!src || size == 0) return fail(ctx, DSM_ERR_INVALID_ARG, "unknown or empty debug buffer");
  if (bytes != size) return fail(ctx, DSM_ERR_INVALID_ARG, "debug buffer size mismatch");
  if (what == 2) {
    // f~ is held as f plus the antialiased values of the listed texels
    const LightBufs& lb = ctx->light[index];
    const int n = lb.res * lb.res;
    if (ctx->params.aa_shadow)
      launch_compose(lb.fmap.as<float2>(), ctx->view[index].hflag.as<uint8_t>(), lb.ftilde.as<float2>(),
                     static_cast<float2*>(dst), n, ctx->stream);
    else
      DSM_CHECK(cudaMemcpyAsync(dst, lb.fmap.p, size, cudaMemcpyDeviceToDevice, ctx->stream));
    DSM_CHECK(cudaGetLastError());
    DSM_CHECK(cudaStreamSynchronize(ctx->stream));
    return DSM_OK;
  }
  DSM_CHECK(cudaMemcpyAsync(dst, src, size, cudaMemcpyDeviceToDevice, ctx->stream));
  DSM_CHECK(cudaStreamSynchronize(ctx->stream));
  return DSM_OK;
}

dsm_status dsm_raster_stats(dsm_ctx* ctx, int32_t view, int64_t* out) {
  if (!ctx || !out) return DSM_ERR_INVALID_ARG;
  if (!ctx->have_fwd) return fail(ctx, DSM_ERR_NO_FORWARD, "raster stats without a forward");
  if (ctx->recompute)
    return fail(ctx, DSM_ERR_INVALID_ARG, "raster stats need the stored mode (recomputation shares view buffers)");
  if (view < 0 || view >= ctx->L + ctx->C) return fail(ctx, DSM_ERR_INVALID_ARG, "raster stats: view out of range");
  ViewBufs& v = vbuf(ctx, view);
  cudaStream_t st = ctx->stream;
  constexpr size_t kBytes = 3 * sizeof(unsigned long long);
  DSM_CHECK(ctx->stats.ensure(kBytes));
  DSM_CHECK(cudaMemsetAsync(ctx->stats.p, 0, kBytes, st));
  launch_raster_stats(v.setup.as<TriSetup>(), v.offset.as<int>(), v.list.as<int>(), v.list_cap, v.tilesX, v.tilesY,
                      v.bs.tile_log2, ctx->stats.as<unsigned long long>(), st);
  DSM_CHECK(cudaGetLastError());
  unsigned long long h[3];
  int listed = 0;
  DSM_CHECK(cudaMemcpyAsync(h, ctx->stats.p, kBytes, cudaMemcpyDeviceToHost, st));
  DSM_CHECK(cudaMemcpyAsync(&listed, v.aa_ctr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSM_CHECK(cudaStreamSynchronize(st));
  for (int k = 0; k < 3; ++k) out[k] = (int64_t)h[k];
  const bool aa_on = view_is_light(ctx, view) ? ctx->params.aa_shadow != 0 : ctx->params.aa_final != 0;
  out[3] = aa_on ? (int64_t)listed : 0;
  return DSM_OK;
}

uint64_t dsm_memory_bytes(dsm_ctx* ctx) {
  if (!ctx) return 0;
  uint64_t n = 0;
  const Buf* bufs[] = {&ctx->adj, &ctx->vf_off, &ctx->vf_list, &ctx->lights_dev, &ctx->viewM, &ctx->viewMlo, &ctx->status,
                       &ctx->vnormal, &ctx->vnlen, &ctx->gnormal, &ctx->gpos, &ctx->gN, &ctx->gface, &ctx->gQ, &ctx->gdirect,
                       &ctx->scratch_dverts, &ctx->scratch_dlight, &ctx->scratch_dalbedo, &ctx->filter_tmp,
                       &ctx->red, &ctx->stats};
  for (const Buf* b : bufs) n += b->cap;
  for (const auto& v : ctx->view) {
    const Buf* vb[] = {&v.clip, &v.snap, &v.depth, &v.setup, &v.orient, &v.sil, &v.count, &v.offset, &v.list,
                       &v.gbuf, &v.gclip, &v.big_index, &v.big_tri, &v.big_acc, &v.aa_list, &v.aa_ctr,
                       &v.hflag, &v.rim, &v.color, &v.gcolor, &v.pgrad, &v.units, &v.tile_done, &v.skey};
    for (const Buf* b : vb) n += b->cap;
  }
  for (const auto& l : ctx->light) {
    const Buf* lb[] = {&l.fmap, &l.ftilde, &l.tmp, &l.mom, &l.gm, &l.gft};
    for (const Buf* b : lb) n += b->cap;
  }
  return n;
}

}  // extern "C"
