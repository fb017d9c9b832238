// C-ABI entry points: context, scratch management and the orchestration of the
// forward (Alg. 1 per light, Alg. 2 + Lambert per camera pixel) and backward
// passes.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {
std::atomic<unsigned long long> g_kernel_launches{0};

static const char* const kStageNames[] = {
    "setup", "bin_fill", "raster", "sm_antialias", "filter", "shade", "final_antialias",
    "bwd_clear", "bwd_final_antialias", "bwd_shade", "bwd_shade_scatter", "bwd_filter", "bwd_sm_antialias",
    "bwd_sm_interp", "bwd_vertex"};
constexpr int kStages = (int)(sizeof(kStageNames) / sizeof(kStageNames[0]));
enum Stage { ST_SETUP, ST_BIN_FILL, ST_RASTER, ST_SM_AA, ST_FILTER, ST_SHADE, ST_FINAL_AA,
             ST_BWD_CLEAR, ST_BWD_FINAL_AA, ST_BWD_SHADE, ST_BWD_SHADE_SCATTER, ST_BWD_FILTER, ST_BWD_SM_AA,
             ST_BWD_SM_INTERP, ST_BWD_VERTEX };

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

struct ViewBufs {
  int W = 0, H = 0, tilesX = 0, tilesY = 0;
  Buf clip, snap, depth, setup, orient, sil, count, offset, list, gbuf, gclip;
  Buf big_index, big_tri, big_acc;
  Buf aa_list, aa_ctr, hflag;   // antialiasing work list, its counter, per-pixel "listed" flag
  int list_cap = 0;
  AAWork aa_work() { return AAWork{aa_list.as<int>(), aa_ctr.as<int>()}; }
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
  ViewBufs view[DSM_MAX_LIGHTS + 1];
  LightBufs light[DSM_MAX_LIGHTS];
  Buf lights_dev, viewM, status, vnormal, vnlen, camcolor, gcolor, gnormal, gN, gface, gQ, gdirect, red, pgrad;
  Buf scratch_dverts, scratch_dlight, scratch_dalbedo, filter_tmp;
  DevStatus* hstatus = nullptr;
  // state of the last forward
  bool have_fwd = false;
  dsm_mesh mesh{};
  dsm_light lights[DSM_MAX_LIGHTS]{};
  int L = 0;
  dsm_camera cam{};
  dsm_params params{};
  cudaStream_t stream = nullptr;
  uint64_t sized_sig = 0;
  // internal streams: one per view (lights, then camera), fork/join events
  cudaStream_t vs[DSM_MAX_LIGHTS + 1] = {};
  cudaEvent_t ev_fork = nullptr, ev_bfork = nullptr, ev_join[DSM_MAX_LIGHTS + 1] = {};
  // per-stage timing
  bool prof = false;
  // views serialised on the caller's stream (batched scenes overlap one another instead)
  bool serial = false;
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

__global__ void set_matrix_kernel(Mat20 m, float* dst) {
  int k = threadIdx.x;
  if (k < 20) dst[k] = m.v[k];
}

// One launch that zeroes several buffers: segment blockIdx.y, 16-byte stores
// over its aligned body, 4-byte stores for an unaligned head and the tail.
constexpr int kMaxClear = 40;
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
  StageTimer(dsm_ctx* c_, int stage_, cudaStream_t st_) : c(c_), st(st_), stage(stage_) {
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
  if ((e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&c->ev_bfork, cudaEventDisableTiming)) != cudaSuccess) return e;
  for (auto& ev : c->ev_join)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Stream of view w: its own stream, or the caller's while stage profiling is
// on (profiling serialises the views so that each stage's events bracket only
// its own kernels).
cudaStream_t view_stream(const dsm_ctx* c, int w, cudaStream_t st) {
  return (c->prof || c->serial) ? st : c->vs[w];
}

// All view streams wait for the work enqueued so far on st.
cudaError_t fork_views(dsm_ctx* c, cudaStream_t st, cudaEvent_t ev, int n_views) {
  if (c->prof || c->serial) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev, st);
  for (int w = 0; w < n_views && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(c->vs[w], ev, 0);
  return e;
}

// st waits for the work enqueued so far on the first n view streams.
cudaError_t join_views(dsm_ctx* c, cudaStream_t st, int n_views) {
  if (c->prof || c->serial) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < n_views && e == cudaSuccess; ++w) {
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
// Batched scenes: each context keeps its views on the caller's stream.
void set_serial_views(dsm_ctx* ctx, bool serial) {
  if (ctx) ctx->serial = serial;
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
  Buf* bufs[] = {&ctx->adj, &ctx->vf_off, &ctx->vf_list, &ctx->lights_dev, &ctx->viewM, &ctx->status,
                 &ctx->vnormal, &ctx->vnlen, &ctx->camcolor, &ctx->gcolor, &ctx->gnormal, &ctx->gN, &ctx->gface,
                 &ctx->gQ, &ctx->gdirect, &ctx->scratch_dverts, &ctx->scratch_dlight, &ctx->scratch_dalbedo,
                 &ctx->filter_tmp, &ctx->red, &ctx->pgrad};
  for (Buf* b : bufs) b->release();
  for (auto& v : ctx->view) {
    Buf* vb[] = {&v.clip, &v.snap, &v.depth, &v.setup, &v.orient, &v.sil, &v.count, &v.offset, &v.list,
                 &v.gbuf, &v.gclip, &v.big_index, &v.big_tri, &v.big_acc, &v.aa_list, &v.aa_ctr,
                 &v.hflag};
    for (Buf* b : vb) b->release();
  }
  for (auto& l : ctx->light) {
    Buf* lb[] = {&l.fmap, &l.ftilde, &l.tmp, &l.mom, &l.gm, &l.gft};
    for (Buf* b : lb) b->release();
  }
  if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto v : ctx->vs) if (v) cudaStreamDestroy(v);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_bfork) cudaEventDestroy(ctx->ev_bfork);
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
  if (n_tris < 0 || n_verts < 0 || (n_tris > 0 && !tris)) return fail(ctx, DSM_ERR_INVALID_ARG, "bad topology arguments");
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
                             const float* light_params, int32_t n_lights, const dsm_camera* cam,
                             const dsm_params* params, float* image) {
  if (!mesh || !cam || !params || !image) return fail(ctx, DSM_ERR_INVALID_ARG, "null argument");
  if (n_lights < 0 || n_lights > DSM_MAX_LIGHTS) return fail(ctx, DSM_ERR_INVALID_ARG, "n_lights out of range");
  if (n_lights > 0 && (!lights || !light_params)) return fail(ctx, DSM_ERR_INVALID_ARG, "null light arrays");
  if (mesh->n_verts < 0 || mesh->n_tris < 0) return fail(ctx, DSM_ERR_INVALID_ARG, "negative mesh size");
  if ((mesh->n_verts > 0 && !mesh->verts) || (mesh->n_tris > 0 && !mesh->tris))
    return fail(ctx, DSM_ERR_INVALID_ARG, "null mesh arrays");
  if (mesh->n_materials < 1 || !mesh->albedo) return fail(ctx, DSM_ERR_INVALID_ARG, "no albedo table");
  if (mesh->n_tris != ctx->topo_T || mesh->n_verts != ctx->topo_V)
    return fail(ctx, DSM_ERR_NO_TOPOLOGY, "dsm_set_topology was not called for this mesh size");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(ctx, DSM_ERR_INVALID_ARG, "camera size out of range");
  for (int l = 0; l < n_lights; ++l) {
    const dsm_light& L = lights[l];
    if (L.type != 0 && L.type != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "unknown light type");
    if (L.res < 1 || L.res > 16384) return fail(ctx, DSM_ERR_INVALID_ARG, "shadow-map size out of range");
    if (!(L.far_plane > L.near_plane)) return fail(ctx, DSM_ERR_INVALID_ARG, "far must exceed near");
    if (L.type == 0 && !(L.ortho_half > 0.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "ortho_half must be positive");
    if (L.type == 1 && !(L.fov_y_deg > 0.f && L.fov_y_deg < 180.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "bad fov");
    if (!(L.sigma > 0.f) && L.radius <= 0) return fail(ctx, DSM_ERR_INVALID_ARG, "filter needs sigma or radius");
    if (L.radius > 32) return fail(ctx, DSM_ERR_INVALID_ARG, "filter radius above 32");
  }
  if (params->filter_kind != 0 && params->filter_kind != 1) return fail(ctx, DSM_ERR_INVALID_ARG, "filter_kind");
  if (params->filter_boundary != 0 && params->filter_boundary != 1)
    return fail(ctx, DSM_ERR_INVALID_ARG, "filter_boundary");
  if (params->recompute_in_backward != 0) return fail(ctx, DSM_ERR_INVALID_ARG, "recompute_in_backward unsupported");
  if (!(params->min_variance >= 0.f)) return fail(ctx, DSM_ERR_INVALID_ARG, "min_variance");
  return DSM_OK;
}

static dsm_status ensure_view(dsm_ctx* ctx, ViewBufs& v, int W, int H, int V, int T, bool is_light) {
  v.W = W;
  v.H = H;
  v.tilesX = (W + kTile - 1) / kTile;
  v.tilesY = (H + kTile - 1) / kTile;
  const size_t tiles = (size_t)v.tilesX * v.tilesY;
  const size_t Vn = std::max(V, 1), Tn = std::max(T, 1);
  DSM_CHECK(v.clip.ensure(Vn * sizeof(float4)));
  DSM_CHECK(v.snap.ensure(Vn * sizeof(VertSnap)));
  DSM_CHECK(v.setup.ensure(Tn * sizeof(TriSetup)));
  DSM_CHECK(v.orient.ensure(Tn));
  DSM_CHECK(v.sil.ensure(Tn));
  DSM_CHECK(v.count.ensure(tiles * 4));
  DSM_CHECK(v.offset.ensure(2 * tiles * 4));
  DSM_CHECK(v.gbuf.ensure((size_t)W * H * sizeof(float4)));
  DSM_CHECK(v.gclip.ensure(Vn * sizeof(float4)));
  DSM_CHECK(v.big_index.ensure(Tn * 4));
  DSM_CHECK(v.big_tri.ensure(kMaxBig * 4));
  DSM_CHECK(v.big_acc.ensure((size_t)kMaxBig * kBigSlots * (is_light ? kBigStrideSm : kBigStrideCam) * 4));
  if (is_light) {
    DSM_CHECK(v.depth.ensure(Vn * 4));
  }
  DSM_CHECK(v.aa_list.ensure((size_t)W * H * 4));
  DSM_CHECK(v.aa_ctr.ensure(sizeof(int)));
  DSM_CHECK(v.hflag.ensure((size_t)W * H));
  if (v.list_cap == 0) {
    const size_t cap = 2 * Tn + 2 * tiles + 1024;
    DSM_CHECK(v.list.ensure(cap * 4));
    v.list_cap = (int)cap;
  }
  return DSM_OK;
}

dsm_status dsm_render(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights, const float* light_params,
                      int32_t n_lights, const dsm_camera* cam, const dsm_params* params, float* image) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  dsm_status s = check_args(ctx, mesh, lights, light_params, n_lights, cam, params, image);
  if (s != DSM_OK) return s;
  ctx->have_fwd = false;
  cudaStream_t st = (cudaStream_t)params->stream;
  const int V = mesh->n_verts, T = mesh->n_tris, L = n_lights;
  const int Wc = cam->width, Hc = cam->height;

  // ---- buffers
  uint64_t sig = mix(mix(mix(1, V), T), L);
  sig = mix(mix(sig, Wc), Hc);
  for (int l = 0; l < L; ++l) {
    s = ensure_view(ctx, ctx->view[l], lights[l].res, lights[l].res, V, T, true);
    if (s != DSM_OK) return s;
    LightBufs& lb = ctx->light[l];
    const size_t R2 = (size_t)lights[l].res * lights[l].res * sizeof(float2);
    DSM_CHECK(lb.fmap.ensure(R2));
    DSM_CHECK(lb.ftilde.ensure(R2));
    DSM_CHECK(lb.tmp.ensure(R2));
    DSM_CHECK(lb.mom.ensure(R2));
    lb.res = lights[l].res;
    make_filter_args(lights[l].sigma, lights[l].radius, params->filter_kind, params->filter_boundary, &lb.fa);
    sig = mix(mix(sig, lights[l].res), lights[l].type);
  }
  s = ensure_view(ctx, ctx->view[L], Wc, Hc, V, T, false);
  if (s != DSM_OK) return s;
  DSM_CHECK(ctx->lights_dev.ensure(sizeof(LightDev) * DSM_MAX_LIGHTS));
  DSM_CHECK(ctx->viewM.ensure(sizeof(float) * 20 * (DSM_MAX_LIGHTS + 1)));
  DSM_CHECK(ctx->vnormal.ensure(sizeof(float) * 3 * std::max(V, 1)));
  DSM_CHECK(ctx->vnlen.ensure(sizeof(float) * std::max(V, 1)));
  DSM_CHECK(ctx->camcolor.ensure((size_t)Wc * Hc * sizeof(float4)));

  // ---- light cameras and the camera matrix
  LightSetupArgs la{};
  la.n = L;
  for (int l = 0; l < L; ++l) {
    const dsm_light& Lh = lights[l];
    LightConst& c = la.c[l];
    c.type = Lh.type;
    c.res = Lh.res;
    c.dist = Lh.dist;
    c.ortho_half = Lh.ortho_half;
    c.near_plane = Lh.near_plane;
    c.far_plane = Lh.far_plane;
    c.persp_c = Lh.type == 1 ? 1.0 / std::tan((double)Lh.fov_y_deg * M_PI / 360.0) : 0.0;
    c.intensity[0] = Lh.intensity[0]; c.intensity[1] = Lh.intensity[1]; c.intensity[2] = Lh.intensity[2];
  }
  float* viewM = ctx->viewM.as<float>();
  LightDev* ldev = ctx->lights_dev.as<LightDev>();
  StageTimer t_setup(ctx, ST_SETUP, st);
  if (L > 0) launch_light_setup(light_params, la, ldev, viewM, st);
  Mat20 cm{};
  for (int k = 0; k < 16; ++k) cm.v[k] = cam->clip[k];
  count_launches(1);
  set_matrix_kernel<<<1, 32, 0, st>>>(cm, viewM + 20 * L);
  // every view at once: transform, triangle setup, silhouettes (and zeroed
  // tile counters for the binning)
  DevStatus* dstat = ctx->status.as<DevStatus>();
  {
    ViewSetupArgs va{};
    va.n = L + 1;
    for (int w = 0; w <= L; ++w) {
      ViewBufs& v = ctx->view[w];
      va.W[w] = v.W; va.H[w] = v.H; va.tiles[w] = v.tilesX * v.tilesY;
      va.clip[w] = v.clip.as<float4>();
      va.snap[w] = v.snap.as<VertSnap>();
      va.depth[w] = w < L ? v.depth.as<float>() : nullptr;
      va.setup[w] = v.setup.as<TriSetup>();
      va.orient[w] = v.orient.as<int8_t>();
      va.sil[w] = v.sil.as<uint8_t>();
      va.count[w] = v.count.as<int>();
      va.aa_count[w] = v.aa_ctr.as<int>();
    }
    launch_setup_all(mesh->verts, V, mesh->tris, T, ctx->adj.as<int>(), viewM, va, dstat, st);
  }
  t_setup.stop();

  // ---- per view on its own stream: bin count, scan (the light views and the
  // camera view are independent until shading)
  DSM_CHECK(ensure_streams(ctx));
  DSM_CHECK(fork_views(ctx, st, ctx->ev_fork, L + 1));
  {
    cudaStream_t cst = view_stream(ctx, L, st);
    StageTimer tn(ctx, ST_SETUP, cst);
    launch_vertex_normals(mesh->verts, V, mesh->tris, ctx->vf_off.as<int>(), ctx->vf_list.as<int>(),
                          ctx->vnormal.as<float>(), ctx->vnlen.as<float>(), cst);
  }
  for (int w = 0; w <= L; ++w) {
    ViewBufs& v = ctx->view[w];
    cudaStream_t vst = view_stream(ctx, w, st);
    StageTimer tw(ctx, ST_SETUP, vst);
    launch_bin_count(v.setup.as<TriSetup>(), T, v.tilesX, v.count.as<int>(), dstat, w, v.big_index.as<int>(),
                     v.big_tri.as<int>(), vst);
    launch_scan(v.count.as<int>(), v.tilesX * v.tilesY, v.offset.as<int>(), dstat, w, vst);
  }
  DSM_CHECK(cudaGetLastError());
  if (ctx->sized_sig != sig) {
    // first frame of this scene size: read the pair counts once and size the lists
    DSM_CHECK(join_views(ctx, st, L + 1));
    DSM_CHECK(cudaMemcpyAsync(ctx->hstatus, dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    DSM_CHECK(cudaStreamSynchronize(st));
    for (int w = 0; w <= L; ++w) {
      ViewBufs& v = ctx->view[w];
      const long long need = ctx->hstatus->needed_pairs[w];
      if (need > v.list_cap) {
        const long long cap = need + need / 2 + 1024;
        if (cap > 0x7fffffffLL) return fail(ctx, DSM_ERR_CAPACITY, "tile list above 2^31 entries");
        DSM_CHECK(v.list.ensure((size_t)cap * 4));
        v.list_cap = (int)cap;
      }
    }
    ctx->sized_sig = sig;
    DSM_CHECK(fork_views(ctx, st, ctx->ev_fork, L + 1));
  }
  // ---- per view: bin fill, raster; per light: Alg. 1 (f, f^2 -> antialias -> filter)
  for (int w = 0; w <= L; ++w) {
    ViewBufs& v = ctx->view[w];
    cudaStream_t vst = view_stream(ctx, w, st);
    {
      StageTimer t(ctx, ST_BIN_FILL, vst);
      launch_bin_fill(v.setup.as<TriSetup>(), T, v.tilesX, v.count.as<int>(), v.offset.as<int>(), v.list.as<int>(),
                      v.list_cap, dstat, w, v.big_index.as<int>(), v.big_tri.as<int>(), vst);
    }
    {
      StageTimer t(ctx, ST_RASTER, vst);
      launch_raster(v.setup.as<TriSetup>(), v.offset.as<int>(), v.list.as<int>(), v.list_cap, v.tilesX, v.tilesY, v.W,
                    v.H, v.clip.as<float4>(), mesh->tris, v.gbuf.as<float4>(), w < L ? v.depth.as<float>() : nullptr,
                    w < L ? ctx->light[w].fmap.as<float2>() : nullptr, vst);
    }
    if (w == L) continue;
    LightBufs& lb = ctx->light[w];
    {
      StageTimer t(ctx, ST_SM_AA, vst);
      if (params->aa_shadow) {
        AAArgs aa{v.gbuf.as<float4>(), v.W, v.H, mesh->tris, v.sil.as<uint8_t>(), v.snap.as<VertSnap>(),
                  v.clip.as<float4>()};
        launch_aa_detect(aa, v.hflag.as<uint8_t>(), v.aa_work(), vst);
        launch_aa_forward2_list(aa, lb.fmap.as<float2>(), lb.ftilde.as<float2>(), v.aa_work(), vst);
      }
    }
    {
      // f~ = f except at the listed texels, whose values the list pass left in ftilde
      StageTimer t(ctx, ST_FILTER, vst);
      launch_filter(lb.fmap.as<float2>(), lb.tmp.as<float2>(), lb.mom.as<float2>(), v.W, lb.fa, vst,
                    params->aa_shadow ? v.hflag.as<uint8_t>() : nullptr, lb.ftilde.as<float2>());
    }
  }
  DSM_CHECK(join_views(ctx, st, L + 1));
  DSM_CHECK(cudaGetLastError());

  // ---- camera: shade (Alg. 2 x Lambert) and the final antialiasing
  ViewBufs& cv = ctx->view[L];
  ShadeArgs sa{};
  sa.gbuf = cv.gbuf.as<float4>();
  sa.W = Wc; sa.H = Hc;
  sa.verts = mesh->verts; sa.tris = mesh->tris; sa.tri_mat = mesh->tri_material;
  sa.albedo = mesh->albedo; sa.n_mat = mesh->n_materials;
  sa.vnormal = ctx->vnormal.as<float>();
  sa.cam_clip = cv.clip.as<float4>();
  sa.lights = ldev; sa.L = L;
  for (int l = 0; l < L; ++l) { sa.mom[l] = ctx->light[l].mom.as<float2>(); sa.res[l] = lights[l].res; }
  sa.min_variance = params->min_variance;
  {
    StageTimer t(ctx, ST_SHADE, st);
    launch_shade(sa, ctx->camcolor.as<float4>(), st);
  }
  StageTimer t_final(ctx, ST_FINAL_AA, st);
  if (params->aa_final) {
    AAArgs aa{cv.gbuf.as<float4>(), Wc, Hc, mesh->tris, cv.sil.as<uint8_t>(), cv.snap.as<VertSnap>(),
              cv.clip.as<float4>()};
    launch_aa_forward4(aa, ctx->camcolor.as<float4>(), reinterpret_cast<float4*>(image), cv.hflag.as<uint8_t>(),
                       cv.aa_work(), st);
  } else {
    DSM_CHECK(cudaMemcpyAsync(image, ctx->camcolor.p, (size_t)Wc * Hc * sizeof(float4), cudaMemcpyDeviceToDevice, st));
  }
  t_final.stop();
  DSM_CHECK(cudaGetLastError());

  ctx->mesh = *mesh;
  for (int l = 0; l < L; ++l) ctx->lights[l] = lights[l];
  ctx->L = L;
  ctx->cam = *cam;
  ctx->params = *params;
  ctx->stream = st;
  ctx->have_fwd = true;
  return DSM_OK;
}

dsm_status dsm_render_backward(dsm_ctx* ctx, const float* dL_dimage, float* dL_dverts, float* dL_dlight,
                               float* dL_dalbedo) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (!ctx->have_fwd) return fail(ctx, DSM_ERR_NO_FORWARD, "dsm_render_backward without a forward");
  if (!dL_dimage) return fail(ctx, DSM_ERR_INVALID_ARG, "null dL_dimage");
  cudaStream_t st = ctx->stream;
  const dsm_mesh& mesh = ctx->mesh;
  const int V = mesh.n_verts, T = mesh.n_tris, L = ctx->L;
  const int Wc = ctx->cam.width, Hc = ctx->cam.height;
  if (!dL_dverts) { DSM_CHECK(ctx->scratch_dverts.ensure(sizeof(float) * 3 * std::max(V, 1))); dL_dverts = ctx->scratch_dverts.as<float>(); }
  if (!dL_dlight) { DSM_CHECK(ctx->scratch_dlight.ensure(sizeof(float) * 6 * DSM_MAX_LIGHTS)); dL_dlight = ctx->scratch_dlight.as<float>(); }
  if (!dL_dalbedo) { DSM_CHECK(ctx->scratch_dalbedo.ensure(sizeof(float) * 3 * mesh.n_materials)); dL_dalbedo = ctx->scratch_dalbedo.as<float>(); }
  DSM_CHECK(ctx->gcolor.ensure((size_t)Wc * Hc * sizeof(float4)));
  DSM_CHECK(ctx->pgrad.ensure((size_t)Wc * Hc * 2 * sizeof(float4)));
  DSM_CHECK(ctx->gnormal.ensure(sizeof(float) * 3 * std::max(V, 1)));
  DSM_CHECK(ctx->gN.ensure(sizeof(float) * 3 * std::max(V, 1)));
  DSM_CHECK(ctx->gface.ensure(sizeof(float) * 3 * std::max(T, 1)));
  DSM_CHECK(ctx->gQ.ensure(sizeof(float) * 20 * DSM_MAX_LIGHTS));
  DSM_CHECK(ctx->gdirect.ensure(sizeof(float) * 3 * DSM_MAX_LIGHTS));
  const int n_mat_red = mesh.n_materials <= kMaxSharedMat ? mesh.n_materials : 0;
  const int red_stride = 23 * L + 3 * n_mat_red;
  DSM_CHECK(ctx->red.ensure(sizeof(float) * kRedSlots * std::max(red_stride, 1)));
  for (int l = 0; l < L; ++l) {
    const size_t R2 = (size_t)ctx->light[l].res * ctx->light[l].res * sizeof(float2);
    DSM_CHECK(ctx->light[l].gm.ensure(R2));
    DSM_CHECK(ctx->light[l].gft.ensure(R2));
  }
  // ---- clear accumulators and outputs
  StageTimer t_clear(ctx, ST_BWD_CLEAR, st);
  {
    Clearer cl;
    cl.add(dL_dverts, sizeof(float) * 3 * V);
    if (L) cl.add(dL_dlight, sizeof(float) * 6 * L);
    cl.add(dL_dalbedo, sizeof(float) * 3 * mesh.n_materials);
    cl.add(ctx->gnormal.p, sizeof(float) * 3 * V);
    cl.add(ctx->gQ.p, sizeof(float) * 20 * DSM_MAX_LIGHTS);
    cl.add(ctx->gdirect.p, sizeof(float) * 3 * DSM_MAX_LIGHTS);
    for (int w = 0; w <= L; ++w) cl.add(ctx->view[w].gclip.p, sizeof(float4) * V);
    for (int l = 0; l < L; ++l)
      cl.add(ctx->light[l].gm.p, (size_t)ctx->light[l].res * ctx->light[l].res * sizeof(float2));
    cl.add(ctx->red.p, sizeof(float) * kRedSlots * red_stride);
    for (int w = 0; w <= L; ++w)
      cl.add(ctx->view[w].big_acc.p, (size_t)kMaxBig * kBigSlots * (w < L ? kBigStrideSm : kBigStrideCam) * 4);
    static_assert(6 + 3 * (DSM_MAX_LIGHTS + 1) <= kMaxClear, "clear list");
    cl.launch(st);
  }
  DSM_CHECK(cudaGetLastError());

  t_clear.stop();
  // ---- final antialiasing adjoint and the shading adjoint
  ViewBufs& cv = ctx->view[L];
  StageTimer t_faa(ctx, ST_BWD_FINAL_AA, st);
  AAArgs caa{cv.gbuf.as<float4>(), Wc, Hc, mesh.tris, cv.sil.as<uint8_t>(), cv.snap.as<VertSnap>(), cv.clip.as<float4>()};
  if (ctx->params.aa_final) {
    launch_aa_backward4(caa, ctx->camcolor.as<float4>(), reinterpret_cast<const float4*>(dL_dimage),
                        ctx->gcolor.as<float4>(), cv.gclip.as<float4>(), cv.hflag.as<uint8_t>(), cv.aa_work(), st);
  } else {
    DSM_CHECK(cudaMemcpyAsync(ctx->gcolor.p, dL_dimage, (size_t)Wc * Hc * sizeof(float4), cudaMemcpyDeviceToDevice,
                              st));
  }
  t_faa.stop();
  ShadeArgs sa{};
  sa.gbuf = cv.gbuf.as<float4>();
  sa.W = Wc; sa.H = Hc;
  sa.verts = mesh.verts; sa.tris = mesh.tris; sa.tri_mat = mesh.tri_material;
  sa.albedo = mesh.albedo; sa.n_mat = mesh.n_materials;
  sa.vnormal = ctx->vnormal.as<float>();
  sa.cam_clip = cv.clip.as<float4>();
  sa.lights = ctx->lights_dev.as<LightDev>(); sa.L = L;
  for (int l = 0; l < L; ++l) { sa.mom[l] = ctx->light[l].mom.as<float2>(); sa.res[l] = ctx->light[l].res; }
  sa.min_variance = ctx->params.min_variance;
  ShadeGradArgs ga{};
  ga.gcolor = ctx->gcolor.as<float4>();
  ga.dverts = dL_dverts;
  ga.gnormal = ctx->gnormal.as<float>();
  ga.gclip = cv.gclip.as<float4>();
  ga.dalbedo = dL_dalbedo;
  for (int l = 0; l < L; ++l) ga.gm[l] = ctx->light[l].gm.as<float2>();
  ga.red = ctx->red.as<float>();
  ga.red_stride = red_stride;
  ga.big = cv.big_index.as<int>();
  ga.big_acc = cv.big_acc.as<float>();
  ga.pgrad = ctx->pgrad.as<float4>();
  {
    StageTimer t(ctx, ST_BWD_SHADE, st);
    launch_shade_backward(sa, ga, st);
  }
  // ---- per light on its own stream: G^T, antialiasing adjoint, interpolation
  // adjoint (they write only that light's buffers), beside the camera scatter
  DSM_CHECK(ensure_streams(ctx));
  DSM_CHECK(fork_views(ctx, st, ctx->ev_bfork, L));
  for (int l = 0; l < L; ++l) {
    ViewBufs& v = ctx->view[l];
    LightBufs& lb = ctx->light[l];
    cudaStream_t vst = view_stream(ctx, l, st);
    AAArgs aa{v.gbuf.as<float4>(), v.W, v.H, mesh.tris, v.sil.as<uint8_t>(), v.snap.as<VertSnap>(), v.clip.as<float4>()};
    {
      StageTimer t(ctx, ST_BWD_FILTER, vst);
      // dL/d(f~, (f^2)~) and, folded through f^2 = f f, dL/df (into tmp)
      launch_filter_adjoint(lb.gm.as<float2>(), lb.tmp.as<float2>(), lb.gft.as<float2>(), v.W, lb.fa, vst,
                            lb.fmap.as<float2>(), lb.tmp.as<float>());
    }
    {
      // the listed texels: dL/df through the antialiasing (overwrites tmp there)
      StageTimer t(ctx, ST_BWD_SM_AA, vst);
      if (ctx->params.aa_shadow)
        launch_sm_aa_adjoint_list(aa, lb.fmap.as<float2>(), lb.gft.as<float2>(), v.gclip.as<float4>(),
                                  lb.tmp.as<float>(), v.aa_work(), vst);
    }
    {
      StageTimer t(ctx, ST_BWD_SM_INTERP, vst);
      BigArgs big{v.big_index.as<int>(), v.big_tri.as<int>(), v.big_acc.as<float>(), ctx->status.as<DevStatus>(), l};
      launch_sm_interp_adjoint(aa, lb.tmp.as<float>(), v.depth.as<float>(), v.gclip.as<float4>(), big, vst);
    }
  }
  {
    StageTimer t(ctx, ST_BWD_SHADE_SCATTER, st);
    launch_shade_scatter(sa, ga, st);
    launch_shade_big_resolve(sa, ga, cv.big_tri.as<int>(), ctx->status.as<DevStatus>(), L, st);
  }
  DSM_CHECK(join_views(ctx, st, L));
  // ---- vertices, normals, lights
  StageTimer t_vert(ctx, ST_BWD_VERTEX, st);
  VertGradPtrs gp{};
  for (int w = 0; w <= L; ++w) gp.gclip[w] = ctx->view[w].gclip.as<float4>();
  launch_vertex_backward(mesh.verts, V, ctx->viewM.as<float>(), L + 1, L, gp, dL_dverts, ctx->red.as<float>(),
                         red_stride, st);
  launch_normals_backward(mesh.verts, V, mesh.tris, T, ctx->vf_off.as<int>(), ctx->vf_list.as<int>(),
                          ctx->vnormal.as<float>(), ctx->vnlen.as<float>(), ctx->gnormal.as<float>(),
                          ctx->gN.as<float>(), ctx->gface.as<float>(), dL_dverts, st);
  launch_red_reduce(ctx->red.as<float>(), red_stride, L, n_mat_red, ctx->gQ.as<float>(), ctx->gdirect.as<float>(),
                    dL_dalbedo, st);
  launch_light_grad(ctx->lights_dev.as<LightDev>(), L, ctx->gQ.as<float>(), ctx->gdirect.as<float>(), dL_dlight, st);
  DSM_CHECK(cudaGetLastError());
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
  if (!in || !out || res < 1 || res > 16384 || (kind != 0 && kind != 1) || (boundary != 0 && boundary != 1) ||
      radius > 32 || (!(sigma > 0.f) && radius <= 0))
    return fail(ctx, DSM_ERR_INVALID_ARG, "bad filter arguments");
  DSM_CHECK(ctx->filter_tmp.ensure((size_t)res * res * sizeof(float2)));
  FilterArgs fa;
  make_filter_args(sigma, radius, kind, boundary, &fa);
  launch_filter(reinterpret_cast<const float2*>(in), ctx->filter_tmp.as<float2>(), reinterpret_cast<float2*>(out), res,
                fa, (cudaStream_t)stream);
  DSM_CHECK(cudaGetLastError());
  return DSM_OK;
}

dsm_status dsm_filter_moments_adjoint(dsm_ctx* ctx, const float* gout, float* gin, int32_t res, float sigma,
                                      int32_t radius, int32_t kind, int32_t boundary, void* stream) {
  if (!ctx) return DSM_ERR_INVALID_ARG;
  if (!gout || !gin || res < 1 || res > 16384 || (kind != 0 && kind != 1) || (boundary != 0 && boundary != 1) ||
      radius > 32 || (!(sigma > 0.f) && radius <= 0))
    return fail(ctx, DSM_ERR_INVALID_ARG, "bad filter arguments");
  DSM_CHECK(ctx->filter_tmp.ensure((size_t)res * res * sizeof(float2)));
  FilterArgs fa;
  make_filter_args(sigma, radius, kind, boundary, &fa);
  launch_filter_adjoint(reinterpret_cast<const float2*>(gout), ctx->filter_tmp.as<float2>(),
                        reinterpret_cast<float2*>(gin), res, fa, (cudaStream_t)stream);
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
  const void* src = nullptr;
  size_t size = 0;
  auto light_ok = [&](int i) { return i >= 0 && i < L; };
  auto view_ok = [&](int i) { return i >= 0 && i <= L; };
  switch (what) {
    case 0: if (view_ok(index)) { src = ctx->view[index].gbuf.p; size = (size_t)ctx->view[index].W * ctx->view[index].H * 16; } break;
    case 1: if (light_ok(index)) { src = ctx->light[index].fmap.p; size = (size_t)ctx->light[index].res * ctx->light[index].res * 8; } break;
    case 2: if (light_ok(index)) { src = ctx->light[index].ftilde.p; size = (size_t)ctx->light[index].res * ctx->light[index].res * 8; } break;
    case 3: if (light_ok(index)) { src = ctx->light[index].mom.p; size = (size_t)ctx->light[index].res * ctx->light[index].res * 8; } break;
    case 4: src = ctx->camcolor.p; size = (size_t)ctx->cam.width * ctx->cam.height * 16; break;
    case 5: src = ctx->viewM.p; size = (size_t)L * 20 * 4; break;
    case 6: if (view_ok(index)) { src = ctx->view[index].snap.p; size = (size_t)V * 16; } break;
    case 7: if (light_ok(index)) { src = ctx->light[index].gm.p; size = (size_t)ctx->light[index].res * ctx->light[index].res * 8; } break;
    case 8: if (view_ok(index)) { src = ctx->view[index].gclip.p; size = (size_t)V * 16; } break;
    case 9: if (light_ok(index)) { src = ctx->light[index].gft.p; size = (size_t)ctx->light[index].res * ctx->light[index].res * 8; } break;
    case 10: src = ctx->gcolor.p; size = (size_t)ctx->cam.width * ctx->cam.height * 16; break;
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

}  // extern "C"
