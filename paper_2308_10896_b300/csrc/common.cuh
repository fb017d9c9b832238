// Device-side definitions shared by the kernels of the shadow-mapping library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dsm {

constexpr int kSubpix = 256;          // 8 sub-pixel bits: 24.8 fixed point
constexpr int kGuard = 1 << 28;       // |snapped coordinate| limit; beyond it a triangle is culled
constexpr float kWMin = 1e-6f;        // clip w below this culls the triangle
constexpr int kMaxLightViews = DSM_MAX_LIGHT_VIEWS;            // shadow-map views (cube faces count one each)
constexpr int kMaxViews = kMaxLightViews + DSM_MAX_CAMERAS;     // light views, then camera views
// Raster tile side 2^tile_log2 pixels: 16 or 32 per view (chosen by the
// tuning of the context; 32 by default).
constexpr int kTileLog2Min = 4, kTileLog2Max = 5, kTileLog2Default = 5;
constexpr unsigned kFull = 0xffffffffu;

// Snapped vertex of one view: 24.8 fixed-point screen position, ndc depth,
// validity (w >= kWMin and inside the guard band).
struct __align__(16) VertSnap {
  int X, Y;
  float z;
  int ok;
};

// Per-triangle raster record of one view (64 bytes, loaded whole into shared
// memory by the tile rasteriser).
struct __align__(16) TriSetup {
  int X[3], Y[3];     // snapped vertices
  float z[3];         // ndc depth of the vertices
  float a2f;          // float(2A), 2A > 0 after orientation normalisation
  int ibox, jbox;     // pixel bbox: i0 | i1 << 16, j0 | j1 << 16 (empty: i0 > i1)
  int tri;            // triangle index
  int flags;          // bit 0..2: top-left flag of edge k; bit 3: s = -1; bit 4: visible
  int pad[2];
};
static_assert(sizeof(TriSetup) == 64, "TriSetup must be 64 bytes");

// Light record written by the light-camera kernel: Q rows 0-3 = clip matrix,
// row 4 = depth row; J = dQ/d(pos, dir) (20 x 6, row-major).
struct LightDev {
  float Q[20];
  float J[120];
  float fwd[3];       // normalised travel direction
  float dir_norm;     // |dir|
  float pos[3];
  int type;           // 0 directional, 1 perspective (spot light or a cube face of a point light)
  int res;
  float intensity[3];
  int face;           // cube face 0..5 (+X, -X, +Y, -Y, +Z, -Z) of a point light, -1 otherwise
  int user;           // index of the light in the caller's arrays
};

// Device status word (errors raised by kernels, read by dsm_sync).
struct DevStatus {
  int capacity_overflow;
  int timeout;
  int needed_pairs[kMaxViews];
  int big_count[kMaxViews];   // triangles of each view flagged as big
  int units[kMaxViews];       // raster work units of each view (record batches of its tiles)
  int split[kMaxViews];       // tiles of each view raster by several units (key slots in use)
};

// Contention control for gradient scatters.  A triangle whose pixel bbox spans
// at least big_tiles raster tiles (a binning parameter of the view, default
// kBigTilesDefault) is "big": it is binned per tile (each tile tests the
// view's few big triangles) rather than per triangle, and in the backward its
// per-triangle sums go to
// kBigSlots private copies (spread over L2) instead of straight onto its three
// vertices, and a resolve kernel adds the copies up.  Block-level reductions
// of the light and albedo gradients likewise go to kRedSlots copies.
constexpr int kBigTilesDefault = 16;
constexpr int kMaxBig = 64;
constexpr int kBigSlots = 64;
constexpr int kBigStrideSm = 32;      // floats per slot copy (15 used), one 128-byte line each
constexpr int kBigStrideCam = 32;     // floats per slot copy (30 used)
constexpr int kRedSlots = 64;
constexpr int kMaxSharedMat = 256;      // albedo tables up to this size are reduced in shared memory

__device__ __forceinline__ int block_slot(int n) {
  return (int)((blockIdx.x * 0x9E3779B1u + blockIdx.y * 0x85EBCA77u) >> 16) & (n - 1);
}

__device__ __forceinline__ int scatter_slot(int n) {
  return (int)((blockIdx.x * 0x9E3779B1u + blockIdx.y * 0x85EBCA77u + threadIdx.y * 0xC2B2AE3Du) >> 16) & (n - 1);
}

// Face normal cross(v1 - v0, v2 - v0) of triangle t (area-weighted, unnormalised).
__device__ __forceinline__ float3 face_normal(const float* __restrict__ verts, const int* __restrict__ tris, int t) {
  const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
  const float3 v0 = make_float3(verts[3 * a], verts[3 * a + 1], verts[3 * a + 2]);
  const float3 e1 = make_float3(verts[3 * b] - v0.x, verts[3 * b + 1] - v0.y, verts[3 * b + 2] - v0.z);
  const float3 e2 = make_float3(verts[3 * c] - v0.x, verts[3 * c + 1] - v0.y, verts[3 * c + 2] - v0.z);
  return make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
}

// Vertex normals: the area-weighted sum of the incident face normals of
// vertex v (faces off[v] .. off[v + 1] of lst), normalised; its length kept
// for the adjoint.
struct VertNormalArgs {
  const float* verts;
  int V;
  const int* tris;
  const int* off;
  const int* lst;
  float* vn;
  float* vlen;
};
__device__ __forceinline__ void vertex_normal_at(const VertNormalArgs& a, int v) {
  float3 s = make_float3(0.f, 0.f, 0.f);
  for (int k = a.off[v]; k < a.off[v + 1]; ++k) {
    const float3 f = face_normal(a.verts, a.tris, a.lst[k]);
    s.x += f.x; s.y += f.y; s.z += f.z;
  }
  const float l = sqrtf(s.x * s.x + s.y * s.y + s.z * s.z);
  const float il = l > 0.f ? 1.f / l : 1.f;
  a.vn[3 * v] = s.x * il; a.vn[3 * v + 1] = s.y * il; a.vn[3 * v + 2] = s.z * il;
  a.vlen[v] = l;
}

// Exact float32 -> float64 widening from the bit fields of the two IEEE 754
// formats (exponent rebiased by 1023 - 127 = 896, the 23 fraction bits at the
// top of the 52), on the integer pipes; zeros keep their sign, and subnormal,
// infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ double widen_exact(float v) {
  const unsigned u = __float_as_uint(v), e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e == 0u || e == 0xffu) return (double)v;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}

__device__ __forceinline__ uint32_t order_bits(float z) {
  uint32_t u = __float_as_uint(z);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ uint64_t depth_key(float z, int tri) {
  return (static_cast<uint64_t>(order_bits(z)) << 32) | static_cast<uint32_t>(tri);
}

// Edge vertex pairs in the order the antialiasing scans them: v0v1, v1v2, v2v0.
__device__ __forceinline__ int edge_p(int e) { return e; }
__device__ __forceinline__ int edge_q(int e) { return e == 2 ? 0 : e + 1; }

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// Moment channels of a shadow-map depth sample f: (w, w^2) with w = f
// (variance shadow maps) or w = exp(ec f) (exponential variance shadow maps,
// ec > 0: the exponent c of the warp).
__device__ __forceinline__ float2 moment_encode(float f, float ec) {
  const float w = ec > 0.f ? expf(ec * f) : f;
  return make_float2(w, w * w);
}

// dL/df of a texel from the gradient g of its channels (w, w^2): the product
// rule of w^2 = w w, times dw/df (1, or ec w for the exponential warp).
__device__ __forceinline__ float moment_fold(float2 g, float w, float ec) {
  const float gw = g.x + 2.f * w * g.y;
  return ec > 0.f ? gw * (ec * w) : gw;
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float dotv(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ float dotv(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return f2add(a, b); }
__device__ __forceinline__ float4 vadd(float4 a, float4 b) { return f4add(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return f2sub(a, b); }
__device__ __forceinline__ float4 vsub(float4 a, float4 b) { return f4sub(a, b); }
__device__ __forceinline__ float2 vscale(float2 a, float s) { return f2scale(a, s); }
__device__ __forceinline__ float4 vscale(float4 a, float s) { return f4scale(a, s); }
template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Error-free float32 transformations: a b = p + e (one fused multiply-add)
// and a + b = s + e (Knuth's two-sum), both exact.  The explicitly rounded
// intrinsics keep the compiler from contracting or reordering them.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Unsnapped screen positions are held per vertex as float-float pairs
// (sx_hi, sx_lo, sy_hi, sy_lo) with sx = (x / w / 2 + 1/2) W and
// sy = (1/2 - y / w / 2) H of the exact clip coordinates: the product of the
// vertex with the view matrix carried exactly, not the pinned float32
// transform that every discrete decision uses (see transform_all_kernel).
// An offset from a pixel centre, (sx_hi - (i + 1/2)) + sx_lo, then keeps
// float32 accuracy relative to the offset itself, even for a vertex ~1000
// pixels from the view's origin next to that centre.
__device__ __forceinline__ float scr_dx(float4 scr, int i) { return (scr.x - ((float)i + 0.5f)) + scr.y; }
__device__ __forceinline__ float scr_dy(float4 scr, int j) { return (scr.z - ((float)j + 0.5f)) + scr.w; }

// Perspective-correct barycentrics at the centre of pixel (i, j) of the
// triangle with clip vertices hi[k] (w) and screen positions scr[k]:
// b ~ a x c with a_k = x_k - px w_k = (2/W) w_k (sx_k - i - 1/2) and
// c_k = y_k - py w_k = -(2/H) w_k (sy_k - j - 1/2) (px, py the centre's ndc).
// The offsets come from the float-float screen positions, so b keeps float32
// accuracy relative to the triangle's own size even for sub-pixel triangles
// far from the view's origin.
struct Bary {
  float b[3];
  float a[3], c[3];
  float beta[3];
  float S;
};

__device__ __forceinline__ Bary bary_at(const float4 (&hi)[3], const float4 (&scr)[3], int i, int j, int W, int H) {
  Bary r;
  const float sx = 2.0f / (float)W, sy = -2.0f / (float)H;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.a[k] = scr_dx(scr[k], i) * (hi[k].w * sx);
    r.c[k] = scr_dy(scr[k], j) * (hi[k].w * sy);
  }
  r.beta[0] = r.a[1] * r.c[2] - r.a[2] * r.c[1];
  r.beta[1] = r.a[2] * r.c[0] - r.a[0] * r.c[2];
  r.beta[2] = r.a[0] * r.c[1] - r.a[1] * r.c[0];
  r.S = r.beta[0] + r.beta[1] + r.beta[2];
  float iS = 1.0f / r.S;
  r.b[0] = r.beta[0] * iS; r.b[1] = r.beta[1] * iS; r.b[2] = r.beta[2] * iS;
  return r;
}

// Adjoint of bary_at, given the centred gradient gbc_k = dL/db_k - sum_j b_j
// dL/db_j (the normalisation b = beta / S removes the mean): the gradient of
// the three clip vertices.  Callers form gbc from differences of vertex
// attributes, gbc_k = sum_j b_j (dL/db_k - dL/db_j), which stay accurate when
// the attributes of a small triangle's corners nearly agree (subtracting the
// mean of nearly equal float32 values would lose those digits).
__device__ __forceinline__ void bary_backward(const Bary& r, const float gbc[3], float px, float py,
                                              float4 gc[3]) {
  float iS = 1.0f / r.S;
  float gbeta[3] = {gbc[0] * iS, gbc[1] * iS, gbc[2] * iS};
  // beta = a x c:  dL/da = c x gbeta,  dL/dc = gbeta x a
  float ga[3] = {r.c[1] * gbeta[2] - r.c[2] * gbeta[1], r.c[2] * gbeta[0] - r.c[0] * gbeta[2],
                 r.c[0] * gbeta[1] - r.c[1] * gbeta[0]};
  float gcc[3] = {gbeta[1] * r.a[2] - gbeta[2] * r.a[1], gbeta[2] * r.a[0] - gbeta[0] * r.a[2],
                  gbeta[0] * r.a[1] - gbeta[1] * r.a[0]};
  for (int k = 0; k < 3; ++k)
    gc[k] = make_float4(ga[k], gcc[k], 0.f, -px * ga[k] - py * gcc[k]);
}

// ndc of the pixel centre: (2i + 1 - W) / W and (H - 2j - 1) / H.
__device__ __forceinline__ float pix_ndc_x(int i, int W) { return (float)(2 * i + 1 - W) / (float)W; }
__device__ __forceinline__ float pix_ndc_y(int j, int H) { return (float)(H - 2 * j - 1) / (float)H; }

// Warp-aggregated append of `value` to list (one atomic on *count per warp)
// for the lanes with `want`; every lane of the warp must call it.
__device__ __forceinline__ void warp_append(int* list, int* count, bool want, int value) {
  const unsigned m = __ballot_sync(kFull, want);
  if (!m) return;
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (want) list[base + __popc(m & ((1u << lane) - 1))] = value;
}

// The same for up to N values per lane (bit k of `mask`: append v[k]), with
// one atomic per warp for all of them.
template <int N>
__device__ __forceinline__ void warp_append_n(int* list, int* count, unsigned mask, const int (&v)[N]) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int n = __popc(mask);
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  int base = 0;
  if (lane == 31) base = atomicAdd(count, total);
  base = __shfl_sync(kFull, base, 31) + incl - n;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if ((mask >> k) & 1u) list[base++] = v[k];
}

__device__ __forceinline__ void atomic_add4(float4* p, float4 v) {
  atomicAdd(p, v);
}
__device__ __forceinline__ void atomic_add2(float2* p, float2 v) {
  atomicAdd(p, v);
}

// Per-lane register sums for up to K big triangles per warp (a big triangle's
// texels are spread over most lanes and rows of a strip, so their
// contributions are summed in registers and reduced across the warp once, at
// the flush).  The triangles held are the same on every lane; a lane whose big
// triangle finds no free slot adds it through `direct`.  Every lane of the
// warp must call add / flush together; add with b < 0 adds nothing.
template <int N, int K>
struct BigRun {
  int big[K];       // big-triangle index held by each slot, -1 = free (warp-uniform)
  float v[K][N];
};

template <int N, int K>
__device__ __forceinline__ void big_run_reset(BigRun<N, K>& r) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    r.big[s] = -1;
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[s][k] = 0.f;
  }
}

template <int N, int K, typename Direct>
__device__ __forceinline__ void big_run_add(BigRun<N, K>& r, int b, const float (&c)[N], Direct& direct) {
  // claim free slots for big triangles not yet held (warp-uniform decisions)
  auto held = [&](int x) {
    bool h = false;
#pragma unroll
    for (int s = 0; s < K; ++s) h |= (x == r.big[s]);
    return h;
  };
  unsigned m = __ballot_sync(kFull, b >= 0 && !held(b));
  while (m) {
    const int bn = __shfl_sync(kFull, b, __ffs(m) - 1);
    int free_slot = -1;
#pragma unroll
    for (int s = K - 1; s >= 0; --s)
      if (r.big[s] < 0) free_slot = s;
    if (free_slot < 0) break;
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (s == free_slot) r.big[s] = bn;
    m = __ballot_sync(kFull, b >= 0 && !held(b));
  }
  if (b < 0) return;
  bool done = false;
#pragma unroll
  for (int s = 0; s < K; ++s)
    if (b == r.big[s]) {
#pragma unroll
      for (int k = 0; k < N; ++k) r.v[s][k] += c[k];
      done = true;
    }
  if (!done) direct(b, c, threadIdx.x & 31);
}

// flush(big index, sums) is called by lane 0 for each held slot.
template <int N, int K, typename Flush>
__device__ __forceinline__ void big_run_flush(BigRun<N, K>& r, Flush& flush) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (r.big[s] < 0) continue;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float x = r.v[s][k];
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      r.v[s][k] = x;
    }
    if ((threadIdx.x & 31) == 0) flush(r.big[s], r.v[s]);
  }
  big_run_reset(r);
}

}  // namespace dsm
