// Deferred shading of the camera G-buffer (supplementary Sec. A: Lambert summed
// over lights) with the visibility of Alg. 2 (Sec. 3 Chebyshev bound), its
// adjoint (Sec. 4), vertex normals, per-vertex gradient gathers and the light
// parameter chain rule.
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {

// ------------------------------------------------------------------ vertex normals
// dL/d(unnormalised vertex normal) from dL/d(unit normal).
// dL/d unnormalised vertex normal N from dL/d unit normal n = N / |N|:
// (g - n (n.g)) / |N|, with n and |N| saved by the forward.
__global__ void normals_bwd_vertex_kernel(const float* __restrict__ vn, const float* __restrict__ vlen, int V,
                                          const float4* __restrict__ gn, float* __restrict__ gN) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float l = vlen[v];
  const float4 g4 = gn[v];
  const float3 g = make_float3(g4.x, g4.y, g4.z);
  float3 r = g;
  if (l > 0.f) {
    const float il = 1.f / l;
    const float3 n = make_float3(vn[3 * v], vn[3 * v + 1], vn[3 * v + 2]);
    const float d = n.x * g.x + n.y * g.y + n.z * g.z;
    r = make_float3((g.x - n.x * d) * il, (g.y - n.y * d) * il, (g.z - n.z * d) * il);
  }
  gN[3 * v] = r.x; gN[3 * v + 1] = r.y; gN[3 * v + 2] = r.z;
}
__global__ void normals_bwd_face_kernel(const int* __restrict__ tris, int T, const float* __restrict__ gN,
                                        float* __restrict__ gface) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  float3 s = make_float3(0.f, 0.f, 0.f);
  for (int k = 0; k < 3; ++k) {
    const int v = tris[3 * t + k];
    s.x += gN[3 * v]; s.y += gN[3 * v + 1]; s.z += gN[3 * v + 2];
  }
  gface[3 * t] = s.x; gface[3 * t + 1] = s.y; gface[3 * t + 2] = s.z;
}

// F = e1 x e2 (e1 = v1 - v0, e2 = v2 - v0):  dL/de1 = e2 x G,  dL/de2 = G x e1.
// Adds the vertex's face-normal gradient and its position gradient gpos.
__global__ void normals_bwd_gather_kernel(const float* __restrict__ verts, int V, const int* __restrict__ tris,
                                          const int* __restrict__ off, const int* __restrict__ lst,
                                          const float* __restrict__ gface, const float4* __restrict__ gpos,
                                          float* __restrict__ dverts) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float4 gp = gpos[v];
  float3 acc = make_float3(gp.x, gp.y, gp.z);
  for (int k = off[v]; k < off[v + 1]; ++k) {
    const int t = lst[k];
    const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    const float3 v0 = make_float3(verts[3 * a], verts[3 * a + 1], verts[3 * a + 2]);
    const float3 e1 = make_float3(verts[3 * b] - v0.x, verts[3 * b + 1] - v0.y, verts[3 * b + 2] - v0.z);
    const float3 e2 = make_float3(verts[3 * c] - v0.x, verts[3 * c + 1] - v0.y, verts[3 * c + 2] - v0.z);
    const float3 G = make_float3(gface[3 * t], gface[3 * t + 1], gface[3 * t + 2]);
    const float3 g1 = make_float3(e2.y * G.z - e2.z * G.y, e2.z * G.x - e2.x * G.z, e2.x * G.y - e2.y * G.x);
    const float3 g2 = make_float3(G.y * e1.z - G.z * e1.y, G.z * e1.x - G.x * e1.z, G.x * e1.y - G.y * e1.x);
    if (v == b) { acc.x += g1.x; acc.y += g1.y; acc.z += g1.z; }
    if (v == c) { acc.x += g2.x; acc.y += g2.y; acc.z += g2.z; }
    if (v == a) { acc.x -= g1.x + g2.x; acc.y -= g1.y + g2.y; acc.z -= g1.z + g2.z; }
  }
  dverts[3 * v] += acc.x; dverts[3 * v + 1] += acc.y; dverts[3 * v + 2] += acc.z;
}

// ------------------------------------------------------------------ shading
struct Surf {
  int tri, v[3];
  float b[3];
  float3 x, nt, n;     // world position, interpolated normal, unit normal
  float nlen;
};

__device__ __forceinline__ bool load_surf(const ShadeArgs& a, size_t p, Surf& s) {
  const float4 g = a.gbuf[p];
  const int id = __float_as_int(g.x);
  if (!id) return false;
  s.tri = id - 1;
  s.b[0] = g.y; s.b[1] = g.z; s.b[2] = 1.f - g.y - g.z;
  s.x = make_float3(0.f, 0.f, 0.f);
  s.nt = make_float3(0.f, 0.f, 0.f);
  for (int k = 0; k < 3; ++k) {
    const int v = a.tris[3 * s.tri + k];
    s.v[k] = v;
    s.x.x += s.b[k] * a.verts[3 * v]; s.x.y += s.b[k] * a.verts[3 * v + 1]; s.x.z += s.b[k] * a.verts[3 * v + 2];
    s.nt.x += s.b[k] * a.vnormal[3 * v];
    s.nt.y += s.b[k] * a.vnormal[3 * v + 1];
    s.nt.z += s.b[k] * a.vnormal[3 * v + 2];
  }
  s.nlen = sqrtf(s.nt.x * s.nt.x + s.nt.y * s.nt.y + s.nt.z * s.nt.z);
  const float il = s.nlen > 0.f ? 1.f / s.nlen : 0.f;
  s.n = make_float3(s.nt.x * il, s.nt.y * il, s.nt.z * il);
  return true;
}

__device__ __forceinline__ int material_of(const ShadeArgs& a, int tri) {
  const int m = a.tri_mat ? a.tri_mat[tri] : 0;
  return min(max(m, 0), a.n_mat - 1);     // out-of-range material ids read the nearest table entry
}

// Vertex data of one triangle, kept in registers while consecutive pixels of a
// strip hit the same triangle.
struct TriCache {
  int tri = -1;
  int v[3];
  float3 p[3], n[3];
  float4 cc[3], cs[3];   // camera clip coordinates (pinned float32) and float-float screen positions
  int mat;
  float3 alb;
};

__device__ __forceinline__ void tri_load(const ShadeArgs& a, int t, TriCache& c) {
  c.tri = t;
  for (int k = 0; k < 3; ++k) {
    const int v = a.tris[3 * t + k];
    c.v[k] = v;
    c.p[k] = make_float3(a.verts[3 * v], a.verts[3 * v + 1], a.verts[3 * v + 2]);
    c.n[k] = make_float3(a.vnormal[3 * v], a.vnormal[3 * v + 1], a.vnormal[3 * v + 2]);
    c.cc[k] = a.cam_clip[v];
    c.cs[k] = a.cam_scr[v];
  }
  c.mat = material_of(a, t);
  c.alb = make_float3(a.albedo[3 * c.mat], a.albedo[3 * c.mat + 1], a.albedo[3 * c.mat + 2]);
}

// Surface point of a covered pixel from its G-buffer texel and the cached triangle.
__device__ __forceinline__ void surf_from(const float4 g, const TriCache& c, Surf& s) {
  s.tri = c.tri;
  s.b[0] = g.y; s.b[1] = g.z; s.b[2] = 1.f - g.y - g.z;
  s.x = make_float3(0.f, 0.f, 0.f);
  s.nt = make_float3(0.f, 0.f, 0.f);
  for (int k = 0; k < 3; ++k) {
    s.v[k] = c.v[k];
    s.x.x += s.b[k] * c.p[k].x; s.x.y += s.b[k] * c.p[k].y; s.x.z += s.b[k] * c.p[k].z;
    s.nt.x += s.b[k] * c.n[k].x; s.nt.y += s.b[k] * c.n[k].y; s.nt.z += s.b[k] * c.n[k].z;
  }
  s.nlen = sqrtf(s.nt.x * s.nt.x + s.nt.y * s.nt.y + s.nt.z * s.nt.z);
  const float il = s.nlen > 0.f ? 1.f / s.nlen : 0.f;
  s.n = make_float3(s.nt.x * il, s.nt.y * il, s.nt.z * il);
}

// Lookup of Alg. 2 for one light at world point x: clip, depth d, texel
// coordinates, bilinear (m1, m2), visibility.  With the exponential warp
// (ec > 0) the receiver depth is compared as dw = exp(ec d) and the variance
// floor is min_var (ec dw)^2 (the depth-unit floor carried by the warp's
// slope at the receiver).
struct Look {
  float4 clip;
  float d;
  float dw;              // receiver depth in the moments' encoding
  int inside;
  float u, v;            // light-space position (clip x, y over w)
  float s, t;            // texel coordinates of the bilinear lookup
  int i0, j0;            // floor of the texel coordinates
  float fs, ft;
  float2 m;
  float var;
  int var_clamped;
  float delta;
  float vis;
};

__device__ __forceinline__ Look lookup(const float* Q, const float2* __restrict__ mom, int R, float3 x,
                                       float min_var, float ec) {
  Look L;
  L.clip = make_float4(Q[0] * x.x + Q[1] * x.y + Q[2] * x.z + Q[3], Q[4] * x.x + Q[5] * x.y + Q[6] * x.z + Q[7],
                       Q[8] * x.x + Q[9] * x.y + Q[10] * x.z + Q[11], Q[12] * x.x + Q[13] * x.y + Q[14] * x.z + Q[15]);
  L.d = Q[16] * x.x + Q[17] * x.y + Q[18] * x.z + Q[19];
  L.dw = ec > 0.f ? expf(ec * L.d) : L.d;
  L.vis = 1.f;
  L.inside = 0;
  if (!(L.clip.w > 0.f)) return L;
  const float u = L.clip.x / L.clip.w, v = L.clip.y / L.clip.w;
  L.u = u;
  L.v = v;
  if (!(fabsf(u) <= 1.f && fabsf(v) <= 1.f)) return L;
  L.inside = 1;
  const float s = (0.5f * u + 0.5f) * R - 0.5f, t = (0.5f - 0.5f * v) * R - 0.5f;
  L.s = s;
  L.t = t;
  const float fi = floorf(s), fj = floorf(t);
  L.i0 = (int)fi; L.j0 = (int)fj;
  L.fs = s - fi; L.ft = t - fj;
  const int i0 = min(max(L.i0, 0), R - 1), i1 = min(max(L.i0 + 1, 0), R - 1);
  const int j0 = min(max(L.j0, 0), R - 1), j1 = min(max(L.j0 + 1, 0), R - 1);
  const float2 m00 = mom[(size_t)j0 * R + i0], m01 = mom[(size_t)j0 * R + i1];
  const float2 m10 = mom[(size_t)j1 * R + i0], m11 = mom[(size_t)j1 * R + i1];
  const float w00 = (1.f - L.fs) * (1.f - L.ft), w01 = L.fs * (1.f - L.ft);
  const float w10 = (1.f - L.fs) * L.ft, w11 = L.fs * L.ft;
  L.m = make_float2(w00 * m00.x + w01 * m01.x + w10 * m10.x + w11 * m11.x,
                    w00 * m00.y + w01 * m01.y + w10 * m10.y + w11 * m11.y);
  const float raw = fmaf(-L.m.x, L.m.x, L.m.y);
  const float floor_var = ec > 0.f ? min_var * (ec * L.dw) * (ec * L.dw) : min_var;
  L.var_clamped = !(raw >= floor_var);
  L.var = L.var_clamped ? floor_var : raw;
  L.delta = L.dw - L.m.x;
  L.vis = L.delta <= 0.f ? 1.f : L.var / (L.var + L.delta * L.delta);
  return L;
}

__device__ __forceinline__ float3 light_omega(const LightDev& Ld, float3 x, float& len) {
  if (Ld.type == 0) {
    len = 1.f;
    return make_float3(-Ld.fwd[0], -Ld.fwd[1], -Ld.fwd[2]);
  }
  const float3 d = make_float3(Ld.pos[0] - x.x, Ld.pos[1] - x.y, Ld.pos[2] - x.z);
  len = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  const float il = 1.f / len;
  return make_float3(d.x * il, d.y * il, d.z * il);
}

// Cube face holding direction d (from a point light to a surface point): the
// axis of largest magnitude and its sign; ties go to x, then y.
__device__ __forceinline__ int cube_face(float3 d) {
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  if (ax >= ay && ax >= az) return d.x >= 0.f ? 0 : 1;
  if (ay >= az) return d.y >= 0.f ? 2 : 3;
  return d.z >= 0.f ? 4 : 5;
}

// Whether light view Ld shades point x: always, except a cube face of a point
// light, which shades the points of its face only (one face per point).
__device__ __forceinline__ bool view_shades(const LightDev& Ld, float3 x) {
  return Ld.face < 0 || cube_face(make_float3(x.x - Ld.pos[0], x.y - Ld.pos[1], x.z - Ld.pos[2])) == Ld.face;
}

__global__ void shade_kernel(ShadeArgs a, float4* __restrict__ color, float4* __restrict__ image,
                             const uint8_t* __restrict__ hflag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.W || j >= a.H) return;
  const size_t p = (size_t)j * a.W + i;
  const bool to_image = image && !(hflag && hflag[p]);
  Surf s;
  if (!load_surf(a, p, s)) {
    color[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (to_image) image[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  float3 rad = make_float3(0.f, 0.f, 0.f);
  for (int l = 0; l < a.L; ++l) {
    const LightDev& Ld = a.lights[l];
    if (!view_shades(Ld, s.x)) continue;
    const Look L = lookup(Ld.Q, a.mom[l], a.res[l], s.x, a.min_variance, a.ec);
    float len;
    const float3 om = light_omega(Ld, s.x, len);
    const float lam = fmaxf(s.n.x * om.x + s.n.y * om.y + s.n.z * om.z, 0.f);
    const float k = L.vis * lam;
    rad.x += k * Ld.intensity[0]; rad.y += k * Ld.intensity[1]; rad.z += k * Ld.intensity[2];
  }
  const int mat = material_of(a, s.tri);
  const float4 c = make_float4(a.albedo[3 * mat] * rad.x, a.albedo[3 * mat + 1] * rad.y, a.albedo[3 * mat + 2] * rad.z,
                               1.f);
  color[p] = c;
  if (to_image) image[p] = c;
}

// Diagnostic copy of the shading stage's intermediate values at every pixel of
// a camera, computed by the same device functions as shade_kernel (so a
// comparison can feed a reference the values this kernel used, stage by
// stage).  l < 0: out[2p] = (x, 0), out[2p + 1] = (n, 0), the interpolated
// world position and unit normal.  l >= 0 (light view l): out[2p] =
// (u, v, s, t), out[2p + 1] = (dw, m1, m2, vis): light-space position, texel
// coordinates, receiver depth in the moments' encoding, bilinear moments and
// visibility.  Values the pixel does not have are NaN: every value of a
// background pixel or of a view that does not shade the point (another cube
// face), (u, v) when the point is behind the light, and (s, t, m1, m2)
// outside the light's window.
__global__ void shade_probe_kernel(ShadeArgs a, int l, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.W || j >= a.H) return;
  const size_t p = (size_t)j * a.W + i;
  const float nan = __int_as_float(0x7fc00000);
  float4 o0 = make_float4(nan, nan, nan, nan), o1 = o0;
  Surf s;
  if (load_surf(a, p, s)) {
    if (l < 0) {
      o0 = make_float4(s.x.x, s.x.y, s.x.z, 0.f);
      o1 = make_float4(s.n.x, s.n.y, s.n.z, 0.f);
    } else if (view_shades(a.lights[l], s.x)) {
      const Look L = lookup(a.lights[l].Q, a.mom[l], a.res[l], s.x, a.min_variance, a.ec);
      const bool front = L.clip.w > 0.f;
      o0 = make_float4(front ? L.u : nan, front ? L.v : nan, L.inside ? L.s : nan, L.inside ? L.t : nan);
      o1 = make_float4(L.dw, L.inside ? L.m.x : nan, L.inside ? L.m.y : nan, L.vis);
    }
  }
  out[2 * p] = o0;
  out[2 * p + 1] = o1;
}

void launch_shade_probe(const ShadeArgs& a, int l, float4* out, cudaStream_t st) {
  dim3 b(32, 8), g((a.W + 31) / 32, (a.H + 7) / 8);
  count_launches(1);
  shade_probe_kernel<<<g, b, 0, st>>>(a, l, out);
}

constexpr int kShadeStrip = 8;

// Warp reduce-scatter of N (16 or 32) values per lane by recursive halving:
// after the exchange steps (N/2 + ... + 1 shuffles, plus one across the half
// warps when N = 16) lane k holds the warp sum of value k mod N.  Far cheaper
// than N separate butterfly reductions.
template <int N>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[N]) {
  static_assert(N == 16 || N == 32, "16 or 32 values");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = N / 2; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = upper ? v[k] : v[k + h];
      const float keep = upper ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, h);
    }
  }
  if (N == 16) v[0] += __shfl_xor_sync(kFull, v[0], 16);
  return v[0];
}

// Adjoint of shade_kernel, one thread per pixel.  Scatters the texel maps
// dL/d(m1, m2) (bilinear adjoint), reduces dL/dQ, the direct light terms and
// the albedo gradient per block (slot copies), and writes the per-pixel
// dL/d world position and dL/d interpolated normal for shade_scatter_kernel.
template <bool kListed>
__global__ void __launch_bounds__(256, 4) shade_backward_kernel(ShadeArgs a, ShadeGradArgs g, AAWork w) {
  __shared__ float sQ[kMaxLightViews * 20];
  __shared__ float sD[kMaxLightViews * 3];
  __shared__ float sA[kMaxSharedMat * 3];
  __shared__ float sL;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) sL = 0.f;
  const bool mat_shared = a.n_mat <= kMaxSharedMat;
  for (int k = tid; k < kMaxLightViews * 20; k += 256) sQ[k] = 0.f;
  for (int k = tid; k < kMaxLightViews * 3; k += 256) sD[k] = 0.f;
  for (int k = tid; k < kMaxSharedMat * 3; k += 256) sA[k] = 0.f;
  __syncthreads();
  // One pixel (every lane of the warp calls it; inb false: no pixel).  The
  // grid pass (kListed false) takes every pixel except those on the final
  // antialiasing's work list, and the squared error of all of them; the list
  // pass (kListed true) takes the listed ones, whose dL/dcolour the
  // antialiasing adjoint writes, so that the grid pass need not wait for it.
  auto pixel = [&](const int i, const int j, const bool inb_) {
  const size_t p = inb_ ? (size_t)j * a.W + i : 0;
  const bool flagged = kListed || (inb_ && g.hflag && g.hflag[p]);
  const bool inb = inb_ && (kListed || !flagged);   // this pass's pixel
  const float4 gb4 = inb ? a.gbuf[p] : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 gcol = make_float4(0.f, 0.f, 0.f, 0.f);
  float sq = 0.f;   // squared error of the pixel (mean squared error backward)
  if (!kListed && inb_ && g.loss_index >= 0) {
    const float4 im = g.gimage.image[p], tg = g.gimage.target[p];
    const float4 d = make_float4(im.x - tg.x, im.y - tg.y, im.z - tg.z, im.w - tg.w);
    sq = d.x * d.x + d.y * d.y + d.z * d.z + d.w * d.w;
    const float sc = g.gimage.scale;
    if (inb) gcol = make_float4(sc * d.x, sc * d.y, sc * d.z, sc * d.w);
  } else if (inb) {
    gcol = flagged ? g.gcolor[p] : g.gimage[p];
  }
  const int id = __float_as_int(gb4.x);
  const bool act = inb && id && (gcol.x != 0.f || gcol.y != 0.f || gcol.z != 0.f);
  Surf s;
  int mat = -1;
  float3 alb = make_float3(0.f, 0.f, 0.f);
  if (act) {
    TriCache tc;
    tri_load(a, id - 1, tc);
    surf_from(gb4, tc, s);
    mat = tc.mat;
    alb = tc.alb;
  }
  const float4 gc4 = act ? gcol : make_float4(0.f, 0.f, 0.f, 0.f);
  float3 gx = make_float3(0.f, 0.f, 0.f), gn = make_float3(0.f, 0.f, 0.f), rad = make_float3(0.f, 0.f, 0.f);
  const float3 grad_rad = make_float3(gc4.x * alb.x, gc4.y * alb.y, gc4.z * alb.z);
  for (int l = 0; l < a.L; ++l) {
    float gq[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) gq[k] = 0.f;
    float3 gdir = make_float3(0.f, 0.f, 0.f);
    bool has_q = false;
    if (act && view_shades(a.lights[l], s.x)) {
      const LightDev& Ld = a.lights[l];
      const int R = a.res[l];
      const Look L = lookup(Ld.Q, a.mom[l], R, s.x, a.min_variance, a.ec);
      float len;
      const float3 om = light_omega(Ld, s.x, len);
      const float ndo = s.n.x * om.x + s.n.y * om.y + s.n.z * om.z;
      const float lam = fmaxf(ndo, 0.f);
      rad.x += L.vis * lam * Ld.intensity[0];
      rad.y += L.vis * lam * Ld.intensity[1];
      rad.z += L.vis * lam * Ld.intensity[2];
      const float sl = grad_rad.x * Ld.intensity[0] + grad_rad.y * Ld.intensity[1] + grad_rad.z * Ld.intensity[2];
      const float gvis = sl * lam, glam = sl * L.vis;
      if (ndo > 0.f && glam != 0.f) {
        gn.x += glam * om.x; gn.y += glam * om.y; gn.z += glam * om.z;
        const float3 gom = make_float3(glam * s.n.x, glam * s.n.y, glam * s.n.z);
        if (Ld.type == 0) {
          gdir = gom;                    // dL/d omega with omega = -fwd (chained in light_sums_kernel)
        } else {
          const float d = om.x * gom.x + om.y * gom.y + om.z * gom.z;
          const float il = 1.f / len;
          const float3 gp = make_float3((gom.x - om.x * d) * il, (gom.y - om.y * d) * il, (gom.z - om.z * d) * il);
          gdir = gp;                     // dL/d position (direct term)
          gx.x -= gp.x; gx.y -= gp.y; gx.z -= gp.z;
        }
      }
      if (L.inside && L.delta > 0.f && gvis != 0.f) {
        has_q = true;
        const float S = L.var + L.delta * L.delta;
        const float iS2 = 1.f / (S * S);
        const float dv_dvar = L.delta * L.delta * iS2;
        const float dv_ddelta = -2.f * L.var * L.delta * iS2;
        const float gdelta = gvis * dv_ddelta;
        float gm1 = -gdelta, gm2 = 0.f, gdw = gdelta;
        if (!L.var_clamped) {
          gm1 += gvis * dv_dvar * (-2.f * L.m.x);
          gm2 = gvis * dv_dvar;
        } else if (a.ec > 0.f) {
          gdw += gvis * dv_dvar * (2.f * a.min_variance * a.ec * a.ec * L.dw);   // the floor follows dw
        }
        const float gd = a.ec > 0.f ? gdw * (a.ec * L.dw) : gdw;   // dL/d depth
        const int i0 = min(max(L.i0, 0), R - 1), i1 = min(max(L.i0 + 1, 0), R - 1);
        const int j0c = min(max(L.j0, 0), R - 1), j1c = min(max(L.j0 + 1, 0), R - 1);
        const float w00 = (1.f - L.fs) * (1.f - L.ft), w01 = L.fs * (1.f - L.ft), w10 = (1.f - L.fs) * L.ft,
                    w11 = L.fs * L.ft;
        float2* gm = g.gm[l];
        atomic_add2(&gm[(size_t)j0c * R + i0], make_float2(w00 * gm1, w00 * gm2));
        atomic_add2(&gm[(size_t)j0c * R + i1], make_float2(w01 * gm1, w01 * gm2));
        atomic_add2(&gm[(size_t)j1c * R + i0], make_float2(w10 * gm1, w10 * gm2));
        atomic_add2(&gm[(size_t)j1c * R + i1], make_float2(w11 * gm1, w11 * gm2));
        const float2* mom = a.mom[l];
        const float2 m00 = mom[(size_t)j0c * R + i0], m01 = mom[(size_t)j0c * R + i1];
        const float2 m10 = mom[(size_t)j1c * R + i0], m11 = mom[(size_t)j1c * R + i1];
        // d(bilinear)/ds, /dt from texel differences (neighbouring moments
        // nearly agree; differencing them first keeps their digits)
        const float gfs = (1.f - L.ft) * ((m01.x - m00.x) * gm1 + (m01.y - m00.y) * gm2) +
                          L.ft * ((m11.x - m10.x) * gm1 + (m11.y - m10.y) * gm2);
        const float gft = (1.f - L.fs) * ((m10.x - m00.x) * gm1 + (m10.y - m00.y) * gm2) +
                          L.fs * ((m11.x - m01.x) * gm1 + (m11.y - m01.y) * gm2);
        // s = (0.5 u + 0.5) R - 0.5,  t = (0.5 - 0.5 v) R - 0.5,  u = cx / cw,  v = cy / cw
        const float gu = gfs * 0.5f * R, gv = -gft * 0.5f * R;
        const float iw = 1.f / L.clip.w;
        const float u = L.clip.x * iw, v = L.clip.y * iw;
        const float gcl[4] = {gu * iw, gv * iw, 0.f, -(gu * u + gv * v) * iw};
        const float xh[4] = {s.x.x, s.x.y, s.x.z, 1.f};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) gq[r * 4 + c] = gcl[r] * xh[c];
#pragma unroll
        for (int c = 0; c < 4; ++c) gq[16 + c] = gd * xh[c];
        const float* Q = Ld.Q;
        gx.x += Q[0] * gcl[0] + Q[4] * gcl[1] + Q[12] * gcl[3] + Q[16] * gd;
        gx.y += Q[1] * gcl[0] + Q[5] * gcl[1] + Q[13] * gcl[3] + Q[17] * gd;
        gx.z += Q[2] * gcl[0] + Q[6] * gcl[1] + Q[14] * gcl[3] + Q[18] * gd;
      }
    }
    // rows 0, 1, 3 and the depth row of dL/dQ (row 2 is zero: the lookup never
    // reads clip z) and the direct light term, one warp reduce-scatter; a warp
    // without a shadowed lookup has only the direct term to sum
    if (!__any_sync(kFull, has_q)) {
      float d0 = gdir.x, d1 = gdir.y, d2 = gdir.z;
      if (__any_sync(kFull, d0 != 0.f || d1 != 0.f || d2 != 0.f)) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          d0 += __shfl_xor_sync(kFull, d0, o);
          d1 += __shfl_xor_sync(kFull, d1, o);
          d2 += __shfl_xor_sync(kFull, d2, o);
        }
        if ((threadIdx.x & 31) == 0) {
          if (d0 != 0.f) atomicAdd(&sD[l * 3], d0);
          if (d1 != 0.f) atomicAdd(&sD[l * 3 + 1], d1);
          if (d2 != 0.f) atomicAdd(&sD[l * 3 + 2], d2);
        }
      }
    } else {
      float v[32];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = gq[k];
#pragma unroll
      for (int k = 8; k < 16; ++k) v[k] = gq[k + 4];
      v[16] = gdir.x; v[17] = gdir.y; v[18] = gdir.z;
#pragma unroll
      for (int k = 19; k < 32; ++k) v[k] = 0.f;
      const float r = warp_reduce_scatter<32>(v);
      const int lane = threadIdx.x & 31;
      if (r != 0.f) {
        if (lane < 8) atomicAdd(&sQ[l * 20 + lane], r);
        else if (lane < 16) atomicAdd(&sQ[l * 20 + lane + 4], r);
        else if (lane < 19) atomicAdd(&sD[l * 3 + lane - 16], r);
      }
    }
  }
  // albedo: warp-reduced when the warp's active pixels share one material
  const float3 ga = make_float3(gc4.x * rad.x, gc4.y * rad.y, gc4.z * rad.z);
  const int m0 = __reduce_max_sync(kFull, mat);
  if (__all_sync(kFull, mat == -1 || mat == m0)) {
    if (m0 >= 0) {
      float v0 = ga.x, v1 = ga.y, v2 = ga.z;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        v0 += __shfl_xor_sync(kFull, v0, o);
        v1 += __shfl_xor_sync(kFull, v1, o);
        v2 += __shfl_xor_sync(kFull, v2, o);
      }
      if ((threadIdx.x & 31) == 0) {
        float* dst = mat_shared ? sA : g.dalbedo;
        atomicAdd(&dst[3 * m0], v0); atomicAdd(&dst[3 * m0 + 1], v1); atomicAdd(&dst[3 * m0 + 2], v2);
      }
    }
  } else if (act) {
    float* dst = mat_shared ? sA : g.dalbedo;
    atomicAdd(&dst[3 * mat], ga.x); atomicAdd(&dst[3 * mat + 1], ga.y); atomicAdd(&dst[3 * mat + 2], ga.z);
  }
  if (g.loss_index >= 0) {
#pragma unroll
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
    if ((threadIdx.x & 31) == 0 && sq != 0.f) atomicAdd(&sL, sq);
  }
  // per-pixel dL/dx and dL/d(interpolated normal) for the scatter pass
  if (inb) {
    float3 gnt = make_float3(0.f, 0.f, 0.f);
    if (act && s.nlen > 0.f) {
      const float d = s.n.x * gn.x + s.n.y * gn.y + s.n.z * gn.z;
      const float il = 1.f / s.nlen;
      gnt = make_float3((gn.x - s.n.x * d) * il, (gn.y - s.n.y * d) * il, (gn.z - s.n.z * d) * il);
    }
    g.pgrad[2 * p] = make_float4(gx.x, gx.y, gx.z, gnt.x);
    g.pgrad[2 * p + 1] = make_float4(gnt.y, gnt.z, act ? 1.f : 0.f, 0.f);
  }
  };
  if (!kListed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    pixel(i, j, i < a.W && j < a.H);
  } else {
    const int n = *w.count;
    for (int k0 = blockIdx.x * 256 + (tid & ~31); k0 < n; k0 += gridDim.x * 256) {
      const int k = k0 + (tid & 31);
      const int q = k < n ? w.list[k] : 0;
      pixel(q % a.W, q / a.W, k < n);
    }
  }
  __syncthreads();
  // block sums into float64 slot copies: the light gradients sum millions of
  // terms of both signs, whose cancellation float32 accumulation would not keep
  double* red = g.red + (size_t)block_slot(kRedSlots) * g.red_stride;
  for (int k = tid; k < a.L * 20; k += 256)
    if (sQ[k] != 0.f) atomicAdd(&red[k], (double)sQ[k]);
  for (int k = tid; k < a.L * 3; k += 256)
    if (sD[k] != 0.f) atomicAdd(&red[a.L * 20 + k], (double)sD[k]);
  if (mat_shared)
    for (int k = tid; k < a.n_mat * 3; k += 256)
      if (sA[k] != 0.f) atomicAdd(&red[a.L * 23 + k], (double)sA[k]);
  if (g.loss_index >= 0 && tid == 0 && sL != 0.f) atomicAdd(&red[g.loss_index], (double)sL);
}

// Per-triangle scatter of the camera interpolation adjoint: from the per-pixel
// dL/dx and dL/dn, x = sum b_k v_k and n~ = sum b_k n_k give 9 dL/dv (b_k dL/dx),
// 9 dL/d unit vertex normal (b_k dL/dn~) and, through the barycentrics, 12
// dL/d camera clip.  Strips of kShadeStrip rows per warp with a run
// accumulator; big triangles go to their slot copies.
struct CamScatter {
  const int* tris;
  float4* gpos;
  float4* gnormal;
  float4* gclip;
  float* big_acc;
  int slot;
  // ordinary triangle: onto its vertices, three 16-byte atomics per vertex
  __device__ __forceinline__ void vertices(int t, const float (&c)[30]) const {
    for (int k = 0; k < 3; ++k) {
      const int v = tris[3 * t + k];
      atomic_add4(&gpos[v], make_float4(c[3 * k], c[3 * k + 1], c[3 * k + 2], 0.f));
      atomic_add4(&gnormal[v], make_float4(c[9 + 3 * k], c[10 + 3 * k], c[11 + 3 * k], 0.f));
      atomic_add4(&gclip[v], make_float4(c[18 + 4 * k], c[19 + 4 * k], c[20 + 4 * k], c[21 + 4 * k]));
    }
  }
  // big triangle b: into one of its slot copies
  __device__ __forceinline__ void operator()(int b, const float (&c)[30], int lane = 0) const {
    float* d = big_acc + ((size_t)b * kBigSlots + ((slot + lane) & (kBigSlots - 1))) * kBigStrideCam;
    for (int k = 0; k < 30; ++k) atomicAdd(&d[k], c[k]);
  }
};

__global__ void __launch_bounds__(256) shade_scatter_kernel(ShadeArgs a, ShadeGradArgs g) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * kShadeStrip;
  const bool col_ok = i < a.W;
  CamScatter sc{a.tris, g.gpos, g.gnormal, g.gclip, g.big_acc, scatter_slot(kBigSlots)};
  BigRun<30, 1> run;
  big_run_reset(run);
  TriCache tc;
  for (int srow = 0; srow < kShadeStrip; ++srow) {
    const int j = j0 + srow;
    float c[30];
#pragma unroll
    for (int k = 0; k < 30; ++k) c[k] = 0.f;
    int t = -1;
    if (col_ok && j < a.H) {
      const size_t p = (size_t)j * a.W + i;
      const float4 q1 = g.pgrad[2 * p + 1];
      if (q1.z != 0.f) {
        const float4 q0 = g.pgrad[2 * p];
        const float4 gb4 = a.gbuf[p];
        t = __float_as_int(gb4.x) - 1;
        if (t != tc.tri) tri_load(a, t, tc);
        const float b[3] = {gb4.y, gb4.z, 1.f - gb4.y - gb4.z};
        const float3 gx = make_float3(q0.x, q0.y, q0.z), gnt = make_float3(q0.w, q1.x, q1.y);
        for (int k = 0; k < 3; ++k) {
          c[3 * k] = b[k] * gx.x; c[3 * k + 1] = b[k] * gx.y; c[3 * k + 2] = b[k] * gx.z;
          c[9 + 3 * k] = b[k] * gnt.x; c[10 + 3 * k] = b[k] * gnt.y; c[11 + 3 * k] = b[k] * gnt.z;
        }
        const float px = pix_ndc_x(i, a.W), py = pix_ndc_y(j, a.H);
        const Bary r = bary_at(tc.cc, tc.cs, i, j, a.W, a.H);
        // x = sum_k b_k p_k, n~ = sum_k b_k n_k: centred dL/db_k from corner differences
        float gb[3];
        for (int k = 0; k < 3; ++k) {
          float acc = 0.f;
          for (int q = 0; q < 3; ++q) {
            const float3 dp = make_float3(tc.p[k].x - tc.p[q].x, tc.p[k].y - tc.p[q].y, tc.p[k].z - tc.p[q].z);
            const float3 dn = make_float3(tc.n[k].x - tc.n[q].x, tc.n[k].y - tc.n[q].y, tc.n[k].z - tc.n[q].z);
            acc += r.b[q] * (dp.x * gx.x + dp.y * gx.y + dp.z * gx.z + dn.x * gnt.x + dn.y * gnt.y + dn.z * gnt.z);
          }
          gb[k] = acc;
        }
        float4 gcv[3];
        bary_backward(r, gb, px, py, gcv);
        for (int k = 0; k < 3; ++k) {
          c[18 + 4 * k] = gcv[k].x; c[19 + 4 * k] = gcv[k].y; c[20 + 4 * k] = gcv[k].z; c[21 + 4 * k] = gcv[k].w;
        }
      }
    }
    const int bi = t >= 0 ? g.big[t] : -1;
    big_run_add(run, bi, c, sc);
    if (t >= 0 && bi < 0) sc.vertices(t, c);
  }
  big_run_flush(run, sc);
}

// Sum the kBigSlots copies of each big camera-view triangle and scatter them.
__global__ void shade_big_resolve_kernel(ShadeArgs a, ShadeGradArgs g, const int* __restrict__ big_tri,
                                         const DevStatus* __restrict__ status, int view) {
  const int b = blockIdx.x;
  if (b >= min(status->big_count[view], kMaxBig)) return;
  __shared__ float sum[30];
  const int k = threadIdx.x;
  if (k < 30) {
    float acc = 0.f;
    for (int q = 0; q < kBigSlots; ++q) acc += g.big_acc[((size_t)b * kBigSlots + q) * kBigStrideCam + k];
    sum[k] = acc;
  }
  __syncthreads();
  if (k < 3) {
    const int v = a.tris[3 * big_tri[b] + k];
    atomic_add4(&g.gpos[v], make_float4(sum[3 * k], sum[3 * k + 1], sum[3 * k + 2], 0.f));
    atomic_add4(&g.gnormal[v], make_float4(sum[9 + 3 * k], sum[10 + 3 * k], sum[11 + 3 * k], 0.f));
    atomic_add4(&g.gclip[v], make_float4(sum[18 + 4 * k], sum[19 + 4 * k], sum[20 + 4 * k], sum[21 + 4 * k]));
  }
}

// ------------------------------------------------------------------ per-vertex gathers
// dL/dv += M^T dL/dclip for every view (+ depth row for lights);
// dL/dQ_l += dL/dclip (x) [v, 1] and dL/dd (x) [v, 1].
__global__ void __launch_bounds__(256) vertex_backward_kernel(const float* __restrict__ verts, int V,
                                                              const float* __restrict__ viewM, int n_views,
                                                              int n_lights, VertGradPtrs gp,
                                                              float* __restrict__ dverts, double* __restrict__ red,
                                                              int red_stride) {
  __shared__ float sQ[kMaxLightViews * 20];
  for (int k = threadIdx.x; k < kMaxLightViews * 20; k += blockDim.x) sQ[k] = 0.f;
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = v < V;
  const float xh[4] = {ok ? verts[3 * v] : 0.f, ok ? verts[3 * v + 1] : 0.f, ok ? verts[3 * v + 2] : 0.f, 1.f};
  float3 acc = make_float3(0.f, 0.f, 0.f);
  for (int w = 0; w < n_views; ++w) {
    const float* M = viewM + 20 * w;
    const float4 gc = ok ? gp.gclip[w][v] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool is_light = w < n_lights;
    // light views carry dL/d vertex depth in the z slot (clip z has no gradient there)
    const float gz = is_light ? 0.f : gc.z;
    const float gd = is_light ? gc.z : 0.f;
    acc.x += M[0] * gc.x + M[4] * gc.y + M[8] * gz + M[12] * gc.w + (is_light ? M[16] * gd : 0.f);
    acc.y += M[1] * gc.x + M[5] * gc.y + M[9] * gz + M[13] * gc.w + (is_light ? M[17] * gd : 0.f);
    acc.z += M[2] * gc.x + M[6] * gc.y + M[10] * gz + M[14] * gc.w + (is_light ? M[18] * gd : 0.f);
    if (is_light) {
      // dL/dQ rows 0, 1, 3 and the depth row (row 2, clip z, has no gradient)
      const float g4[4] = {gc.x, gc.y, gc.w, gd};
      float q[16];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) q[r * 4 + c] = g4[r] * xh[c];
      const float sum = warp_reduce_scatter<16>(q);
      const int lane = threadIdx.x & 31, r = lane >> 2;
      if (lane < 16 && sum != 0.f) atomicAdd(&sQ[w * 20 + (r < 2 ? r : r + 1) * 4 + (lane & 3)], sum);
    }
  }
  if (ok) {
    dverts[3 * v] += acc.x; dverts[3 * v + 1] += acc.y; dverts[3 * v + 2] += acc.z;
  }
  __syncthreads();
  double* dst = red + (size_t)block_slot(kRedSlots) * red_stride;
  for (int k = threadIdx.x; k < n_lights * 20; k += blockDim.x)
    if (sQ[k] != 0.f) atomicAdd(&dst[k], (double)sQ[k]);
}

// One block of 1024 threads, the end of the backward: the kRedSlots float64
// copies of the light-matrix gradient, the direct light terms and the albedo
// block sums reduced (four threads per entry, 16 slots each, all loads issued
// at once, then two shuffles; dQ and the direct terms overwritten, the albedo
// added), then dL/d(pos, dir) of every caller light u: four threads
// per (view l, parameter j) form view l's share J^T dL/dQ (five terms each)
// plus the direct term of the shading direction omega (directional
// omega = -dir / |dir|, spot and point omega = normalize(pos - x)), and thread
// (u, j) adds the shares of u's views in view order (a point light's six cube
// faces; their J has no direction columns).  float64 keeps the cancellation of
// both sums.  float64 has a long latency here, so the views' J, direction and
// type are staged in shared memory first (their loads overlap the slot
// reduction's) and every float64 chain is kept short.
__global__ void __launch_bounds__(1024) light_sums_kernel(const double* __restrict__ red, int stride, int L,
                                                          int n_mat_red, const LightDev* __restrict__ lights,
                                                          int n_user, double* __restrict__ gQ,
                                                          double* __restrict__ gdirect, float* __restrict__ dalbedo,
                                                          float* __restrict__ dlight, float* __restrict__ loss,
                                                          double inv_n) {
  static_assert(kRedSlots % 4 == 0, "four threads per entry");
  __shared__ double sred[kMaxLightViews * 23];   // dL/dQ (20 per view), then the direct terms (3 per view)
  __shared__ double sshare[kMaxLightViews * 6];
  __shared__ float sJ[kMaxLightViews * 120];
  __shared__ float sdir[kMaxLightViews * 4];     // fwd xyz, |dir|
  __shared__ int suser[kMaxLightViews], stype[kMaxLightViews];
  const int t = threadIdx.x;
  for (int i = t; i < L * 120; i += blockDim.x) sJ[i] = lights[i / 120].J[i % 120];
  if (t < L) {
    const LightDev& Ld = lights[t];
    suser[t] = Ld.user;
    stype[t] = Ld.type;
    sdir[4 * t] = Ld.fwd[0];
    sdir[4 * t + 1] = Ld.fwd[1];
    sdir[4 * t + 2] = Ld.fwd[2];
    sdir[4 * t + 3] = Ld.dir_norm;
  }
  const int n = L * 23 + n_mat_red * 3 + (loss ? 1 : 0);
  for (int base = 0; base < 4 * n; base += blockDim.x) {
    const int e = base + t, k = e >> 2, part = e & 3;
    double acc = 0.0;
    if (k < n)
#pragma unroll
      for (int q = 0; q < kRedSlots / 4; ++q) acc += red[(size_t)(4 * q + part) * stride + k];
    acc += __shfl_xor_sync(kFull, acc, 1);
    acc += __shfl_xor_sync(kFull, acc, 2);
    if (k < n && part == 0) {
      if (k < L * 20) {
        gQ[k] = acc;
        sred[k] = acc;
      } else if (k < L * 23) {
        gdirect[k - L * 20] = acc;
        sred[k] = acc;
      } else if (k < L * 23 + n_mat_red * 3) {
        dalbedo[k - L * 23] += (float)acc;
      } else {
        *loss = (float)(acc * inv_n);   // the mean squared error
      }
    }
  }
  __syncthreads();   // sred and the staged views
  {
    // thread t: view l, parameter j, terms k = part, part + 4, ... of J^T dL/dQ;
    // part 1 adds the direct term
    const int l = t / 24, j = (t % 24) >> 2, part = t & 3;
    const bool ok = t < L * 24;
    double acc = 0.0;
    if (ok) {
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const int k = part + 4 * m;
        acc += sred[l * 20 + k] * widen_exact(sJ[l * 120 + k * 6 + j]);
      }
      const double* gd = sred + L * 20 + 3 * l;
      if (part == 1) {
        if (stype[l] == 1) {
          if (j < 3) acc += gd[j];
        } else if (j >= 3) {
          const int c = j - 3;
          const float* fw = sdir + 4 * l;
          const double f0 = widen_exact(fw[0]), f1 = widen_exact(fw[1]), f2 = widen_exact(fw[2]);
          const double fc = c == 0 ? f0 : (c == 1 ? f1 : f2);
          const double fg = f0 * gd[0] + f1 * gd[1] + f2 * gd[2];
          acc += -(gd[c] - fc * fg) / widen_exact(fw[3]);
        }
      }
    }
    acc += __shfl_xor_sync(kFull, acc, 1);
    acc += __shfl_xor_sync(kFull, acc, 2);
    if (ok && part == 0) sshare[l * 6 + j] = acc;
  }
  __syncthreads();   // sshare
  if (t < n_user * 6) {
    const int u = t / 6, j = t - 6 * u;
    double acc = 0.0;
    for (int l = 0; l < L; ++l)
      if (suser[l] == u) acc += sshare[l * 6 + j];
    dlight[t] = (float)acc;
  }
}

__global__ void l2_kernel(const float* __restrict__ img, const float* __restrict__ tgt, int64_t n,
                          float* __restrict__ loss, float* __restrict__ grad) {
  float acc = 0.f;
  const float sc = 2.0f / (float)n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[k] - tgt[k];
    grad[k] = sc * d;
    acc += d * d;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  __shared__ float ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v / (float)n);
  }
}

// ------------------------------------------------------------------ launchers
static inline dim3 grid2(int W, int H, dim3 b) { return dim3((W + b.x - 1) / b.x, (H + b.y - 1) / b.y); }

void launch_normals_backward(const float* verts, int V, const int* tris, int T, const int* vf_off,
                             const int* vf_list, const float* vnormal, const float* vlen, const float4* gnormal,
                             const float4* gpos, float* gN, float* gface, float* dverts, cudaStream_t st) {
  if (V == 0 || T == 0) return;
  count_launches(1);
  normals_bwd_vertex_kernel<<<(V + 255) / 256, 256, 0, st>>>(vnormal, vlen, V, gnormal, gN);
  count_launches(1);
  normals_bwd_face_kernel<<<(T + 255) / 256, 256, 0, st>>>(tris, T, gN, gface);
  count_launches(1);
  normals_bwd_gather_kernel<<<(V + 255) / 256, 256, 0, st>>>(verts, V, tris, vf_off, vf_list, gface, gpos,
                                                             dverts);
}

void launch_shade(const ShadeArgs& a, float4* color, float4* image, const uint8_t* hflag, cudaStream_t st) {
  dim3 b(32, 8);
  count_launches(1);
  shade_kernel<<<grid2(a.W, a.H, b), b, 0, st>>>(a, color, image, hflag);
}

void launch_shade_backward(const ShadeArgs& a, const ShadeGradArgs& g, cudaStream_t st) {
  dim3 b(32, 8);
  count_launches(1);
  shade_backward_kernel<false><<<grid2(a.W, a.H, b), b, 0, st>>>(a, g, AAWork{});
}

void launch_shade_backward_listed(const ShadeArgs& a, const ShadeGradArgs& g, const AAWork& w, cudaStream_t st) {
  count_launches(1);
  shade_backward_kernel<true><<<148 * 4, 256, 0, st>>>(a, g, w);
}

void launch_shade_scatter(const ShadeArgs& a, const ShadeGradArgs& g, cudaStream_t st) {
  dim3 b(32, 8), grid((a.W + 31) / 32, (a.H + 8 * kShadeStrip - 1) / (8 * kShadeStrip));
  count_launches(1);
  shade_scatter_kernel<<<grid, b, 0, st>>>(a, g);
}

void launch_vertex_backward(const float* verts, int V, const float* viewM, int n_views, int n_lights,
                            const VertGradPtrs& gp, float* dverts, double* red, int red_stride, cudaStream_t st) {
  if (V == 0) return;
  count_launches(1);
  vertex_backward_kernel<<<(V + 255) / 256, 256, 0, st>>>(verts, V, viewM, n_views, n_lights, gp, dverts, red,
                                                          red_stride);
}

void launch_shade_big_resolve(const ShadeArgs& a, const ShadeGradArgs& g, const int* big_tri,
                              const DevStatus* status, int view, cudaStream_t st) {
  count_launches(1);
  shade_big_resolve_kernel<<<kMaxBig, 32, 0, st>>>(a, g, big_tri, status, view);
}

void launch_light_sums(const double* red, int red_stride, int L, int n_mat_red, const LightDev* lights, int n_user,
                       double* gQ, double* gdirect, float* dalbedo, float* dlight, float* loss, int64_t n_img,
                       cudaStream_t st) {
  if (L * 23 + n_mat_red * 3 == 0 && n_user == 0 && !loss) return;
  count_launches(1);
  light_sums_kernel<<<1, 1024, 0, st>>>(red, red_stride, L, n_mat_red, lights, n_user, gQ, gdirect, dalbedo, dlight,
                                        loss, loss ? 1.0 / (double)n_img : 0.0);
}

void launch_l2(const float* img, const float* tgt, int64_t n, float* loss, float* grad, cudaStream_t st) {
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (n == 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  count_launches(1);
  l2_kernel<<<blocks, 256, 0, st>>>(img, tgt, n, loss, grad);
}

}  // namespace dsm
