// Light cameras, pinned vertex transform, triangle setup, binning and the tile
// rasteriser (Eq. 1: nearest surface per pixel centre).
#include <algorithm>
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {

// ------------------------------------------------------------------ light camera
// The float32 light matrix Q (supplementary Sec. A light cameras: clip rows
// 0-3, depth row 4) must be reproducible bit for bit, so its entries are
// formed in float64 with explicitly rounded operations (no contraction) in a
// fixed order and rounded to float32 once.  The derivatives J = dQ/d theta
// (theta = pos xyz, dir xyz) only feed gradients and use float32 dual numbers.
// The frame and the entries are stated once, as templates over the number
// type (light_frame, q_entry), which the duals instantiate; the float64
// values take the same operations spread over a warp's lanes
// (light_q64_lanes).
struct F1 {    // float32 value with its derivative w.r.t. one light parameter
  float v, d;
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ F1 operator-(F1 a) { return {-a.v, -a.d}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ F1 operator/(F1 a, F1 b) {
  const float q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ F1 tsqrt(F1 a) {
  const float r = sqrtf(a.v);
  return {r, a.d / (2.f * r)};
}
__device__ __forceinline__ double val(F1 a) { return a.v; }

template <class T> struct V3 { T x, y, z; };
template <class T> __device__ __forceinline__ T dot3(const V3<T>& a, const V3<T>& b) {
  return (a.x * b.x + a.y * b.y) + a.z * b.z;
}
template <class T> __device__ __forceinline__ V3<T> cross3(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> __device__ __forceinline__ V3<T> normalize3(const V3<T>& a) {
  const T n = tsqrt((a.x * a.x + a.y * a.y) + a.z * a.z);
  return {a.x / n, a.y / n, a.z / n};
}

// Light frame: forward f, right r, up u, eye e, and the scalars every entry uses.
template <class T> struct Frame {
  V3<T> f, r, u, e;
  T fe, rng, nfe_near;   // f.e, far - near, -f.e - near
};
template <class T> __device__ __forceinline__ Frame<T> light_frame(const T (&th)[6], const LightConst& L, T zero,
                                                                   T one) {
  Frame<T> F;
  const V3<T> dir = {th[3], th[4], th[5]};
  F.f = normalize3(dir);
  const V3<T> up = fabs(val(F.f.y)) > 0.99 ? V3<T>{zero, zero, one} : V3<T>{zero, one, zero};
  F.r = normalize3(cross3(F.f, up));
  F.u = cross3(F.r, F.f);
  if (L.type == 0) {
    const T md = -(one * T{(decltype(one.v))L.dist});
    F.e = {md * F.f.x, md * F.f.y, md * F.f.z};
  } else {
    F.e = {th[0], th[1], th[2]};
  }
  F.fe = dot3(F.f, F.e);
  const T nearp = one * T{(decltype(one.v))L.near_plane}, farp = one * T{(decltype(one.v))L.far_plane};
  F.rng = farp - nearp;
  F.nfe_near = -F.fe - nearp;
  return F;
}

// Entry k of Q as mult * op (+ add for the spot's [2][3]) / den, in the order
// the entry is defined: directional rows r/h, u/h, depth row, (0 0 0 1);
// spot rows c r, c u, A f (+B), f; both: depth row f / (far - near).
template <class T> __device__ __forceinline__ T q_entry(int k, const Frame<T>& F, const LightConst& L, T zero, T one) {
  using S = decltype(one.v);
  const T nearp = one * T{(S)L.near_plane}, farp = one * T{(S)L.far_plane};
  const V3<T>& f = F.f;
  if (k >= 16) {
    const T op = k == 16 ? f.x : k == 17 ? f.y : k == 18 ? f.z : F.nfe_near;
    return op / F.rng;
  }
  const int row = k >> 2, c = k & 3;
  if (L.type == 0) {
    const T h = one * T{(S)L.ortho_half};
    if (row == 0) return (c == 0 ? F.r.x : c == 1 ? F.r.y : c == 2 ? F.r.z : -dot3(F.r, F.e)) / h;
    if (row == 1) return (c == 0 ? F.u.x : c == 1 ? F.u.y : c == 2 ? F.u.z : -dot3(F.u, F.e)) / h;
    if (row == 2) return (c == 0 ? f.x : c == 1 ? f.y : c == 2 ? f.z : F.nfe_near) / F.rng;
    return c == 3 ? one : zero;
  }
  const T cc = one * T{(S)L.persp_c};
  if (row == 0) return c < 3 ? cc * (c == 0 ? F.r.x : c == 1 ? F.r.y : F.r.z) : -(cc * dot3(F.r, F.e));
  if (row == 1) return c < 3 ? cc * (c == 0 ? F.u.x : c == 1 ? F.u.y : F.u.z) : -(cc * dot3(F.u, F.e));
  if (row == 2) {
    const T A = farp / F.rng;
    if (c < 3) return A * (c == 0 ? f.x : c == 1 ? f.y : f.z);
    const T B = (-(farp * nearp)) / F.rng;
    return (-(A * F.fe)) + B;
  }
  return c == 0 ? f.x : c == 1 ? f.y : c == 2 ? f.z : -F.fe;
}

// Axis component k of cube face `face` (+X, -X, +Y, -Y, +Z, -Z): the fixed
// viewing direction of that face of a point light's cube map.
__device__ __forceinline__ float face_axis(int face, int k) {
  return (face >> 1) == k ? ((face & 1) ? -1.f : 1.f) : 0.f;
}

// The float64 frame and Q of one light view, spread over the lanes of one
// warp.  Every operation is one that light_frame and q_entry state, on the
// same operands in the same order, each separately rounded (explicit
// intrinsics, no contraction), so Q is the same to the bit as their float64
// evaluation; only the lane that performs an operation differs.  float64 issues at a small fraction of the
// float32 rate here, so the warp's time is its count of float64 instructions:
// lane i forms component i mod 3 of each frame vector (one division or cross
// product term per lane where every lane formed all three), the sums of
// squares and the dot products f.e, r.e, u.e gather their terms from lanes
// 0-8 by shuffles, and the divisions of all twenty entries, with the spot
// light's A = far / (far - near) in lane 20 and B = -far near / (far - near)
// in lane 21, are one lane-parallel division.  thd: this lane's direction
// component theta[3 + i mod 3]; thp: its position component theta[i mod 3].
struct LightQ64 {
  double q;    // Q entry `lane` (lanes < 20)
  double fc;   // component lane mod 3 of the normalised direction f
  double n;    // |dir|
};
__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(kFull, v, src); }

__device__ __forceinline__ LightQ64 light_q64_lanes(double thd, double thp, const LightConst& L, int lane) {
  const int c = lane % 3, c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  // f = dir / |dir|, |dir| = sqrt((x x + y y) + z z)
  const double d2 = __dmul_rn(thd, thd);
  const double n = __dsqrt_rn(__dadd_rn(__dadd_rn(shfl_d(d2, 0), shfl_d(d2, 1)), shfl_d(d2, 2)));
  const double fc = __ddiv_rn(thd, n);
  const double fc1 = shfl_d(fc, c1), fc2 = shfl_d(fc, c2);
  // r = normalize(f x up), up = z when |f.y| > 0.99, else y; (a x b)_c = a_c1 b_c2 - a_c2 b_c1
  const int upk = fabs(shfl_d(fc, 1)) > 0.99 ? 2 : 1;
  const double up1 = c1 == upk ? 1.0 : 0.0, up2 = c2 == upk ? 1.0 : 0.0;
  const double rr = __dsub_rn(__dmul_rn(fc1, up2), __dmul_rn(fc2, up1));
  const double r2 = __dmul_rn(rr, rr);
  const double nr = __dsqrt_rn(__dadd_rn(__dadd_rn(shfl_d(r2, 0), shfl_d(r2, 1)), shfl_d(r2, 2)));
  const double rc = __ddiv_rn(rr, nr);
  // u = r x f
  const double uc = __dsub_rn(__dmul_rn(shfl_d(rc, c1), fc2), __dmul_rn(shfl_d(rc, c2), fc1));
  // eye: -dist f (directional) or the position
  const double ec = L.type == 0 ? __dmul_rn(-L.dist, fc) : thp;
  // f.e, r.e, u.e: lanes 0-2, 3-5 and 6-8 hold the products of one each
  const double pv = __dmul_rn(lane < 3 ? fc : (lane < 6 ? rc : uc), ec);
  const int g0 = lane < 3 ? 0 : (lane < 6 ? 3 : 6);
  const double dsum = __dadd_rn(__dadd_rn(shfl_d(pv, g0), shfl_d(pv, g0 + 1)), shfl_d(pv, g0 + 2));
  const double fe = shfl_d(dsum, 0), re = shfl_d(dsum, 3), ue = shfl_d(dsum, 6);
  const double nearp = L.near_plane, farp = L.far_plane;
  const double rng = __dsub_rn(farp, nearp), nfe_near = __dsub_rn(-fe, nearp);
  // entry k = lane: row k / 4, column cq = k mod 4 (the depth row, k >= 16, has column k - 16)
  const int k = lane, row = k >> 2, cq = k & 3, ci = cq < 3 ? cq : 0;
  const double fq = shfl_d(fc, ci), rq = shfl_d(rc, ci), uq = shfl_d(uc, ci);
  const bool spot = L.type != 0;
  // the spot light's products before its divisions: c r, c u (rows 0, 1), far near (lane 21)
  const double pm = __dmul_rn(k == 21 ? farp : L.persp_c,
                              k == 21 ? nearp : (row == 0 ? (cq < 3 ? rq : re) : (cq < 3 ? uq : ue)));
  double num = 1.0, den = 1.0;
  if (k >= 16 && k < 20) {
    num = cq < 3 ? fq : nfe_near;
    den = rng;
  } else if (!spot && k < 12) {
    num = row == 0 ? (cq < 3 ? rq : -re) : row == 1 ? (cq < 3 ? uq : -ue) : (cq < 3 ? fq : nfe_near);
    den = row == 2 ? rng : L.ortho_half;
  } else if (spot && (k == 20 || k == 21)) {
    num = k == 20 ? farp : -pm;
    den = rng;
  }
  const double qd = __ddiv_rn(num, den);
  // the spot light's depth row: A f_c, and (-(A f.e)) + B
  const double A = shfl_d(qd, 20), B = shfl_d(qd, 21);
  const double am = __dmul_rn(A, cq < 3 ? fq : fe);
  const double ab = __dadd_rn(-am, B);
  double q;
  if (k >= 16) q = qd;
  else if (!spot) q = row == 3 ? (cq == 3 ? 1.0 : 0.0) : qd;
  else if (row < 2) q = cq < 3 ? pm : -pm;
  else if (row == 2) q = cq < 3 ? am : ab;
  else q = cq < 3 ? fq : -fe;
  return {q, fc, n};
}

// One CTA per light view.  Warp 0 forms Q in float64 (light_q64_lanes; lane
// k < 20 writes Q[k]) and the view's other fields; warp 1: lane j < 6 forms
// all of Q with float32 duals in direction theta_j and writes column j of J.
// A cube face takes the light's position and the face axis as its direction
// (a constant: its J has no direction columns).  CTA a.n copies the C camera
// matrices after the light views' (a camera's float32 matrix is exact: its
// residual rows are zero).  The CTAs after it form the vertex normals, one
// thread per vertex: the light CTAs' float64 chains occupy a few SMs for
// several microseconds, and in one launch the normals run beside them for
// certain (as a kernel of their own on another stream they were seen to start
// only after it).
constexpr int kLightSetupThreads = 128;
__global__ void __launch_bounds__(kLightSetupThreads) light_setup_kernel(const float* __restrict__ params,
                                                                         LightSetupArgs a, LightDev* out,
                                                                         float* viewM, float* viewMlo, CamMats cams,
                                                                         int C, VertNormalArgs vn) {
  const int l = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (l > a.n) {
    const int v = (l - a.n - 1) * kLightSetupThreads + threadIdx.x;
    if (v < vn.V) vertex_normal_at(vn, v);
    return;
  }
  if (l == a.n) {
    for (int k = threadIdx.x; k < 20 * C; k += blockDim.x) viewM[20 * a.n + k] = cams.v[k];
    for (int k = threadIdx.x; k < 16 * C; k += blockDim.x) viewMlo[16 * a.n + k] = 0.f;
    return;
  }
  const LightConst& L = a.c[l];
  LightDev& o = out[l];
  const float* pl = params + L.user * 6;
  if (warp == 0) {
    const int c = lane % 3;
    const float thd = L.face >= 0 ? face_axis(L.face, c) : pl[3 + c];
    const LightQ64 r = light_q64_lanes(widen_exact(thd), widen_exact(pl[c]), L, lane);
    if (lane < 20) {
      const float q = __double2float_rn(r.q);
      o.Q[lane] = q;
      viewM[l * 20 + lane] = q;
      // the clip rows' rounding residual: the unsnapped clip coordinates that
      // interpolation and antialiasing use are those of the float64 matrix
      if (lane < 16) viewMlo[l * 16 + lane] = __double2float_rn(r.q - widen_exact(q));
    }
    if (lane < 3) {
      o.fwd[lane] = __double2float_rn(r.fc);
      o.pos[lane] = pl[lane];
    }
    if (lane == 0) {
      o.dir_norm = __double2float_rn(r.n);
      o.type = L.type;
      o.res = L.res;
      o.intensity[0] = L.intensity[0]; o.intensity[1] = L.intensity[1]; o.intensity[2] = L.intensity[2];
      o.face = L.face;
      o.user = L.user;
    }
  } else if (warp == 1 && lane < 6) {
    F1 th[6];
    for (int k = 0; k < 6; ++k)
      th[k] = (k >= 3 && L.face >= 0) ? F1{face_axis(L.face, k - 3), 0.f} : F1{pl[k], k == lane ? 1.f : 0.f};
    const F1 zero{0.f, 0.f}, one{1.f, 0.f};
    const Frame<F1> F = light_frame(th, L, zero, one);
    for (int k = 0; k < 20; ++k) o.J[k * 6 + lane] = q_entry(k, F, L, zero, one).d;
  }
}

// ------------------------------------------------------------------ vertex transform
__device__ __forceinline__ float pinned_row(const float* M, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[0], x), __fmul_rn(M[1], y)), __fmul_rn(M[2], z)), M[3]);
}

// Screen position of a clip-space vertex snapped to 24.8 fixed point, ndc z,
// and validity (w >= kWMin and inside the guard band).
__device__ __forceinline__ VertSnap snap_vertex(float c0, float c1, float c2, float c3, int W, int H) {
  const float nx = __fdiv_rn(c0, c3), ny = __fdiv_rn(c1, c3), nz = __fdiv_rn(c2, c3);
  const float sx = __fmul_rn(__fadd_rn(__fmul_rn(0.5f, nx), 0.5f), (float)W);
  const float sy = __fmul_rn(__fsub_rn(0.5f, __fmul_rn(0.5f, ny)), (float)H);
  const float fx = __fmul_rn(sx, (float)kSubpix), fy = __fmul_rn(sy, (float)kSubpix);
  const bool ok = (c3 >= kWMin) && (fabsf(fx) <= (float)kGuard) && (fabsf(fy) <= (float)kGuard);
  VertSnap s;
  s.X = ok ? __float2int_rn(fx) : 0;
  s.Y = ok ? __float2int_rn(fy) : 0;
  s.z = nz;
  s.ok = ok ? 1 : 0;
  return s;
}

// ------------------------------------------------------------------ triangle setup
// Setup record of triangle t in one view from its snapped corners: bbox,
// orientation-normalised top-left flags, float 2A; orient = sign of 2A (0:
// culled).
__device__ __forceinline__ TriSetup setup_triangle(int t, VertSnap s0, VertSnap s1, VertSnap s2, int W, int H,
                                                   TriSetup* __restrict__ out, int8_t* __restrict__ orient) {
  long long area2 = (long long)(s1.X - s0.X) * (s2.Y - s0.Y) - (long long)(s1.Y - s0.Y) * (s2.X - s0.X);
  bool culled = !(s0.ok && s1.ok && s2.ok) || area2 == 0;
  int sg = area2 > 0 ? 1 : -1;
  *orient = culled ? 0 : (int8_t)sg;
  TriSetup r;
  r.X[0] = s0.X; r.X[1] = s1.X; r.X[2] = s2.X;
  r.Y[0] = s0.Y; r.Y[1] = s1.Y; r.Y[2] = s2.Y;
  r.z[0] = s0.z; r.z[1] = s1.z; r.z[2] = s2.z;
  r.a2f = __ll2float_rn((long long)sg * area2);
  r.tri = t;
  r.pad[0] = r.pad[1] = 0;
  int i0 = 1, i1 = 0, j0 = 1, j1 = 0;
  int flags = (sg < 0) ? 8 : 0;
  if (!culled) {
    long long mnx = min(s0.X, min(s1.X, s2.X)), mxx = max(s0.X, max(s1.X, s2.X));
    long long mny = min(s0.Y, min(s1.Y, s2.Y)), mxy = max(s0.Y, max(s1.Y, s2.Y));
    long long a0 = -((128 - mnx) >> 8), a1 = (mxx - 128) >> 8;
    long long b0 = -((128 - mny) >> 8), b1 = (mxy - 128) >> 8;
    i0 = (int)max(a0, 0LL); i1 = (int)min(a1, (long long)(W - 1));
    j0 = (int)max(b0, 0LL); j1 = (int)min(b1, (long long)(H - 1));
    const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};
    for (int k = 0; k < 3; ++k) {
      int Xa = r.X[ea[k]], Ya = r.Y[ea[k]], Xb = r.X[eb[k]], Yb = r.Y[eb[k]];
      long long ca = -(long long)sg * (Yb - Ya), cb = (long long)sg * (Xb - Xa);
      if (ca > 0 || (ca == 0 && cb > 0)) flags |= 1 << k;
    }
    if (i0 <= i1 && j0 <= j1) flags |= 16;
  }
  if (!(flags & 16)) { i0 = 1; i1 = 0; j0 = 1; j1 = 0; }
  r.ibox = (i0 & 0xffff) | (i1 << 16);
  r.jbox = (j0 & 0xffff) | (j1 << 16);
  r.flags = flags;
  *out = r;
  return r;
}


// Silhouette edge mask per triangle: bit e set when edge e (v0v1, v1v2, v2v0)
// is a boundary / non-manifold edge, the triangle across it is culled, or the
// two triangles have opposite screen orientation.
// Silhouette edges of triangle t (bit e): boundary or non-manifold edge, a
// culled neighbour across it, or the neighbour's opposite screen orientation.
__device__ __forceinline__ uint8_t silhouette_mask(const int8_t* __restrict__ orient, int t, int a0, int a1, int a2) {
  const int8_t o = orient[t];
  const int adj[3] = {a0, a1, a2};
  int m = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int a = adj[e];
    if (a < 0) { m |= 1 << e; continue; }
    const int8_t oa = orient[a];
    if (oa == 0 || oa != o) m |= 1 << e;
  }
  return (uint8_t)m;
}


// ------------------------------------------------------------------ all views at once
// The per-view setup kernels above, fused over the views of one frame: each
// vertex / triangle is read once and processed for every view (the view loop
// is unrolled so that the per-view pointers stay in parameter space).
// Rounding residual of a pinned row: the exact value of
// ((Mh + Ml) . [x, y, z, 1]) minus `pinned`, with Mh the float32 matrix row and
// Ml its own residual against the float64 row it was rounded from (zero for a
// camera, whose float32 matrix is the definition).  The Mh products and their
// sum are carried exactly as float-float (two_prod, two_sum); Ml's small
// terms in plain float32.
__device__ __forceinline__ float row_residual(const float* Mh, const float* Ml, float x, float y, float z,
                                              float pinned) {
  float p0, e0, p1, e1, p2, e2, s, t;
  two_prod(Mh[0], x, p0, e0);
  two_prod(Mh[1], y, p1, e1);
  two_prod(Mh[2], z, p2, e2);
  two_sum(p0, p1, s, t);
  float err = __fadd_rn(__fadd_rn(e0, e1), t);
  two_sum(s, p2, s, t);
  err = __fadd_rn(err, __fadd_rn(e2, t));
  two_sum(s, Mh[3], s, t);
  err = __fadd_rn(err, t);
  err = __fadd_rn(err, __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(Ml[0], x), __fmul_rn(Ml[1], y)),
                                           __fmul_rn(Ml[2], z)), Ml[3]));
  // s and `pinned` approximate the same value to a few ulps: their difference is exact
  return __fadd_rn(__fsub_rn(s, pinned), err);
}

// sx = (x / w / 2 + 1/2) S (sign = 1) or sy = (1/2 - y / w / 2) S (sign = -1)
// of clip coordinates x = xh + xl, w = wh + wl, as a float-float pair: the
// quotient's remainder is exact (one fused multiply-add), the scalings by 1/2
// exact, the final products and sums split exactly (two_prod, two_sum).
__device__ __forceinline__ float2 screen_ff(float xh, float xl, float wh, float wl, float sign, float S) {
  const float q1 = __fdiv_rn(xh, wh);
  const float rem = __fadd_rn(__fmaf_rn(-q1, wh, xh), __fmaf_rn(-q1, wl, xl));
  const float q2 = __fdiv_rn(rem, wh);                    // x / w = q1 + q2
  float s, e;
  two_sum(0.5f, __fmul_rn(sign * 0.5f, q1), s, e);         // 1/2 +- q1 / 2
  e = __fadd_rn(e, __fmul_rn(sign * 0.5f, q2));
  float p, pe;
  two_prod(s, S, p, pe);
  pe = __fmaf_rn(e, S, pe);
  float hi, lo;
  two_sum(p, pe, hi, lo);
  return make_float2(hi, lo);
}

__global__ void transform_all_kernel(const float* __restrict__ verts, int V, const float* __restrict__ viewM,
                                     const float* __restrict__ viewMlo, ViewSetupArgs a, DevStatus* status) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  // the binning's tile counters, big-triangle counts and list and unit
  // totals, and the antialiasing work lists of these views start this frame
  // empty (other views' entries may be in use by a concurrent setup)
  for (int w = 0; w < a.n; ++w)
    for (int k = v; k < a.tiles[w]; k += gridDim.x * blockDim.x) a.count[w][k] = 0;
  if (v < a.n) {
    status->big_count[a.view0 + v] = 0;
    status->needed_pairs[a.view0 + v] = 0;
    status->units[a.view0 + v] = 0;
    status->split[a.view0 + v] = 0;
  }
  if (v < a.n && a.aa_count[v]) *a.aa_count[v] = 0;
  if (v >= V) return;
  const float x = verts[3 * v], y = verts[3 * v + 1], z = verts[3 * v + 2];
#pragma unroll
  for (int w = 0; w < kMaxViews; ++w) {
    if (w >= a.n) break;
    const float* M20 = viewM + 20 * w;
    const float* L16 = viewMlo + 16 * w;
    const float c0 = pinned_row(M20 + 0, x, y, z);
    const float c1 = pinned_row(M20 + 4, x, y, z);
    const float c2 = pinned_row(M20 + 8, x, y, z);
    const float c3 = pinned_row(M20 + 12, x, y, z);
    a.clip[w][v] = make_float4(c0, c1, c2, c3);
    const float l0 = row_residual(M20 + 0, L16 + 0, x, y, z, c0);
    const float l1 = row_residual(M20 + 4, L16 + 4, x, y, z, c1);
    const float l3 = row_residual(M20 + 12, L16 + 12, x, y, z, c3);
    const float2 sx = screen_ff(c0, l0, c3, l3, 1.f, (float)a.W[w]);
    const float2 sy = screen_ff(c1, l1, c3, l3, -1.f, (float)a.H[w]);
    a.scr[w][v] = make_float4(sx.x, sx.y, sy.x, sy.y);
    if (a.depth[w]) a.depth[w][v] = pinned_row(M20 + 16, x, y, z);
    a.snap[w][v] = snap_vertex(c0, c1, c2, c3, a.W[w], a.H[w]);
  }
}

__global__ void silhouette_all_kernel(const int* __restrict__ adj, int T, ViewSetupArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = t < T;
  const int a0 = ok ? adj[3 * t] : -1, a1 = ok ? adj[3 * t + 1] : -1, a2 = ok ? adj[3 * t + 2] : -1;
#pragma unroll
  for (int w = 0; w < kMaxViews; ++w) {
    if (w >= a.n) break;
    const uint8_t m = ok ? silhouette_mask(a.orient[w], t, a0, a1, a2) : 0;
    if (ok) a.sil[w][t] = m;
    // the packed copy: one word per warp of 32 consecutive triangles
    const unsigned bits = __ballot_sync(kFull, m != 0);
    if ((threadIdx.x & 31) == 0 && t < T) a.silbits[w][t >> 5] = bits;
  }
}

// ------------------------------------------------------------------ binning
// Tile range of a setup record: its bbox in tiles of side 2^tl (origin tx0,
// ty0, width ntx); returns the number of tiles (0 for a record with no pixel
// centre in its bbox).
__device__ __forceinline__ int tile_range(int flags, int ibox, int jbox, int tl, int& tx0, int& ty0, int& ntx) {
  if (!(flags & 16)) return 0;
  const int i0 = ibox & 0xffff, i1 = (unsigned)ibox >> 16, j0 = jbox & 0xffff, j1 = (unsigned)jbox >> 16;
  tx0 = i0 >> tl;
  ty0 = j0 >> tl;
  ntx = (i1 >> tl) - tx0 + 1;
  return ntx * ((j1 >> tl) - ty0 + 1);
}

// Warp-cooperative emission of (triangle, tile) pairs: the 32 triangles of a
// warp pool their tile ranges and the lanes stride over the pooled pairs, so a
// triangle spanning thousands of tiles is spread over 32 lanes.  Lanes that
// hit the same tile (neighbouring triangles usually share tiles) take one
// atomic through their lowest lane.  Count pass: adds to the tile's counter;
// fill pass: takes list slots of the tile's segment by counting the counter
// back down (to zero).  Every lane of the warp calls it; n = 0 emits nothing.
template <bool kFill>
__device__ __forceinline__ void emit_pairs(int t, int n, int tx0, int ty0, int ntx, int tilesX,
                                           int* __restrict__ counter, const int* __restrict__ offset,
                                           int* __restrict__ list, int capacity, DevStatus* status) {
  const int lane = threadIdx.x & 31;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  int total = __shfl_sync(kFull, incl, 31);
  int excl = incl - n;
  for (int base = 0; base < total; base += 32) {
    int p = base + lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      int e = __shfl_sync(kFull, excl, lo + step);
      if (e <= p) lo += step;
    }
    int o_excl = __shfl_sync(kFull, excl, lo);
    int o_tx0 = __shfl_sync(kFull, tx0, lo);
    int o_ty0 = __shfl_sync(kFull, ty0, lo);
    int o_ntx = __shfl_sync(kFull, ntx, lo);
    int o_t = __shfl_sync(kFull, t, lo);
    int tile = -1;
    if (p < total) {
      int q = p - o_excl;
      tile = (o_ty0 + q / o_ntx) * tilesX + o_tx0 + q % o_ntx;
    }
    const unsigned peers = __match_any_sync(kFull, tile);
    const int leader = __ffs(peers) - 1;
    const int cnt = __popc(peers);
    if (!kFill) {
      if (tile >= 0 && lane == leader) atomicAdd(&counter[tile], cnt);
    } else {
      int base_slot = 0;
      if (tile >= 0 && lane == leader) base_slot = offset[tile] + atomicSub(&counter[tile], cnt) - cnt;
      base_slot = __shfl_sync(kFull, base_slot, leader);
      if (tile >= 0) {
        const int slot = base_slot + __popc(peers & ((1u << lane) - 1));
        if (slot >= 0 && slot < capacity) list[slot] = o_t;
        else atomicExch(&status->capacity_overflow, 1);
      }
    }
  }
}

// Triangle setup of one view (blockIdx.y) with the binning's count pass: the
// record stays in registers for the tile counts.  A triangle spanning at least
// big_tiles tiles is listed as big (at most kMaxBig per view) and binned per
// tile by alloc_units_kernel instead.
__global__ void setup_bin_kernel(const int* __restrict__ tris, int T, ViewSetupArgs a, DevStatus* status) {
  const int w = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const BinShape bs = a.bs[w];
  int n = 0, tx0 = 0, ty0 = 0, ntx = 1;
  if (t < T) {
    const int v0 = tris[3 * t], v1 = tris[3 * t + 1], v2 = tris[3 * t + 2];
    const VertSnap* snap = a.snap[w];
    const TriSetup r = setup_triangle(t, snap[v0], snap[v1], snap[v2], a.W[w], a.H[w], a.setup[w] + t,
                                      a.orient[w] + t);
    n = tile_range(r.flags, r.ibox, r.jbox, bs.tile_log2, tx0, ty0, ntx);
    int b = -1;
    if (n >= bs.big_tiles) {
      b = atomicAdd(&status->big_count[a.view0 + w], 1);
      if (b < kMaxBig) a.big_tri[w][b] = t;
      else b = -1;
    }
    a.big_index[w][t] = b;
    if (b >= 0) n = 0;
  }
  emit_pairs<false>(t, n, tx0, ty0, ntx, a.tilesX[w], a.count[w], nullptr, nullptr, 0, status);
}

// Fill pass of one view: the same pairs as the count pass, into the list.
__global__ void bin_fill_kernel(const TriSetup* __restrict__ setup, int T, int tilesX, BinShape bs,
                                int* __restrict__ counter, const int* __restrict__ offset, int* __restrict__ list,
                                int capacity, DevStatus* status, const int* __restrict__ big_index) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int n = 0, tx0 = 0, ty0 = 0, ntx = 1;
  if (t < T && big_index[t] < 0) n = tile_range(setup[t].flags, setup[t].ibox, setup[t].jbox, bs.tile_log2, tx0, ty0, ntx);
  emit_pairs<true>(t, n, tx0, ty0, ntx, tilesX, counter, offset, list, capacity, status);
}

// A tile can hold a covered pixel centre of the triangle only if no edge
// function is negative at all four corner pixel centres of the tile.
__device__ __forceinline__ bool tile_may_cover(const TriSetup& r, int tx, int ty, int tl) {
  const int tile = 1 << tl;
  const long long x0 = (long long)(tx << tl) * kSubpix + 128, x1 = x0 + (long long)(tile - 1) * kSubpix;
  const long long y0 = (long long)(ty << tl) * kSubpix + 128, y1 = y0 + (long long)(tile - 1) * kSubpix;
  const int sg = (r.flags & 8) ? -1 : 1;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int a = e == 0 ? 1 : (e == 1 ? 2 : 0), b = e == 0 ? 2 : (e == 1 ? 0 : 1);
    const long long dx = (long long)sg * (r.X[b] - r.X[a]), dy = (long long)sg * (r.Y[b] - r.Y[a]);
    // E = dx (Py - Ya) - dy (Px - Xa): maximise over the corner pixel centres
    const long long py = dx >= 0 ? y1 : y0, px = dy >= 0 ? x0 : x1;
    if (dx * (py - r.Y[a]) - dy * (px - r.X[a]) < 0) return false;
  }
  return true;
}

// Whether big triangle r may cover tile (tx, ty): inside its bbox's tile
// range and not excluded by the corner test.  The big triangles (at most
// kMaxBig per view, listed by the count pass) are binned per tile by
// alloc_units_kernel instead of per triangle.
__device__ __forceinline__ bool big_covers_tile(const TriSetup& r, int tx, int ty, int tl) {
  const int i0 = r.ibox & 0xffff, i1 = (unsigned)r.ibox >> 16, j0 = r.jbox & 0xffff, j1 = (unsigned)r.jbox >> 16;
  if (tx < (i0 >> tl) || tx > (i1 >> tl) || ty < (j0 >> tl) || ty > (j1 >> tl)) return false;
  return tile_may_cover(r, tx, ty, tl);
}

// Per tile of one view: its list segment [offset[k], offset[n + k]), the
// ordinary triangles of the count pass then the big triangles that may cover
// the tile.  Segments are handed out by one atomic per warp on the view's
// running total (status->needed_pairs, zeroed by the transform), so they are
// not in tile order (nothing depends on that order); the total tells the host
// the list size.  With `write`: the big triangles go into the segment after
// its ordinary part (which the fill pass takes), and the raster work units
// follow, one per kRasterBatch records (at least one per tile), handed out by
// one atomic per warp on status->units, with a key slot for a tile of several
// units; each unit carries its record range and the tile's slot and unit
// count, so the raster starts from one 16-byte entry.  (The bounds hold
// whenever the list fits its capacity; a frame that overflows it is reported
// and only has to stay in bounds.)
__global__ void alloc_units_kernel(const int* __restrict__ count, int n, int* __restrict__ offset,
                                   DevStatus* status, int view, const TriSetup* __restrict__ setup,
                                   const int* __restrict__ big_tri, int tilesX, int tl, int* __restrict__ list,
                                   int capacity, RasterUnits ru, bool write) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  int c_ord = 0, c = 0;
  unsigned long long covers = 0ull;   // bit b: big triangle b may cover the tile
  if (tile < n) {
    c_ord = count[tile];
    const int nbig = min(status->big_count[view], kMaxBig);
    for (int b = 0; b < nbig; ++b)
      if (big_covers_tile(setup[big_tri[b]], tile % tilesX, tile / tilesX, tl)) covers |= 1ull << b;
    c = c_ord + __popcll(covers);
  }
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  int base = 0;
  if (lane == 31 && incl > 0) base = atomicAdd(&status->needed_pairs[view], incl);
  base = __shfl_sync(kFull, base, 31);
  const int beg = base + incl - c;
  if (tile < n) {
    offset[tile] = beg;
    offset[n + tile] = base + incl;
  }
  if (!write) return;   // (uniform over the grid)
  if (tile < n) {
    int k = beg + c_ord;
    for (unsigned long long m = covers; m; m &= m - 1) {
      if (k < capacity) list[k] = big_tri[__ffsll((long long)m) - 1];
      else atomicExch(&status->capacity_overflow, 1);
      ++k;
    }
  }
  const int nb = tile < n ? max(1, (c + kRasterBatch - 1) / kRasterBatch) : 0;
  incl = nb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += u;
  }
  base = 0;
  if (lane == 31 && incl > 0) base = atomicAdd(&status->units[view], incl);
  base = __shfl_sync(kFull, base, 31);
  if (tile < n) {
    const int u0 = base + incl - nb;
    int slot = -1;
    if (nb > 1) {
      slot = atomicAdd(&status->split[view], 1);
      if (slot >= ru.slot_cap) slot = -1;
    }
    // slots past the list capacity were never written (the fill pass flagged the overflow)
    const int end = min(beg + c, capacity);
    for (int b = 0; b < nb && u0 + b < ru.units_cap; ++b) {
      // without a key slot the tile's first unit takes all its records and the others none (-1)
      const int ub = slot >= 0 ? min(beg + kRasterBatch * b, end) : (b == 0 ? min(beg, end) : -1);
      const int ue = slot >= 0 ? min(end, ub + kRasterBatch) : (b == 0 ? end : -1);
      ru.units[u0 + b] = make_int4(tile, ub, ue, (slot + 1) | (nb << 20));
    }
  }
}

// ------------------------------------------------------------------ tile rasteriser
// Coverage of pixel centre (Px, Py) by a setup record: integer edge functions
// with the top-left rule; returns the depth key or ~0.  The record is read as
// words in TriSetup order (X[3], Y[3], z[3], a2f, ibox, jbox, tri, flags).
// Correctly rounded int64 -> float32 without the 64-bit conversion (which
// runs on the slow double-precision pipe).  For |v| < 2^48: v = h 2^24 + l
// with h = v >> 24 and 0 <= l < 2^24 both exact in float32, and one fused
// multiply-add rounds the exact sum once, to nearest even.
__device__ __forceinline__ float ll_to_float(long long v) {
  const float h = __int2float_rn((int)(v >> 24));
  const float l = __int2float_rn((int)(v & 0xffffff));
  return __fmaf_rn(h, 16777216.f, l);
}
// Any int64 (h above is no longer exact in float32 from 2^48 on; edge
// functions this large need vertices tens of thousands of pixels off
// screen): IEEE rounding written out on the integer pipes, |v| shifted so
// that its leading one is bit 63, the top 24 bits kept and rounded to nearest
// even on the 40 below them.
__device__ __forceinline__ float ll_to_float_wide(long long v) {
  if (v == 0) return 0.f;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll(a);
  const unsigned long long m = a << lz;
  unsigned mant = (unsigned)(m >> 40);
  const unsigned long long rest = m & ((1ull << 40) - 1), half = 1ull << 39;
  if (rest > half || (rest == half && (mant & 1u))) ++mant;
  int e = 63 - lz;
  if (mant == (1u << 24)) {   // the rounding carried into a new leading bit
    mant >>= 1;
    ++e;
  }
  return __uint_as_float((v < 0 ? 0x80000000u : 0u) | ((unsigned)(e + 127) << 23) | (mant & 0x7fffffu));
}

__device__ __forceinline__ float key_depth(uint64_t key) {
  const uint32_t k = (uint32_t)(key >> 32);
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Shared-memory form of a setup record inside one tile: for each edge e the
// orientation-normalised edge function at the tile's first pixel centre, E0_e
// (int64), and the edge's orientation-normalised snapped extent (dx_e, dy_e)
// (int32: snapped coordinates lie within +-2^28), so that
// E_e(x, y) = E0_e + 256 (y dx_e - x dy_e) is the exact integer edge function
// of Eq. 1's coverage test at tile pixel (x, y); then z[3], 2A (float),
// triangle, flags.  19 words; the stride is odd so that records of different
// lanes sit in different banks.
// E0_e is stored biased by the top-left rule, E0_e - (1 - tl_e): the pixel is
// covered iff every biased edge function is >= 0 (E > 0, or E = 0 on a
// top-left edge), which one sign test of their bitwise OR decides.  Records
// whose biased edge functions stay within int32 over the whole tile (every
// triangle a few tiles across) are flagged kRecSmall and stepped in int32;
// the coverage and the depth key are the same integers either way.
constexpr int kRecE0 = 0, kRecD = 6, kRecZ = 12, kRecA2 = 15, kRecTri = 16, kRecFlags = 17;
constexpr int kRecStride = 19;

__device__ __forceinline__ long long rec_ll(const int* w, int o) {
  return (long long)(((unsigned long long)(unsigned)w[o + 1] << 32) | (unsigned)w[o]);
}
__device__ __forceinline__ void rec_set_ll(int* w, int o, long long v) {
  w[o] = (int)(unsigned)(unsigned long long)v;
  w[o + 1] = (int)(unsigned)((unsigned long long)v >> 32);
}

constexpr int kRecSmall = 32;   // the biased edge functions fit int32 over the tile
constexpr int kRecWide = 64;    // 2A >= 2^48: a covered pixel's edge functions (0 <= E_k <= 2A) may exceed 2^48
constexpr int kSpan = 4;
__device__ __forceinline__ void rec_stage(const TriSetup& r, long long Px0, long long Py0, int* w) {
  const int sg = (r.flags & 8) ? -1 : 1;
  bool small = true;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int a = e == 0 ? 1 : (e == 1 ? 2 : 0);
    const int b = e == 0 ? 2 : (e == 1 ? 0 : 1);
    const int dx = sg * (r.X[b] - r.X[a]), dy = sg * (r.Y[b] - r.Y[a]);
    // biased by the top-left rule: covered iff E'_e = E_e - (1 - tl_e) >= 0
    const long long E0 = (long long)dx * (Py0 - r.Y[a]) - (long long)dy * (Px0 - r.X[a]) - (((r.flags >> e) & 1) ^ 1);
    rec_set_ll(w, kRecE0 + 2 * e, E0);
    w[kRecD + 2 * e] = dx;
    w[kRecD + 2 * e + 1] = dy;
    // |E| over tile pixels x <= 31 + kSpan (a span steps once past its end), y <= 31
    small = small && llabs(E0) + 256LL * (31LL * llabs((long long)dx) + (31LL + kSpan) * llabs((long long)dy)) <
                         (1LL << 31);
  }
  w[kRecZ] = __float_as_int(r.z[0]);
  w[kRecZ + 1] = __float_as_int(r.z[1]);
  w[kRecZ + 2] = __float_as_int(r.z[2]);
  w[kRecA2] = __float_as_int(r.a2f);
  w[kRecTri] = r.tri;
  w[kRecFlags] = r.flags | (small ? kRecSmall : 0) | (r.a2f >= 281474976710656.f ? kRecWide : 0);
}

// Coverage of the span of pixels xs..xe of row y by a staged record: the
// biased edge functions at (xs, y), then one step per pixel along x; a pixel
// is covered iff no biased edge function is negative (one sign test of their
// OR).  TE is int when the record's edge functions fit int32 over the tile.
template <typename TE, bool kWide>
__device__ __forceinline__ float edge_float(TE v) {
  if constexpr (sizeof(TE) == 4) return __int2float_rn(v);
  else if constexpr (kWide) return ll_to_float_wide(v);
  else return ll_to_float(v);
}

template <typename TE, int kTileT, bool kWide = false>
__device__ __forceinline__ void cover_span(const int* w, int xs, int xe, int y, unsigned long long* sbest) {
  const int flags = w[kRecFlags];
  TE E[3], S[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int dx = w[kRecD + 2 * e], dy = w[kRecD + 2 * e + 1];
    if constexpr (sizeof(TE) == 4)
      E[e] = w[kRecE0 + 2 * e] + 256 * (y * dx - xs * dy);
    else
      E[e] = rec_ll(w, kRecE0 + 2 * e) + 256LL * ((long long)y * dx - (long long)xs * dy);
    S[e] = -256 * (TE)dy;
  }
#pragma unroll
  for (int k = 0; k < kSpan; ++k) {
    if (xs + k <= xe && (E[0] | E[1] | E[2]) >= 0) {
      // the unbiased edge functions weight the corner depths (Eq. 1's key)
      const float e0 = edge_float<TE, kWide>(E[0] + (TE)((flags & 1) ^ 1));
      const float e1 = edge_float<TE, kWide>(E[1] + (TE)(((flags >> 1) & 1) ^ 1));
      const float e2 = edge_float<TE, kWide>(E[2] + (TE)(((flags >> 2) & 1) ^ 1));
      const float z = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(e0, __int_as_float(w[kRecZ])),
                                                    __fmul_rn(e1, __int_as_float(w[kRecZ + 1]))),
                                          __fmul_rn(e2, __int_as_float(w[kRecZ + 2]))),
                                __int_as_float(w[kRecA2]));
        atomicMin(&sbest[y * kTileT + xs + k], (unsigned long long)depth_key(z, w[kRecTri]));
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) E[e] += S[e];
  }
}

// One 256-thread CTA per work unit: up to kRasterBatch records of the list of
// one tile of kTile x kTile pixels (kTile = 2^kTL, 16 or 32); a tile with
// more records has several units, which merge their minima in the tile's key
// slot.  The unit's records are read 256 at a time.  Every record
// contributes the spans of its bbox-in-tile (kSpan pixels of one row each) as
// work items; a block prefix sum turns them into one flat list that all
// threads stride over (balanced whatever the triangle sizes), and each
// covered pixel centre folds (depth key, triangle) into the pixel's
// shared-memory 64-bit minimum.  The minimum is order independent, so the
// result is deterministic.  A thread finds the record of its item by a binary
// search of the records' first items (eight shared-memory reads; records
// without items share their successor's first item, so the search lands on
// the one that owns it).
// Each pixel then writes one 16-byte G-buffer texel: id + 1,
// perspective-correct b0, b1, depth key.
template <int kTL>
__global__ void __launch_bounds__(256, 6) raster_kernel(const TriSetup* __restrict__ setup,
                                                     const int* __restrict__ list, int tilesX,
                                                     int W, int H, const float4* __restrict__ clip,
                                                     const float4* __restrict__ scr,
                                                     const int* __restrict__ tris, float4* __restrict__ gbuf,
                                                     const float* __restrict__ depth, float2* __restrict__ fmap,
                                                     float ec, RasterUnits ru, const DevStatus* __restrict__ status,
                                                     int view, const uint32_t* __restrict__ silbits,
                                                     uint8_t* __restrict__ hflag, AAWork aa, RimBufs rim) {
  constexpr int kTile = 1 << kTL;
  constexpr int kPix = kTile * kTile;
  static_assert(kTile <= 32, "tile-local coordinates are packed in 5 bits");
  __shared__ int sq[256 * kRecStride];
  __shared__ unsigned long long sbest[kPix];
  __shared__ int spre[257];          // exclusive prefix of the work items (spans) per record
  __shared__ int sbox[256];          // bbox in tile: x0 | x1 << 5 | y0 << 10 | y1 << 15 (tile-local)
  __shared__ int sinv[256];          // ceil(2^16 / spans per bbox row)
  __shared__ unsigned char spair[kPix];     // the detection's pair map
  __shared__ int swarp[8];
  __shared__ int slast;
  __shared__ unsigned srim[4];       // flagged rim pixels of the tile: top row, bottom row, left, right column
  // this CTA's work unit: records [beg, lim) of one tile
  if ((int)blockIdx.x >= min(status->units[view], ru.units_cap)) return;
  const int4 unit = ru.units[blockIdx.x];
  const int tile = unit.x, beg = unit.y, lim = unit.z;
  const int slot = (unit.w & 0xfffff) - 1, nb = unit.w >> 20;
  if (lim < 0) return;   // no key slot: the tile's first unit takes all its records
  const int ti = tile % tilesX, tj = tile / tilesX;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ti0 = ti * kTile, tj0 = tj * kTile;
  const long long Px0 = (long long)ti0 * kSubpix + 128, Py0 = (long long)tj0 * kSubpix + 128;
  for (int q = tid; q < kPix; q += 256) sbest[q] = ~0ull;
  if (tid < 4) srim[tid] = 0u;
  for (int base = beg; base < lim; base += 256) {
    const int k = base + tid;
    int area = 0, box = 0, inv = 0;
    if (k < lim) {
      const TriSetup r = setup[list[k]];
      const int i0 = max(r.ibox & 0xffff, ti0), i1 = min((int)((unsigned)r.ibox >> 16), ti0 + kTile - 1);
      const int j0 = max(r.jbox & 0xffff, tj0), j1 = min((int)((unsigned)r.jbox >> 16), tj0 + kTile - 1);
      if (i0 <= i1 && j0 <= j1) {
        const int wd = (i1 - i0 + kSpan) / kSpan;   // spans per row
        area = wd * (j1 - j0 + 1);
        box = (i0 - ti0) | ((i1 - ti0) << 5) | ((j0 - tj0) << 10) | ((j1 - tj0) << 15);
        inv = (65536 + wd - 1) / wd;
        rec_stage(r, Px0, Py0, sq + tid * kRecStride);
      }
    }
    sbox[tid] = box;
    sinv[tid] = inv;
    // block exclusive scan of the areas
    int incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) swarp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int w = lane < 8 ? swarp[lane] : 0;
      int wi = w;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += v;
      }
      if (lane < 8) swarp[lane] = wi - w;
      if (lane == 7) spre[256] = wi;
    }
    __syncthreads();
    const int my_start = swarp[warp] + incl - area;
    spre[tid] = my_start;
    __syncthreads();
    const int total = spre[256];
    // the owner of item q: the last record whose first item is at most q
    for (int q = tid; q < total; q += 256) {
      int rec = 0;
#pragma unroll
      for (int step = 128; step; step >>= 1)
        if (spre[rec + step] <= q) rec += step;
      const int b = sbox[rec];
      const int x0 = b & 31, x1 = (b >> 5) & 31, y0 = (b >> 10) & 31;
      const int it = q - spre[rec], wd = (x1 - x0 + kSpan) / kSpan;
      const int qy = (it * sinv[rec]) >> 16;   // it / wd (exact for it <= 256 spans, wd <= 8)
      const int xs = x0 + kSpan * (it - qy * wd), y = y0 + qy;
      const int* rw = sq + rec * kRecStride;
      const int rf = rw[kRecFlags];
      if (rf & kRecSmall) cover_span<int, kTile>(rw, xs, min(xs + kSpan - 1, x1), y, sbest);
      else if (!(rf & kRecWide)) cover_span<long long, kTile>(rw, xs, min(xs + kSpan - 1, x1), y, sbest);
      else cover_span<long long, kTile, true>(rw, xs, min(xs + kSpan - 1, x1), y, sbest);
    }
    __syncthreads();
  }
  if (slot >= 0) {
    // fold this unit's minima into the tile's key slot; the last unit of the
    // tile takes the merged keys (and empties the slot for the next frame)
    unsigned long long* kb = ru.skey + (size_t)slot * 1024;
    for (int px = tid; px < kPix; px += 256) {
      const unsigned long long v = sbest[px];
      if (v != ~0ull) atomicMax(&kb[px], ~v);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) slast = atomicAdd(&ru.tile_done[tile], 1) == nb - 1;
    __syncthreads();
    if (!slast) return;
    __threadfence();
    for (int px = tid; px < kPix; px += 256) {
      sbest[px] = ~__ldcg(&kb[px]);
      kb[px] = 0ull;
    }
    if (tid == 0) ru.tile_done[tile] = 0;
    __syncthreads();
  }
  __syncthreads();   // every pixel's final key is visible to the detection
  // antialiasing detection of the pairs inside the tile (both pixels in the
  // image): a pair of different ids (the keys' low words: triangle, or all
  // ones for the background) whose occluder (the smaller key; the
  // background's is the largest) has a silhouette edge flags both its
  // pixels.  A detecting thread takes four consecutive pixels of one row,
  // tests their right and lower pairs (spair: bits 0-3 and 4-7), then ORs in
  // the pairs of its left and upper neighbours' threads.  The flagged pixels
  // are listed after the G-buffer writes (one atomic per warp, its latency
  // behind them); the rim's keys and flags go to rim for the seam pass
  // (aa_seam_kernel).
  constexpr int kRowThreads = kTile / 4, kDetThreads = kPix / 4;
  unsigned hbits = 0u;   // bit q: pixel q of the thread's four is flagged
  if (hflag) {
    auto pair_heavy = [&](unsigned long long kp, unsigned long long kq) -> unsigned {
      if ((unsigned)kp == (unsigned)kq) return 0u;
      const unsigned occ = (unsigned)(kp < kq ? kp : kq);
      return (silbits[occ >> 5] >> (occ & 31)) & 1u;
    };
    const int ly = tid / kRowThreads, x0 = (tid % kRowThreads) * 4;
    const int i0 = ti0 + x0, j = tj0 + ly;
    unsigned long long k[4];
    if (tid < kDetThreads) {
      const unsigned long long* row = sbest + ly * kTile + x0;
#pragma unroll
      for (int q = 0; q < 4; ++q) k[q] = row[q];
      const bool down = ly + 1 < kTile && j + 1 < H;
      unsigned pr = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool right = (q < 3 || x0 + 4 < kTile) && i0 + q + 1 < W && j < H;
        if (right) pr |= pair_heavy(k[q], q < 3 ? k[q + 1] : row[4]) << q;
        if (down && i0 + q < W) pr |= pair_heavy(k[q], row[kTile + q]) << (4 + q);
      }
      spair[tid] = (unsigned char)pr;
    }
    __syncthreads();
    if (tid < kDetThreads) {
      const unsigned me = spair[tid];
      const unsigned left = x0 > 0 ? spair[tid - 1] : 0u;
      const unsigned up = ly > 0 ? spair[tid - kRowThreads] : 0u;
      // pixel q: its right and lower pair, the right pair of pixel q - 1, the lower pair of the pixel above
      hbits = (me | (me >> 4) | (me << 1) | ((left >> 3) & 1u) | (up >> 4)) & 15u;
      unsigned inimg = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) inimg |= (i0 + q < W && j < H ? 1u : 0u) << q;
      hbits &= inimg;
      const size_t p0 = (size_t)j * W + i0;
      if (inimg == 15u && (p0 & 3) == 0) {
        *reinterpret_cast<unsigned*>(hflag + p0) =
            (hbits & 1u) | ((hbits & 2u) << 7) | ((hbits & 4u) << 14) | ((hbits & 8u) << 21);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if ((inimg >> q) & 1u) hflag[p0 + q] = (hbits >> q) & 1u;
      }
      unsigned long long* rk = rim.key + (size_t)tile * 4 * kTile;
      if (ly == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) rk[x0 + q] = k[q];
        if (hbits) atomicOr(&srim[0], hbits << x0);
      }
      if (ly == kTile - 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) rk[kTile + x0 + q] = k[q];
        if (hbits) atomicOr(&srim[1], hbits << x0);
      }
      if (x0 == 0) {
        rk[2 * kTile + ly] = k[0];
        if (hbits & 1u) atomicOr(&srim[2], 1u << ly);
      }
      if (x0 == kTile - 4) {
        rk[3 * kTile + ly] = k[3];
        if (hbits & 8u) atomicOr(&srim[3], 1u << ly);
      }
    }
  }
  for (int px = tid; px < kPix; px += 256) {
    const int i = ti0 + (px & (kTile - 1)), j = tj0 + (px >> kTL);
    const uint64_t best = sbest[px];
    if (i >= W || j >= H) continue;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float f = 1.f;   // shadow-map depth sample; background: 1
    if (best != ~0ull) {
      const int t = (int)(best & 0xffffffffu);
      const int v0 = tris[3 * t], v1 = tris[3 * t + 1], v2 = tris[3 * t + 2];
      const float4 ch[3] = {clip[v0], clip[v1], clip[v2]};
      const float4 cs[3] = {scr[v0], scr[v1], scr[v2]};
      const Bary r = bary_at(ch, cs, i, j, W, H);
      out = make_float4(__int_as_float(t + 1), r.b[0], r.b[1], key_depth(best));
      if (fmap) {
        // f = sum_k b_k d_k with b_2 = 1 - b_0 - b_1 of the stored barycentrics
        const float b2 = 1.f - r.b[0] - r.b[1];
        f = r.b[0] * depth[v0] + r.b[1] * depth[v1] + b2 * depth[v2];
      }
    }
    gbuf[(size_t)j * W + i] = out;
    if (fmap) fmap[(size_t)j * W + i] = moment_encode(f, ec);
  }
  if (hflag) {
    __syncthreads();
    if (tid < 4) rim.flags[(size_t)tile * 4 + tid] = srim[tid];
    const int p0 = (tj0 + tid / kRowThreads) * W + ti0 + (tid % kRowThreads) * 4;
    const int dpix[4] = {p0, p0 + 1, p0 + 2, p0 + 3};
    warp_append_n<4>(aa.list, aa.count, hbits, dpix);
  }
}

// ------------------------------------------------------------------ work counts
// The raster's integer work for one view, from the same lists and records the
// raster reads: tile-triangle pairs, spans of kSpan pixels (its work items) and
// pixel-centre coverage tests (three edge-function steps each).  One warp per
// tile; a diagnostic, off the frame's path.
__global__ void raster_stats_kernel(const TriSetup* __restrict__ setup, const int* __restrict__ offset,
                                    const int* __restrict__ list, int capacity, int n_tiles, int tilesX, int tl,
                                    unsigned long long* __restrict__ out) {
  const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (tile >= n_tiles) return;
  const int ts = 1 << tl;
  const int ti0 = (tile % tilesX) * ts, tj0 = (tile / tilesX) * ts;
  const int beg = min(offset[tile], capacity), end = min(offset[n_tiles + tile], capacity);
  unsigned long long pairs = 0, spans = 0, tests = 0;
  for (int k = beg + lane; k < end; k += 32) {
    const TriSetup r = setup[list[k]];
    const int i0 = max(r.ibox & 0xffff, ti0), i1 = min((int)((unsigned)r.ibox >> 16), ti0 + ts - 1);
    const int j0 = max(r.jbox & 0xffff, tj0), j1 = min((int)((unsigned)r.jbox >> 16), tj0 + ts - 1);
    if (i0 > i1 || j0 > j1) continue;
    pairs += 1;
    spans += (unsigned long long)((i1 - i0 + kSpan) / kSpan) * (j1 - j0 + 1);
    tests += (unsigned long long)(i1 - i0 + 1) * (j1 - j0 + 1);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    pairs += __shfl_xor_sync(kFull, pairs, o);
    spans += __shfl_xor_sync(kFull, spans, o);
    tests += __shfl_xor_sync(kFull, tests, o);
  }
  if (lane == 0 && pairs) {
    atomicAdd(&out[0], pairs);
    atomicAdd(&out[1], spans);
    atomicAdd(&out[2], tests);
  }
}

// ------------------------------------------------------------------ launchers
void launch_light_setup(const float* params, const LightSetupArgs& a, LightDev* out, float* viewM, float* viewMlo,
                        const CamMats& cams, int C, const VertNormalArgs& vn, cudaStream_t st) {
  count_launches(1);
  const int nv = (vn.V + kLightSetupThreads - 1) / kLightSetupThreads;
  light_setup_kernel<<<a.n + 1 + nv, kLightSetupThreads, 0, st>>>(params, a, out, viewM, viewMlo, cams, C, vn);
}

void launch_setup_all(const float* verts, int V, const int* tris, int T, const int* adj, const float* viewM,
                      const float* viewMlo,
                      const ViewSetupArgs& a, DevStatus* status, bool silhouettes, cudaStream_t st) {
  // (launched for V = 0 too: it zeroes the binning's counters)
  count_launches(1);
  transform_all_kernel<<<std::max((V + 255) / 256, 16), 256, 0, st>>>(verts, V, viewM, viewMlo, a, status);
  if (T > 0 && a.n > 0) {
    count_launches(1);
    setup_bin_kernel<<<dim3((T + 255) / 256, a.n), 256, 0, st>>>(tris, T, a, status);
  }
  if (silhouettes) launch_silhouettes_all(adj, T, a, st);
}

void launch_silhouettes_all(const int* adj, int T, const ViewSetupArgs& a, cudaStream_t st) {
  if (T == 0) return;
  count_launches(1);
  silhouette_all_kernel<<<(T + 255) / 256, 256, 0, st>>>(adj, T, a);
}

void launch_alloc_units(const int* count, int n, int* offset, DevStatus* status, int view, const TriSetup* setup,
                        const int* big_tri, int tilesX, int tile_log2, int* list, int capacity,
                        const RasterUnits& ru, bool write, cudaStream_t st) {
  count_launches(1);
  alloc_units_kernel<<<(n + 255) / 256, 256, 0, st>>>(count, n, offset, status, view, setup, big_tri, tilesX,
                                                      tile_log2, list, capacity, ru, write);
}

void launch_bin_fill(const TriSetup* setup, int T, int tilesX, BinShape bs, int* counter, const int* offset,
                     int* list, int capacity, DevStatus* status, const int* big_index, cudaStream_t st) {
  if (T == 0) return;
  count_launches(1);
  bin_fill_kernel<<<(T + 255) / 256, 256, 0, st>>>(setup, T, tilesX, bs, counter, offset, list, capacity, status,
                                                   big_index);
}

void launch_raster(const TriSetup* setup, const int* list, int tilesX, int tile_log2, int W, int H,
                   const float4* clip, const float4* scr, const int* tris, float4* gbuf, const float* depth,
                   float2* fmap, float ec, const RasterUnits& ru, DevStatus* status, int view,
                   const uint32_t* silbits, uint8_t* hflag, const AAWork& aa, const RimBufs& rim, cudaStream_t st) {
  count_launches(1);
  if (tile_log2 == 4)
    raster_kernel<4><<<ru.units_cap, 256, 0, st>>>(setup, list, tilesX, W, H, clip, scr, tris, gbuf, depth, fmap, ec,
                                                  ru, status, view, silbits, hflag, aa, rim);
  else
    raster_kernel<5><<<ru.units_cap, 256, 0, st>>>(setup, list, tilesX, W, H, clip, scr, tris, gbuf, depth, fmap, ec,
                                                  ru, status, view, silbits, hflag, aa, rim);
}

void launch_raster_stats(const TriSetup* setup, const int* offset, const int* list, int capacity, int tilesX,
                         int tilesY, int tile_log2, unsigned long long* out, cudaStream_t st) {
  const int n = tilesX * tilesY;
  if (n == 0) return;
  count_launches(1);
  raster_stats_kernel<<<(n + 7) / 8, 256, 0, st>>>(setup, offset, list, capacity, n, tilesX, tile_log2, out);
}

}  // namespace dsm
