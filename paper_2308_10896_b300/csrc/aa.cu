// Shadow-map depth interpolation (f, f^2) and the analytic edge antialiasing
// that makes silhouettes differentiable (Sec. 4/5: f, f^2 -> f~, (f^2)~; the
// same pass smooths the final image), with their adjoints.
#include "dsm.h"
#include "common.cuh"
#include "kernels.h"

namespace dsm {

// Crossing of a silhouette edge of triangle `tri` with the segment between the
// centres of the occluder pixel O = (io, jo) and its neighbour N = (in, jn).
// Decisions on the exact snapped coordinates; t from the unsnapped edge.
struct Cross {
  int found;
  int va, vb;
  float t;          // crossing parameter from O towards N, clamped to [0, 1]
  int active;       // t strictly inside (0, 1): it depends on the edge
  float dt[4];      // dt / d(xa, ya, xb, yb) in screen pixels (when active)
};

// Unsnapped screen position (pixels, y down) of vertex v relative to the
// centre of pixel (i, j), from its float-float screen position.
__device__ __forceinline__ float2 rel_screen(const AAArgs& a, int v, int i, int j) {
  const float4 s = a.scr[v];
  return make_float2(scr_dx(s, i), scr_dy(s, j));
}

template <bool kGrad>
__device__ __forceinline__ Cross find_crossing(const AAArgs& a, int tri, int io, int jo, int in, int jn,
                                               bool vertical) {
  Cross c;
  c.found = 0;
  const int m = a.sil[tri];
  if (!m) return c;
  long long line, lo;
  if (vertical) {
    line = (long long)io * kSubpix + 128;
    lo = (long long)min(jo, jn) * kSubpix + 128;
  } else {
    line = (long long)jo * kSubpix + 128;
    lo = (long long)min(io, in) * kSubpix + 128;
  }
  const long long hi = lo + kSubpix;
  for (int e = 0; e < 3; ++e) {
    if (!((m >> e) & 1)) continue;
    const int va = a.tris[3 * tri + edge_p(e)], vb = a.tris[3 * tri + edge_q(e)];
    const VertSnap A = a.snap[va], B = a.snap[vb];
    long long ua, ub, wa, wb;
    if (vertical) { ua = A.X; ub = B.X; wa = A.Y; wb = B.Y; }
    else          { ua = A.Y; ub = B.Y; wa = A.X; wb = B.X; }
    if ((ua >= line) == (ub >= line)) continue;
    const long long D = ub - ua;
    const long long along = llabs(wb - wa);
    if (vertical ? !(llabs(D) >= along) : !(llabs(D) > along)) continue;   // one axis per edge
    const long long num = wa * D + (line - ua) * (wb - wa);
    const bool inside = D > 0 ? (lo * D <= num && num <= hi * D) : (lo * D >= num && num >= hi * D);
    if (!inside) continue;
    c.found = 1;
    c.va = va;
    c.vb = vb;
    // unsnapped screen positions of the endpoints relative to O's pixel centre,
    // from their float-float screen positions: accurate to float32 relative to
    // these small offsets, not to the view's size
    const float2 sa = rel_screen(a, va, io, jo), sb = rel_screen(a, vb, io, jo);
    // along-coordinate p, across-coordinate q (q = 0 is the line through both
    // centres, p = 0 is O's centre)
    float pa, qa, pb, qb, step;
    if (vertical) {
      pa = sa.y; qa = sa.x; pb = sb.y; qb = sb.x;
      step = (jn > jo) ? 1.f : -1.f;
    } else {
      pa = sa.x; qa = sa.y; pb = sb.x; qb = sb.y;
      step = (in > io) ? 1.f : -1.f;
    }
    const float dq = qb - qa;
    if (dq == 0.f) {
      c.t = 0.5f;
      c.active = 0;
      return c;
    }
    const float s = -qa / dq;
    const float r = (pb - pa) / dq;
    const float cross = pa + s * (pb - pa);
    const float traw = cross * step;
    c.t = fminf(fmaxf(traw, 0.f), 1.f);
    c.active = (traw > 0.f && traw < 1.f);
    if (kGrad) {
      // d cross / d(pa, qa, pb, qb)
      const float dpa = 1.f - s, dpb = s, dqa = -r * (1.f - s), dqb = -r * s;
      if (vertical) {  // p = y, q = x
        c.dt[0] = step * dqa; c.dt[1] = step * dpa; c.dt[2] = step * dqb; c.dt[3] = step * dpb;
      } else {
        c.dt[0] = step * dpa; c.dt[1] = step * dqa; c.dt[2] = step * dpb; c.dt[3] = step * dqb;
      }
    }
    return c;
  }
  return c;
}

// dL/d clip of a vertex from dL/d of its screen position (sx, sy).
__device__ __forceinline__ float4 screen_to_clip_grad(float4 c, float gx, float gy, int W, int H) {
  const float iw = 1.0f / c.w;
  const float ax = 0.5f * W * iw, ay = -0.5f * H * iw;
  return make_float4(gx * ax, gy * ay, 0.f, -(gx * ax * c.x + gy * ay * c.y) * iw);
}

__device__ __forceinline__ int gid(float4 g) { return __float_as_int(g.x); }

// Pair bookkeeping for pixel p=(i,j) and its neighbour q.  Returns false when
// the pair has no antialiasing crossing.
struct PairInfo {
  bool p_occ;       // p is the occluder pixel O
  bool p_is_first;  // p is the left / top pixel of the pair
  Cross c;
};

// Whether p is the occluder O of the pair (p, q) (ids differ): the nearer
// surface by depth key; the background never occludes.
__device__ __forceinline__ bool pair_p_occ(int i, int j, int ni, int nj, float4 gp, float4 gq) {
  const int idp = gid(gp), idq = gid(gq);
  const bool p_first = (ni > i) || (nj > j);
  const int idA = p_first ? idp : idq, idB = p_first ? idq : idp;
  const float zA = p_first ? gp.w : gq.w, zB = p_first ? gq.w : gp.w;
  const bool a_occ = (idB == 0) || (idA != 0 && depth_key(zA, idA - 1) < depth_key(zB, idB - 1));
  return p_first ? a_occ : !a_occ;
}

template <bool kGrad>
__device__ __forceinline__ bool pair_info(const AAArgs& a, int i, int j, int ni, int nj, float4 gp, float4 gq,
                                          PairInfo& pi) {
  const int idp = gid(gp), idq = gid(gq);
  if (idp == idq) return false;
  const bool p_first = (ni > i) || (nj > j);
  const bool p_occ = pair_p_occ(i, j, ni, nj, gp, gq);
  const int tri = (p_occ ? idp : idq) - 1;
  const int io = p_occ ? i : ni, jo = p_occ ? j : nj, in = p_occ ? ni : i, jn = p_occ ? nj : j;
  pi.c = find_crossing<kGrad>(a, tri, io, jo, in, jn, nj != j);
  pi.p_occ = p_occ;
  pi.p_is_first = p_first;
  return pi.c.found;
}

// Neighbour d of pixel (i, j): left, right, up, down.
__device__ __forceinline__ int nb_dx(int d) { return d == 0 ? -1 : d == 1 ? 1 : 0; }
__device__ __forceinline__ int nb_dy(int d) { return d == 2 ? -1 : d == 3 ? 1 : 0; }

// Antialiasing runs as a detection step and a list pass.  Only a pair whose
// occluder triangle has a silhouette edge can have a crossing, and such pairs
// are few (about 1 % of pixels in the benchmark scenes); the code that finds
// and differentiates crossings needs many registers.  So the detection only
// flags the pixels with such a pair (hflag) and appends them to the view's
// work list, and the list passes run the full pair logic for the listed
// pixels only.  The raster detects the pairs inside one of its tiles from the
// tile's final keys (a pair's occluder is the smaller depth key, the
// background's key being the largest), and aa_seam_kernel the pairs across
// tile edges.  Every other pixel's antialiased value is its own value, so the
// consumers read the unmodified map there: the moment filter substitutes the
// list pass's values at flagged texels, the camera's shading writes the image
// at unflagged pixels, the backward's filter transpose writes dL/df directly
// and the shading adjoint reads dL/dimage there.  The list depends only on the
// G-buffer, so the backward reuses the forward's list; the transform of the
// next frame clears its counter.
// Warp-aggregated append to the view's work list; every lane of the warp must call it.
__device__ __forceinline__ void list_append(const AAWork& w, bool want, int value) {
  warp_append(w.list, w.count, want, value);
}

// ------------------------------------------------------------------ forward
// Every pixel gathers the gains of the (up to 4) pairs it belongs to: if t > 1/2
// the neighbour-side pixel N gains (t - 1/2)(c_O - c_N), else O gains
// (1/2 - t)(c_N - c_O).  aa_pair_gain: the gain of pixel (i, j) from its pair
// in direction d.
template <typename V>
__device__ __forceinline__ V aa_pair_gain(const AAArgs& a, int i, int j, int d, float4 gp, V cp,
                                          const V* __restrict__ color) {
  const int ni = i + nb_dx(d), nj = j + nb_dy(d);
  if (ni < 0 || nj < 0 || ni >= a.W || nj >= a.H) return V{};
  const size_t q = (size_t)nj * a.W + ni;
  const float4 gq = a.gbuf[q];
  PairInfo pi;
  if (!pair_info<false>(a, i, j, ni, nj, gp, gq, pi)) return V{};
  const float tt = pi.c.t;
  if (tt > 0.5f) {
    if (!pi.p_occ) return vscale(vsub(color[q], cp), tt - 0.5f);   // p = N, cq = c_O
  } else {
    if (pi.p_occ) return vscale(vsub(color[q], cp), 0.5f - tt);    // p = O, cq = c_N
  }
  return V{};
}

__device__ __forceinline__ float2 shfl_xor_v(float2 v, int m) {
  return make_float2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}
__device__ __forceinline__ float4 shfl_xor_v(float4 v, int m) {
  return make_float4(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m), __shfl_xor_sync(kFull, v.z, m),
                     __shfl_xor_sync(kFull, v.w, m));
}

// Second passes: four consecutive lanes take one listed pixel, one pair
// direction each, and sum their terms with two shuffles.  `body(k, d, act)`
// runs for every lane (act: the lane has an item).
template <typename Body>
__device__ __forceinline__ void for_listed_pairs(const AAWork& w, Body body) {
  const int n = *(volatile int*)w.count;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_sweep = gridDim.x * blockDim.x / 4;
  for (int k0 = 0; k0 < n; k0 += per_sweep) {
    const int k = k0 + gtid / 4;
    body(k, gtid & 3, k < n);
  }
}

// Detection across tile seams.  The raster tested the pairs inside each of
// its tiles (side T = 2^tl) and left each tile's rim (final keys, flagged
// pixels) in rim; this pass tests the pairs across tile edges from the rims
// alone and flags and lists the rim pixels the raster left unflagged.  One
// thread per rim entry: side s (top, bottom, left, right) and position k;
// the top and bottom rows hold the corners, with both of their neighbours
// across the tile's edges, and the columns skip them.  A pair of different
// ids has the smaller key as its occluder (the background's is the largest).
constexpr int kSeamThreads = 128;
__device__ __forceinline__ bool seam_pair_heavy(unsigned long long kp, unsigned long long kq,
                                                const uint32_t* __restrict__ silbits) {
  const unsigned idp = kp == ~0ull ? 0u : (unsigned)kp + 1u, idq = kq == ~0ull ? 0u : (unsigned)kq + 1u;
  if (idp == idq) return false;
  const unsigned occ = (unsigned)(kp < kq ? kp : kq);
  return (silbits[occ >> 5] >> (occ & 31)) & 1u;
}
__global__ void __launch_bounds__(kSeamThreads) aa_seam_kernel(int W, int H, int tilesX, int n_tiles, int tl,
                                                               RimBufs rim, const uint32_t* __restrict__ silbits,
                                                               uint8_t* __restrict__ hflag, AAWork w) {
  const int T = 1 << tl;
  const int g = blockIdx.x * kSeamThreads + threadIdx.x;
  const int tile = g >> (tl + 2), r = g & (4 * T - 1), side = r >> tl, k = r & (T - 1);
  const int tx = tile % tilesX, ty = tile / tilesX;
  const int x = side == 0 || side == 1 ? k : (side == 2 ? 0 : T - 1);
  const int y = side == 0 ? 0 : (side == 1 ? T - 1 : k);
  const int i = (tx << tl) + x, j = (ty << tl) + y;
  const bool in = tile < n_tiles && !(side >= 2 && (k == 0 || k == T - 1)) && i < W && j < H;
  bool want = false;
  if (in && !((rim.flags[(size_t)tile * 4 + side] >> k) & 1u)) {
    const unsigned long long kp = rim.key[(size_t)tile * 4 * T + r];
    // the neighbour across the edge of side `side`: the facing side of the adjacent tile
    const int ntx = tx + (side == 2 ? -1 : side == 3 ? 1 : 0), nty = ty + (side == 0 ? -1 : side == 1 ? 1 : 0);
    const int ni = i + (side == 2 ? -1 : side == 3 ? 1 : 0), nj = j + (side == 0 ? -1 : side == 1 ? 1 : 0);
    if (ni >= 0 && nj >= 0 && ni < W && nj < H) {
      const int facing = side ^ 1;   // top <-> bottom, left <-> right
      const unsigned long long kq = rim.key[((size_t)(nty * tilesX + ntx) * 4 + facing) * T + k];
      want = seam_pair_heavy(kp, kq, silbits);
    }
    // a corner of the top or bottom row: also its neighbour across the side edge
    // (the adjacent tile's same row, its far end)
    if (side < 2 && (k == 0 || k == T - 1)) {
      const int d = k == 0 ? -1 : 1;
      if (i + d >= 0 && i + d < W) {
        const unsigned long long kq = rim.key[((size_t)(ty * tilesX + tx + d) * 4 + side) * T + (T - 1 - k)];
        want = want || seam_pair_heavy(kp, kq, silbits);
      }
    }
    if (want) hflag[(size_t)j * W + i] = 1;
  }
  warp_append(w.list, w.count, want, j * W + i);
}

template <typename V>
__global__ void __launch_bounds__(256) aa_forward_list_kernel(AAArgs a, const V* __restrict__ color,
                                                              V* __restrict__ out, AAWork w) {
  for_listed_pairs(w, [&](int k, int d, bool act) {
    V g{};
    V cp{};
    int p = 0;
    if (act) {
      p = w.list[k];
      const int j = p / a.W, i = p - j * a.W;
      cp = color[p];
      g = aa_pair_gain<V>(a, i, j, d, a.gbuf[p], cp, color);
    }
    g = vadd(g, shfl_xor_v(g, 1));
    g = vadd(g, shfl_xor_v(g, 2));
    if (act && d == 0) out[p] = vadd(cp, g);
  });
}

// ------------------------------------------------------------------ adjoint
// dL/dc_p = g_p + the pair terms; the t-gradient of each pair is scattered once
// (by its left / top pixel) onto the clip coordinates of the edge endpoints.
// aa_pair_adjoint: the term of pixel (i, j) from its pair in direction d;
// gout[q] gives the output gradient of pixel q.
template <typename V, typename G>
__device__ __forceinline__ V aa_pair_adjoint(const AAArgs& a, int i, int j, int d, float4 gp, V g_p, const V* color,
                                             const G& gout, float4* gclip) {
  const int ni = i + nb_dx(d), nj = j + nb_dy(d);
  if (ni < 0 || nj < 0 || ni >= a.W || nj >= a.H) return V{};
  const size_t p = (size_t)j * a.W + i, q = (size_t)nj * a.W + ni;
  const float4 gq = a.gbuf[q];
  PairInfo pi;
  if (!pair_info<true>(a, i, j, ni, nj, gp, gq, pi)) return V{};
  const V g_q = gout[q];
  const float tt = pi.c.t;
  const V gO = pi.p_occ ? g_p : g_q, gN = pi.p_occ ? g_q : g_p;
  V term;
  float dLdt = 0.f;
  if (tt > 0.5f) {            // Delta_N = (t - 1/2)(c_O - c_N)
    term = vscale(gN, pi.p_occ ? (tt - 0.5f) : -(tt - 0.5f));
    if (pi.p_is_first && pi.c.active) {
      const V cp = color[p], cq = color[q];
      const V cO = pi.p_occ ? cp : cq, cN = pi.p_occ ? cq : cp;
      dLdt = dotv(gN, vsub(cO, cN));
    }
  } else {                   // Delta_O = (1/2 - t)(c_N - c_O)
    term = vscale(gO, pi.p_occ ? -(0.5f - tt) : (0.5f - tt));
    if (pi.p_is_first && pi.c.active) {
      const V cp = color[p], cq = color[q];
      const V cO = pi.p_occ ? cp : cq, cN = pi.p_occ ? cq : cp;
      dLdt = dotv(gO, vsub(cO, cN));
    }
  }
  if (dLdt != 0.f) {
    const float4 ca = a.clip[pi.c.va], cb = a.clip[pi.c.vb];
    atomic_add4(&gclip[pi.c.va], screen_to_clip_grad(ca, dLdt * pi.c.dt[0], dLdt * pi.c.dt[1], a.W, a.H));
    atomic_add4(&gclip[pi.c.vb], screen_to_clip_grad(cb, dLdt * pi.c.dt[2], dLdt * pi.c.dt[3], a.W, a.H));
  }
  return term;
}

__global__ void __launch_bounds__(256) aa_backward4_list_kernel(AAArgs a, const float4* __restrict__ color,
                                                                ImageGrad gout, float4* __restrict__ gcolor,
                                                                float4* __restrict__ gclip, AAWork w) {
  for_listed_pairs(w, [&](int k, int d, bool act) {
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f), g_p = g;
    int p = 0;
    if (act) {
      p = w.list[k];
      const int j = p / a.W, i = p - j * a.W;
      g_p = gout[p];
      g = aa_pair_adjoint<float4>(a, i, j, d, a.gbuf[p], g_p, color, gout, gclip);
    }
    g = vadd(g, shfl_xor_v(g, 1));
    g = vadd(g, shfl_xor_v(g, 2));
    if (act && d == 0) gcolor[p] = vadd(g_p, g);
  });
}

// Adjoint of the shadow-map antialiasing at the listed texels: dL/d(f, f^2)
// (the pair t-gradients go to the light-space clip coordinates of the edge
// endpoints), folded into dL/df by moment_fold (the product rule of the
// second channel, times the warp's slope).  The filter transpose already
// wrote dL/df at every other texel.
__global__ void __launch_bounds__(256) sm_aa_adjoint_list_kernel(AAArgs a, const float2* __restrict__ fmap,
                                                                 const float2* __restrict__ gft,
                                                                 float4* __restrict__ gclip,
                                                                 float* __restrict__ gf_out, float ec, AAWork w) {
  for_listed_pairs(w, [&](int k, int d, bool act) {
    float2 g = make_float2(0.f, 0.f), g_p = g;
    int p = 0;
    if (act) {
      p = w.list[k];
      const int j = p / a.W, i = p - j * a.W;
      g_p = gft[p];
      g = aa_pair_adjoint<float2>(a, i, j, d, a.gbuf[p], g_p, fmap, gft, gclip);
    }
    g = vadd(g, shfl_xor_v(g, 1));
    g = vadd(g, shfl_xor_v(g, 2));
    if (act && d == 0) {
      const float2 gc = vadd(g_p, g);
      gf_out[p] = moment_fold(gc, fmap[p].x, ec);
    }
  });
}


// Adjoint of the interpolation f = sum_k b_k d_k: dL/dd_k = b_k dL/df onto the
// vertex depths and, through the perspective-correct barycentrics, onto the
// light-space clip coordinates.  Each warp walks a strip of kStrip rows over 32
// columns; per-triangle sums go through a run accumulator (a large triangle
// costs one set of atomics per strip), the current triangle's vertex data stay
// in registers, and the next row's texel data are fetched one row ahead.
constexpr int kStrip = 8;

// Scatter of 12 per-triangle values: for each vertex (dL/dclip_x, dL/dclip_y,
// dL/dd, dL/dclip_w).  A light view's barycentrics never depend on clip z, so
// the z slot of the clip gradient carries the vertex-depth gradient instead.
struct SmScatter {
  const int* tris;
  float4* gclip;
  float* big_acc;        // kMaxBig x kBigSlots x kBigStrideSm
  int slot;
  // ordinary triangle: onto its vertices
  __device__ __forceinline__ void vertices(int t, const float (&c)[12]) const {
    for (int k = 0; k < 3; ++k)
      atomic_add4(&gclip[tris[3 * t + k]], make_float4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]));
  }
  // big triangle b: into one of its slot copies
  __device__ __forceinline__ void operator()(int b, const float (&c)[12], int lane = 0) const {
    float* d = big_acc + ((size_t)b * kBigSlots + ((slot + lane) & (kBigSlots - 1))) * kBigStrideSm;
    for (int k = 0; k < 12; ++k) atomicAdd(&d[k], c[k]);
  }
};

__global__ void __launch_bounds__(256) sm_interp_adjoint_kernel(AAArgs a, const float* __restrict__ gf_map,
                                                                const float* __restrict__ depth,
                                                                float4* __restrict__ gclip,
                                                                const int* __restrict__ big,
                                                                float* __restrict__ big_acc) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * kStrip;
  const bool col_ok = i < a.W;
  SmScatter sc{a.tris, gclip, big_acc, scatter_slot(kBigSlots)};
  BigRun<12, 1> run;
  big_run_reset(run);
  float4 cc[3];
  float cd[3];
  // prefetch of row j0
  // the texel gradients of the strip first; a G-buffer texel is read only
  // where its gradient is nonzero
  float gfs[kStrip];
#pragma unroll
  for (int s = 0; s < kStrip; ++s) gfs[s] = (col_ok && j0 + s < a.H) ? gf_map[(size_t)(j0 + s) * a.W + i] : 0.f;
  for (int s = 0; s < kStrip; ++s) {
    const int j = j0 + s;
    const float gf = gfs[s];
    const float4 g = gf != 0.f ? a.gbuf[(size_t)j * a.W + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float c[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) c[k] = 0.f;
    int t = -1;
    const int id = gid(g);
    if (col_ok && j < a.H && id && gf != 0.f) {
      t = id - 1;
      // the triangle's corners are reloaded per texel (L1 hits): keeping them
      // live across rows costs more in occupancy than the loads
      float4 cs[3];
      for (int k = 0; k < 3; ++k) {
        const int v = a.tris[3 * t + k];
        cc[k] = a.clip[v];
        cs[k] = a.scr[v];
        cd[k] = depth[v];
      }
      const float px = pix_ndc_x(i, a.W), py = pix_ndc_y(j, a.H);
      const Bary r = bary_at(cc, cs, i, j, a.W, a.H);
      const float b[3] = {g.y, g.z, 1.f - g.y - g.z};
      // f = sum_k b_k d_k: centred dL/db_k = gf sum_j b_j (d_k - d_j)
      float gb[3];
      for (int k = 0; k < 3; ++k)
        gb[k] = gf * (r.b[0] * (cd[k] - cd[0]) + r.b[1] * (cd[k] - cd[1]) + r.b[2] * (cd[k] - cd[2]));
      float4 gcv[3];
      bary_backward(r, gb, px, py, gcv);
      for (int k = 0; k < 3; ++k) {
        c[4 * k] = gcv[k].x; c[4 * k + 1] = gcv[k].y; c[4 * k + 2] = b[k] * gf; c[4 * k + 3] = gcv[k].w;
      }
    }
    const int bi = t >= 0 ? big[t] : -1;
    big_run_add(run, bi, c, sc);
    if (t >= 0 && bi < 0) sc.vertices(t, c);
  }
  big_run_flush(run, sc);
}

// Sum the kBigSlots copies of each big triangle and scatter the result onto its
// vertices' light-space clip gradients (z slot: vertex depth).
__global__ void sm_big_resolve_kernel(const int* __restrict__ tris, const int* __restrict__ big_tri,
                                      const DevStatus* __restrict__ status, int view,
                                      const float* __restrict__ big_acc, float4* __restrict__ gclip) {
  const int b = blockIdx.x;
  if (b >= min(status->big_count[view], kMaxBig)) return;
  __shared__ float sum[12];
  const int k = threadIdx.x;
  if (k < 12) {
    float acc = 0.f;
    for (int q = 0; q < kBigSlots; ++q) acc += big_acc[((size_t)b * kBigSlots + q) * kBigStrideSm + k];
    sum[k] = acc;
  }
  __syncthreads();
  if (k < 3)
    atomic_add4(&gclip[tris[3 * big_tri[b] + k]],
                make_float4(sum[4 * k], sum[4 * k + 1], sum[4 * k + 2], sum[4 * k + 3]));
}

// ------------------------------------------------------------------ launchers

constexpr int kListGrid = 148 * 8;   // CTAs of a second pass (grid-stride over the list)

void launch_aa_seam(const AAArgs& a, int tilesX, int tilesY, int tile_log2, const RimBufs& rim,
                    const uint32_t* silbits, uint8_t* hflag, const AAWork& w, cudaStream_t st) {
  const int n = tilesX * tilesY;
  if (n == 0) return;
  count_launches(1);
  const int threads = n << (tile_log2 + 2);
  aa_seam_kernel<<<(threads + kSeamThreads - 1) / kSeamThreads, kSeamThreads, 0, st>>>(
      a.W, a.H, tilesX, n, tile_log2, rim, silbits, hflag, w);
}
void launch_aa_forward2_list(const AAArgs& a, const float2* color, float2* out, const AAWork& w, cudaStream_t st) {
  count_launches(1);
  aa_forward_list_kernel<float2><<<kListGrid, 256, 0, st>>>(a, color, out, w);
}
void launch_aa_forward4_list(const AAArgs& a, const float4* color, float4* out, const AAWork& w, cudaStream_t st) {
  count_launches(1);
  aa_forward_list_kernel<float4><<<kListGrid, 256, 0, st>>>(a, color, out, w);
}
void launch_sm_aa_adjoint_list(const AAArgs& a, const float2* fmap, const float2* gft, float4* gclip, float* gf_out,
                               float ec, const AAWork& w, cudaStream_t st) {
  count_launches(1);
  sm_aa_adjoint_list_kernel<<<kListGrid, 256, 0, st>>>(a, fmap, gft, gclip, gf_out, ec, w);
}

void launch_sm_interp_adjoint(const AAArgs& a, const float* gf, const float* depth, float4* gclip,
                              const BigArgs& big, cudaStream_t st) {
  dim3 b(32, 8), g((a.W + 31) / 32, (a.H + 8 * kStrip - 1) / (8 * kStrip));
  count_launches(1);
  sm_interp_adjoint_kernel<<<g, b, 0, st>>>(a, gf, depth, gclip, big.index, big.acc);
  count_launches(1);
  sm_big_resolve_kernel<<<kMaxBig, 32, 0, st>>>(a.tris, big.tri, big.status, big.view, big.acc, gclip);
}

void launch_aa_backward4_list(const AAArgs& a, const float4* color, const ImageGrad& gout, float4* gcolor,
                              float4* gclip, const AAWork& w, cudaStream_t st) {
  count_launches(1);
  aa_backward4_list_kernel<<<kListGrid, 256, 0, st>>>(a, color, gout, gcolor, gclip, w);
}

// Diagnostic (dsm_set_grad_mask): zero dL/df~ and dL/df at the texels of the
// shadow map's silhouette band, the texels the detection pass flagged: those
// with a 4-neighbour of another triangle id whose pair's nearer surface has a
// silhouette edge in this view.  Every antialiasing crossing lies in that
// band, so with the mask the backward carries no edge-antialiasing term of the
// map and no interpolation term of a band texel.
__global__ void sm_band_mask_kernel(const uint8_t* __restrict__ hflag, int n, float2* __restrict__ gft,
                                    float* __restrict__ gf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && hflag[p]) {
    gft[p] = make_float2(0.f, 0.f);
    gf[p] = 0.f;
  }
}

void launch_sm_band_mask(const uint8_t* hflag, int n, float2* gft, float* gf, cudaStream_t st) {
  count_launches(1);
  sm_band_mask_kernel<<<(n + 255) / 256, 256, 0, st>>>(hflag, n, gft, gf);
}

}  // namespace dsm
