// Launchers of the device kernels (host-callable).  Every launcher enqueues on
// the given stream and returns immediately.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>
#include "dsm.h"
#include "common.cuh"

namespace dsm {

// Process-wide count of launched kernels (reported by dsm_kernel_launches).
extern std::atomic<unsigned long long> g_kernel_launches;
inline void count_launches(int n) { g_kernel_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

struct LightConst {
  int type;                // 0 directional, 1 perspective (spot, or a cube face: persp_c = 1)
  int res;
  int user;                // the caller's light index (its row of the parameter array)
  int face;                // cube face 0..5 of a point light (fixed axis direction), -1 otherwise
  double dist, ortho_half, near_plane, far_plane;
  double persp_c;          // 1 / tan(fov / 2), computed on the host in float64
  float intensity[3];
};

struct Mat20 {
  float v[20];
};

struct LightSetupArgs {
  LightConst c[kMaxLightViews];
  int n;
};

// Camera matrices, 20 floats each (the clip matrix, then an unused depth row).
struct CamMats {
  float v[20 * DSM_MAX_CAMERAS];
};

// Filter weights and the clamp-boundary fold coefficients of the adjoint.
struct FilterArgs {
  float w[65];             // taps w[k + r], |k| <= r
  float fold[33];          // fold[i] = sum of w over taps that leave the map by more than i texels
  int r;
  int boundary;            // 0 clamp, 1 zero
  int shape;               // 0 TMA-staged persistent kernel (radius <= 8, side a multiple of 16, and no
                           //   antialiased patch to substitute; else 2),
                           // 1 two 1-D passes, 2 one fused tile kernel with plain loads (radius <= 15, else 1)
};

// Extras of the shadow-map path (NULL for a plain filter):
//   forward: the input is (f, f^2) except where hflag marks a texel whose
//     antialiased value the antialiasing pass wrote into patch;
//   adjoint: also writes dL/df of the output g (moment_fold of g with the
//     first channel of fmap and the warp exponent ec).
struct FilterExtras {
  const uint8_t* hflag;
  const float2* patch;
  const float2* fmap;
  float* gf;
  float ec;
};

// Binning and raster shape of one view: tile side 2^tile_log2 pixels, and the
// tile count from which a triangle takes the big-triangle binning.
struct BinShape {
  int tile_log2;
  int big_tiles;
};

struct ShadeArgs {
  const float4* gbuf;
  int W, H;
  const float* verts;
  const int* tris;
  const int* tri_mat;
  const float* albedo;
  int n_mat;
  const float* vnormal;    // V x 3, unit vertex normals
  const float4* cam_clip;  // V, camera clip coordinates
  const float4* cam_scr;   // V, float-float unsnapped screen positions (sx hi, lo, sy hi, lo)
  const LightDev* lights;
  int L;
  const float2* mom[kMaxLightViews];
  int res[kMaxLightViews];
  float min_variance;
  float ec;                           // exponential warp of the moments (0: variance shadow maps)
};

// dL/dimage of a camera: given (g), or, for g NULL, that of the mean squared
// error L = sum (image - target)^2 / n over the n floats of the image, whose
// gradient 2 / n (image - target) is formed in the arithmetic of
// dsm_l2_loss_grad (scale = 2 / n rounded to float32, then one product).
struct ImageGrad {
  const float4* g;
  const float4* image;
  const float4* target;
  float scale;
  __device__ __forceinline__ float4 operator[](size_t p) const {
    if (g) return g[p];
    const float4 a = image[p], b = target[p];
    return make_float4(scale * (a.x - b.x), scale * (a.y - b.y), scale * (a.z - b.z), scale * (a.w - b.w));
  }
};

struct ShadeGradArgs {
  // dL/d colour before the final antialiasing: gcolor at the pixels flagged by
  // the camera's antialiasing detection (hflag), dL/dimage gimage elsewhere
  // (hflag NULL: gimage everywhere)
  const float4* gcolor;
  ImageGrad gimage;
  const uint8_t* hflag;
  int loss_index;                     // with the mean squared error: its sum of squares goes to red[loss_index]
                                      // (per block slot); -1 otherwise
  float4* gpos;                       // V, dL/d vertex position through the camera's interpolation (xyz)
  float4* gnormal;                    // V, dL/d unit vertex normal (xyz)
  float4* gclip;                      // V, dL/d camera clip
  float* dalbedo;                     // M x 3
  float2* gm[kMaxLightViews];         // dL/d(m1, m2) texel maps
  double* red;                        // kRedSlots x red_stride: [dQ (L x 20) | direct (L x 3) | albedo (M x 3) |
                                      //   squared error (1)]
  int red_stride;
  const int* big;                     // camera view big-triangle index per triangle
  float* big_acc;                     // kMaxBig x kBigSlots x kBigStrideCam
  float4* pgrad;                      // per pixel: (dL/dx, dL/dn~ x) (dL/dn~ y, z, active, 0)
};

struct VertGradPtrs {
  const float4* gclip[kMaxViews];   // per view (lights, then cameras); lights: z = dL/d vertex depth
};

// Big-triangle bookkeeping of one view (see kBigTilesDefault).
struct BigArgs {
  const int* index;          // per triangle: big index or -1
  const int* tri;            // per big index: triangle
  float* acc;                // kMaxBig x kBigSlots x N accumulators
  const DevStatus* status;   // holds the number of big triangles
  int view;
};

// Antialiasing work list of a view: pixel indices appended by the detection
// (the raster and the seam pass); the counter is cleared by the transform of
// each frame.
struct AAWork {
  int* list;
  int* count;
};

// The raster tiles' rims for the seam pass of the antialiasing detection:
// per tile (side T), the final keys of its top row, bottom row, left and right
// column (4 T entries), and four words with the pixels of each the raster
// flagged (bit k: entry k of that side).
struct RimBufs {
  unsigned long long* key;   // tiles x 4 T
  unsigned* flags;           // tiles x 4
};

struct AAArgs {
  const float4* gbuf;
  int W, H;
  const int* tris;
  const uint8_t* sil;
  const VertSnap* snap;
  const float4* clip;
  const float4* scr;       // V, float-float unsnapped screen positions (sx hi, lo, sy hi, lo)
};

// Per-view pointers and sizes for the fused setup of all views of a frame.
struct ViewSetupArgs {
  int n;
  int view0;                      // frame view index of entry 0 (the device status is indexed by frame view)
  int W[kMaxViews], H[kMaxViews], tiles[kMaxViews];
  float4* clip[kMaxViews];
  float4* scr[kMaxViews];         // float-float unsnapped screen positions (see transform_all_kernel)
  VertSnap* snap[kMaxViews];
  float* depth[kMaxViews];        // light views only (camera: NULL)
  TriSetup* setup[kMaxViews];
  int8_t* orient[kMaxViews];
  uint8_t* sil[kMaxViews];
  uint32_t* silbits[kMaxViews];   // the same, one bit per triangle (bit t & 31 of word t >> 5: any silhouette edge)
  int* count[kMaxViews];          // tile counters, zeroed by the transform
  int* aa_count[kMaxViews];       // antialiasing work-list counters, zeroed by the transform
  int tilesX[kMaxViews];
  BinShape bs[kMaxViews];
  int* big_index[kMaxViews];      // per triangle: its index in big_tri, or -1
  int* big_tri[kMaxViews];        // the view's big triangles (at most kMaxBig)
};
// Transform and triangle setup of every view, with the binning's count pass
// (per-tile counts of the ordinary triangles, the list of big ones) in the
// setup kernel; the transform first zeroes the tile counters, the view
// totals of the device status and the antialiasing work lists.  With
// `silhouettes`, the silhouettes follow (needed only by the antialiasing,
// they may instead follow later through launch_silhouettes_all).
void launch_setup_all(const float* verts, int V, const int* tris, int T, const int* adj, const float* viewM,
                      const float* viewMlo,
                      const ViewSetupArgs& a, DevStatus* status, bool silhouettes, cudaStream_t st);
void launch_silhouettes_all(const int* adj, int T, const ViewSetupArgs& a, cudaStream_t st);
// The light views' matrices and derivatives (one CTA per light view), the
// C camera matrices after them, and in the same launch the vertex normals
// (vn.V vertices; none when vn.V = 0), which need neither.
void launch_light_setup(const float* params, const LightSetupArgs& a, LightDev* out, float* viewM, float* viewMlo,
                        const CamMats& cams, int C, const VertNormalArgs& vn, cudaStream_t st);
// Raster work units of one view.  A tile's list is rastered kRasterBatch
// records per unit (one CTA each); a tile of several units merges their
// per-pixel minimum keys in a key slot (global 64-bit maxima of the inverted
// keys, 0 = empty) and its last unit to finish writes the G-buffer, then
// empties the slot and its counter again.
constexpr int kRasterBatch = 1024;   // records per unit (four batches of 256)
struct RasterUnits {
  // per unit: tile, the list range of its records [begin, end) (-1, -1 for a
  // unit with nothing to do), and the tile's key slot + 1 (0: none) with the
  // tile's unit count << 20
  int4* units;
  int units_cap;               // tiles + list capacity / kRasterBatch + 1 (an upper bound)
  int slot_cap;                // list capacity / (kRasterBatch + 1) + 1 (an upper bound)
  int* tile_done;              // units finished per tile (zero between frames)
  unsigned long long* skey;    // slot_cap x 1024 inverted keys (zero between frames)
};
// Segment of every tile of one view in its triangle list (begin, end): the
// count pass's ordinary triangles, then the big triangles that may cover the
// tile.  With `write`, also appends those big triangles to the segments and
// hands out the raster work units and key slots; without it (a first frame,
// whose list capacity is sized from the segments' total first), only the
// segments and their total.
void launch_alloc_units(const int* count, int n, int* offset, DevStatus* status, int view, const TriSetup* setup,
                        const int* big_tri, int tilesX, int tile_log2, int* list, int capacity,
                        const RasterUnits& ru, bool write, cudaStream_t st);
// Fill pass: the ordinary triangles into their tiles' segments, by taking
// slots down from the count pass's per-tile counts (which end at zero).
void launch_bin_fill(const TriSetup* setup, int T, int tilesX, BinShape bs, int* counter, const int* offset,
                     int* list, int capacity, DevStatus* status, const int* big_index, cudaStream_t st);
// Raster work counts of one view into out[0..2] (added): tile-triangle pairs,
// spans, pixel-centre coverage tests.
void launch_raster_stats(const TriSetup* setup, const int* offset, const int* list, int capacity, int tilesX,
                         int tilesY, int tile_log2, unsigned long long* out, cudaStream_t st);
// Light views (fmap != NULL) also write the shadow-map depth sample (f, f^2)
// of every texel, f interpolated from the per-vertex light depths.  With
// hflag (the view's antialiasing on), also the antialiasing detection of the
// pixel pairs inside each tile (silbits: the view's packed silhouette flags):
// hflag at every pixel and the flagged pixels appended to aa; the tiles' rims
// go to rim.
void launch_raster(const TriSetup* setup, const int* list, int tilesX, int tile_log2, int W, int H,
                   const float4* clip, const float4* scr, const int* tris, float4* gbuf, const float* depth,
                   float2* fmap, float ec, const RasterUnits& ru, DevStatus* status, int view,
                   const uint32_t* silbits, uint8_t* hflag, const AAWork& aa, const RimBufs& rim, cudaStream_t st);

// shadow-map interpolation and antialiasing
// Antialiasing (detection + list passes, see aa.cu).
// The detection's pairs across the edges of the raster's tiles (after the
// raster of the view, which detects the pairs inside its tiles and leaves
// their rims in rim).
void launch_aa_seam(const AAArgs& a, int tilesX, int tilesY, int tile_log2, const RimBufs& rim,
                    const uint32_t* silbits, uint8_t* hflag, const AAWork& w, cudaStream_t st);
void launch_aa_forward2_list(const AAArgs& a, const float2* color, float2* out, const AAWork& w, cudaStream_t st);
void launch_aa_forward4_list(const AAArgs& a, const float4* color, float4* out, const AAWork& w, cudaStream_t st);
void launch_sm_aa_adjoint_list(const AAArgs& a, const float2* fmap, const float2* gft, float4* gclip, float* gf_out,
                               float ec, const AAWork& w, cudaStream_t st);
// dL/dcolour at the listed pixels (every other pixel's is dL/dimage itself).
void launch_aa_backward4_list(const AAArgs& a, const float4* color, const ImageGrad& gout, float4* gcolor,
                              float4* gclip, const AAWork& w, cudaStream_t st);
void launch_sm_interp_adjoint(const AAArgs& a, const float* gf, const float* depth, float4* gclip,
                              const BigArgs& big, cudaStream_t st);

// separable filter
// Whether (sigma, radius, kind, boundary) describe a filter: kind and boundary
// 0 or 1, radius <= 32, and a finite sigma > 0 for the Gaussian (kind 0) and
// whenever the radius is derived from sigma (radius <= 0).
bool filter_args_ok(float sigma, int radius, int kind, int boundary);
void make_filter_args(double sigma, int radius, int kind, int boundary, FilterArgs* fa);
// m = G g; with hflag (shadow-map path) g is (f, f^2) except at flagged texels,
// where the antialiasing pass left (f~, (f^2)~) in patch.
// The TMA-staged filter (filter_tma.cu); false when the map or the radius does
// not qualify (the caller then takes another shape).  A bounded wait that runs
// out sets status->timeout.
bool launch_filter_tma(bool adjoint, const float2* in, float2* out, int R, const FilterArgs& fa,
                       const FilterExtras& ex, DevStatus* status, cudaStream_t st);
// One CTA waiting on an mbarrier with the bounded wait of the TMA filter;
// without `arrive` nothing completes the phase and the wait records a timeout.
void launch_bounded_wait_probe(DevStatus* status, bool arrive, cudaStream_t st);
void launch_filter(const float2* in, float2* tmp, float2* out, int R, const FilterArgs& fa, cudaStream_t st,
                   const uint8_t* hflag = nullptr, const float2* patch = nullptr, DevStatus* status = nullptr);
// out = hflag ? patch : fmap per texel (the antialiased shadow map, materialised
// on request).
void launch_compose(const float2* fmap, const uint8_t* hflag, const float2* patch, float2* out, int n,
                    cudaStream_t st);
// gin = G^T gout; with gf (shadow-map path) also dL/df = gin.x + 2 f gin.y.
// With fmap and gf: also writes gf = dL/df of every texel from the result
// (moment_fold with the warp exponent ec).
void launch_filter_adjoint(const float2* gout, float2* tmp, float2* gin, int R, const FilterArgs& fa, cudaStream_t st,
                           const float2* fmap = nullptr, float* gf = nullptr, float ec = 0.f,
                           DevStatus* status = nullptr);

// normals, shading, vertex gradients
// dL/dv of the cameras' interpolation: the unit vertex normals' gradient
// gnormal through the normalisation and the area-weighted face normals, plus
// the positions' gradient gpos, added to dverts.
void launch_normals_backward(const float* verts, int V, const int* tris, int T, const int* vf_off,
                             const int* vf_list, const float* vnormal, const float* vlen, const float4* gnormal,
                             const float4* gpos, float* gN, float* gface, float* dverts, cudaStream_t st);
// Colour of every pixel (Alg. 2 x Lambert); with image, also the image at the
// pixels that hflag leaves unflagged (all of them for hflag NULL), whose
// antialiased value is their colour.
void launch_shade(const ShadeArgs& a, float4* color, float4* image, const uint8_t* hflag, cudaStream_t st);
void launch_shade_probe(const ShadeArgs& a, int l, float4* out, cudaStream_t st);
void launch_sm_band_mask(const uint8_t* hflag, int n, float2* gft, float* gf, cudaStream_t st);
// The shading adjoint in two passes that may run side by side: the grid pass
// over every pixel that the final antialiasing did not list (and the squared
// error of every pixel), and the pass over the listed pixels, after the
// antialiasing adjoint wrote their dL/dcolour.  Without the final
// antialiasing (g.hflag NULL) the grid pass takes every pixel.
void launch_shade_backward(const ShadeArgs& a, const ShadeGradArgs& g, cudaStream_t st);
void launch_shade_backward_listed(const ShadeArgs& a, const ShadeGradArgs& g, const AAWork& w, cudaStream_t st);
void launch_shade_scatter(const ShadeArgs& a, const ShadeGradArgs& g, cudaStream_t st);
void launch_vertex_backward(const float* verts, int V, const float* viewM, int n_views, int n_lights,
                            const VertGradPtrs& gp, float* dverts, double* red, int red_stride, cudaStream_t st);
void launch_shade_big_resolve(const ShadeArgs& a, const ShadeGradArgs& g, const int* big_tri,
                              const DevStatus* status, int view, cudaStream_t st);
// With loss (the mean squared error of a backward against a target): also
// the loss, the block sums' squared error over the n_img floats of the image.
void launch_light_sums(const double* red, int red_stride, int L, int n_mat_red, const LightDev* lights, int n_user,
                       double* gQ, double* gdirect, float* dalbedo, float* dlight, float* loss, int64_t n_img,
                       cudaStream_t st);
void launch_l2(const float* img, const float* tgt, int64_t n, float* loss, float* grad, cudaStream_t st);

}  // namespace dsm
