/*
 * dsm.h -- C ABI of the differentiable variance-shadow-mapping library (sm_103a).
 *
 * Method: Worchel & Alexa, "Differentiable Shadow Mapping for Efficient Inverse
 * Graphics" (CVPR 2023).  Per light, Alg. 1 renders the light-view depth map f
 * (Eq. 1), smooths f and f^2 by edge antialiasing (Sec. 4/5) and filters them
 * into the moment maps m1 = G f~, m2 = G (f^2)~ (Eqs. moment1, moment2).  The
 * camera pass shades every pixel with Lambert times the visibility of Alg. 2
 * (Chebyshev bound of Sec. 3) per light, and the image is antialiased again.
 * The backward pass returns dL/d vertices, dL/d light (position, direction) and
 * dL/d albedo (Sec. 4: chain rule through G, the moments and the visibility).
 *
 * Conventions shared by every call
 *  - Matrices are row-major 4x4 float: clip = M [x y z 1]^T.
 *  - Screen: sx = (0.5 ndc_x + 0.5) W, sy = (0.5 - 0.5 ndc_y) H, row 0 at the top.
 *    Pixel (i, j) is column i, row j; its centre is (i + 0.5, j + 0.5).
 *  - Images and maps are row-major, pixel (i, j) at index j * W + i.
 *  - All pointers named "device" are CUDA device pointers on the current device;
 *    the caller owns them.  The context owns its scratch memory and the state
 *    saved by dsm_render for dsm_render_backward; that state stays valid until
 *    the next dsm_render on the same context.
 *  - Every call enqueues work on params->stream (the stream given to the last
 *    dsm_render for dsm_render_backward) and returns without waiting, except
 *    where stated.  Errors found on the device are reported by dsm_sync.
 *  - Nothing throws across this boundary; every call returns a dsm_status and
 *    dsm_last_error() gives a one-line description of the last failure.
 */
#ifndef DSM_H
#define DSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSM_MAX_LIGHTS 8         /* lights per call                                     */
#define DSM_MAX_LIGHT_VIEWS 24   /* shadow-map views of those lights: one per directional
                                    or spot light, six per point light (cube map)        */
#define DSM_MAX_CAMERAS 8

typedef enum dsm_status {
  DSM_OK = 0,
  DSM_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range          */
  DSM_ERR_CAPACITY = 2,      /* an internal list overflowed; the result is invalid     */
  DSM_ERR_CUDA = 3,          /* a CUDA runtime call failed                             */
  DSM_ERR_TIMEOUT = 4,       /* a bounded device wait gave up                          */
  DSM_ERR_NO_FORWARD = 5,    /* backward called without a matching forward             */
  DSM_ERR_OOM = 6,           /* device allocation failed                               */
  DSM_ERR_NO_TOPOLOGY = 7    /* dsm_set_topology was not called for this mesh          */
} dsm_status;

typedef struct dsm_ctx dsm_ctx;   /* opaque */

/* Triangle mesh.  verts: device, n_verts x 3 float, world space.  tris: device,
 * n_tris x 3 int32 vertex indices.  tri_material: device, n_tris int32 indices
 * into albedo (NULL: material 0 everywhere).  albedo: device, n_materials x 3
 * float Lambert albedo (supplementary Sec. A). */
typedef struct dsm_mesh {
  const float*   verts;
  int32_t        n_verts;
  const int32_t* tris;
  int32_t        n_tris;
  const int32_t* tri_material;
  const float*   albedo;
  int32_t        n_materials;
} dsm_mesh;

/* Constant description of one light (supplementary Sec. A).  The differentiable
 * light parameters are NOT here: they are passed as a device array
 * light_params[l * 6 + 0..2] = position, [l * 6 + 3..5] = direction of travel.
 *  type 0, directional: orthographic shadow camera at -dist * normalize(dir),
 *          looking along dir, window +-ortho_half;
 *  type 1, spot: perspective shadow camera at the position looking along dir,
 *          full vertical field of view fov_y_deg;
 *  type 2, point (omnidirectional, Sec. 3: several shadow-map planes arranged
 *          as a box): a cube map of six perspective faces at the position,
 *          90-degree field of view, looking along +X, -X, +Y, -Y, +Z, -Z
 *          (light views in that order), res x res texels each; dir and
 *          fov_y_deg are unused (zero direction gradient).  Each face is
 *          antialiased and filtered on its own (the filter boundary applies
 *          at the face edges) and a point x is shaded by the face of the
 *          largest component of x - position (ties: x, then y).
 * The map stores the normalised depth d = (z_view - near) / (far - near), with
 * z_view the distance along normalize(dir) (along the face axis for a cube
 * face; Sec. 3: distance from a plane for a directional light).  Up vector +Y,
 * or +Z when |dir_y| > 0.99 |dir|. */
typedef struct dsm_light {
  int32_t type;
  int32_t res;            /* shadow-map side in texels, 1..16384                   */
  float   fov_y_deg;      /* spot only                                             */
  float   ortho_half;     /* directional only                                      */
  float   dist;           /* directional only                                      */
  float   near_plane;
  float   far_plane;
  float   intensity[3];
  float   sigma;          /* Gaussian filter sigma in texels                       */
  int32_t radius;         /* filter radius r (kernel size k = 2r + 1); <= 0: ceil(2 sigma) */
} dsm_light;

/* Camera: row-major world -> clip matrix (OpenGL-style: ndc z grows with depth)
 * and the image size. */
typedef struct dsm_camera {
  float   clip[16];
  int32_t width;
  int32_t height;
} dsm_camera;

typedef struct dsm_params {
  float   min_variance;     /* floor of sigma^2 in the Chebyshev bound (normalised depth^2) */
  int32_t filter_kind;      /* 0 Gaussian, 1 box (kernel size 2r + 1)                        */
  int32_t filter_boundary;  /* 0 clamp to edge, 1 zero outside                              */
  int32_t aa_shadow;        /* 1: antialias (f, f^2) before filtering (Sec. 5 ablation: 0)  */
  int32_t aa_final;         /* 1: antialias the shaded image                                */
  int32_t recompute_in_backward; /* 0: keep every view's buffers from forward to backward;
                                   * 1: views share one light and one camera buffer set and
                                   * the backward rebuilds what it reads (see dsm_render_cameras) */
  int32_t moments;          /* pre-filtered moment family: 0 variance shadow maps (f, f^2);
                             * 1 exponential variance shadow maps (w, w^2), w = exp(c f):
                             * the same antialiasing and filter, the Chebyshev bound on the
                             * warped depth exp(c d) with the floor min_variance (c exp(c d))^2
                             * (less light bleeding where occluder depths vary)          */
  float   exponent;         /* c of moments = 1, in (0, 40] (w^2 stays finite in float32)   */
  void*   stream;           /* cudaStream_t; NULL = legacy default stream                   */
} dsm_params;

/* Create / destroy a context bound to the current CUDA device.  dsm_create
 * returns DSM_ERR_CUDA when no device is usable. */
dsm_status dsm_create(dsm_ctx** out);
void       dsm_destroy(dsm_ctx* ctx);

/* Mesh topology (edge adjacency for the silhouette test of the antialiasing,
 * vertex -> face lists for the vertex normals).  tris: device, n_tris x 3.
 * Synchronous: copies tris to the host and builds the tables there.  Call once
 * per topology, before dsm_render; it may allocate. */
dsm_status dsm_set_topology(dsm_ctx* ctx, const int32_t* tris, int32_t n_tris, int32_t n_verts);

/* Forward pass (Alg. 1 per light, Alg. 2 + Lambert per camera pixel, final
 * antialiasing).  light_params: device, n_lights x 6 float (see dsm_light).
 * image: device, height x width x 4 float, RGB and coverage alpha, overwritten.
 * Synchronises once with the stream on the first call for a new scene size (to
 * size the tile lists); later calls do not wait. */
dsm_status dsm_render(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights,
                      const float* light_params, int32_t n_lights,
                      const dsm_camera* camera, const dsm_params* params, float* image);

/* Backward pass of the last dsm_render on ctx.  dL_dimage: device, H x W x 4.
 * Outputs (device, overwritten, any may be NULL to skip): dL_dverts n_verts x 3,
 * dL_dlight n_lights x 6 (position, direction; zero position gradient for
 * directional lights), dL_dalbedo n_materials x 3.  The mesh, light and
 * albedo buffers of that dsm_render must still hold the same values.
 * DSM_ERR_INVALID_ARG when the last forward had several cameras. */
dsm_status dsm_render_backward(dsm_ctx* ctx, const float* dL_dimage, float* dL_dverts,
                               float* dL_dlight, float* dL_dalbedo);

/* Backward pass of the last dsm_render on ctx for the mean squared error
 * L = sum (image - target)^2 / n over the n = H x W x 4 floats of its image
 * (the loss of dsm_l2_loss_grad): the same gradients as dsm_l2_loss_grad
 * followed by dsm_render_backward with its dL/dimage, whose arithmetic it
 * uses (dL/dimage = 2 / n (image - target), 2 / n rounded to float), without
 * writing dL/dimage; the kernels that read dL/dimage form it from image and
 * target.  image: device, the image that dsm_render wrote (unchanged since);
 * target: device, H x W x 4; loss: device, one float, overwritten with L (the
 * squared errors summed in float64 over per-block float sums, so it agrees
 * with dsm_l2_loss_grad's float sum to rounding).  Outputs as in
 * dsm_render_backward.  DSM_ERR_INVALID_ARG when image, target or loss is
 * NULL or the last forward had several cameras. */
dsm_status dsm_render_backward_l2(dsm_ctx* ctx, const float* image, const float* target, float* loss,
                                  float* dL_dverts, float* dL_dlight, float* dL_dalbedo);

/* Forward pass seen by n_cameras cameras (1..DSM_MAX_CAMERAS) under the same
 * lights: each light's moment maps (Alg. 1) are built once and every camera
 * is shaded with all of them (Alg. 2 + Lambert, final antialiasing).
 * cameras: host array of n_cameras; images: host array of n_cameras device
 * pointers, image c height_c x width_c x 4 (as in dsm_render).  dsm_render is
 * this call with one camera; the result of camera c equals a dsm_render with
 * camera c alone.
 * With params->recompute_in_backward = 1 the views go one at a time through
 * one light buffer set and one camera buffer set (device memory of one light
 * view and one camera view instead of all of them, plus every light's moment
 * maps); the backward then rasterises every view again and filters the
 * moment maps again instead of reading stored ones.  Results are the same in
 * both modes; with recomputation the debug copies of per-view buffers are
 * unavailable. */
dsm_status dsm_render_cameras(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights,
                              const float* light_params, int32_t n_lights,
                              const dsm_camera* cameras, int32_t n_cameras,
                              const dsm_params* params, float* const* images);

/* Backward pass of the last dsm_render_cameras (or dsm_render) on ctx for the
 * loss summed over the cameras.  dL_dimages: host array of that call's
 * n_cameras device pointers, each height_c x width_c x 4.  Outputs as in
 * dsm_render_backward (gradients summed over the cameras). */
dsm_status dsm_render_cameras_backward(dsm_ctx* ctx, const float* const* dL_dimages,
                                       float* dL_dverts, float* dL_dlight, float* dL_dalbedo);

/* Device memory held by ctx (its scratch and saved state), in bytes. */
uint64_t dsm_memory_bytes(dsm_ctx* ctx);

/* Integer work of the raster of view `view` (lights' views first, then the
 * cameras, as in dsm_render_cameras) in the last forward on ctx, counted from
 * the tile lists and setup records that raster read (Eq. 1's coverage test):
 * out[0] tile-triangle pairs, out[1] spans of 4 pixels of one row (the raster's
 * work items), out[2] pixel-centre coverage tests (three edge-function steps
 * each), and out[3] the pixels on the view's antialiasing work list (those
 * with a neighbour pair whose nearer triangle has a silhouette edge; 0 when
 * that view's antialiasing is off).  out: host array of 4.  A diagnostic:
 * launches one kernel on the last
 * forward's stream and synchronises it.  DSM_ERR_NO_FORWARD without a forward;
 * DSM_ERR_INVALID_ARG for a view out of range or a recomputing context (its
 * views share one buffer set). */
dsm_status dsm_raster_stats(dsm_ctx* ctx, int32_t view, int64_t* out);

/* ---- Kernel shapes of a context.  The results do not depend on them (the
 * raster is exact and order independent; the filter is the same sums), only
 * the speed does.  Defaults: 32, 32, 16, 0. */
typedef struct dsm_tuning {
  int32_t light_tile;    /* raster tile side of the light views, pixels: 16 or 32                 */
  int32_t camera_tile;   /* raster tile side of the camera views: 16 or 32                        */
  int32_t big_tiles;     /* bin depth: a triangle whose bbox spans at least this many tiles is
                            "big" (the first 64 of a view): binned per tile, each tile testing
                            the view's big triangles, and its backward sums go to private
                            copies; 2..4096                                                       */
  int32_t filter_shape;  /* 0: input tiles staged by the TMA in a persistent double-buffered kernel
                            (radius <= 8, map side a multiple of 16, no antialiased patch to
                            substitute; otherwise shape 2); 1: two 1-D passes; 2: both passes
                            in one kernel on 32x32 output tiles with plain loads (radius <= 15,
                            larger radii take two passes)                                       */
} dsm_tuning;

/* Set / read the shapes used by the next calls on ctx.  DSM_ERR_INVALID_ARG
 * for a value out of range. */
dsm_status dsm_set_tuning(dsm_ctx* ctx, const dsm_tuning* tuning);
dsm_status dsm_get_tuning(dsm_ctx* ctx, dsm_tuning* tuning);

/* Autotuner: times forward + backward steps of the given frame (arguments as
 * in dsm_render_cameras; the images double as dL/dimage of the timed
 * backward, whose gradients go to context scratch) for candidate shapes and
 * keeps the fastest on ctx.  Coordinate search from the current shapes: each
 * knob in turn (light tile, camera tile, bin depth from {4, 16, 64}, filter
 * shape from {0, 1, 2}) is set to each of its other values and kept when the step gets
 * faster; each candidate runs one untimed step (sizing) and `reps` timed
 * steps (1..100) with CUDA events on params->stream.  Synchronous.  best and
 * best_ms (host, may be NULL) receive the chosen shapes and their time per
 * step in milliseconds.  The state of the last forward is that of the last
 * candidate: render again before a backward. */
dsm_status dsm_autotune(dsm_ctx* ctx, const dsm_mesh* mesh, const dsm_light* lights,
                        const float* light_params, int32_t n_lights,
                        const dsm_camera* cameras, int32_t n_cameras, const dsm_params* params,
                        float* const* images, int32_t reps, dsm_tuning* best, float* best_ms);

/* One Adam step (Kingma & Ba 2015, Algorithm 1) in place, for optimising the
 * vertices (or any float parameters) with the gradients of the backward pass;
 * the paper optimises its scene parameters with Adam.  params, m, v: device,
 * n floats, read and overwritten (m, v start at zero before step 1); grads:
 * device, n floats; step: 1-based step count t (bias corrections 1 - beta^t).
 * params -= lr * m^ / (sqrt(v^) + eps) with m^ = m / (1 - beta1^t),
 * v^ = v / (1 - beta2^t).  DSM_ERR_INVALID_ARG for a bad argument (beta outside
 * [0, 1), eps <= 0, step < 1).  stream: cudaStream_t. */
dsm_status dsm_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int32_t step,
                         float lr, float beta1, float beta2, float eps, void* stream);

/* L = mean((image - target)^2) over n floats and dL/dimage = 2 (image - target) / n.
 * image, target, dL_dimage: device, n floats; loss: device, one float (overwritten).
 * stream: cudaStream_t. */
dsm_status dsm_l2_loss_grad(const float* image, const float* target, int64_t n,
                            float* loss, float* dL_dimage, void* stream);

/* Separable filter of a two-channel map (Eqs. moment1/moment2: m = G g), the
 * same arithmetic as inside dsm_render: G filters along x, then along y, with
 * 2 radius + 1 normalised taps.  in, out: device, res x res float2 (row-major,
 * 8-byte aligned), caller-owned, must not overlap.  sigma: Gaussian standard
 * deviation in texels (kind 0); radius: taps on each side, 0 = ceil(2 sigma),
 * at most 32; kind: 0 Gaussian, 1 box (equal taps); boundary: 0 clamp to the
 * edge texel, 1 zero outside the map.  Radii up to 15 take one tiled kernel;
 * larger radii take two 1-D passes through ctx scratch (may allocate).
 * DSM_ERR_INVALID_ARG for bad arguments: kind or boundary not 0 or 1, radius
 * above 32, or no finite sigma > 0 where one is needed (always for the
 * Gaussian, and for the box when radius <= 0).  DSM_ERR_CUDA on a launch error.
 * stream: cudaStream_t (NULL = legacy default stream). */
dsm_status dsm_filter_moments(dsm_ctx* ctx, const float* in, float* out, int32_t res,
                              float sigma, int32_t radius, int32_t kind, int32_t boundary,
                              void* stream);

/* Transpose of dsm_filter_moments for the same arguments: gin = G^T gout
 * (Sec. 4: the gradient with respect to the filtered moments is carried back
 * to the unfiltered texels; for the clamp boundary the weight of the taps that
 * G clamped onto an edge texel returns to that texel).  gout, gin: device,
 * res x res float2, caller-owned, must not overlap.  Same errors and scratch
 * rule as dsm_filter_moments. */
dsm_status dsm_filter_moments_adjoint(dsm_ctx* ctx, const float* gout, float* gin, int32_t res,
                                      float sigma, int32_t radius, int32_t kind, int32_t boundary,
                                      void* stream);

/* Allocation-free variant of dsm_filter_moments.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory while
 * they run, such as a real-time loop that works inside a fixed, preallocated
 * memory budget, or a host application that owns the device memory pool and
 * lets no other allocator touch the device.  (dsm_filter_moments may grow its
 * context's scratch with cudaMalloc.)  It computes the same separable filter
 * with the same result as dsm_filter_moments for the same arguments.
 * in, out: device, res x res float2, must not overlap; the caller owns both.
 * No call allocates or frees memory.  Radii up to 15 run as one tiled kernel
 * with no intermediate map.  Radii 16 to 32 run as two 1-D passes whose
 * intermediate map lives in a static device array of the library (1024 x 1024
 * texels, 8 MiB, held by every GPU that loads the library until the process
 * exits).  The first call on a device looks up that array's device address
 * and caches it; make that first call before any stream capture on the
 * device, and do not use the library on a device again after cudaDeviceReset.
 * For radii 16 to 32 every call shares the array: such calls whose work
 * overlaps on the GPU (two streams, or two threads) race on it, so serialise
 * them.  Returns DSM_ERR_CAPACITY when res * res exceeds 1024 * 1024,
 * DSM_ERR_INVALID_ARG for other bad arguments (the rules of
 * dsm_filter_moments), DSM_ERR_CUDA when the device lookup or the launch
 * fails.  stream: cudaStream_t (NULL = legacy default stream). */
dsm_status dsm_filter_moments_noalloc(const float* in, float* out, int32_t res, float sigma,
                                      int32_t radius, int32_t kind, int32_t boundary, void* stream);

/* ---- Batched frames.  n independent scenes (each a mesh, lights, a camera and
 * an L2 target) advanced by one call per step: forward, L2 loss and backward
 * of every scene.  The paper renders one view at a time and has no batch
 * call; per scene the step is exactly dsm_render and dsm_render_backward_l2
 * (the gradients of dsm_l2_loss_grad followed by dsm_render_backward).
 *
 * Each scene has its own context (dsm_batch_context: set its topology there
 * before the first step; its debug copies work as usual) and its own stream,
 * its views on the context's own streams forked from it; the scenes, and the
 * views within each scene, overlap.  The
 * first step with a given set of items and params runs eagerly (it sizes
 * every context; this is the only step with host synchronisation) and then
 * records the same step into one CUDA graph; a later step whose items
 * (pointers, sizes, light and camera descriptions) and params are unchanged
 * replays that graph with one launch.  The contents of the device buffers
 * (vertices, light parameters, albedo, targets) may change between steps.
 * One params serves every scene; params->stream must not be the legacy
 * default stream (graph capture).  With params->recompute_in_backward = 1
 * each scene's context holds one light and one camera buffer set (see
 * dsm_render_cameras). */
typedef struct dsm_batch dsm_batch;
typedef struct dsm_batch_item {
  dsm_mesh          mesh;
  const dsm_light*  lights;        /* host, n_lights (read at every step)          */
  const float*      light_params;  /* device, n_lights x 6 (see dsm_render)        */
  int32_t           n_lights;
  dsm_camera        camera;
  float*            image;         /* device, H x W x 4, written                   */
  const float*      target;        /* device, H x W x 4                             */
  float*            loss;          /* device, 1 float, written                      */
  float*            dL_dimage;     /* unused (the loss backward forms dL/dimage where
                                      it reads it); may be NULL                       */
  float*            dL_dverts;     /* device, n_verts x 3, written (NULL: skipped)  */
  float*            dL_dlight;     /* device, n_lights x 6, written (NULL: skipped) */
  float*            dL_dalbedo;    /* device, n_materials x 3, written (NULL: skip) */
  /* Optional host staging, pinned host memory (cudaHostAlloc / registered),
   * NULL to skip each.  The step first copies host_verts into mesh.verts,
   * host_light_params into light_params and host_albedo into mesh.albedo
   * (the same sizes; those device buffers are overwritten), and ends by
   * copying the loss into host_loss (1 float), all inside the recorded step:
   * a host loop then needs only dsm_batch_step and a stream synchronisation. */
  const void*       host_verts;
  const void*       host_light_params;
  const void*       host_albedo;
  void*             host_loss;
} dsm_batch_item;

/* Create a batch for up to n scenes (n contexts and streams); destroy frees
 * them all.  DSM_ERR_CUDA / DSM_ERR_OOM when the device objects cannot be made. */
dsm_status dsm_batch_create(dsm_batch** out, int32_t n);
void       dsm_batch_destroy(dsm_batch* b);
/* The context of scene i (owned by the batch), NULL when i is out of range. */
dsm_ctx*   dsm_batch_context(dsm_batch* b, int32_t i);
/* One step of scenes 0..n-1 (n <= the batch size).  Asynchronous on
 * params->stream except for the eager first step.  Errors: DSM_ERR_INVALID_ARG
 * for bad items, a scene's own error (dsm_batch_last_error names the scene),
 * DSM_ERR_CUDA for stream, capture or graph failures. */
dsm_status dsm_batch_step(dsm_batch* b, const dsm_batch_item* items, int32_t n, const dsm_params* params);
/* dsm_sync of every scene's context. */
dsm_status dsm_batch_sync(dsm_batch* b);
/* Kernels one recorded step launches (counted while recording). */
uint64_t   dsm_batch_kernels_per_step(dsm_batch* b);
/* Autotuner of the batch: the same coordinate search as dsm_autotune over
 * shapes shared by every scene, each candidate timed as whole batched steps
 * (an eager step that records the graph and one replay untimed, then `reps`
 * timed replays on params->stream), since the scenes overlap one another in a
 * step.  Synchronous; leaves the fastest shapes on every scene's context and
 * its graph recorded. */
dsm_status dsm_batch_autotune(dsm_batch* b, const dsm_batch_item* items, int32_t n, const dsm_params* params,
                              int32_t reps);
const char* dsm_batch_last_error(dsm_batch* b);

/* Wait for the context's stream and report device-side errors (capacity
 * overflow, timeouts) raised since the last dsm_sync. */
dsm_status dsm_sync(dsm_ctx* ctx);

/* Check of the failure path of the bounded device waits (the TMA-staged
 * filter waits on mbarriers with an iteration limit): one CTA on the
 * context's stream waits on an mbarrier.  With arrive = 1 a thread completes
 * the phase and the wait ends; with arrive = 0 nothing completes it, the wait
 * gives up after a short limit and records a timeout, which the next dsm_sync
 * reports as DSM_ERR_TIMEOUT.  No fault is raised and the context stays
 * usable.  DSM_ERR_CUDA on a launch error. */
dsm_status dsm_bounded_wait_probe(dsm_ctx* ctx, int32_t arrive);

/* One-line description of the last error on ctx (static storage, never NULL). */
const char* dsm_last_error(dsm_ctx* ctx);

/* Copy an internal buffer of the last dsm_render / dsm_render_backward into a
 * caller device buffer (stage-wise testing and profiling).  what:
 *  0 G-buffer of view index (lights 0..n-1, then cameras n..): per pixel int32 id+1
 *    (0 = background), float b0, float b1, float depth key; 16 B per pixel
 *  1 f, f^2 before antialiasing (light index), float2 per texel
 *  2 f~, (f^2)~ after antialiasing (light), float2
 *  3 m1, m2 moment maps (light), float2
 *  4 colour of camera index (0..n_cameras-1) before the final antialiasing, float4
 *  5 light matrices Q (20 floats per light: clip rows 0-3, depth row 4)
 *  6 snapped vertices of view index: int32 X, Y (24.8 fixed point), float ndc z,
 *    int32 valid; 16 B per vertex
 *  7 dL/d(m1, m2) texel gradients (light), float2
 *  8 dL/d clip coordinates of view index, float4 per vertex (light views: the
 *    z slot holds dL/d vertex depth d, since clip z carries no gradient there)
 *  9 dL/d(f~, (f^2)~) (light), float2
 * 10 dL/d colour of camera index before the final antialiasing, float4 per pixel,
 *    at the pixels on the final antialiasing's work list (every other pixel's
 *    dL/d colour is its dL/d image, which the shading adjoint reads directly;
 *    the buffer holds no defined value there)
 * 11 shading-stage surface of camera index (Alg. 2 inputs, recomputed by the
 *    shading kernel's own device functions): two float4 per pixel,
 *    (x, y, z, 0) world position and (nx, ny, nz, 0) unit normal
 * 12 shading-stage lookup of camera index / 64 in light view index % 64:
 *    two float4 per pixel, (u, v, s, t) light-space position and texel
 *    coordinates, (dw, m1, m2, vis) receiver depth in the moments' encoding,
 *    bilinear moments and visibility (Alg. 2, Sec. 3)
 *    11, 12: NaN where the pixel has no such value (background, a cube face
 *    that does not shade the point, (u, v) behind the light, (s, t, m1, m2)
 *    outside its window)
 * bytes must equal the buffer size; returns DSM_ERR_INVALID_ARG otherwise.
 * After a forward with recompute_in_backward = 1 only 3, 5 and 7 are kept. */
dsm_status dsm_debug_copy(dsm_ctx* ctx, int32_t what, int32_t index, void* dst, size_t bytes);

/* Diagnostic gradient masks for comparisons that judge gradients away from
 * silhouettes (the paper's edge antialiasing, Sec. 5, acts only there).
 * flags: 0 (default) or DSM_GRAD_MASK_SM_BAND: every later dsm_render_backward
 * on ctx zeroes dL/d(f~, (f^2)~) at the shadow maps' silhouette-band texels,
 * so no gradient flows from them.  The band: texels with a 4-neighbour of
 * another triangle id (background included) such that the nearer surface of
 * the pair (by depth key, ties to the lower id; the background never is) is a
 * triangle with a silhouette edge in that view.  Every antialiasing crossing
 * lies in it.  Only with params.aa_shadow = 1 (without antialiasing there is
 * no band to mask).  DSM_ERR_INVALID_ARG for unknown flags. */
#define DSM_GRAD_MASK_SM_BAND 1
dsm_status dsm_set_grad_mask(dsm_ctx* ctx, int32_t flags);

/* Per-stage device timing: while enabled, dsm_render and dsm_render_backward
 * run every view on the caller's stream (instead of one internal stream per
 * view) and record a CUDA event pair around every stage of every view (stage
 * names: dsm_profile_stage_name).  dsm_profile_read waits for the recorded
 * events, writes the accumulated milliseconds and the number of timed calls of
 * each of the first n stages (ms, calls: host arrays of n entries) and clears
 * the records. */
dsm_status  dsm_profile_enable(dsm_ctx* ctx, int32_t enable);
int32_t     dsm_profile_stage_count(void);
const char* dsm_profile_stage_name(int32_t stage);   /* NULL when out of range */
dsm_status  dsm_profile_read(dsm_ctx* ctx, double* ms, int64_t* calls, int32_t n);

/* Number of kernels this library has launched in this process (all contexts). */
uint64_t dsm_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DSM_H */
