"""Thin Python binding of the C ABI in ``include/dsm.h`` (ctypes).

Argument marshalling only: every step of the shadow-mapping path runs in the
CUDA kernels of ``libdsm.so``.  Torch provides device memory and streams.  The
library must be built (``python -m paper_2308_10896_b300.build``); there is no
fallback when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsm.so")

DSM_OK, DSM_ERR_INVALID_ARG, DSM_ERR_CAPACITY, DSM_ERR_CUDA, DSM_ERR_TIMEOUT, DSM_ERR_NO_FORWARD, DSM_ERR_OOM, \
    DSM_ERR_NO_TOPOLOGY = range(8)
MAX_LIGHTS = 8
MAX_CAMERAS = 8

# debug_copy buffer codes (see include/dsm.h)
DBG_GBUF, DBG_F, DBG_FTILDE, DBG_MOMENTS, DBG_COLOR, DBG_Q, DBG_SNAP, DBG_GM, DBG_GCLIP, DBG_GFT, DBG_GCOLOR, \
    DBG_SURF, DBG_LOOKUP = range(13)
GRAD_MASK_SM_BAND = 1

EXPORTED = ["dsm_create", "dsm_destroy", "dsm_set_topology", "dsm_render", "dsm_render_backward",
            "dsm_l2_loss_grad", "dsm_filter_moments", "dsm_sync", "dsm_last_error", "dsm_debug_copy",
            "dsm_profile_enable", "dsm_profile_stage_count", "dsm_profile_stage_name", "dsm_profile_read",
            "dsm_kernel_launches", "dsm_filter_moments_noalloc", "dsm_filter_moments_adjoint",
            "dsm_batch_create", "dsm_batch_destroy", "dsm_batch_context", "dsm_batch_step", "dsm_batch_sync",
            "dsm_batch_kernels_per_step", "dsm_batch_last_error", "dsm_render_cameras",
            "dsm_render_cameras_backward", "dsm_memory_bytes", "dsm_adam_step", "dsm_set_tuning",
            "dsm_get_tuning", "dsm_autotune", "dsm_batch_autotune", "dsm_bounded_wait_probe",
            "dsm_raster_stats", "dsm_set_grad_mask", "dsm_render_backward_l2"]


class DsmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dsm status {status}: {msg}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int32), ("tris", ctypes.c_void_p),
                ("n_tris", ctypes.c_int32), ("tri_material", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("n_materials", ctypes.c_int32)]


class Light(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("res", ctypes.c_int32), ("fov_y_deg", ctypes.c_float),
                ("ortho_half", ctypes.c_float), ("dist", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("far_plane", ctypes.c_float), ("intensity", ctypes.c_float * 3), ("sigma", ctypes.c_float),
                ("radius", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("clip", ctypes.c_float * 16), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("min_variance", ctypes.c_float), ("filter_kind", ctypes.c_int32),
                ("filter_boundary", ctypes.c_int32), ("aa_shadow", ctypes.c_int32), ("aa_final", ctypes.c_int32),
                ("recompute_in_backward", ctypes.c_int32), ("moments", ctypes.c_int32), ("exponent", ctypes.c_float),
                ("stream", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("light_tile", ctypes.c_int32), ("camera_tile", ctypes.c_int32), ("big_tiles", ctypes.c_int32),
                ("filter_shape", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("mesh", Mesh), ("lights", ctypes.c_void_p), ("light_params", ctypes.c_void_p),
                ("n_lights", ctypes.c_int32), ("camera", Camera), ("image", ctypes.c_void_p),
                ("target", ctypes.c_void_p), ("loss", ctypes.c_void_p), ("dL_dimage", ctypes.c_void_p),
                ("dL_dverts", ctypes.c_void_p), ("dL_dlight", ctypes.c_void_p), ("dL_dalbedo", ctypes.c_void_p),
                ("host_verts", ctypes.c_void_p), ("host_light_params", ctypes.c_void_p),
                ("host_albedo", ctypes.c_void_p), ("host_loss", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdsm.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2308_10896_b300.build`")
    lib = ctypes.CDLL(path)
    P, I32, I64, S = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "dsm_create": ([ctypes.POINTER(P)], I32),
        "dsm_destroy": ([P], None),
        "dsm_set_topology": ([P, P, I32, I32], I32),
        "dsm_render": ([P, ctypes.POINTER(Mesh), ctypes.POINTER(Light), P, I32, ctypes.POINTER(Camera),
                        ctypes.POINTER(Params), P], I32),
        "dsm_render_backward": ([P, P, P, P, P], I32),
        "dsm_render_backward_l2": ([P, P, P, P, P, P, P], I32),
        "dsm_l2_loss_grad": ([P, P, I64, P, P, P], I32),
        "dsm_filter_moments": ([P, P, P, I32, ctypes.c_float, I32, I32, I32, P], I32),
        "dsm_sync": ([P], I32),
        "dsm_last_error": ([P], ctypes.c_char_p),
        "dsm_debug_copy": ([P, I32, I32, P, S], I32),
        "dsm_profile_enable": ([P, I32], I32),
        "dsm_profile_stage_count": ([], I32),
        "dsm_profile_stage_name": ([I32], ctypes.c_char_p),
        "dsm_profile_read": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), I32], I32),
        "dsm_kernel_launches": ([], ctypes.c_uint64),
        "dsm_filter_moments_noalloc": ([P, P, I32, ctypes.c_float, I32, I32, I32, P], I32),
        "dsm_filter_moments_adjoint": ([P, P, P, I32, ctypes.c_float, I32, I32, I32, P], I32),
        "dsm_batch_create": ([ctypes.POINTER(P), I32], I32),
        "dsm_batch_destroy": ([P], None),
        "dsm_batch_context": ([P, I32], P),
        "dsm_batch_step": ([P, P, I32, P], I32),
        "dsm_batch_sync": ([P], I32),
        "dsm_batch_kernels_per_step": ([P], ctypes.c_uint64),
        "dsm_batch_last_error": ([P], ctypes.c_char_p),
        "dsm_render_cameras": ([P, ctypes.POINTER(Mesh), ctypes.POINTER(Light), P, I32, ctypes.POINTER(Camera), I32,
                                ctypes.POINTER(Params), ctypes.POINTER(P)], I32),
        "dsm_render_cameras_backward": ([P, ctypes.POINTER(P), P, P, P], I32),
        "dsm_memory_bytes": ([P], ctypes.c_uint64),
        "dsm_raster_stats": ([P, I32, P], I32),
        "dsm_set_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "dsm_get_tuning": ([P, ctypes.POINTER(Tuning)], I32),
        "dsm_autotune": ([P, ctypes.POINTER(Mesh), ctypes.POINTER(Light), P, I32, ctypes.POINTER(Camera), I32,
                          ctypes.POINTER(Params), ctypes.POINTER(P), I32, ctypes.POINTER(Tuning),
                          ctypes.POINTER(ctypes.c_float)], I32),
        "dsm_batch_autotune": ([P, P, I32, P, I32], I32),
        "dsm_bounded_wait_probe": ([P, I32], I32),
        "dsm_set_grad_mask": ([P, I32], I32),
        "dsm_adam_step": ([P, P, P, P, I64, I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, P],
                          I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def light_struct(d: dict) -> Light:
    L = Light()
    L.type = int(d["type"])
    L.res = int(d["res"])
    L.fov_y_deg = float(d.get("fov_y_deg", 0.0))
    L.ortho_half = float(d.get("ortho_half", 0.0))
    L.dist = float(d.get("dist", 0.0))
    L.near_plane = float(d["near"])
    L.far_plane = float(d["far"])
    for k in range(3):
        L.intensity[k] = float(d["intensity"][k])
    L.sigma = float(d["sigma"])
    L.radius = int(d.get("radius", 0))
    return L


def camera_struct(cam: dict) -> Camera:
    c = Camera()
    m = np.asarray(cam["clip"], np.float32).reshape(-1)
    for k in range(16):
        c.clip[k] = float(m[k])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def params_struct(p: dict, stream=None) -> Params:
    q = Params()
    q.min_variance = float(p.get("min_variance", 1e-6))
    q.filter_kind = int(p.get("filter_kind", 0))
    q.filter_boundary = int(p.get("filter_boundary", 0))
    q.aa_shadow = int(p.get("aa_shadow", 1))
    q.aa_final = int(p.get("aa_final", 1))
    q.recompute_in_backward = int(p.get("recompute_in_backward", 0))
    q.moments = int(p.get("moments", 0))
    q.exponent = float(p.get("exponent", 0.0))
    q.stream = _stream_ptr(stream)
    return q


class Context:
    """Owner of one dsm_ctx (scratch memory and the state of the last forward)."""

    def __init__(self, handle=None):
        self.lib = load_library()
        self.owned = handle is None
        if handle is not None:
            self.h = ctypes.c_void_p(handle) if not isinstance(handle, ctypes.c_void_p) else handle
            return
        h = ctypes.c_void_p()
        self._check(self.lib.dsm_create(ctypes.byref(h)), None)
        self.h = h

    @classmethod
    def wrap(cls, handle) -> "Context":
        """A non-owning view of a context created elsewhere (a batch's scene,
        dsm_batch_context): its debug copies, backward and masks; closing it
        leaves the context alone."""
        return cls(handle)

    def _check(self, status: int, h=None):
        if status != DSM_OK:
            msg = self.lib.dsm_last_error(h if h is not None else getattr(self, "h", None))
            raise DsmError(status, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "owned", True):
                self.lib.dsm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_topology(self, tris: torch.Tensor, n_verts: int):
        self._check(self.lib.dsm_set_topology(self.h, _ptr(tris), tris.shape[0], n_verts), self.h)

    def render(self, mesh: Mesh, lights, light_params: torch.Tensor, camera: Camera, params: Params,
               image: torch.Tensor):
        arr = (Light * max(1, len(lights)))(*lights)
        self._check(self.lib.dsm_render(self.h, ctypes.byref(mesh), arr, _ptr(light_params), len(lights),
                                        ctypes.byref(camera), ctypes.byref(params), _ptr(image)), self.h)

    def render_backward(self, dL_dimage, dverts=None, dlight=None, dalbedo=None):
        self._check(self.lib.dsm_render_backward(self.h, _ptr(dL_dimage), _ptr(dverts), _ptr(dlight),
                                                 _ptr(dalbedo)), self.h)

    def render_backward_l2(self, image, target, loss, dverts=None, dlight=None, dalbedo=None):
        self._check(self.lib.dsm_render_backward_l2(self.h, _ptr(image), _ptr(target), _ptr(loss), _ptr(dverts),
                                                    _ptr(dlight), _ptr(dalbedo)), self.h)

    def render_cameras(self, mesh: Mesh, lights, light_params: torch.Tensor, cameras, params: Params, images):
        arr = (Light * max(1, len(lights)))(*lights)
        cams = (Camera * len(cameras))(*cameras)
        ptrs = (ctypes.c_void_p * len(images))(*[_ptr(im) for im in images])
        self._check(self.lib.dsm_render_cameras(self.h, ctypes.byref(mesh), arr, _ptr(light_params), len(lights),
                                                cams, len(cameras), ctypes.byref(params), ptrs), self.h)

    def render_cameras_backward(self, dL_dimages, dverts=None, dlight=None, dalbedo=None):
        ptrs = (ctypes.c_void_p * len(dL_dimages))(*[_ptr(g) for g in dL_dimages])
        self._check(self.lib.dsm_render_cameras_backward(self.h, ptrs, _ptr(dverts), _ptr(dlight), _ptr(dalbedo)),
                    self.h)

    def memory_bytes(self) -> int:
        """Device memory held by this context (scratch and saved state)."""
        return int(self.lib.dsm_memory_bytes(self.h))

    def raster_stats(self, view: int) -> dict:
        """Raster work of one view in the last forward (see dsm_raster_stats)."""
        out = (ctypes.c_int64 * 4)()
        self._check(self.lib.dsm_raster_stats(self.h, int(view), ctypes.cast(out, ctypes.c_void_p)), self.h)
        return {"pairs": int(out[0]), "spans": int(out[1]), "pixel_tests": int(out[2]), "aa_listed": int(out[3])}

    def set_tuning(self, light_tile=32, camera_tile=32, big_tiles=16, filter_shape=0):
        t = Tuning(light_tile, camera_tile, big_tiles, filter_shape)
        self._check(self.lib.dsm_set_tuning(self.h, ctypes.byref(t)), self.h)

    def get_tuning(self) -> dict:
        t = Tuning()
        self._check(self.lib.dsm_get_tuning(self.h, ctypes.byref(t)), self.h)
        return t.as_dict()

    def autotune(self, mesh: Mesh, lights, light_params, cameras, params: Params, images, reps: int = 3):
        arr = (Light * max(1, len(lights)))(*lights)
        cams = (Camera * len(cameras))(*cameras)
        ptrs = (ctypes.c_void_p * len(images))(*[_ptr(im) for im in images])
        best, ms = Tuning(), ctypes.c_float()
        self._check(self.lib.dsm_autotune(self.h, ctypes.byref(mesh), arr, _ptr(light_params), len(lights), cams,
                                          len(cameras), ctypes.byref(params), ptrs, int(reps), ctypes.byref(best),
                                          ctypes.byref(ms)), self.h)
        return best.as_dict(), float(ms.value)

    def filter_moments(self, inp: torch.Tensor, out: torch.Tensor, sigma: float, radius: int = 0, kind: int = 0,
                       boundary: int = 0, stream=None):
        self._check(self.lib.dsm_filter_moments(self.h, _ptr(inp), _ptr(out), inp.shape[0], float(sigma),
                                                int(radius), int(kind), int(boundary), _stream_ptr(stream)), self.h)

    def filter_moments_adjoint(self, gout: torch.Tensor, gin: torch.Tensor, sigma: float, radius: int = 0,
                               kind: int = 0, boundary: int = 0, stream=None):
        self._check(self.lib.dsm_filter_moments_adjoint(self.h, _ptr(gout), _ptr(gin), gout.shape[0], float(sigma),
                                                        int(radius), int(kind), int(boundary),
                                                        _stream_ptr(stream)), self.h)

    def sync(self):
        self._check(self.lib.dsm_sync(self.h), self.h)

    def set_grad_mask(self, flags: int):
        """Diagnostic gradient masks (dsm_set_grad_mask): GRAD_MASK_SM_BAND
        zeroes dL/df~ at the shadow maps' silhouette-band texels."""
        self._check(self.lib.dsm_set_grad_mask(self.h, int(flags)), self.h)

    def probe_surface(self, cam: int, W: int, H: int) -> torch.Tensor:
        """(H, W, 2, 4): world position and unit normal the shading used."""
        return self.debug(DBG_SURF, cam, (H, W, 2, 4))

    def probe_lookup(self, cam: int, view: int, W: int, H: int) -> torch.Tensor:
        """(H, W, 2, 4): (u, v, s, t) and (dw, m1, m2, vis) of light view `view`."""
        return self.debug(DBG_LOOKUP, 64 * cam + view, (H, W, 2, 4))

    def bounded_wait_probe(self, arrive: bool):
        """One CTA waiting on an mbarrier (see dsm_bounded_wait_probe)."""
        self._check(self.lib.dsm_bounded_wait_probe(self.h, 1 if arrive else 0), self.h)

    def profile(self, enable: bool):
        self._check(self.lib.dsm_profile_enable(self.h, 1 if enable else 0), self.h)

    def profile_read(self) -> dict:
        n = self.lib.dsm_profile_stage_count()
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_int64 * n)()
        self._check(self.lib.dsm_profile_read(self.h, ms, calls, n), self.h)
        return {self.lib.dsm_profile_stage_name(i).decode(): (ms[i], calls[i]) for i in range(n)}

    def debug(self, what: int, index: int, shape, dtype=torch.float32) -> torch.Tensor:
        out = torch.empty(shape, dtype=dtype, device="cuda")
        self._check(self.lib.dsm_debug_copy(self.h, what, index, _ptr(out), out.numel() * out.element_size()),
                    self.h)
        return out


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().dsm_kernel_launches())


def l2_loss_grad(image: torch.Tensor, target: torch.Tensor, loss: torch.Tensor, grad: torch.Tensor, stream=None):
    """Fused L = mean((image - target)^2) and dL/dimage on the device."""
    lib = load_library()
    st = lib.dsm_l2_loss_grad(_ptr(image), _ptr(target), image.numel(), _ptr(loss), _ptr(grad), _stream_ptr(stream))
    if st != DSM_OK:
        raise DsmError(st, "dsm_l2_loss_grad")


def adam_step(params: torch.Tensor, grads: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
              lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8, stream=None):
    """In-place Adam step on float32 device tensors (m, v zero before step 1)."""
    lib = load_library()
    n = params.numel()
    for t in (grads, m, v):
        if t.numel() != n:
            raise ValueError("adam_step: params, grads, m and v must have the same size")
    st = lib.dsm_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), n, int(step), float(lr), float(betas[0]),
                           float(betas[1]), float(eps), _stream_ptr(stream))
    if st != DSM_OK:
        raise DsmError(st, "dsm_adam_step")


class Renderer:
    """Scene held on the device plus a context: forward / backward of the
    differentiable shadow-mapping renderer for one camera."""

    def __init__(self, scene: dict, device: str = "cuda"):
        self.ctx = Context()
        self.device = device
        self.verts = torch.as_tensor(scene["verts"], dtype=torch.float32, device=device).contiguous()
        self.tris = torch.as_tensor(scene["tris"], dtype=torch.int32, device=device).contiguous()
        self.tri_mat = torch.as_tensor(scene["tri_mat"], dtype=torch.int32, device=device).contiguous()
        self.albedo = torch.as_tensor(scene["albedo"], dtype=torch.float32, device=device).contiguous()
        self.light_params = torch.as_tensor(
            np.stack([np.concatenate([l["pos"], l["dir"]]) for l in scene["lights"]]).astype(np.float32)
            if scene["lights"] else np.zeros((0, 6), np.float32), device=device).contiguous()
        self.lights = [light_struct(l) for l in scene["lights"]]
        self.camera_dict = scene["camera"]
        self.camera = camera_struct(scene["camera"])
        self.params_dict = dict(scene["params"])
        self.W, self.H = int(scene["camera"]["width"]), int(scene["camera"]["height"])
        self.ctx.set_topology(self.tris, self.verts.shape[0])

    def set_camera(self, cam: dict):
        self.camera_dict = cam
        self.camera = camera_struct(cam)
        self.W, self.H = int(cam["width"]), int(cam["height"])

    def mesh_struct(self, verts=None, albedo=None) -> Mesh:
        v = self.verts if verts is None else verts
        a = self.albedo if albedo is None else albedo
        self._keep = (v, a)
        return Mesh(_ptr(v), v.shape[0], _ptr(self.tris), self.tris.shape[0], _ptr(self.tri_mat), _ptr(a),
                    a.shape[0])

    def forward(self, verts=None, light_params=None, albedo=None, image=None, stream=None) -> torch.Tensor:
        lp = self.light_params if light_params is None else light_params
        if image is None:
            image = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        self.ctx.render(self.mesh_struct(verts, albedo), self.lights, lp, self.camera,
                        params_struct(self.params_dict, stream), image)
        return image

    def _grads(self, dverts, dlight, dalbedo):
        V, L, M = self.verts.shape[0], len(self.lights), self.albedo.shape[0]
        dverts = torch.empty((V, 3), dtype=torch.float32, device=self.device) if dverts is None else dverts
        dlight = torch.empty((max(L, 1), 6), dtype=torch.float32, device=self.device) if dlight is None else dlight
        dalbedo = torch.empty((M, 3), dtype=torch.float32, device=self.device) if dalbedo is None else dalbedo
        return dverts, dlight, dalbedo

    def backward(self, dL_dimage: torch.Tensor, dverts=None, dlight=None, dalbedo=None):
        dverts, dlight, dalbedo = self._grads(dverts, dlight, dalbedo)
        self.ctx.render_backward(dL_dimage.contiguous(), dverts, dlight, dalbedo)
        return dverts, dlight[:len(self.lights)], dalbedo

    def backward_l2(self, image: torch.Tensor, target: torch.Tensor, loss: torch.Tensor, dverts=None, dlight=None,
                    dalbedo=None):
        """Backward of the mean squared error of the last forward's image
        against target (dsm_render_backward_l2); loss (one float on the device)
        receives its value."""
        dverts, dlight, dalbedo = self._grads(dverts, dlight, dalbedo)
        self.ctx.render_backward_l2(image.contiguous(), target.contiguous(), loss, dverts, dlight, dalbedo)
        return dverts, dlight[:len(self.lights)], dalbedo

    def forward_cameras(self, cameras: list, verts=None, light_params=None, albedo=None, images=None,
                        stream=None) -> list:
        """One forward seen by several cameras (dicts like scene["camera"]):
        each light's maps are built once; returns one image per camera."""
        lp = self.light_params if light_params is None else light_params
        if images is None:
            images = [torch.empty((int(c["height"]), int(c["width"]), 4), dtype=torch.float32, device=self.device)
                      for c in cameras]
        self.ctx.render_cameras(self.mesh_struct(verts, albedo), self.lights, lp,
                                [camera_struct(c) for c in cameras], params_struct(self.params_dict, stream), images)
        return images

    def shape_class(self, cameras: list | None = None) -> str:
        """Key of the autotuner's cache: triangle count (rounded to a power of
        two), light view sizes, camera sizes and the recompute mode."""
        cams = cameras if cameras is not None else [self.camera_dict]
        t = 1 << max(0, int(self.tris.shape[0]) - 1).bit_length()
        lights = ",".join(f"{l.type}:{l.res}" for l in self.lights)
        views = ",".join(f"{int(c['width'])}x{int(c['height'])}" for c in cams)
        return f"T{t}|L{lights}|C{views}|R{int(self.params_dict.get('recompute_in_backward', 0))}"

    def autotune(self, cameras: list | None = None, reps: int = 3, stream=None, cache: str | None = None):
        """Choose the kernel shapes of this renderer's context by timing
        forward + backward steps of its scene (dsm_autotune); returns the
        chosen shapes and the time per step in ms (None when taken from the
        cache).  With `cache` (a JSON file path) the shapes chosen for this
        scene's shape class are read from it when present, and stored in it
        after a search otherwise."""
        import json
        key = self.shape_class(cameras)
        if cache and os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
            if key in known:
                self.ctx.set_tuning(**known[key])
                return self.ctx.get_tuning(), None
        cams = cameras if cameras is not None else [self.camera_dict]
        images = [torch.empty((int(c["height"]), int(c["width"]), 4), dtype=torch.float32, device=self.device)
                  for c in cams]
        best, ms = self.ctx.autotune(self.mesh_struct(), self.lights, self.light_params,
                                     [camera_struct(c) for c in cams], params_struct(self.params_dict, stream),
                                     images, reps)
        if cache:
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = best
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return best, ms

    def backward_cameras(self, dL_dimages: list, dverts=None, dlight=None, dalbedo=None):
        """Backward of the last forward_cameras for the loss summed over the cameras."""
        dverts, dlight, dalbedo = self._grads(dverts, dlight, dalbedo)
        self.ctx.render_cameras_backward([g.contiguous() for g in dL_dimages], dverts, dlight, dalbedo)
        return dverts, dlight[:len(self.lights)], dalbedo


class DSMFunction(torch.autograd.Function):
    """image = render(verts, light_params, albedo) with the library's own
    backward.  The renderer's context keeps the forward state: call backward
    before the next forward on the same renderer."""

    @staticmethod
    def forward(ctx, verts, light_params, albedo, renderer: Renderer):
        image = renderer.forward(verts.contiguous(), light_params.contiguous(), albedo.contiguous())
        ctx.renderer = renderer
        return image

    @staticmethod
    def backward(ctx, grad_image):
        dv, dl, da = ctx.renderer.backward(grad_image.contiguous())
        return dv, dl, da, None


def render(verts, light_params, albedo, renderer: Renderer):
    return DSMFunction.apply(verts, light_params, albedo, renderer)


class Batch:
    """Batched frames (dsm_batch_*): every scene's forward, L2 loss against its
    target and backward in one call per step, replayed from a CUDA graph after
    the first step.  Device copies of each scene and its output buffers are
    held here; `step` runs on a dedicated non-default stream."""

    def __init__(self, scenes: list, targets: list, device: str = "cuda"):
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.dsm_batch_create(ctypes.byref(h), len(scenes))
        if st != DSM_OK:
            raise DsmError(st, "dsm_batch_create")
        self.h = h
        self.stream = torch.cuda.Stream()
        self.params = params_struct(scenes[0]["params"], self.stream)
        self.scenes = []
        items = []
        for i, (sc, tgt) in enumerate(zip(scenes, targets)):
            d = {"verts": torch.as_tensor(sc["verts"], dtype=torch.float32, device=device).contiguous(),
                 "tris": torch.as_tensor(sc["tris"], dtype=torch.int32, device=device).contiguous(),
                 "tri_mat": torch.as_tensor(sc["tri_mat"], dtype=torch.int32, device=device).contiguous(),
                 "albedo": torch.as_tensor(sc["albedo"], dtype=torch.float32, device=device).contiguous(),
                 "light_params": torch.as_tensor(
                     np.stack([np.concatenate([l["pos"], l["dir"]]) for l in sc["lights"]]).astype(np.float32),
                     device=device).contiguous()}
            W, H = int(sc["camera"]["width"]), int(sc["camera"]["height"])
            V, L, M = d["verts"].shape[0], len(sc["lights"]), d["albedo"].shape[0]
            d["image"] = torch.zeros((H, W, 4), dtype=torch.float32, device=device)
            d["target"] = torch.as_tensor(tgt, dtype=torch.float32, device=device).contiguous()
            d["loss"] = torch.zeros(1, dtype=torch.float32, device=device)
            d["gimg"] = torch.empty((H, W, 4), dtype=torch.float32, device=device)
            d["dverts"] = torch.empty((V, 3), dtype=torch.float32, device=device)
            d["dlight"] = torch.empty((max(L, 1), 6), dtype=torch.float32, device=device)
            d["dalbedo"] = torch.empty((M, 3), dtype=torch.float32, device=device)
            d["lights"] = (Light * max(1, L))(*[light_struct(l) for l in sc["lights"]])
            ctx = self.lib.dsm_batch_context(self.h, i)
            st = self.lib.dsm_set_topology(ctx, _ptr(d["tris"]), d["tris"].shape[0], V)
            if st != DSM_OK:
                raise DsmError(st, self.lib.dsm_last_error(ctx).decode())
            it = BatchItem()
            it.mesh = Mesh(_ptr(d["verts"]), V, _ptr(d["tris"]), d["tris"].shape[0], _ptr(d["tri_mat"]),
                           _ptr(d["albedo"]), M)
            it.lights = ctypes.cast(d["lights"], ctypes.c_void_p)
            it.light_params, it.n_lights = _ptr(d["light_params"]), L
            it.camera = camera_struct(sc["camera"])
            it.image, it.target, it.loss, it.dL_dimage = (_ptr(d["image"]), _ptr(d["target"]), _ptr(d["loss"]),
                                                          _ptr(d["gimg"]))
            it.dL_dverts, it.dL_dlight, it.dL_dalbedo = _ptr(d["dverts"]), _ptr(d["dlight"]), _ptr(d["dalbedo"])
            items.append(it)
            self.scenes.append(d)
        self.items = (BatchItem * len(items))(*items)
        torch.cuda.synchronize()

    def step(self):
        st = self.lib.dsm_batch_step(self.h, ctypes.cast(self.items, ctypes.c_void_p), len(self.scenes),
                                     ctypes.byref(self.params))
        if st != DSM_OK:
            raise DsmError(st, self.lib.dsm_batch_last_error(self.h).decode())

    def sync(self):
        st = self.lib.dsm_batch_sync(self.h)
        if st != DSM_OK:
            raise DsmError(st, self.lib.dsm_batch_last_error(self.h).decode())

    def kernels_per_step(self) -> int:
        return int(self.lib.dsm_batch_kernels_per_step(self.h))

    def context(self, i: int) -> Context:
        """Scene i's context (non-owning): its debug copies and, after a step,
        further backward passes of that step's forward."""
        return Context.wrap(self.lib.dsm_batch_context(self.h, i))

    def set_host_io(self, i: int, verts=None, light_params=None, albedo=None, loss=None):
        """Pinned host tensors that scene i's recorded step uploads first
        (vertices, light parameters, albedo) and the loss it downloads last;
        None leaves that copy out.  The next step records a new graph."""
        for t in (verts, light_params, albedo, loss):
            if t is not None and (t.is_cuda or not t.is_pinned() or not t.is_contiguous()):
                raise ValueError("host staging tensors must be contiguous pinned host memory")
        it = self.items[i]
        self._host = getattr(self, "_host", {})
        self._host[i] = (verts, light_params, albedo, loss)
        it.host_verts = verts.data_ptr() if verts is not None else None
        it.host_light_params = light_params.data_ptr() if light_params is not None else None
        it.host_albedo = albedo.data_ptr() if albedo is not None else None
        it.host_loss = loss.data_ptr() if loss is not None else None

    def autotune(self, reps: int = 2):
        """Shapes shared by every scene, chosen by timing whole batched steps
        (dsm_batch_autotune, synchronous)."""
        st = self.lib.dsm_batch_autotune(self.h, ctypes.cast(self.items, ctypes.c_void_p), len(self.scenes),
                                         ctypes.byref(self.params), int(reps))
        if st != DSM_OK:
            raise DsmError(st, self.lib.dsm_batch_last_error(self.h).decode())

    def tunings(self) -> list:
        out = []
        for i in range(len(self.scenes)):
            t = Tuning()
            self.lib.dsm_get_tuning(self.lib.dsm_batch_context(self.h, i), ctypes.byref(t))
            out.append(t.as_dict())
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.dsm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
