"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded scene, stage by stage."""
from __future__ import annotations

import numpy as np
import torch

import scenes
from oracle import dsm_oracle as O

F64 = torch.float64

# Floating-point tolerance for depths, moments, shadow factors and pixels.
ATOL, RTOL = 1e-5, 1e-4


def close(gpu, ref, atol=ATOL, rtol=RTOL):
    """|g - o| <= atol + rtol |o| elementwise; returns (ok, worst excess, index)."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ref, np.float64)
    err = np.abs(g - o) - (atol + rtol * np.abs(o))
    if err.size == 0:
        return True, 0.0, ()
    k = int(np.argmax(err))
    return err.max() <= 0, float(err.max()), np.unravel_index(k, err.shape)


def assert_close(gpu, ref, what, atol=ATOL, rtol=RTOL):
    ok, worst, idx = close(gpu, ref, atol, rtol)
    if not ok:
        g = np.asarray(gpu)[idx]
        o = np.asarray(ref)[idx]
        raise AssertionError(f"{what}: excess {worst:.3g} at {idx}: gpu {g} oracle {o}")


def loss_tolerance(n: int, loss: float) -> float:
    """Bound on |a - b| for two float32 evaluations of the mean squared error
    over n floats: dsm_l2_loss_grad (a float sum per thread over its
    grid-stride elements, a 256-lane tree of 8 levels, the block sums divided
    by n and added by float atomics, one per block of at most 148 * 8 blocks)
    and dsm_render_backward_l2 (four squares per pixel, a warp tree of 5
    levels, at most 8 float atomics per block, float64 above).  All terms are
    non-negative, so each float addition along a chain adds at most one unit
    roundoff u = 2^-24 of the total: |error| <= (additions in the longest
    chain) u loss per evaluation."""
    blocks = min((n + 255) // 256, 148 * 8)
    per_thread = -(-n // (blocks * 256))
    chain_l2 = per_thread + 1 + 8 + 1 + blocks
    chain_fused = 4 + 1 + 5 + 8 + 2
    return (chain_l2 + chain_fused) * 2.0 ** -24 * abs(loss) + 1e-12


def report(record: dict):
    """Append one JSON line of measured parity figures to the file named by the
    environment variable DSM_PARITY_REPORT (nothing when it is unset)."""
    import json
    import os
    path = os.environ.get("DSM_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(record, default=float) + "\n")


def grad_stats(gpu, ref) -> dict:
    """Relative L2 error, and the per-element relative error over the elements
    with |o| > 1e-3 max|o| (max, 99th percentile, share above 1e-3), of a
    gradient against the oracle's."""
    g = np.asarray(gpu, np.float64).ravel()
    o = np.asarray(ref, np.float64).ravel()
    scale = np.abs(o).max() if o.size else 0.0
    if scale == 0.0:
        return {"rel_l2": 0.0 if not g.size or np.abs(g).max() == 0 else float("inf"), "rel_max": 0.0,
                "rel_p99": 0.0, "share_above_1e-3": 0.0, "n": int(o.size)}
    big = np.abs(o) > 1e-3 * scale
    elem = np.abs(g - o)[big] / np.abs(o)[big]
    return {"rel_l2": float(np.linalg.norm(g - o) / np.linalg.norm(o)),
            "rel_max": float(elem.max()) if elem.size else 0.0,
            "rel_p99": float(np.percentile(elem, 99)) if elem.size else 0.0,
            "share_above_1e-3": float(np.mean(elem > 1e-3)) if elem.size else 0.0,
            "small_abs_max_over_scale": float((np.abs(g - o)[~big]).max() / scale) if (~big).any() else 0.0,
            "n": int(o.size)}


def grad_close_strict(gpu, ref, what, rel=1e-3):
    """Gradient parity outside the silhouette band: relative L2 <= rel and
    every element with |o| > 1e-3 max|o| within rel |o| (the smaller elements
    count through the relative L2; their largest error is reported).  Returns
    grad_stats."""
    g = np.asarray(gpu, np.float64).ravel()
    o = np.asarray(ref, np.float64).ravel()
    st = grad_stats(g, o)
    scale = np.abs(o).max() if o.size else 0.0
    if scale == 0.0:
        assert not g.size or np.abs(g).max() <= 1e-12, f"{what}: oracle is zero, gpu {np.abs(g).max()}"
        return st
    big = np.abs(o) > 1e-3 * scale
    bound = np.where(big, rel * np.abs(o), np.inf)
    over = np.abs(g - o) > bound
    k = int(np.argmax(np.where(big, np.abs(g - o) / np.where(big, np.abs(o), 1.0), 0.0)))
    assert st["rel_l2"] <= rel, f"{what}: relative L2 {st['rel_l2']:.3g} > {rel}"
    assert not over.any(), (f"{what}: {int(over.sum())} of {o.size} elements outside rel {rel}; worst at {k}: "
                            f"gpu {g[k]:.6g} oracle {o[k]:.6g}")
    return st


def grad_close(gpu, ref, what, rel=1e-3):
    """Gradient parity: per element where |o| > 1e-3 max|o| (relative error
    <= rel, with an absolute floor of rel * 1e-3 max|o|) and relative L2 of the
    whole vector <= rel."""
    g = np.asarray(gpu, np.float64).ravel()
    o = np.asarray(ref, np.float64).ravel()
    scale = np.abs(o).max() if o.size else 0.0
    if scale == 0.0:
        assert np.abs(g).max() <= 1e-12, f"{what}: oracle is zero, gpu {np.abs(g).max()}"
        return 0.0
    l2 = np.linalg.norm(g - o) / np.linalg.norm(o)
    big = np.abs(o) > 1e-3 * scale
    elem = np.abs(g - o)[big] / np.abs(o)[big]
    worst = float(elem.max()) if elem.size else 0.0
    assert l2 <= rel, f"{what}: relative L2 {l2:.3g} > {rel}"
    assert worst <= 10 * rel or np.mean(elem > rel) < 0.01, \
        f"{what}: per-element relative error {worst:.3g}, {np.mean(elem > rel):.3%} above {rel}"
    return l2


class GpuFrame:
    """Forward (and optionally backward) of the CUDA path on one scene."""

    def __init__(self, scene: dict, target=None, ctx=None, image=None):
        """Render `scene` with a new Renderer, or (ctx given) view the last
        forward of an existing context, e.g. a batched scene's, whose image is
        `image`."""
        from paper_2308_10896_b300 import dsm
        self.dsm = dsm
        self.scene = scene
        if ctx is not None:
            self.r = None
            self.ctx = ctx
            self.image = image
        else:
            self.r = dsm.Renderer(scene)
            self.ctx = self.r.ctx
            self.image = self.r.forward()
            self.ctx.sync()
        # light views: one per directional or spot light, six cube faces per point light
        self.view_light = [l for l, Lt in enumerate(scene["lights"]) for _ in range(6 if Lt["type"] == 2 else 1)]
        self.L = len(self.view_light)
        self.target = target
        if target is not None:
            tgt = torch.as_tensor(np.asarray(target, np.float32), device="cuda").contiguous()
            self.loss = torch.zeros(1, device="cuda")
            self.gimg = torch.empty_like(self.image)
            dsm.l2_loss_grad(self.image, tgt, self.loss, self.gimg)
            self.dverts, self.dlight, self.dalbedo = self.r.backward(self.gimg)
            self.r.ctx.sync()

    def view_size(self, w):
        if w < self.L:
            R = self.scene["lights"][self.view_light[w]]["res"]
            return R, R
        return self.scene["camera"]["width"], self.scene["camera"]["height"]

    def gbuf(self, w):
        W, H = self.view_size(w)
        g = self.ctx.debug(self.dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
        return ids, g[..., 1].numpy(), g[..., 2].numpy(), g[..., 3].numpy()

    def snap(self, w):
        V = self.scene["verts"].shape[0]
        s = self.ctx.debug(self.dsm.DBG_SNAP, w, (V, 4)).cpu()
        si = s.view(torch.int32).numpy()
        return si[:, 0].astype(np.int64), si[:, 1].astype(np.int64), s[:, 2].numpy(), si[:, 3]

    def light_map(self, what, l):
        R = self.scene["lights"][self.view_light[l]]["res"]
        return self.ctx.debug(what, l, (R, R, 2)).cpu().numpy()

    def color(self):
        W, H = self.view_size(self.L)
        return self.ctx.debug(self.dsm.DBG_COLOR, 0, (H, W, 4)).cpu().numpy()

    def Q(self):
        return self.ctx.debug(self.dsm.DBG_Q, 0, (self.L, 20)).cpu().numpy()

    def surface(self, cam=0):
        """(x, n) the shading used at every pixel: two (H, W, 3) arrays (NaN off the mesh)."""
        W, H = self.view_size(self.L + cam)
        s = self.ctx.probe_surface(cam, W, H).cpu().numpy()
        return s[:, :, 0, :3], s[:, :, 1, :3]

    def lookup(self, view, cam=0):
        """(H, W, 8): u, v, s, t, dw, m1, m2, vis of light view `view` (NaN where absent)."""
        W, H = self.view_size(self.L + cam)
        return self.ctx.probe_lookup(cam, view, W, H).cpu().numpy().reshape(H, W, 8)

    def shading_teacher(self, cam=0) -> dict:
        """The shading stages' values as an oracle teacher (x, n, lookup per light view)."""
        x, n = self.surface(cam)
        return {"x": x, "n": n, "lookup": [self.lookup(v, cam) for v in range(self.L)]}

    def full_teacher(self) -> dict:
        """Every float32 stage of the forward as an oracle teacher."""
        t = {"ftilde": [self.light_map(self.dsm.DBG_FTILDE, l) for l in range(self.L)],
             "moments": [self.light_map(self.dsm.DBG_MOMENTS, l) for l in range(self.L)],
             "color": self.color()}
        t.update(self.shading_teacher())
        return t

    def backward_with(self, gimg: torch.Tensor, sm_band: bool):
        """Another backward of the same forward for dL/dimage = gimg, with or
        without the shadow maps' silhouette-band mask; returns host float64
        (dverts, dlight, dalbedo)."""
        torch.cuda.synchronize()     # gimg is ready before the context's own stream reads it
        self.ctx.set_grad_mask(self.dsm.GRAD_MASK_SM_BAND if sm_band else 0)
        try:
            sc = self.scene
            dv = torch.empty((sc["verts"].shape[0], 3), device="cuda")
            dl = torch.empty((max(len(sc["lights"]), 1), 6), device="cuda")
            da = torch.empty((np.asarray(sc["albedo"]).shape[0], 3), device="cuda")
            self.ctx.render_backward(gimg.contiguous(), dv, dl, da)
            self.ctx.sync()
        finally:
            self.ctx.set_grad_mask(0)
        return tuple(t.double().cpu().numpy() for t in (dv, dl[:len(self.scene["lights"])], da))


def camera_band(scene: dict, ref: dict) -> np.ndarray:
    """The camera view's silhouette band (H, W) from the oracle's raster."""
    tris = scene["tris"].astype(np.int64)
    st = ref["camera_setup"]
    return O.silhouette_band(ref["camera_raster"], O.silhouette_table(O.edge_adjacency(tris), st))


def stage_excess(gpu, ref, atol=ATOL, rtol=RTOL, mask=None):
    """(worst excess over atol + rtol |o|, count compared) where both are finite (and mask)."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ref, np.float64)
    m = np.isfinite(g) & np.isfinite(o)
    if mask is not None:
        m &= mask
    if not m.any():
        return 0.0, 0
    return float((np.abs(g[m] - o[m]) - (atol + rtol * np.abs(o[m]))).max()), int(m.sum())


def oracle_shading_maps(ref: dict, H: int, W: int, nviews: int):
    """The oracle's recorded shading stages laid out as GPU probe arrays:
    (x, n) (H, W, 3) and per light view (H, W, 8) (u, v, s, t, dw, m1, m2, vis),
    NaN where the oracle has no value."""
    sh = ref["shading"]
    jj, ii = sh["pixels"]
    x = np.full((H, W, 3), np.nan)
    n = np.full((H, W, 3), np.nan)
    x[jj, ii] = sh["x"].numpy()
    n[jj, ii] = sh["n"].numpy()
    looks = []
    for v in range(nviews):
        r = sh["lookup"][v]
        a = np.full((H, W, 8), np.nan)
        uv = r["uv"].numpy().copy()
        uv[~r["front"]] = np.nan
        st = r["st"].numpy().copy()
        st[~r["inside"]] = np.nan
        mm = r["mm"].numpy().copy()
        mm[~r["inside"]] = np.nan
        a[jj, ii, 0:2] = uv
        a[jj, ii, 2:4] = st
        a[jj, ii, 4] = r["dw"].numpy()
        a[jj, ii, 5:7] = mm
        a[jj, ii, 7] = np.where(r["inside"], r["vis"].numpy(), 1.0)
        looks.append(a)
    return x, n, looks


def oracle_target(scene: dict, sigma=0.01, seed=1):
    v = scenes.jitter_vertices(scene, sigma, seed)
    return O.render(scene, verts=torch.as_tensor(v, dtype=F64), keep=False)["image"].detach().numpy()
