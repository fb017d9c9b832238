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

    def __init__(self, scene: dict, target=None):
        from paper_2308_10896_b300 import dsm
        self.dsm = dsm
        self.scene = scene
        self.r = dsm.Renderer(scene)
        self.image = self.r.forward()
        self.r.ctx.sync()
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
        g = self.r.ctx.debug(self.dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
        return ids, g[..., 1].numpy(), g[..., 2].numpy(), g[..., 3].numpy()

    def snap(self, w):
        V = self.scene["verts"].shape[0]
        s = self.r.ctx.debug(self.dsm.DBG_SNAP, w, (V, 4)).cpu()
        si = s.view(torch.int32).numpy()
        return si[:, 0].astype(np.int64), si[:, 1].astype(np.int64), s[:, 2].numpy(), si[:, 3]

    def light_map(self, what, l):
        R = self.scene["lights"][self.view_light[l]]["res"]
        return self.r.ctx.debug(what, l, (R, R, 2)).cpu().numpy()

    def color(self):
        W, H = self.view_size(self.L)
        return self.r.ctx.debug(self.dsm.DBG_COLOR, 0, (H, W, 4)).cpu().numpy()

    def Q(self):
        return self.r.ctx.debug(self.dsm.DBG_Q, 0, (self.L, 20)).cpu().numpy()


def oracle_target(scene: dict, sigma=0.01, seed=1):
    v = scenes.jitter_vertices(scene, sigma, seed)
    return O.render(scene, verts=torch.as_tensor(v, dtype=F64), keep=False)["image"].detach().numpy()
