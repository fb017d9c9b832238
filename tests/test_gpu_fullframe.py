"""Whole frames of the benchmark-size configurations against the oracle
(slow: the oracle rasterises every view by brute force, about a minute for the
330k-triangle scene).

- Configs 2 and 3 (the benchmark workload), every view whole: triangle ids and
  depth keys bit-identical; the shading stages with the GPU's earlier stages
  taught, within 1e-5 + 1e-4 |o|; and the gradients of a seeded dL/dimage
  (camera band zeroed, shadow-map bands masked) with every forward stage
  taught: each element within 1e-3 relative.  The same dL/dimage without the
  masks is reported (relative L2 <= 1e-3).
- Config 4 (64 batched scenes): the smallest, the largest and the smallest
  three-light scene of one dsm_batch_step, each against the oracle: ids and
  keys, colour and image, loss, the step's own gradients (relative L2 <= 1e-3)
  and, through the scene's context, the banded backward element by element.
- Config 5's mesh (1M triangles) under its first light from its first camera,
  stored mode: ids, the colour stage and the banded gradients.  The full
  configuration's recomputing backward is checked against the stored mode in
  test_gpu_fullsize.py.

Targets and dL/dimage here are seeded synthetic images, so nothing the oracle
takes as input is produced by the GPU, apart from the taught stage values of
the stage-wise comparison."""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O
from parity_util import (ATOL, GpuFrame, assert_close, camera_band, grad_close, grad_close_strict, grad_stats,
                         oracle_shading_maps, report, stage_excess)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _seeded_grad_image(H, W, seed):
    """A seeded dL/dimage: standard normal per channel, divided by the entry count."""
    return np.random.default_rng(seed).normal(size=(H, W, 4)) / (H * W * 4)


def _check_ids(gpu: GpuFrame, out: dict, what: str):
    rasters = [L["raster"] for L in out["lights"]] + [out["camera_raster"]]
    for w, ras in enumerate(rasters):
        ids, _, _, zk = gpu.gbuf(w)
        assert np.array_equal(ids, ras["ids"]), f"{what} view {w}: {int(np.sum(ids != ras['ids']))} ids differ"
        cov = ids > 0
        assert np.array_equal(zk[cov].view(np.uint32), ras["zkey"][cov].view(np.uint32)), f"{what} view {w} keys"


def _check_shading(gpu: GpuFrame, out: dict, what: str) -> dict:
    """Shading stages of the oracle (fed the GPU's x, n, lookups and moments)
    against the GPU's, and the colour."""
    W, H = gpu.view_size(gpu.L)
    ox, on, olook = oracle_shading_maps(out, H, W, gpu.L)
    gx, gn = gpu.surface()
    worst = {}
    for name, g, o in (("x", gx, ox), ("n", gn, on)):
        worst[name], _ = stage_excess(g, o)
    for v in range(gpu.L):
        g, o = gpu.lookup(v), olook[v]
        R = gpu.scene["lights"][gpu.view_light[v]]["res"]
        for name, cols, atol, rtol in (("uv", slice(0, 2), ATOL, 1e-4), ("st", slice(2, 4), 8 * R * 2.0 ** -24, 0.0),
                                       ("dw", slice(4, 5), ATOL, 1e-4), ("m", slice(5, 7), ATOL, 1e-4),
                                       ("vis", slice(7, 8), ATOL, 1e-4)):
            worst[f"{name}[{v}]"], _ = stage_excess(g[..., cols], o[..., cols], atol, rtol)
    for k, e in worst.items():
        assert e <= 0, f"{what}: shading stage {k} excess {e:.3g}"
    assert_close(gpu.color(), out["color"].detach().numpy(), f"{what}: colour")
    return worst


def _teacher_without_colour(gpu: GpuFrame) -> dict:
    t = gpu.full_teacher()
    t.pop("color")        # the oracle's colour is computed from the taught shading stages
    return t


@pytest.fixture(scope="module", params=["config2", "config3"])
def whole(request):
    from paper_2308_10896_b300 import dsm  # noqa: F401
    torch.cuda.set_device(0)
    sc = {"config2": scenes.config2, "config3": scenes.config3}[request.param]()
    gpu = GpuFrame(sc)
    W, H = gpu.view_size(gpu.L)
    G = _seeded_grad_image(H, W, 31)
    band = camera_band_from_gpu(gpu)
    Gm = G.copy()
    Gm[band] = 0.0
    masked = gpu.backward_with(torch.as_tensor(Gm, dtype=torch.float32, device="cuda"), sm_band=True)
    full = gpu.backward_with(torch.as_tensor(G, dtype=torch.float32, device="cuda"), sm_band=False)
    # the oracle zeroes the camera band from its own raster
    out = O.render_and_grad(sc, None, teacher=_teacher_without_colour(gpu),
                            objectives=[(G, True, True), (G, False, False)])
    assert np.array_equal(out["camera_band"], band), "camera silhouette bands differ"
    return {"name": request.param, "sc": sc, "gpu": gpu, "out": out, "masked": masked, "full": full,
            "band_pixels": int(band.sum())}


def camera_band_from_gpu(gpu: GpuFrame) -> np.ndarray:
    """The camera's silhouette band from the GPU's G-buffer (ids and depth keys
    are bit-identical to the oracle's, which the tests check)."""
    sc = gpu.scene
    tris = sc["tris"].astype(np.int64)
    ids, _, _, zk = gpu.gbuf(gpu.L)
    order = zk.astype(np.float32).view(np.uint32).astype(np.uint64)
    neg = (order & 0x80000000) != 0
    order = np.where(neg, (~order) & 0xFFFFFFFF, order | 0x80000000)
    key = np.where(ids > 0, (order << np.uint64(32)) | (ids - 1).clip(0).astype(np.uint64),
                   np.iinfo(np.uint64).max)
    V32 = sc["verts"].astype(np.float32)
    st = O.setup_view(O.clip_pinned(np.asarray(sc["camera"]["clip"], np.float32), V32), tris,
                      int(sc["camera"]["width"]), int(sc["camera"]["height"]))
    return O.silhouette_band({"ids": ids, "key": key}, O.silhouette_table(O.edge_adjacency(tris), st))


def test_whole_frame_ids_and_depth_keys(whole):
    _check_ids(whole["gpu"], whole["out"], whole["name"])


def test_whole_frame_shading_stagewise(whole):
    worst = _check_shading(whole["gpu"], whole["out"], whole["name"])
    report({"test": "whole_frame_shading_stagewise", "case": whole["name"], "worst_excess": worst})


def test_whole_frame_gradients_outside_band(whole):
    out, (dv, dl, da) = whole["out"], whole["masked"]
    gv, gl, ga = out["objective_grads"][0]
    rec = {"test": "whole_frame_gradients_outside_band", "case": whole["name"],
           "camera_band_pixels": whole["band_pixels"]}
    for name, g, o in (("albedo", da, ga), ("light", dl, gl), ("verts", dv, gv)):
        rec[name] = grad_close_strict(g, o.numpy(), f"{whole['name']} dL/d{name} outside the band")
    report(rec)


def test_whole_frame_gradients_with_band(whole):
    out, (dv, dl, da) = whole["out"], whole["full"]
    gv, gl, ga = out["objective_grads"][1]
    rec = {"test": "whole_frame_gradients_with_band", "case": whole["name"]}
    for name, g, o in (("albedo", da, ga), ("light", dl, gl), ("verts", dv, gv)):
        rec[name] = grad_stats(g, o.numpy())
        grad_close(g, o.numpy(), f"{whole['name']} dL/d{name}")
    report(rec)


def _config4_picks(scs):
    T = [int(s["tris"].shape[0]) for s in scs]
    three = [k for k, s in enumerate(scs) if len(s["lights"]) == 3]
    return sorted({int(np.argmin(T)), int(np.argmax(T)), min(three, key=lambda k: T[k])})


def test_config4_batched_scenes_against_oracle():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    scs = scenes.config4()
    for sc in scs[1:]:
        sc["params"] = dict(scs[0]["params"])
    targets = [np.random.default_rng(4100 + k).uniform(0.0, 0.6, size=(int(s["camera"]["height"]),
                                                                       int(s["camera"]["width"]), 4))
               for k, s in enumerate(scs)]
    b = dsm.Batch(scs, targets)
    b.step()
    b.stream.synchronize()
    b.sync()
    for k in _config4_picks(scs):
        sc, d = scs[k], b.scenes[k]
        what = f"config4 scene {k} ({int(sc['tris'].shape[0])} triangles, {len(sc['lights'])} lights)"
        gpu = GpuFrame(sc, ctx=b.context(k), image=d["image"])
        W, H = gpu.view_size(gpu.L)
        band = camera_band_from_gpu(gpu)
        G = _seeded_grad_image(H, W, 400 + k)
        out = O.render_and_grad(sc, targets[k], teacher=_teacher_without_colour(gpu), objectives=[(G, True, True)])
        _check_ids(gpu, out, what)
        assert np.array_equal(out["camera_band"], band), f"{what}: camera silhouette bands differ"
        G[band] = 0.0
        _check_shading(gpu, out, what)
        # the final antialiasing of the oracle's (stage-checked) colour against
        # the batched image.  The antialiasing blends by the crossing parameter t
        # of an edge whose unsnapped screen position the GPU holds in float32:
        # a few ulps of the image side, so t carries up to 4 2^-24 max(W, H)
        # and a blended value that times the colour step it blends across.
        img = d["image"].cpu().numpy()
        blend_tol = 4.0 * 2.0 ** -24 * max(W, H) * float(np.abs(img).max())
        assert_close(img, out["image"].detach().numpy(), f"{what}: image", atol=ATOL + blend_tol)
        loss_o = float(out["loss"])
        assert abs(float(d["loss"].item()) - loss_o) <= 1e-5 + 1e-4 * abs(loss_o), f"{what}: loss"
        L = len(sc["lights"])
        rec = {"test": "config4_batched_vs_oracle", "case": what}
        for name, g, o in (("verts", d["dverts"], out["grad_verts"]), ("light", d["dlight"][:L], out["grad_light"]),
                           ("albedo", d["dalbedo"], out["grad_albedo"])):
            rec[name] = grad_stats(g.cpu().numpy(), o.numpy())
            grad_close(g.cpu().numpy(), o.numpy(), f"{what}: batched dL/d{name}")
        dv, dl, da = gpu.backward_with(torch.as_tensor(G, dtype=torch.float32, device="cuda"), sm_band=True)
        gv, gl, ga = out["objective_grads"][0]
        for name, g, o in (("verts", dv, gv), ("light", dl, gl), ("albedo", da, ga)):
            rec[f"{name}_outside_band"] = grad_close_strict(g, o.numpy(), f"{what}: dL/d{name} outside the band")
        report(rec)
    b.close()


def test_config5_mesh_one_light_one_camera_against_oracle():
    """Config 5's 1M-triangle mesh, stored mode, its first light and camera."""
    torch.cuda.set_device(0)
    sc = scenes.config5()
    sc = dict(sc, lights=sc["lights"][:1], camera=sc["cameras"][0],
              params=dict(sc["params"], recompute_in_backward=0))
    sc.pop("cameras", None)
    gpu = GpuFrame(sc)
    W, H = gpu.view_size(gpu.L)
    G = _seeded_grad_image(H, W, 55)
    band = camera_band_from_gpu(gpu)
    out = O.render_and_grad(sc, None, teacher=_teacher_without_colour(gpu), objectives=[(G, True, True)])
    _check_ids(gpu, out, "config5 mesh")
    assert np.array_equal(out["camera_band"], band), "config5 mesh: camera silhouette bands differ"
    G[band] = 0.0
    dv, dl, da = gpu.backward_with(torch.as_tensor(G, dtype=torch.float32, device="cuda"), sm_band=True)
    out["grad_verts"], out["grad_light"], out["grad_albedo"] = out["objective_grads"][0]
    worst = _check_shading(gpu, out, "config5 mesh")
    rec = {"test": "config5_mesh_vs_oracle", "worst_excess": worst}
    for name, g, o in (("verts", dv, out["grad_verts"]), ("light", dl, out["grad_light"]),
                       ("albedo", da, out["grad_albedo"])):
        rec[name] = grad_close_strict(g, o.numpy(), f"config5 mesh dL/d{name} outside the band")
    report(rec)
