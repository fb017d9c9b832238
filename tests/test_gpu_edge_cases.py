"""Degenerate inputs and the maximum sizes, through the C ABI.

- An empty mesh: every pixel is background (colour and coverage 0, as the
  oracle gives), the gradients are zero and the raster has no work.
- No lights: the shading sum is empty, so RGB is 0 while the coverage channel
  and the camera's ids follow the oracle; dL/dalbedo is zero and dL/dverts
  (through the coverage antialiasing) follows the oracle.
- The maximum number of views: four point lights (24 cube faces) seen by 8
  cameras in one dsm_render_cameras call, every view's ids and depth keys
  bit-identical to the oracle's rasters; one view more is rejected.
(Culled and degenerate triangles and one-texel maps are parity cases of
test_gpu_parity.py.)"""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def _empty_scene():
    sc = scenes.tiny_scene(13, res=24, img=20, kind="mixed", n_lights=2)
    sc = dict(sc, verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.int32),
              tri_mat=np.zeros((0,), np.int32))
    sc["camera"] = scenes.look_at_perspective((0.0, 3.0, 4.0), (0.0, 0.5, 0.0), 45.0, 21, 17)
    return sc


def test_empty_mesh():
    from paper_2308_10896_b300 import dsm
    from oracle import dsm_oracle as O
    torch.cuda.set_device(0)
    sc = _empty_scene()
    r = dsm.Renderer(sc)
    img = r.forward()
    gimg = torch.randn(img.shape, generator=torch.Generator().manual_seed(3)).cuda()
    dv, dl, da = r.backward(gimg)
    r.ctx.sync()
    ref = O.render(sc)["image"].numpy()
    assert not ref.any()
    assert not img.cpu().numpy().any(), "an empty scene renders background only"
    assert dv.numel() == 0
    assert not dl.cpu().numpy().any() and not da.cpu().numpy().any()
    for w in range(len(sc["lights"]) + 1):
        assert r.ctx.raster_stats(w) == {"pairs": 0, "spans": 0, "pixel_tests": 0, "aa_listed": 0}


def test_no_lights():
    from paper_2308_10896_b300 import dsm
    from oracle import dsm_oracle as O
    from parity_util import assert_close, grad_close, oracle_target
    torch.cuda.set_device(0)
    sc = dict(scenes.tiny_scene(14, res=32, img=36, kind="directional"), lights=[])
    tgt = oracle_target(sc, 0.01, 5)
    r = dsm.Renderer(sc)
    img = r.forward()
    loss = torch.zeros(1, device="cuda")
    gimg = torch.empty_like(img)
    dsm.l2_loss_grad(img, torch.as_tensor(tgt, dtype=torch.float32, device="cuda"), loss, gimg)
    dv, dl, da = r.backward(gimg)
    r.ctx.sync()
    H, W = img.shape[:2]
    g = r.ctx.debug(dsm.DBG_GBUF, 0, (H, W, 4)).cpu()
    ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
    ref = O.render(sc)
    assert np.array_equal(ids, ref["camera_raster"]["ids"])
    out = img.cpu().numpy()
    assert not out[..., :3].any(), "no light: the shading sum is empty"
    assert_close(out, ref["image"].detach().numpy(), "image without lights")
    teach = {"color": r.ctx.debug(dsm.DBG_COLOR, 0, (H, W, 4)).cpu().numpy()}
    res = O.render_and_grad(sc, tgt, teacher=teach)
    assert abs(float(loss.item()) - float(res["loss"])) <= 1e-5 + 1e-4 * abs(float(res["loss"]))
    assert not da.cpu().numpy().any()
    grad_close(dv.cpu().numpy(), res["grad_verts"].numpy(), "dL/dverts without lights")


def _four_point_lights(n):
    sc = scenes.tiny_scene(15, res=16, img=24, kind="point")
    base = sc["lights"][0]
    offs = [(0.0, 0.0, 0.0), (-1.6, 0.2, 0.3), (0.4, 0.5, -1.5), (-0.8, 0.9, -0.9), (0.9, 0.3, 0.9)]
    lights = []
    for k in range(n):
        L = dict(base)
        L["pos"] = (np.asarray(base["pos"]) + np.asarray(offs[k], np.float32)).astype(np.float32)
        lights.append(L)
    sc["lights"] = lights
    cams = [scenes.look_at_perspective((3.5 * np.cos(a), 2.5, 3.5 * np.sin(a)), (0.0, 0.6, 0.0), 50.0,
                                       24 + 2 * c, 20 + c)
            for c, a in enumerate(np.linspace(0.0, 2 * np.pi, 8, endpoint=False))]
    return sc, cams


def test_maximum_views_bit_exact():
    from paper_2308_10896_b300 import dsm
    from oracle import dsm_oracle as O
    torch.cuda.set_device(0)
    sc, cams = _four_point_lights(4)
    assert len(cams) == dsm.MAX_CAMERAS
    r = dsm.Renderer(sc)
    r.forward_cameras(cams)
    r.ctx.sync()
    L = 6 * len(sc["lights"])
    assert L == 24
    for c, cam in enumerate(cams):
        ref = O.render(dict(sc, camera=cam))
        if c == 0:
            for w, Lv in enumerate(ref["lights"]):
                R = sc["lights"][Lv["light"]]["res"]
                g = r.ctx.debug(dsm.DBG_GBUF, w, (R, R, 4)).cpu()
                ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
                assert np.array_equal(ids, Lv["raster"]["ids"]), f"light view {w}"
                cov = ids > 0
                assert np.array_equal(g[..., 3].numpy()[cov].view(np.uint32),
                                      Lv["raster"]["zkey"][cov].view(np.uint32)), f"light view {w} keys"
        H, W = cam["height"], cam["width"]
        g = r.ctx.debug(dsm.DBG_GBUF, L + c, (H, W, 4)).cpu()
        ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
        assert np.array_equal(ids, ref["camera_raster"]["ids"]), f"camera {c}"
    sc5, _ = _four_point_lights(5)
    with pytest.raises(dsm.DsmError):
        dsm.Renderer(sc5).forward_cameras(cams[:1])


def test_list_overflow_reported_and_recovered():
    """A frame whose tile-triangle pairs exceed the lists sized by an earlier
    frame of the same mesh is reported (DSM_ERR_CAPACITY at the next sync,
    every write of the frame kept in bounds); rendering again re-sizes and
    gives the G-buffers and image of a fresh context.  (A sphere of 180
    triangles grown 4x about its centre: 1175 -> 4563 pairs in the 1024^2
    light view, against lists of 3436 entries.)"""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = scenes.tiny_scene(18, res=1024, img=64, kind="directional", n_lights=1, freq=3)
    shape = dict(light_tile=32, camera_tile=32, big_tiles=64)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(**shape)
    r.forward()
    r.ctx.sync()
    pairs_before = r.ctx.raster_stats(0)["pairs"]
    big = np.asarray(sc["verts"], np.float32).copy()
    centre = np.array([0.1, 1.0, -0.1], np.float32)
    big[:-4] = (big[:-4] - centre) * 4.0 + centre          # the sphere; the last four are the ground
    vbig = torch.as_tensor(big, device="cuda")
    r.forward(verts=vbig)
    with pytest.raises(dsm.DsmError) as err:
        r.ctx.sync()
    assert err.value.status == dsm.DSM_ERR_CAPACITY
    img = r.forward(verts=vbig).cpu()
    r.ctx.sync()
    fresh = dsm.Renderer(dict(sc, verts=big))
    fresh.ctx.set_tuning(**shape)
    img_f = fresh.forward().cpu()
    fresh.ctx.sync()
    assert fresh.ctx.raster_stats(0)["pairs"] > pairs_before
    for w, (W, H) in enumerate([(1024, 1024), (64, 64)]):
        a = r.ctx.debug(dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        b = fresh.ctx.debug(dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        assert torch.equal(a, b), f"view {w}"
    assert torch.equal(img, img_f)
