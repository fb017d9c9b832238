"""Several cameras under the same lights (dsm_render_cameras) and the
recompute-in-backward mode.

- Each camera's image from one multi-camera forward is bit-identical to a
  single-camera dsm_render of that camera (the light maps do not depend on the
  camera and the forward has no order-dependent arithmetic).
- The multi-camera backward of sum_c <g_c, image_c> equals the sum of the
  single-camera backwards up to the order of float atomics.
- With recompute_in_backward = 1 (views share one light and one camera buffer
  set; the backward rasterises every view again and filters the moment maps
  again) images are bit-identical and gradients equal up to atomic order, and
  the context holds less device memory once there are several views."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def _scene():
    sc = scenes.tiny_scene(21, res=48, img=40, kind="mixed", n_lights=3, freq=3)
    sc["lights"][1]["res"] = 64
    sc["lights"][2]["res"] = 33
    cams = [scenes.look_at_perspective((0.0, 3.0, 4.0), (0.0, 0.5, 0.0), 45.0, 40, 40),
            scenes.look_at_perspective((3.5, 2.5, -1.0), (0.0, 0.6, 0.0), 50.0, 56, 36),
            scenes.look_at_perspective((-2.0, 4.0, 2.5), (0.2, 0.4, 0.0), 40.0, 33, 47)]
    return sc, cams


def _rel(a, b):
    a, b = a.double().reshape(-1), b.double().reshape(-1)
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def _grads(seed, cams):
    g = torch.Generator().manual_seed(seed)
    return [torch.randn((int(c["height"]), int(c["width"]), 4), generator=g).cuda() for c in cams]


def _multi(dsm, sc, cams, gimgs, recompute):
    sc = dict(sc)
    sc["params"] = dict(sc["params"], recompute_in_backward=recompute)
    r = dsm.Renderer(sc)
    imgs = [im.clone() for im in r.forward_cameras(cams)]
    dv, dl, da = r.backward_cameras(gimgs)
    torch.cuda.synchronize()
    r.ctx.sync()
    return r, [im.cpu() for im in imgs], dv.cpu(), dl.cpu(), da.cpu()


def test_cameras_match_single_renders():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, cams = _scene()
    gimgs = _grads(5, cams)
    _, imgs, dv, dl, da = _multi(dsm, sc, cams, gimgs, 0)
    r1 = dsm.Renderer(sc)
    sv, sl, sa = 0, 0, 0
    for c, cam in enumerate(cams):
        r1.set_camera(cam)
        img = r1.forward()
        assert torch.equal(imgs[c], img.cpu()), f"camera {c}: image differs from a single-camera render"
        v, l, a = r1.backward(gimgs[c])
        sv, sl, sa = sv + v.double().cpu(), sl + l.double().cpu(), sa + a.double().cpu()
    for name, got, exp in (("verts", dv, sv), ("light", dl, sl), ("albedo", da, sa)):
        assert _rel(got, exp) <= 1e-4, f"dL/d{name}: rel {_rel(got, exp)}"


@pytest.mark.parametrize("n_cams", [1, 3])
def test_recompute_matches_stored(n_cams):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, cams = _scene()
    cams = cams[:n_cams]
    gimgs = _grads(9, cams)
    rs, imgs_s, dv_s, dl_s, da_s = _multi(dsm, sc, cams, gimgs, 0)
    rr, imgs_r, dv_r, dl_r, da_r = _multi(dsm, sc, cams, gimgs, 1)
    for c in range(n_cams):
        assert torch.equal(imgs_s[c], imgs_r[c]), f"camera {c}: recomputation changed the image"
    for name, got, exp in (("verts", dv_r, dv_s), ("light", dl_r, dl_s), ("albedo", da_r, da_s)):
        assert _rel(got, exp) <= 1e-4, f"dL/d{name}: rel {_rel(got, exp)}"
    # the moment maps kept for the debug copy are the same maps
    for l, Lt in enumerate(sc["lights"]):
        R = Lt["res"]
        assert torch.equal(rs.ctx.debug(dsm.DBG_MOMENTS, l, (R, R, 2)), rr.ctx.debug(dsm.DBG_MOMENTS, l, (R, R, 2)))
    with pytest.raises(dsm.DsmError):
        rr.ctx.debug(dsm.DBG_GBUF, 0, (sc["lights"][0]["res"],) * 2 + (4,))
    if n_cams > 1:
        assert rr.ctx.memory_bytes() < rs.ctx.memory_bytes()


def test_recompute_second_step_follows_new_vertices():
    """Two steps on one context: the recomputing backward reads the current
    vertex buffer, like the stored mode."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, cams = _scene()
    gimgs = _grads(13, cams)
    out = {}
    for mode in (0, 1):
        s2 = dict(sc)
        s2["params"] = dict(sc["params"], recompute_in_backward=mode)
        r = dsm.Renderer(s2)
        v = r.verts.clone()
        imgs = []
        for step in range(2):
            imgs = [im.cpu() for im in r.forward_cameras(cams, verts=v)]
            dv, _, _ = r.backward_cameras(gimgs)
            v.mul_(1.01)   # same buffer, new values
        torch.cuda.synchronize()
        out[mode] = (imgs, dv.cpu())
    for c in range(len(cams)):
        assert torch.equal(out[1][0][c], out[0][0][c])
    assert _rel(out[1][1], out[0][1]) <= 1e-4


def test_camera_count_checked():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, cams = _scene()
    r = dsm.Renderer(sc)
    with pytest.raises(dsm.DsmError):
        r.forward_cameras([cams[0]] * (dsm.MAX_CAMERAS + 1))
    r.forward_cameras(cams[:2])
    with pytest.raises(dsm.DsmError):   # the single-camera backward after a two-camera forward
        r.backward(torch.zeros((40, 40, 4), device="cuda"))


def test_cameras_against_oracle():
    """Three cameras, two lights, against the oracle's summed loss: each
    camera's colour stage-wise (1e-5 + 1e-4 |o|), images end to end (the
    derived image bound) and gradients with the GPU's stage values as teachers
    (the oracle's derivatives of every stage)."""
    from paper_2308_10896_b300 import dsm
    from oracle import dsm_oracle as O
    from parity_util import assert_close, grad_close
    torch.cuda.set_device(0)
    sc = scenes.tiny_scene(22, res=40, img=32, kind="mixed", n_lights=2)
    cams = [sc["camera"],
            scenes.look_at_perspective((3.0, 2.5, -1.5), (0.0, 0.6, 0.0), 50.0, 36, 28),
            scenes.look_at_perspective((-2.0, 3.5, 2.0), (0.1, 0.4, 0.0), 45.0, 30, 41)]
    jit = scenes.jitter_vertices(sc, 0.01, 17)
    tg = [O.render(dict(sc, camera=c), verts=torch.as_tensor(jit, dtype=torch.float64), keep=False)["image"]
          .detach().numpy() for c in cams]
    r = dsm.Renderer(sc)
    imgs = r.forward_cameras(cams)
    gimgs, loss = [], 0.0
    for im, t in zip(imgs, tg):
        l1 = torch.zeros(1, device="cuda")
        g = torch.empty_like(im)
        dsm.l2_loss_grad(im, torch.as_tensor(t, dtype=torch.float32, device="cuda"), l1, g)
        loss += float(l1.item())
        gimgs.append(g)
    dv, dl, da = r.backward_cameras(gimgs)
    r.ctx.sync()
    L = len(sc["lights"])
    light = [(Lt["res"],) * 2 + (2,) for Lt in sc["lights"]]
    ftilde = [r.ctx.debug(dsm.DBG_FTILDE, l, light[l]).cpu().numpy() for l in range(L)]
    mom = [r.ctx.debug(dsm.DBG_MOMENTS, l, light[l]).cpu().numpy() for l in range(L)]
    teach = [{"ftilde": ftilde, "moments": mom,
              "color": r.ctx.debug(dsm.DBG_COLOR, c, (cam["height"], cam["width"], 4)).cpu().numpy()}
             for c, cam in enumerate(cams)]
    ref = O.render_cameras_and_grad(sc, cams, tg, teachers=teach)
    plain = O.render_cameras_and_grad(sc, cams, tg)
    for c, cam in enumerate(cams):
        # stage-wise: each camera's colour from the GPU's moment maps and shading-stage values
        W, H = int(cam["width"]), int(cam["height"])
        surf = r.ctx.probe_surface(c, W, H).cpu().numpy()
        st_teach = {"moments": mom, "x": surf[:, :, 0, :3], "n": surf[:, :, 1, :3],
                    "lookup": [r.ctx.probe_lookup(c, l, W, H).cpu().numpy().reshape(H, W, 8) for l in range(L)]}
        out = O.render(dict(sc, camera=cam), teacher=st_teach)
        assert_close(teach[c]["color"], out["color"].detach().numpy(), f"camera {c} colour")
        # end to end: the derived image bound (float32 sigma^2 near its floor)
        assert_close(imgs[c].cpu().numpy(), plain["images"][c].numpy(), f"camera {c} image", atol=2e-3, rtol=1e-3)
    assert abs(loss - float(ref["loss"])) <= 1e-5 + 1e-4 * abs(float(ref["loss"]))
    grad_close(da.cpu().numpy(), ref["grad_albedo"].numpy(), "dL/dalbedo")
    grad_close(dl.cpu().numpy(), ref["grad_light"].numpy(), "dL/dlight")
    grad_close(dv.cpu().numpy(), ref["grad_verts"].numpy(), "dL/dverts")


def test_adam_step_against_oracle():
    from paper_2308_10896_b300 import dsm
    from oracle import dsm_oracle as O
    torch.cuda.set_device(0)
    rng = np.random.default_rng(31)
    n = 100_003   # ragged against the block size
    p0 = rng.normal(size=n)
    gs = rng.normal(size=(5, n)) * np.logspace(-4, 1, n)
    p = torch.as_tensor(p0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    po, mo, vo = p.double().cpu().numpy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g32 = torch.as_tensor(gs[t - 1], dtype=torch.float32)
        dsm.adam_step(p, g32.cuda(), m, v, t, lr=1e-3)
        po, mo, vo = O.adam_step(po, g32.double().numpy(), mo, vo, t, lr=1e-3)
    torch.cuda.synchronize()
    # float32 moments: m is a sum of terms of size |g|, so its rounding is
    # relative to the gradient scale of the element (m may cancel to ~0)
    scale = np.abs(gs).max(0)
    np.testing.assert_allclose(p.cpu().double().numpy(), po, rtol=0, atol=2e-6)
    assert np.all(np.abs(m.cpu().double().numpy() - mo) <= 1e-6 * scale + 1e-5 * np.abs(mo))
    assert np.all(np.abs(v.cpu().double().numpy() - vo) <= 1e-6 * scale ** 2 + 1e-5 * np.abs(vo))
    with pytest.raises(dsm.DsmError):
        dsm.adam_step(p, m, m, v, 0)


def test_second_backward_after_one_forward():
    """The forward zeroes the shadow-map gradient accumulators for the first
    backward; a second backward of the same forward zeroes them itself and
    gives the same gradients (up to the order of float atomics)."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, cams = _scene()
    r = dsm.Renderer(sc)
    imgs = r.forward_cameras(cams)
    gimgs = _grads(21, cams)
    first = [t.clone() for t in r.backward_cameras(gimgs)]
    second = [t.clone() for t in r.backward_cameras(gimgs)]
    torch.cuda.synchronize()
    for a, b, name in zip(first, second, ("verts", "light", "albedo")):
        assert _rel(b.cpu(), a.cpu()) <= 1e-5, f"dL/d{name} differs on the second backward"
