"""The torch.autograd.Function over the C ABI (``dsm.DSMFunction`` through
``dsm.render``): the paper obtains its gradients with PyTorch's reverse mode
(Sec. 5), and this is the same interface over the library's own backward.

- ``.grad`` of a torch loss equals the C ABI backward of that loss's dL/dimage;
- with every forward stage taught and the silhouette bands masked, ``.grad``
  matches the oracle's gradient element by element within 1e-3;
- a directional central difference of the GPU forward (float32, h = 1e-3 world
  units) along vertex displacements away from silhouettes equals the
  directional derivative from ``.grad``."""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O
from parity_util import GpuFrame, camera_band, grad_close_strict, loss_tolerance, oracle_target, report

pytestmark = pytest.mark.gpu

SCENES = {
    "tiny_mixed": lambda: scenes.tiny_scene(2, res=33, img=40, kind="mixed", n_lights=2),
    "tiny_point": lambda: scenes.tiny_scene(5, res=32, img=48, kind="point"),
}


def _inputs(r):
    v = r.verts.clone().requires_grad_(True)
    lp = r.light_params.clone().requires_grad_(True)
    al = r.albedo.clone().requires_grad_(True)
    return v, lp, al


@pytest.mark.parametrize("name", list(SCENES))
def test_autograd_grad_equals_c_abi_backward(name):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = SCENES[name]()
    tgt = torch.as_tensor(oracle_target(sc, 0.01, 7).astype(np.float32), device="cuda")
    r = dsm.Renderer(sc)
    v, lp, al = _inputs(r)
    img = dsm.render(v, lp, al, r)
    loss = ((img - tgt) ** 2).mean()
    loss.backward()
    # the same loss through the C ABI: dsm_l2_loss_grad, then dsm_render_backward
    image = r.forward()
    lbuf = torch.zeros(1, device="cuda")
    gimg = torch.empty_like(image)
    dsm.l2_loss_grad(image, tgt, lbuf, gimg)
    dv, dl, da = r.backward(gimg)
    r.ctx.sync()
    assert torch.equal(img.detach(), image), "forward differs between the autograd and the C ABI call"
    assert abs(float(loss.detach()) - float(lbuf.item())) <= 1e-6 * abs(float(loss.detach())) + 1e-12
    rec = {"test": "autograd_vs_c_abi", "case": name}
    for nm, a, b in (("verts", v.grad, dv), ("light", lp.grad, dl), ("albedo", al.grad, da)):
        assert a is not None and a.shape == b.shape, nm
        rel = float((a - b).norm() / max(float(b.norm()), 1e-30))
        rec[nm] = rel
        # the two dL/dimage differ only in the rounding of 2 (image - target) / N,
        # and the backward's float atomics sum in a run-dependent order
        assert rel <= 1e-5, f"dL/d{nm}: autograd vs C ABI relative L2 {rel:.3g}"
    report(rec)


@pytest.mark.parametrize("name", list(SCENES))
def test_autograd_grad_matches_oracle_outside_silhouette_band(name):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = SCENES[name]()
    tgt = oracle_target(sc, 0.01, 7)
    gpu = GpuFrame(sc)
    ref = O.render(sc)
    band = torch.as_tensor(camera_band(sc, ref), device="cuda")
    v, lp, al = _inputs(gpu.r)
    img = dsm.render(v, lp, al, gpu.r)
    # dL/dimage of the mean squared error, zero on the camera's silhouette band
    G = (2.0 * (img.detach() - torch.as_tensor(tgt.astype(np.float32), device="cuda")) / img.numel())
    G[band] = 0.0
    teach = gpu.full_teacher()
    gpu.r.ctx.set_grad_mask(dsm.GRAD_MASK_SM_BAND)
    try:
        (img * G).sum().backward()
        gpu.r.ctx.sync()
    finally:
        gpu.r.ctx.set_grad_mask(0)
    res = O.render_and_grad(sc, tgt, teacher=teach, grad_image=G.cpu().numpy(), grad_mask_sm_band=True)
    rec = {"test": "autograd_vs_oracle_outside_band", "case": name}
    for nm, a, o in (("verts", v.grad, res["grad_verts"]), ("light", lp.grad, res["grad_light"]),
                     ("albedo", al.grad, res["grad_albedo"])):
        rec[nm] = grad_close_strict(a.double().cpu().numpy(), o.numpy(), f"autograd dL/d{nm}")
    report(rec)


def _loss64(img, tgt):
    d = img.double() - tgt
    return float((d * d).mean())


FD_SCENES = {
    "tiny_freq3": lambda: scenes.tiny_scene(4, res=70, img=64, freq=3),
    "tiny_mixed_f3": lambda: scenes.tiny_scene(2, res=48, img=48, kind="mixed", n_lights=2, freq=3),
    "tiny_point": lambda: scenes.tiny_scene(5, res=32, img=48, kind="point"),
    "config1": scenes.config1,
}


def _free_direction(sc, ref, seed):
    """A random normal displacement of the vertices away from silhouettes:
    zero on every vertex of a triangle that owns a pixel of a silhouette band
    (camera or shadow map), and on the one-ring around them, so that no moving
    edge reaches a band pixel (where a new owner would switch an antialiasing
    crossing on or off)."""
    tris = sc["tris"].astype(np.int64)
    adj = O.edge_adjacency(tris)
    touched = set()
    for ras, st in [(L["raster"], L["setup"]) for L in ref["lights"]] + [(ref["camera_raster"],
                                                                         ref["camera_setup"])]:
        band = O.silhouette_band(ras, O.silhouette_table(adj, st))
        touched |= set(int(t) - 1 for t in np.unique(ras["ids"][band]) if t > 0)
    frozen = np.zeros(sc["verts"].shape[0], bool)
    if touched:
        frozen[tris[sorted(touched)].ravel()] = True
    frozen[tris[frozen[tris].any(1)].ravel()] = True
    rng = np.random.default_rng(100 + seed)
    return rng.normal(size=sc["verts"].shape) * (~frozen)[:, None], int((~frozen).sum())


@pytest.mark.parametrize("name,seed", [("tiny_freq3", 0), ("tiny_mixed_f3", 1), ("tiny_mixed_f3", 2),
                                       ("tiny_point", 1), ("config1", 0), ("config1", 2)])
def test_central_difference_of_gpu_forward(name, seed):
    """(L(v + h e) - L(v - h e)) / 2h of the GPU forward against grad . e from
    DSMFunction, with L the mean squared error evaluated in float64 from the
    float32 images and h = 1e-3 world units (well above float32 rounding).
    e moves only vertices away from silhouettes (``_free_direction``).  The
    method still has non-smooth events (reading 4: a triangle edge crossing a
    point-light cube-face boundary, a sub-pixel triangle taking a pixel), so
    the oracle first confirms in float64 that none lies within h along e: its
    own central difference at the same h equals its gradient within 1e-2.
    Bound for the GPU: 1e-2 relative (the same O(h^2) truncation) plus the
    float32 rounding of the two images, 2^-22 sum |dL/dimage| |image| / 2h."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = FD_SCENES[name]()
    tgt_np = oracle_target(sc, 0.01, 7)
    tgt = torch.as_tensor(tgt_np, device="cuda")
    ref = O.render(sc)
    e, free = _free_direction(sc, ref, seed)
    assert free >= 8, "too few vertices away from the silhouettes"
    h = 1e-3
    # the oracle: no non-smooth event within h along e
    go = O.render_and_grad(sc, tgt_np)["grad_verts"].numpy()
    dd_o = float((go * e).sum())
    fd_o = (float(O.mse_loss(O.render(sc, verts=torch.as_tensor(sc["verts"] + h * e), keep=False)["image"], tgt_np))
            - float(O.mse_loss(O.render(sc, verts=torch.as_tensor(sc["verts"] - h * e), keep=False)["image"],
                               tgt_np))) / (2 * h)
    assert abs(fd_o - dd_o) <= 1e-2 * abs(dd_o), f"oracle: a non-smooth event within h ({fd_o:.6g} vs {dd_o:.6g})"
    r = dsm.Renderer(sc)
    v, lp, al = _inputs(r)
    img = dsm.render(v, lp, al, r)
    ((img.double() - tgt) ** 2).mean().backward()
    dd = float((v.grad.double().cpu().numpy() * e).sum())
    et = torch.as_tensor(e, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        lp_ = _loss64(r.forward(verts=(r.verts + h * et).contiguous()), tgt)
        lm_ = _loss64(r.forward(verts=(r.verts - h * et).contiguous()), tgt)
    fd = (lp_ - lm_) / (2 * h)
    gl = (2.0 * (img.detach().double() - tgt) / img.numel()).abs()
    noise = 2.0 ** -22 * float((gl * img.detach().double().abs()).sum()) / (2 * h)
    report({"test": "central_difference", "case": name, "seed": seed, "fd": fd, "grad_dot_e": dd,
            "oracle_fd": fd_o, "oracle_grad_dot_e": dd_o, "rounding_bound": noise, "free_vertices": free})
    assert abs(fd - dd) <= 1e-2 * abs(dd) + noise, f"central difference {fd:.6g} vs grad . e {dd:.6g}"
    assert abs(fd - fd_o) <= 1e-2 * abs(fd_o) + noise, f"GPU central difference {fd:.6g} vs oracle's {fd_o:.6g}"


@pytest.mark.parametrize("name", list(SCENES))
def test_l2_backward_equals_loss_then_backward(name):
    """dsm_render_backward_l2 (the mean squared error's backward, dL/dimage
    formed where it is read) against dsm_l2_loss_grad followed by
    dsm_render_backward: the same loss within the two float sums' rounding
    bound (parity_util.loss_tolerance), the same gradients up to the order of
    the float atomics."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = SCENES[name]()
    tgt = torch.as_tensor(oracle_target(sc, 0.01, 7).astype(np.float32), device="cuda")
    r = dsm.Renderer(sc)
    image = r.forward()
    lbuf = torch.zeros(1, device="cuda")
    gimg = torch.empty_like(image)
    dsm.l2_loss_grad(image, tgt, lbuf, gimg)
    ref = [x.clone() for x in r.backward(gimg)]
    loss = torch.full((1,), -1.0, device="cuda")
    got = r.backward_l2(image, tgt, loss)
    r.ctx.sync()
    rec = {"test": "l2_backward", "case": name, "loss": float(loss.item()), "loss_ref": float(lbuf.item())}
    assert abs(float(loss.item()) - float(lbuf.item())) <= loss_tolerance(image.numel(), float(lbuf.item()))
    for nm, a, b in zip(("verts", "light", "albedo"), got, ref):
        rel = float((a - b).norm() / max(float(b.norm()), 1e-30))
        rec[nm] = rel
        assert rel <= 1e-5, f"dL/d{nm}: fused loss backward vs loss then backward, relative L2 {rel:.3g}"
    report(rec)
