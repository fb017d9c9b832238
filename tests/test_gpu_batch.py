"""Batched frames (dsm_batch_step): every scene's forward, L2 loss and backward
in one call, replayed from a CUDA graph after the first step, give the same
results as rendering each scene on its own (dsm_render, dsm_l2_loss_grad,
dsm_render_backward): images identical (the forward has no order-dependent
arithmetic), losses equal within the rounding bound of their two float sums
(the batch takes the loss from dsm_render_backward_l2), gradients equal up to
the order of float atomics.
Device data changed between steps is picked up by the replayed graph."""
import numpy as np
import pytest
import torch

import scenes
from parity_util import loss_tolerance

pytestmark = pytest.mark.gpu


def _scenes():
    sc = [scenes.tiny_scene(11, res=40, img=48, kind="mixed", n_lights=2),
          scenes.tiny_scene(12, res=64, img=32, kind="spot"),
          scenes.config1(),
          scenes.tiny_scene(13, res=33, img=40, freq=3)]
    for s in sc:          # one dsm_params serves the whole batch
        s["params"] = dict(sc[0]["params"])
    return sc


def _single(dsm, sc, verts, target):
    r = dsm.Renderer(sc)
    img = r.forward(verts=verts)
    loss = torch.zeros(1, device="cuda")
    gimg = torch.empty_like(img)
    dsm.l2_loss_grad(img, target, loss, gimg)
    dv, dl, da = r.backward(gimg)
    torch.cuda.synchronize()
    return img.cpu(), float(loss.item()), dv.cpu(), dl.cpu(), da.cpu()


def _rel(a, b):
    a, b = a.double().reshape(-1), b.double().reshape(-1)
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def test_batch_matches_single_renders_and_follows_device_data():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    scs = _scenes()
    targets = []
    for k, sc in enumerate(scs):
        r = dsm.Renderer(sc)
        jit = torch.as_tensor(scenes.jitter_vertices(sc, 0.01, 50 + k), device="cuda")
        targets.append(r.forward(verts=jit).clone().cpu().numpy())
    b = dsm.Batch(scs, targets)
    for step in range(3):
        if step == 2:
            # new vertex positions in the same device buffers: the replayed graph must see them
            with torch.cuda.stream(b.stream):
                for d in b.scenes:
                    d["verts"].mul_(1.01)
        b.step()
        b.stream.synchronize()
        b.sync()
        for k, (sc, d) in enumerate(zip(scs, b.scenes)):
            tgt = torch.as_tensor(targets[k], device="cuda")
            img, loss, dv, dl, da = _single(dsm, sc, d["verts"].clone(), tgt)
            assert torch.equal(d["image"].cpu(), img), f"step {step} scene {k}: image differs"
            assert abs(float(d["loss"].item()) - loss) <= loss_tolerance(img.numel(), loss), \
                f"step {step} scene {k}: loss"
            L = len(sc["lights"])
            for name, g, o in (("verts", d["dverts"].cpu(), dv), ("light", d["dlight"][:L].cpu(), dl),
                               ("albedo", d["dalbedo"].cpu(), da)):
                assert _rel(g, o) <= 1e-4, f"step {step} scene {k}: dL/d{name} rel {_rel(g, o)}"
    assert b.kernels_per_step() > 0
    b.close()


def test_batch_autotune_keeps_results():
    """Per-scene autotuning, then a recorded step: images as single renders
    with the default shapes, gradients up to atomic order."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    scs = _scenes()[:3]
    targets = []
    for k, sc in enumerate(scs):
        r = dsm.Renderer(sc)
        jit = torch.as_tensor(scenes.jitter_vertices(sc, 0.01, 70 + k), device="cuda")
        targets.append(r.forward(verts=jit).clone().cpu().numpy())
    b = dsm.Batch(scs, targets)
    b.step()
    b.autotune(reps=1)
    assert len(b.tunings()) == len(scs)
    for _ in range(2):
        b.step()
    b.stream.synchronize()
    b.sync()
    for k, (sc, d) in enumerate(zip(scs, b.scenes)):
        tgt = torch.as_tensor(targets[k], device="cuda")
        img, loss, dv, dl, da = _single(dsm, sc, d["verts"].clone(), tgt)
        assert torch.equal(d["image"].cpu(), img), f"scene {k}: image differs"
        assert _rel(d["dverts"].cpu(), dv) <= 1e-4
    b.close()


def test_single_scene_batch_records_its_view_streams():
    """A batch of one scene records its views on their own streams (fork and
    join events inside the graph): same images as single renders, gradients up
    to atomic order, and replays follow changed vertex buffers."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = scenes.tiny_scene(14, res=48, img=40, kind="mixed3", n_lights=3)
    r = dsm.Renderer(sc)
    jit = torch.as_tensor(scenes.jitter_vertices(sc, 0.01, 81), device="cuda")
    target = r.forward(verts=jit).clone().cpu().numpy()
    b = dsm.Batch([sc], [target])
    d = b.scenes[0]
    for step in range(3):
        if step == 2:
            with torch.cuda.stream(b.stream):
                d["verts"].mul_(0.99)
        b.step()
        b.stream.synchronize()
        b.sync()
        img, loss, dv, dl, da = _single(dsm, sc, d["verts"].clone(), torch.as_tensor(target, device="cuda"))
        assert torch.equal(d["image"].cpu(), img), f"step {step}: image differs"
        assert abs(float(d["loss"].item()) - loss) <= loss_tolerance(img.numel(), loss)
        assert _rel(d["dverts"].cpu(), dv) <= 1e-4 and _rel(d["dlight"][:3].cpu(), dl) <= 1e-4
    b.close()


def test_host_staging_inside_the_recorded_step():
    """Pinned host inputs are uploaded by the recorded step itself and the
    loss is downloaded by it: new host values are picked up by a replay, and
    the result equals a step on the same values uploaded by hand."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = scenes.tiny_scene(15, res=40, img=36, kind="mixed", n_lights=2)
    r = dsm.Renderer(sc)
    target = r.forward(verts=torch.as_tensor(scenes.jitter_vertices(sc, 0.01, 5), device="cuda")).clone()
    b = dsm.Batch([sc], [target.cpu().numpy()])
    d = b.scenes[0]
    h_verts = torch.as_tensor(sc["verts"], dtype=torch.float32).contiguous().pin_memory()
    h_lp = d["light_params"].cpu().contiguous().pin_memory()
    h_alb = d["albedo"].cpu().contiguous().pin_memory()
    h_loss = torch.full((1,), -1.0).pin_memory()
    b.set_host_io(0, verts=h_verts, light_params=h_lp, albedo=h_alb, loss=h_loss)
    for step in range(3):
        h_verts.mul_(1.0 + 0.01 * step)       # new host values before every step
        h_alb.mul_(0.98)
        b.step()
        b.stream.synchronize()
        b.sync()
        assert torch.equal(d["verts"].cpu(), h_verts) and torch.equal(d["albedo"].cpu(), h_alb)
        img, loss, dv, dl, da = _single(dsm, dict(sc, albedo=h_alb.numpy()), h_verts.cuda(), target)
        assert torch.equal(d["image"].cpu(), img), f"step {step}: image differs"
        assert float(h_loss[0]) == float(d["loss"].item())
        assert abs(float(h_loss[0]) - loss) <= loss_tolerance(img.numel(), loss)
        assert _rel(d["dverts"].cpu(), dv) <= 1e-4
    with pytest.raises(ValueError):
        b.set_host_io(0, verts=torch.zeros(3))   # not pinned
    b.close()
