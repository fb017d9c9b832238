"""Kernel shapes (dsm_tuning) and the autotuner.

The shapes change only the speed: the raster is exact and order independent
and both filter shapes take the taps in the same order, so every image is
bit-identical whatever the raster tile (16 or 32 per view kind), the bin
depth (big-triangle threshold) or the filter shape; gradients agree up to the
order of float atomics (the big-triangle scatter and the adjoint filter's
pass order change the summation order)."""
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

SHAPES = [dict(light_tile=16, camera_tile=16, big_tiles=16, filter_shape=0),
          dict(light_tile=32, camera_tile=16, big_tiles=4, filter_shape=1),
          dict(light_tile=16, camera_tile=32, big_tiles=64, filter_shape=1),
          dict(light_tile=32, camera_tile=32, big_tiles=2, filter_shape=0),
          dict(light_tile=32, camera_tile=16, big_tiles=16, filter_shape=2)]


def _ragged(sc, W, H):
    sc["camera"] = scenes.look_at_perspective((0.0, 3.0, 4.0), (0.0, 0.5, 0.0), 45.0, W, H)
    return sc


SCENES = {
    "tiny_mixed": lambda: scenes.tiny_scene(2, res=33, img=40, kind="mixed", n_lights=2),
    "tiny_spot_ragged": lambda: _ragged(scenes.tiny_scene(1, res=70, img=48, kind="spot", freq=3), 37, 29),
    "config1": scenes.config1,
}


def _rel(a, b):
    a, b = a.double().reshape(-1), b.double().reshape(-1)
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def _step(dsm, r, gseed):
    img = r.forward().clone()
    g = torch.randn(img.shape, generator=torch.Generator().manual_seed(gseed)).cuda()
    dv, dl, da = r.backward(g)
    r.ctx.sync()
    return img.cpu(), dv.cpu(), dl.cpu(), da.cpu()


@pytest.mark.parametrize("name", list(SCENES))
def test_shapes_do_not_change_results(name):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    r = dsm.Renderer(SCENES[name]())
    assert r.ctx.get_tuning() == dict(light_tile=32, camera_tile=32, big_tiles=16, filter_shape=0)
    ref = _step(dsm, r, 3)
    for shape in SHAPES:
        r.ctx.set_tuning(**shape)
        assert r.ctx.get_tuning() == shape
        got = _step(dsm, r, 3)
        assert torch.equal(got[0], ref[0]), f"{shape}: image differs"
        for k, what in ((1, "verts"), (2, "light"), (3, "albedo")):
            assert _rel(got[k], ref[k]) <= 1e-4, f"{shape}: dL/d{what} rel {_rel(got[k], ref[k])}"


def test_bad_shapes_rejected():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    r = dsm.Renderer(SCENES["tiny_mixed"]())
    for bad in (dict(light_tile=8), dict(camera_tile=64), dict(big_tiles=1), dict(filter_shape=3)):
        with pytest.raises(dsm.DsmError):
            r.ctx.set_tuning(**bad)


def test_autotune_picks_valid_shapes_and_keeps_results():
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = SCENES["config1"]()
    r = dsm.Renderer(sc)
    ref = _step(dsm, r, 5)
    best, ms = r.autotune(reps=2)
    assert best["light_tile"] in (16, 32) and best["camera_tile"] in (16, 32)
    assert best["big_tiles"] in (4, 16, 64) and best["filter_shape"] in (0, 1, 2)
    assert ms > 0.0
    assert r.ctx.get_tuning() == best
    got = _step(dsm, r, 5)
    assert torch.equal(got[0], ref[0])
    assert _rel(got[1], ref[1]) <= 1e-4


def test_autotune_cache_round_trip(tmp_path):
    """Shapes found by the search are stored under the scene's shape class and
    read back by the next renderer of that class without a search."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    cache = str(tmp_path / "shapes.json")
    r = dsm.Renderer(SCENES["tiny_mixed"]())
    best, ms = r.autotune(reps=1, cache=cache)
    assert ms is not None and ms > 0.0
    r2 = dsm.Renderer(SCENES["tiny_mixed"]())
    r2.ctx.set_tuning(light_tile=16, camera_tile=16, big_tiles=4, filter_shape=1)
    got, ms2 = r2.autotune(reps=1, cache=cache)
    assert ms2 is None and got == best and r2.ctx.get_tuning() == best
