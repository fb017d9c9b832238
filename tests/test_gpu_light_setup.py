"""Light matrices of many seeded random lights against the oracle, bit for bit.

The light setup forms every entry of Q (supplementary Sec. A light cameras:
clip rows 0-3, the depth row of Sec. 3) in float64 with separately rounded
operations and rounds it to float32 once; the oracle's `light_matrix` states
the same operations in the same order.  The per-scene parity cases hold a few
lights each; this sweep draws directional, spot and point lights over the
whole range of their parameters, with a quarter of the directional lights'
directions near the up-vector switch (|f_y| around 0.99), and fills every
light slot and every shadow-map view a call allows (8 lights, 24 views).
"""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O


F64 = torch.float64


def _unit(rng):
    d = rng.normal(size=3)
    return d / np.linalg.norm(d)


def _near_switch(rng):
    # |f_y| drawn around the 0.99 threshold that selects the up vector
    fy = rng.uniform(0.985, 0.995) * rng.choice([-1.0, 1.0])
    phi = rng.uniform(0.0, 2.0 * np.pi)
    s = np.sqrt(1.0 - fy * fy)
    return np.array([s * np.cos(phi), fy, s * np.sin(phi)])


def _directional(rng, i):
    d = _near_switch(rng) if i % 4 == 0 else _unit(rng)
    near = rng.uniform(0.1, 2.0)
    return scenes.directional_light(d, 32, ortho_half=rng.uniform(1.0, 8.0), dist=rng.uniform(4.0, 20.0),
                                    near=near, far=near + rng.uniform(4.0, 40.0), sigma=1.0)


def _spot(rng, i):
    p = rng.uniform(-6.0, 6.0, 3) + np.array([0.0, 6.0, 0.0])
    d = _near_switch(rng) if i % 4 == 0 else _unit(rng)
    near = rng.uniform(0.05, 1.0)
    return scenes.spot_light(p, d, 32, rng.uniform(20.0, 150.0), near=near, far=near + rng.uniform(3.0, 60.0),
                             sigma=1.0)


def _point(rng, i):
    near = rng.uniform(0.05, 0.5)
    return scenes.point_light(rng.uniform(-3.0, 3.0, 3) + np.array([0.0, 2.0, 0.0]), 32, near=near,
                              far=near + rng.uniform(3.0, 30.0), sigma=1.0)


def _light_sets():
    rng = np.random.default_rng(20_231_008)
    sets = []
    for _ in range(3):
        sets.append(("directional", [_directional(rng, i) for i in range(8)]))
        sets.append(("spot", [_spot(rng, i) for i in range(8)]))
    for _ in range(2):
        sets.append(("point", [_point(rng, i) for i in range(4)]))
    sets.append(("mixed", [_directional(rng, 0), _directional(rng, 1), _spot(rng, 0), _spot(rng, 1),
                           _point(rng, 0), _point(rng, 1), _point(rng, 2)]))
    return sets


LIGHT_SETS = _light_sets()


def test_light_sets_fill_the_limits():
    """The sweep reaches the call's limits: 8 lights and 24 views."""
    views = [sum(len(O.light_views(l)) for l in ls) for _, ls in LIGHT_SETS]
    assert max(len(ls) for _, ls in LIGHT_SETS) == 8 and max(views) == 24 and all(v <= 24 for v in views)


@pytest.mark.gpu
@pytest.mark.parametrize("k", range(len(LIGHT_SETS)), ids=[f"{n}{k}" for k, (n, _) in enumerate(LIGHT_SETS)])
def test_random_light_matrices_bit_exact(k):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    kind, lights = LIGHT_SETS[k]
    sc = scenes.tiny_scene(k, 32, 32, "directional", 1)
    sc["lights"] = lights
    r = dsm.Renderer(sc)
    r.forward()
    r.ctx.sync()
    n_views = sum(len(O.light_views(l)) for l in lights)
    Qg = r.ctx.debug(dsm.DBG_Q, 0, (n_views, 20)).cpu().numpy()
    r.ctx.close()
    w = 0
    for li, light in enumerate(lights):
        pos = torch.as_tensor(np.asarray(light["pos"], np.float64), dtype=F64)
        direction = torch.as_tensor(np.asarray(light["dir"], np.float64), dtype=F64)
        for face in O.light_views(light):
            Q32 = O.light_matrix(light, pos, direction, face).numpy().astype(np.float32).reshape(-1)
            assert np.array_equal(Qg[w].view(np.uint32), Q32.view(np.uint32)), (
                f"{kind} light {li} face {face}: entries {np.flatnonzero(Qg[w] != Q32).tolist()} differ")
            w += 1
