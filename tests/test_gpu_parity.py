"""GPU (CUDA path through the C ABI) against the CPU oracle, stage by stage.

Discrete results (light matrices, snapped vertices, triangle ids, depth keys)
must be bit-identical.  Floating-point stages are compared with the oracle fed
the GPU's previous-stage float32 output (a stage-wise comparison): |g - o| <=
1e-5 + 1e-4 |o|.  Gradients: 1e-3 relative (per element above 1e-3 of the
largest, and relative L2)."""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O
from parity_util import ATOL, F64, GpuFrame, assert_close, grad_close, oracle_target

pytestmark = pytest.mark.gpu


def _ragged_camera(sc, W, H):
    sc["camera"] = scenes.look_at_perspective((0.0, 3.0, 4.0), (0.0, 0.5, 0.0), 45.0, W, H)
    return sc


def _evsm(sc, c):
    sc["params"] = dict(sc["params"], moments=1, exponent=c)
    return sc


SCENES = {
    "tiny_dir_ragged": lambda: _ragged_camera(scenes.tiny_scene(0, res=45, img=37), 37, 29),
    "tiny_spot": lambda: scenes.tiny_scene(1, res=40, img=48, kind="spot"),
    "tiny_mixed": lambda: scenes.tiny_scene(2, res=33, img=40, kind="mixed", n_lights=2),
    "tiny_freq3": lambda: _ragged_camera(scenes.tiny_scene(4, res=70, img=64, freq=3), 64, 50),
    "config1": scenes.config1,
    "tiny_point": lambda: scenes.tiny_scene(5, res=32, img=48, kind="point"),
    "tiny_mixed3": lambda: _ragged_camera(scenes.tiny_scene(6, res=40, img=44, kind="mixed3", n_lights=3), 44, 37),
    "tiny_mixed_evsm": lambda: _evsm(scenes.tiny_scene(7, res=40, img=40, kind="mixed", n_lights=2), 10.0),
    "tiny_point_evsm": lambda: _evsm(scenes.tiny_scene(8, res=32, img=40, kind="point"), 20.0),
    # culled and degenerate triangles: zero area, a non-manifold edge, a corner behind the camera, off-screen
    "tiny_degenerate": lambda: scenes.with_degenerate_triangles(
        scenes.tiny_scene(10, res=40, img=44, kind="mixed", n_lights=2)),
    # the smallest sizes: one-texel maps and a one-pixel camera; three-texel maps and a 5x3 camera
    "tiny_res1": lambda: dict(scenes.tiny_scene(11, res=1, img=1, kind="mixed", n_lights=2),
                              camera=scenes.look_at_perspective((0.0, 3.0, 4.0), (0.1, 1.0, -0.1), 45.0, 1, 1)),
    "tiny_res3": lambda: _ragged_camera(scenes.tiny_scene(12, res=3, img=5, kind="mixed", n_lights=2), 5, 3),
    # a dense sphere (2880 triangles within a few tiles): tiles of thousands of records, rastered by
    # several work units whose minima merge in a key slot
    "tiny_dense": lambda: scenes.tiny_scene(16, res=64, img=48, kind="mixed", n_lights=2, freq=12),
}

_cache = {}


def _case(name):
    if name not in _cache:
        sc = SCENES[name]()
        tgt = oracle_target(sc, 0.01, 7)
        gpu = GpuFrame(sc, tgt)
        ref = O.render(sc)
        _cache[name] = (sc, tgt, gpu, ref)
    return _cache[name]


@pytest.fixture(scope="module", params=list(SCENES))
def case(request):
    return _case(request.param)


def test_light_matrices_bit_exact(case):
    sc, _, gpu, ref = case
    if not sc["lights"]:
        return
    Qg = gpu.Q()
    for l, L in enumerate(ref["lights"]):
        assert np.array_equal(Qg[l].view(np.uint32), L["Q32"].reshape(-1).view(np.uint32)), f"light {l}"


def test_snapped_vertices_bit_exact(case):
    sc, _, gpu, ref = case
    setups = [L["setup"] for L in ref["lights"]] + [ref["camera_setup"]]
    for w, st in enumerate(setups):
        X, Y, z, ok = gpu.snap(w)
        vert_ok = np.asarray(ok, bool)
        # the oracle marks invalid vertices through the triangle cull flags; valid ones must agree exactly
        assert np.array_equal(X[vert_ok], st["X"][vert_ok]) and np.array_equal(Y[vert_ok], st["Y"][vert_ok]), w
        assert np.array_equal(z.view(np.uint32), st["zndc"].view(np.uint32)), w


def test_raster_ids_and_keys_bit_exact(case):
    sc, _, gpu, ref = case
    rasters = [L["raster"] for L in ref["lights"]] + [ref["camera_raster"]]
    for w, ras in enumerate(rasters):
        ids, b0, b1, zk = gpu.gbuf(w)
        assert np.array_equal(ids, ras["ids"]), f"view {w}: {np.sum(ids != ras['ids'])} ids differ"
        cov = ids > 0
        assert np.array_equal(zk[cov].view(np.uint32), ras["zkey"][cov].view(np.uint32)), f"view {w} keys"


def test_shadow_map_depth(case):
    sc, _, gpu, ref = case
    for l, L in enumerate(ref["lights"]):
        f = gpu.light_map(gpu.dsm.DBG_F, l)
        assert_close(f, L["f"].detach().numpy(), f"f light {l}")


def test_shadow_map_antialias_stagewise(case):
    sc, _, gpu, ref = case
    tris = sc["tris"].astype(np.int64)
    adj = O.edge_adjacency(tris)
    for l, L in enumerate(ref["lights"]):
        fg = gpu.light_map(gpu.dsm.DBG_F, l)
        ftg = gpu.light_map(gpu.dsm.DBG_FTILDE, l)
        R = sc["lights"][L["light"]]["res"]
        vh = torch.cat([torch.as_tensor(sc["verts"], dtype=F64), torch.ones((len(sc["verts"]), 1), dtype=F64)], 1)
        clip = vh @ L["Q"].detach()[:4].T
        sx, sy = O.screen_coords(clip, R, R)
        exp = O.antialias(torch.as_tensor(fg, dtype=F64), L["raster"], L["setup"],
                          O.silhouette_table(adj, L["setup"]), tris, sx, sy).numpy()
        # the blend weight's float32 error multiplies a channel difference, so
        # the absolute term scales with each channel's magnitude (<= 1 for
        # (f, f^2); up to exp(2c) for the exponential moments)
        scale = np.maximum(np.abs(exp).reshape(-1, 2).max(0), 1.0)
        assert_close(ftg, exp, f"f~ light {l}", atol=ATOL * scale)


def test_moment_filter_stagewise(case):
    sc, _, gpu, ref = case
    for l, L in enumerate(ref["lights"]):
        ftg = gpu.light_map(gpu.dsm.DBG_FTILDE, l)
        mg = gpu.light_map(gpu.dsm.DBG_MOMENTS, l)
        exp = O.separable_filter(torch.as_tensor(ftg, dtype=F64), L["weights"], sc["params"]["filter_boundary"])
        assert_close(mg, exp.numpy(), f"moments light {l}")


def test_shading_stagewise(case):
    sc, _, gpu, ref = case
    teach = {"moments": [gpu.light_map(gpu.dsm.DBG_MOMENTS, l) for l in range(gpu.L)]}
    out = O.render(sc, teacher=teach)
    assert_close(gpu.color(), out["color"].detach().numpy(), "colour before final AA")


def test_final_antialias_stagewise(case):
    sc, _, gpu, ref = case
    tris = sc["tris"].astype(np.int64)
    cam = sc["camera"]
    vh = torch.cat([torch.as_tensor(sc["verts"], dtype=F64), torch.ones((len(sc["verts"]), 1), dtype=F64)], 1)
    clip = vh @ torch.as_tensor(np.asarray(cam["clip"], np.float32), dtype=F64).T
    sx, sy = O.screen_coords(clip, cam["width"], cam["height"])
    st = ref["camera_setup"]
    exp = O.antialias(torch.as_tensor(gpu.color(), dtype=F64), ref["camera_raster"], st,
                      O.silhouette_table(O.edge_adjacency(tris), st), tris, sx, sy).numpy()
    assert_close(gpu.image.cpu().numpy(), exp, "image")


def test_gradients_stagewise(case):
    sc, tgt, gpu, ref = case
    teach = {"ftilde": [gpu.light_map(gpu.dsm.DBG_FTILDE, l) for l in range(gpu.L)],
             "moments": [gpu.light_map(gpu.dsm.DBG_MOMENTS, l) for l in range(gpu.L)],
             "color": gpu.color()}
    res = O.render_and_grad(sc, tgt, teacher=teach)
    assert abs(float(gpu.loss.item()) - float(res["loss"])) <= 1e-5 + 1e-4 * abs(float(res["loss"]))
    grad_close(gpu.dalbedo.cpu().numpy(), res["grad_albedo"].numpy(), "dL/dalbedo")
    grad_close(gpu.dlight.cpu().numpy(), res["grad_light"].numpy(), "dL/dlight")
    grad_close(gpu.dverts.cpu().numpy(), res["grad_verts"].numpy(), "dL/dverts")


def test_end_to_end_image(case):
    """Whole forward with no stage substitution.  Tolerance derived from float32
    moments: sigma^2 = m2 - m1^2 inherits ~3e-8 absolute error, and
    |dv/dsigma^2|, |dv/dmu| <= 0.65 / sigma_min, so pixels may differ by
    ~1e-3 where sigma^2 sits at its floor."""
    sc, _, gpu, ref = case
    assert_close(gpu.image.cpu().numpy(), ref["image"].detach().numpy(), "end-to-end image", atol=2e-3, rtol=1e-3)
