"""The rasteriser's ids and depth keys on adversarial geometry, bit for bit
against the oracle (Eq. 1: the nearest surface per pixel centre, with the
top-left fill rule and the (depth, triangle) key).

A directional light looking straight down with ortho_half = 4 maps world x
and z onto a 64 x 64 shadow map by exact float32 operations: a vertex whose x
and z are multiples of 1/16 snaps exactly onto a texel centre or a texel edge.
Each scene mixes:
- a grid of quads split into triangles with alternating diagonals: shared
  edges through texel centres, every centre covered exactly once;
- small random triangles on the same dyadic grid at three heights, so that
  coplanar overlaps tie on depth and the triangle index decides;
- slivers (one edge a sixteenth of a texel) and a few triangles spanning
  most of the map (the int64 edge steps, the big-triangle binning);
and is rastered with 32- and 16-texel tiles, and with every large triangle
binned as big.  The camera rasters the same soup in perspective, and a
48 x 48 map (texels of 1/6) gives ragged tiles without exact alignment.
"""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O


SHAPES = [(32, 16), (16, 16), (32, 2), (16, 2)]   # (tile side, big_tiles)
_refs = {}


def _ref(seed):
    if seed not in _refs:
        sc = scenes.triangle_soup(seed)
        _refs[seed] = (sc, O.render(sc))
    return _refs[seed]


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("tile,big", SHAPES, ids=[f"tile{t}_big{b}" for t, b in SHAPES])
def test_adversarial_raster_bit_exact(seed, tile, big):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, ref = _ref(seed)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(light_tile=tile, camera_tile=tile, big_tiles=big)
    r.forward()
    r.ctx.sync()
    rasters = [L["raster"] for L in ref["lights"]] + [ref["camera_raster"]]
    sizes = [(L["res"], L["res"]) for L in sc["lights"]] + [(sc["camera"]["width"], sc["camera"]["height"])]
    for w, (ras, (W, H)) in enumerate(zip(rasters, sizes)):
        g = r.ctx.debug(dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
        zk = g[..., 3].numpy()
        assert np.array_equal(ids, ras["ids"]), f"view {w}: {int(np.sum(ids != ras['ids']))} ids differ"
        cov = ids > 0
        assert np.array_equal(zk[cov].view(np.uint32), ras["zkey"][cov].view(np.uint32)), f"view {w} keys"
    r.ctx.close()


def test_soup_has_exact_ties():
    """The straight-down light's snapped texel coordinates land on texel
    centres (shared edges through them) and coplanar triangles overlap."""
    sc, ref = _ref(0)
    st = ref["lights"][0]["setup"]
    X = np.asarray(st["X"], np.int64)
    assert np.mean((X % 256) == 128) > 0.25     # vertices exactly on a texel centre column
    assert np.mean((X % 128) == 0) > 0.9        # and nearly all on the half-texel grid
    ids = ref["lights"][0]["raster"]["ids"]
    assert (ids > 0).mean() > 0.5


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("tile", [32, 16])
def test_adversarial_antialias_detection(seed, tile):
    """The antialiasing detection, fused into the raster's epilogue with a seam
    pass for the pairs across tile edges (which pairs are which depends on the
    tile side): every view lists exactly as many pixels as the oracle's
    silhouette band holds, and f~ of each light (taught the GPU's f) matches the
    oracle's antialiasing at the stage bar."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc, ref = _ref(seed)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(light_tile=tile, camera_tile=tile)
    r.forward()
    r.ctx.sync()
    tris = np.asarray(sc["tris"], np.int64)
    adj = O.edge_adjacency(tris)
    views = [(L["raster"], L["setup"]) for L in ref["lights"]] + [(ref["camera_raster"], ref["camera_setup"])]
    for w, (ras, st) in enumerate(views):
        band = O.silhouette_band(ras, O.silhouette_table(adj, st))
        assert r.ctx.raster_stats(w)["aa_listed"] == int(band.sum()), f"view {w}"
    for l, L in enumerate(ref["lights"]):
        R = sc["lights"][L["light"]]["res"]
        fg = r.ctx.debug(dsm.DBG_F, l, (R, R, 2)).cpu().numpy()
        ftg = r.ctx.debug(dsm.DBG_FTILDE, l, (R, R, 2)).cpu().numpy()
        vh = torch.cat([torch.as_tensor(sc["verts"], dtype=torch.float64),
                        torch.ones((len(sc["verts"]), 1), dtype=torch.float64)], 1)
        sx, sy = O.screen_coords(vh @ L["Q"].detach()[:4].T, R, R)
        exp = O.antialias(torch.as_tensor(fg, dtype=torch.float64), L["raster"], L["setup"],
                          O.silhouette_table(adj, L["setup"]), tris, sx, sy).numpy()
        bad = np.abs(ftg - exp) > 1e-5 + 1e-4 * np.abs(exp)
        assert not bad.any(), f"f~ light {l}: {int(bad.sum())} texels off, max {np.abs(ftg - exp).max():.3g}"
    r.ctx.close()


def _huge_scene():
    """Two crossing triangles whose corners lie about 25,000 map widths off
    the map, inside the guard band: their edge functions at the texel centres
    reach 2^56, beyond the exact range of the raster's fast int64-to-float
    split (2^48), and the two surfaces' depth keys decide the nearest one."""
    X, k = 100_000.0, 4e-6
    # planes y = 0.5 + k x and y = 0.5 + k z, crossing along x = z through the map
    a = [(-X, -X), (X, -0.9 * X), (0.3 * X, X)]
    b = [(-0.8 * X, X), (X, 0.7 * X), (-0.2 * X, -X)]
    verts = np.array([(x, 0.5 + k * x, z) for x, z in a] + [(x, 0.5 + k * z, z) for x, z in b], np.float32)
    tris = np.array([[0, 2, 1], [3, 5, 4]], np.int32)
    light = scenes.directional_light((0.0, -1.0, 0.0), 64, ortho_half=4.0, dist=8.0, near=1.0, far=16.0, sigma=1.0)
    cam = scenes.look_at_perspective((0.3, 5.0, 3.0), (0.0, 0.0, 0.0), 50.0, 32, 24)
    return {"name": "huge", "verts": verts, "tris": tris, "tri_mat": np.zeros(2, np.int32),
            "albedo": np.array([[0.8, 0.8, 0.8]], np.float32), "lights": [light], "camera": cam,
            "params": scenes._default_params()}


def test_huge_triangles_reach_wide_edge_functions():
    """The scene does what it is for: the oracle's edge functions at covered
    texel centres exceed 2^55, and both triangles win some texels."""
    sc = _huge_scene()
    ref = O.render(sc)
    st, ras = ref["lights"][0]["setup"], ref["lights"][0]["raster"]
    X, Y = np.asarray(st["X"], np.int64), np.asarray(st["Y"], np.int64)
    assert np.abs(X).max() < (1 << 28) and np.abs(Y).max() < (1 << 28) and np.abs(X).max() > (1 << 27)
    ids = ras["ids"]
    assert set(np.unique(ids)) == {1, 2}
    t = sc["tris"][0]
    j, i = np.nonzero(ids == 1)
    px, py = 256 * i[0] + 128, 256 * j[0] + 128
    a, b = t[1], t[2]
    e = (int(X[b]) - int(X[a])) * (py - int(Y[a])) - (int(Y[b]) - int(Y[a])) * (px - int(X[a]))
    assert abs(e) >= 1 << 55


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [32, 16])
def test_huge_triangles_bit_exact(tile):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = _huge_scene()
    ref = O.render(sc)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(light_tile=tile, camera_tile=tile)
    r.forward()
    r.ctx.sync()
    ras = ref["lights"][0]["raster"]
    g = r.ctx.debug(dsm.DBG_GBUF, 0, (64, 64, 4)).cpu()
    ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
    zk = g[..., 3].numpy()
    assert np.array_equal(ids, ras["ids"]), f"{int(np.sum(ids != ras['ids']))} ids differ"
    assert np.array_equal(zk.view(np.uint32), ras["zkey"].view(np.uint32)), "keys differ"
    r.ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(2))
@pytest.mark.parametrize("kind", ["spot", "point"])
@pytest.mark.parametrize("tile", [32, 16])
def test_adversarial_soup_under_perspective_lights(seed, kind, tile):
    """The soups under a perspective light: a spot light above them, or a
    point light among them whose six cube faces each raster a part (faces
    that see nothing included); ids and depth keys of every view bit for bit."""
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = scenes.triangle_soup(seed)
    if kind == "spot":
        sc["lights"] = [scenes.spot_light((0.4, 6.0, -0.3), (-0.05, -1.0, 0.04), 48, 70.0, near=0.5, far=12.0,
                                          sigma=1.0)]
    else:
        sc["lights"] = [scenes.point_light((0.2, 1.2, -0.1), 40, near=0.05, far=10.0, sigma=1.0)]
    ref = O.render(sc)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(light_tile=tile, camera_tile=tile)
    r.forward()
    r.ctx.sync()
    R = sc["lights"][0]["res"]
    views = [(L["raster"], R, R) for L in ref["lights"]] + [(ref["camera_raster"], sc["camera"]["width"],
                                                              sc["camera"]["height"])]
    for w, (ras, W, H) in enumerate(views):
        g = r.ctx.debug(dsm.DBG_GBUF, w, (H, W, 4)).cpu()
        ids = g[..., 0].contiguous().view(torch.int32).numpy().astype(np.int64)
        zk = g[..., 3].numpy()
        assert np.array_equal(ids, ras["ids"]), f"view {w}: {int(np.sum(ids != ras['ids']))} ids differ"
        cov = ids > 0
        assert np.array_equal(zk[cov].view(np.uint32), ras["zkey"][cov].view(np.uint32)), f"view {w} keys"
    r.ctx.close()
