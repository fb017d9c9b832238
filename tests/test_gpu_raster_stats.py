"""Raster work counts (dsm_raster_stats) against a brute-force count from the
oracle's setup records.

Every visible triangle is paired with each tile its pixel-centre bbox touches;
a big triangle (at least `big_tiles` tiles) skips the tiles whose four corner
pixel centres all lie outside one of its edges.  Per pair the bbox within the
tile gives the spans (4 pixels of one row) and the pixel-centre tests.  The
counts are integers and must match exactly."""
import numpy as np
import pytest
import torch

import scenes
from oracle import dsm_oracle as O

pytestmark = pytest.mark.gpu

SPAN = 4


def _views(sc):
    from oracle import dsm_oracle as O
    out = []
    for L in sc["lights"]:
        Q = O.light_matrix(L, torch.as_tensor(L["pos"], dtype=torch.float64),
                           torch.as_tensor(L["dir"], dtype=torch.float64)).numpy().astype(np.float32)
        out.append((Q[:4], L["res"], L["res"]))
    cam = sc["camera"]
    out.append((np.asarray(cam["clip"], np.float32).reshape(4, 4), cam["width"], cam["height"]))
    return out


def _may_cover(X, Y, tri, sg, tx, ty, ts):
    x0 = tx * ts * 256 + 128
    y0 = ty * ts * 256 + 128
    x1, y1 = x0 + (ts - 1) * 256, y0 + (ts - 1) * 256
    for a, b in ((1, 2), (2, 0), (0, 1)):
        va, vb = tri[a], tri[b]
        dx, dy = sg * (X[vb] - X[va]), sg * (Y[vb] - Y[va])
        py = y1 if dx >= 0 else y0
        px = x0 if dy >= 0 else x1
        if dx * (py - Y[va]) - dy * (px - X[va]) < 0:
            return False
    return True


def _expected(M, W, H, verts, tris, ts, big_tiles):
    from oracle import dsm_oracle as O
    st = O.setup_view(O.clip_pinned(M, verts.astype(np.float32)), tris, W, H)
    X, Y = st["X"].astype(np.int64), st["Y"].astype(np.int64)
    pairs = spans = tests = 0
    for t in range(tris.shape[0]):
        if st["culled"][t]:
            continue
        xs, ys = X[tris[t]], Y[tris[t]]
        i0, i1 = max(0, -((128 - int(xs.min())) // 256)), min(W - 1, (int(xs.max()) - 128) // 256)
        j0, j1 = max(0, -((128 - int(ys.min())) // 256)), min(H - 1, (int(ys.max()) - 128) // 256)
        if i0 > i1 or j0 > j1:
            continue
        txs, tys = range(i0 // ts, i1 // ts + 1), range(j0 // ts, j1 // ts + 1)
        big = len(txs) * len(tys) >= big_tiles
        sg = 1 if st["area2"][t] > 0 else -1
        for ty in tys:
            for tx in txs:
                if big and not _may_cover(X, Y, tris[t], sg, tx, ty, ts):
                    continue
                w = min(i1, tx * ts + ts - 1) - max(i0, tx * ts) + 1
                h = min(j1, ty * ts + ts - 1) - max(j0, ty * ts) + 1
                pairs += 1
                spans += (w + SPAN - 1) // SPAN * h
                tests += w * h
    return {"pairs": pairs, "spans": spans, "pixel_tests": tests}


@pytest.mark.parametrize("tile,big_tiles", [(32, 16), (16, 4)])
def test_raster_stats_match_brute_force(tile, big_tiles):
    from paper_2308_10896_b300 import dsm
    torch.cuda.set_device(0)
    sc = scenes.tiny_scene(4, res=70, img=64, kind="mixed", n_lights=2, freq=3)
    r = dsm.Renderer(sc)
    r.ctx.set_tuning(light_tile=tile, camera_tile=tile, big_tiles=big_tiles)
    r.forward()
    r.ctx.sync()
    tris = np.asarray(sc["tris"], np.int64)
    ref = O.render(sc)
    adj = O.edge_adjacency(tris)
    rasters = [(L["raster"], L["setup"]) for L in ref["lights"]] + [(ref["camera_raster"], ref["camera_setup"])]
    for w, (M, W, H) in enumerate(_views(sc)):
        got = r.ctx.raster_stats(w)
        exp = _expected(M, W, H, np.asarray(sc["verts"]), tris, tile, big_tiles)
        # the antialiasing detection lists exactly the silhouette band
        ras, st = rasters[w]
        exp["aa_listed"] = int(O.silhouette_band(ras, O.silhouette_table(adj, st)).sum())
        assert got == exp, f"view {w}: {got} != {exp}"
        assert exp["pairs"] > 0 and exp["aa_listed"] > 0
    with pytest.raises(dsm.DsmError):
        r.ctx.raster_stats(len(sc["lights"]) + 1)
