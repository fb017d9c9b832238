"""Pins of the CPU oracle against closed forms, invariants, library routines and
finite differences (no GPU).  Each test names the passage of the paper (Worchel &
Alexa 2023) whose arithmetic it pins."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import scenes
from oracle import dsm_oracle as O

F64 = torch.float64


# ----------------------------------------------------------------------------- helpers
def _scene(parts, lights, cam=None, **params):
    verts, tris, mat = scenes.merge_meshes(parts)
    nm = int(mat.max()) + 1
    if cam is None:
        cam = scenes.look_at_perspective((0.0, 4.0, 4.0), (0.0, 0.0, 0.0), 45.0, 24, 24)
    p = {"min_variance": 1e-6, "filter_kind": 0, "filter_boundary": 0, "aa_shadow": 1, "aa_final": 1}
    p.update(params)
    return {"verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.full((nm, 3), 0.8, np.float32), "lights": lights, "camera": cam, "params": p}


def _frame(direction):
    """Independent numpy construction of the light frame (right, up, forward)."""
    f = np.asarray(direction, np.float64)
    f = f / np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0]) if abs(f[1]) > 0.99 else np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    return r, np.cross(r, f), f


def _quad(corners):
    """Corners listed (-x,-z), (+x,-z), (+x,+z), (-x,+z): wound with normal +Y."""
    return np.asarray(corners, np.float64), np.array([[0, 2, 1], [0, 3, 2]], np.int64)


def _down_light(res=48, half=3.0, sigma=1.0, radius=0):
    return scenes.directional_light((0.0, -1.0, 0.0), res, ortho_half=half, dist=10.0, near=1.0, far=20.0,
                                    sigma=sigma, radius=radius)


def _light_screen_to_world(light, sx, sy, y):
    """World point at height y whose light-screen position is (sx, sy) pixels
    for the straight-down orthographic light (closed form of Sec. A's camera)."""
    r, u, f = _frame(light["dir"])
    R, h = light["res"], light["ortho_half"]
    e = -light["dist"] * f
    ndc_x = 2.0 * sx / R - 1.0
    ndc_y = 1.0 - 2.0 * sy / R
    p = e + h * ndc_x * r + h * ndc_y * u
    p = p + ((y - p[1]) / f[1]) * f
    return p


# ----------------------------------------------------------------------------- P1: plane depth
@pytest.mark.parametrize("kind", ["directional", "spot"])
def test_plane_depth_closed_form(kind):
    """Eq. 1 and Sec. A light cameras: for a single plane, every covered texel
    stores the analytic depth of the plane along the texel-centre ray."""
    n = np.array([0.2, 1.0, -0.3])
    n /= np.linalg.norm(n)
    c0 = 0.1
    t1 = np.cross(n, [1.0, 0.0, 0.0]); t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    ext = 30.0 if kind == "directional" else 6.0      # every vertex in front of the spot light
    corners = [c0 * n + ext * (a * t1 + b * t2) for a, b in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    v, t = _quad(corners)
    if kind == "directional":
        light = scenes.directional_light((0.3, -1.0, 0.45), 40, ortho_half=2.5, dist=10.0, near=1.0,
                                         far=20.0, sigma=1.0)
    else:
        light = scenes.spot_light((0.7, 4.0, 0.4), (-0.1, -1.0, -0.05), 40, 70.0, near=0.5, far=9.0, sigma=1.0)
    sc = _scene([(v, t, 0)], [light])
    out = O.render(sc)
    L = out["lights"][0]
    ids = L["raster"]["ids"]
    f = L["f"][..., 0].detach().numpy()
    r, u, fw = _frame(light["dir"])
    R = light["res"]
    jj, ii = np.nonzero(ids)
    # plane of the (float32-stored) triangle that covers each texel
    vs = sc["verts"].astype(np.float64)
    tv = vs[sc["tris"][ids[jj, ii] - 1]]
    n = np.cross(tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    c0 = (n * tv[:, 0]).sum(1)
    assert len(jj) == R * R
    px = (2 * ii + 1) / R - 1
    py = 1 - (2 * jj + 1) / R
    near, far = light["near"], light["far"]
    if kind == "directional":
        e = -light["dist"] * fw
        h = light["ortho_half"]
        p0 = e + (h * px)[:, None] * r + (h * py)[:, None] * u
        s = (c0 - (p0 * n).sum(1)) / (n @ fw)
    else:
        e = light["pos"].astype(np.float64)
        cc = 1.0 / math.tan(math.radians(light["fov_y_deg"]) / 2)
        dirv = fw + (px / cc)[:, None] * r + (py / cc)[:, None] * u
        s = (c0 - n @ e) / (dirv * n).sum(1)
    d = (s - near) / (far - near)
    np.testing.assert_allclose(f[jj, ii], d, rtol=0, atol=1e-12)
    # the clip/depth matrix itself maps points of the frame as stated
    Q = L["Q"].detach().numpy()
    p = e + 0.3 * r - 0.2 * u + 2.5 * fw
    q = Q @ np.append(p, 1.0)
    assert abs(q[4] - (2.5 - near) / (far - near)) < 1e-12
    if kind == "directional":
        np.testing.assert_allclose(q[:4], [0.3 / h, -0.2 / h, (2.5 - near) / (far - near), 1.0], atol=1e-12)
    else:
        np.testing.assert_allclose(q[0] / q[3], cc * 0.3 / 2.5, atol=1e-12)
        np.testing.assert_allclose(q[1] / q[3], -cc * 0.2 / 2.5, atol=1e-12)
        np.testing.assert_allclose(q[2] / q[3], far / (far - near) * (1 - near / 2.5), atol=1e-12)


# ----------------------------------------------------------------------------- raster pins
def _raster_only(verts, tris, M, W, H):
    st = O.setup_view(O.clip_pinned(M, verts.astype(np.float32)), tris, W, H)
    return st, O.raster(st, tris)


def _ortho_screen_matrix(W, H):
    """clip = identity-like map so that world (x, y) in pixels -> screen pixels."""
    M = np.zeros((4, 4), np.float32)
    M[0, 0], M[0, 3] = 2.0 / W, -1.0
    M[1, 1], M[1, 3] = -2.0 / H, 1.0
    M[2, 2] = 1.0
    M[3, 3] = 1.0
    return M


def _is_sqrt_rn(s: float, r: float) -> bool:
    """r is sqrt(s) rounded to nearest: s lies between the squares of the
    midpoints to r's float64 neighbours (exact rational arithmetic)."""
    from fractions import Fraction
    lo, hi = Fraction(math.nextafter(r, 0.0)), Fraction(math.nextafter(r, math.inf))
    m_lo, m_hi = (lo + Fraction(r)) / 2, (Fraction(r) + hi) / 2
    return m_lo * m_lo <= Fraction(s) <= m_hi * m_hi


def test_frame_norm_is_correctly_rounded():
    """Supplementary Sec. A light cameras: Q's entries are formed in float64
    with every operation rounded once, so the frame's norms are IEEE square
    roots.  Pinned in exact rational arithmetic on random sums of squares and
    on the light direction whose float64 norm torch.sqrt rounds one ulp off;
    the derivative is torch.sqrt's."""
    rng = np.random.default_rng(31)
    for s in list(rng.uniform(0.25, 4.0, 2000)) + [float.fromhex("0x1.0000007822024p+0"), 1.0, 2.0, 0.5]:
        r = float(O._sqrt_rn(torch.tensor(s, dtype=F64)))
        assert _is_sqrt_rn(s, r), s.hex()
    x = torch.tensor(float.fromhex("0x1.0000007822024p+0"), dtype=F64, requires_grad=True)
    O._sqrt_rn(x).backward()
    assert abs(float(x.grad) - 0.5 / math.sqrt(float(x.detach()))) < 1e-15
    # the direction whose norm exposed it: Q's translation column of rows 0 and 1
    # (a cancellation, r.e and u.e with e = -dist f) then matches a plain-float
    # evaluation of the same operations
    d = np.array([np.float32(-0.80092883), np.float32(-0.49904314), np.float32(-0.33086097)], np.float64)
    n = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    assert _is_sqrt_rn((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2], n)
    f = torch.as_tensor(d, dtype=F64)
    fo = O._normalize(f).numpy()
    assert np.array_equal(fo, d / n)


def test_edge_function_to_float32_is_correctly_rounded():
    """Eq. 1's depth key interpolates the corner depths with the integer edge
    functions converted to float32; for triangles far off screen these reach
    2^58.  The oracle's int64 -> float32 cast rounds each to the nearest
    float32, ties to even: checked in exact integer arithmetic against both
    float32 neighbours, on random magnitudes up to 2^62 and on exact ties."""
    rng = np.random.default_rng(7)
    vals = []
    for k in range(24, 63):
        vals += [int(x) for x in rng.integers(1 << k, 1 << (k + 1), 200, dtype=np.int64)]
    for k in range(25, 62):        # halfway between two float32 neighbours, both mantissa parities
        for odd in (0, 1):
            base = (1 << k) | (odd << (k - 23))
            vals += [base | (1 << (k - 24)), (base | (1 << (k - 24))) + 1, (base | (1 << (k - 24))) - 1]
    vals += [-v for v in vals]
    f = np.asarray(vals, np.int64).astype(np.float32)
    for v, g in zip(vals, f):
        gi = int(g)
        lo, hi = int(np.nextafter(g, np.float32(-np.inf))), int(np.nextafter(g, np.float32(np.inf)))
        d = abs(v - gi)
        assert d <= abs(v - lo) and d <= abs(v - hi), v
        if d == abs(v - lo) or d == abs(v - hi):   # a tie: the even mantissa wins
            assert (np.float32(g).view(np.uint32) & 1) == 0, v


def test_top_left_rule_rectangle():
    """A rectangle with corners exactly on pixel centres covers the half-open
    set [i0, i1) x [j0, j1): left/top edges in, right/bottom edges out."""
    W = H = 16
    M = _ortho_screen_matrix(W, H)
    i0, i1, j0, j1 = 3, 11, 2, 9
    v = np.array([[i0 + .5, j0 + .5, .5], [i1 + .5, j0 + .5, .5], [i1 + .5, j1 + .5, .5], [i0 + .5, j1 + .5, .5]])
    for tris in (np.array([[0, 1, 2], [0, 2, 3]]), np.array([[0, 2, 1], [0, 3, 2]]), np.array([[1, 2, 3], [1, 3, 0]])):
        _, ras = _raster_only(v, tris, M, W, H)
        cov = ras["ids"] > 0
        exp = np.zeros((H, W), bool)
        exp[j0:j1, i0:i1] = True
        assert (cov == exp).all()


def test_watertight_jittered_grid():
    """Triangles sharing edges cover every pixel centre of their union exactly
    once (fill rule), also with vertices on pixel centres."""
    rng = np.random.default_rng(5)
    W = H = 24
    M = _ortho_screen_matrix(W, H)
    n = 5
    g = np.linspace(2.0, 22.0, n + 1)
    P = np.stack(np.meshgrid(g, g, indexing="xy"), -1).reshape(-1, 2)
    interior = (P[:, 0] > 2.0) & (P[:, 0] < 22.0) & (P[:, 1] > 2.0) & (P[:, 1] < 22.0)
    jit = rng.uniform(-1.5, 1.5, P.shape)
    jit[rng.random(len(P)) < 0.4] = np.round(jit[rng.random(len(P)) < 0.4].mean()) if False else 0.0
    P = P + np.where(interior[:, None], jit, 0.0)
    P[interior] = np.where(rng.random((interior.sum(), 1)) < 0.3, np.floor(P[interior]) + 0.5, P[interior])
    tris = []
    for a in range(n):
        for b in range(n):
            p00 = a * (n + 1) + b
            p01, p10, p11 = p00 + 1, p00 + n + 1, p00 + n + 2
            if (a + b) % 2:
                tris += [[p00, p01, p11], [p00, p11, p10]]
            else:
                tris += [[p00, p01, p10], [p01, p11, p10]]
    tris = np.array(tris)
    v = np.concatenate([P, np.full((len(P), 1), 0.5)], 1)
    count = np.zeros((H, W), int)
    for t in range(len(tris)):
        _, ras = _raster_only(v, tris[t:t + 1], M, W, H)
        count += ras["ids"] > 0
    ci = np.arange(W) + 0.5
    inside = (ci[None, :] > 2.0) & (ci[None, :] < 22.0) & (ci[:, None] > 2.0) & (ci[:, None] < 22.0)
    assert count.max() == 1
    assert (count[inside] == 1).all()


def test_coverage_matches_float_point_in_triangle():
    """Strictly interior / exterior pixel centres agree with a float64
    point-in-triangle test on the snapped vertices."""
    rng = np.random.default_rng(9)
    W = H = 32
    M = _ortho_screen_matrix(W, H)
    for _ in range(20):
        v = np.concatenate([rng.uniform(-2, 34, (3, 2)), np.full((3, 1), 0.5)], 1)
        tris = np.array([[0, 1, 2]])
        st, ras = _raster_only(v, tris, M, W, H)
        if st["culled"][0]:
            continue
        q = np.stack([st["X"], st["Y"]], 1).astype(np.float64) / 256.0
        cx, cy = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        def e(a, b):
            return (q[b, 0] - q[a, 0]) * (cy - q[a, 1]) - (q[b, 1] - q[a, 1]) * (cx - q[a, 0])
        E = np.stack([e(1, 2), e(2, 0), e(0, 1)])
        s = np.sign(E.sum(0))
        strict_in = (E * s > 1e-9).all(0)
        strict_out = (E * s < -1e-9).any(0)
        cov = ras["ids"] > 0
        assert cov[strict_in].all() and not cov[strict_out].any()


def test_nearest_surface_and_tie_break():
    """Eq. 1: the nearest surface wins; on an exact depth tie the smaller
    triangle index wins."""
    W = H = 12
    M = _ortho_screen_matrix(W, H)
    quad = np.array([[1.0, 1.0], [11.0, 1.0], [11.0, 11.0], [1.0, 11.0]])
    far_v = np.concatenate([quad, np.full((4, 1), 0.7)], 1)
    near_v = np.concatenate([quad, np.full((4, 1), 0.2)], 1)
    v = np.concatenate([far_v, near_v])
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]])
    _, ras = _raster_only(v, tris, M, W, H)
    ids = ras["ids"][ras["ids"] > 0]
    assert set(np.unique(ids)) <= {3, 4}
    same = np.concatenate([near_v, near_v])
    _, ras = _raster_only(same, tris, M, W, H)
    ids = ras["ids"][ras["ids"] > 0]
    assert set(np.unique(ids)) <= {1, 2}


# ----------------------------------------------------------------------------- filter / lookup pins
@pytest.mark.parametrize("boundary,mode", [(0, "nearest"), (1, "constant")])
def test_filter_equals_2d_convolution(boundary, mode):
    """Eqs. moment1/moment2: the separable filter equals the 2-D convolution with
    outer(w, w) (scipy.ndimage), clamp = 'nearest', zero = 'constant'."""
    rng = np.random.default_rng(1)
    g = rng.random((19, 23, 2))
    w = O.filter_weights(1.5, 0)
    assert len(w) == 7 and abs(w.sum() - 1) < 1e-15
    m = O.separable_filter(torch.as_tensor(g), w, boundary).numpy()
    k2 = np.outer(w, w)
    for c in range(2):
        ref = ndi.convolve(g[..., c], k2, mode=mode, cval=0.0)
        np.testing.assert_allclose(m[..., c], ref, atol=1e-14)


def test_filter_invariants():
    """A constant map stays constant (clamp); interior mass is preserved."""
    w = O.filter_weights(2.0, 0)
    assert len(w) == 9
    c = torch.full((10, 13, 2), 0.37, dtype=F64)
    np.testing.assert_allclose(O.separable_filter(c, w, 0).numpy(), 0.37, atol=1e-15)
    g = torch.zeros((30, 30, 2), dtype=F64)
    g[10:20, 12:17] = torch.rand(10, 5, 2, dtype=F64)
    assert abs(float(O.separable_filter(g, w, 1).sum() - g.sum())) < 1e-12
    b = O.filter_weights(1.0, 2, kind=1)
    np.testing.assert_allclose(b, 0.2)


def test_bilinear_matches_map_coordinates():
    """Alg. 2 SampleShadowMap: bilinear with clamped indices equals
    scipy.ndimage.map_coordinates(order=1, mode='nearest')."""
    rng = np.random.default_rng(2)
    m = rng.random((17, 17, 2))
    s = rng.uniform(-1.5, 17.5, 200)
    t = rng.uniform(-1.5, 17.5, 200)
    out = O.bilinear(torch.as_tensor(m), torch.as_tensor(s), torch.as_tensor(t)).numpy()
    for c in range(2):
        ref = ndi.map_coordinates(m[..., c], [t, s], order=1, mode="nearest")
        np.testing.assert_allclose(out[:, c], ref, atol=1e-14)


# ----------------------------------------------------------------------------- Chebyshev pins
def test_chebyshev_invariants_and_paper_derivative():
    """Sec. 3 (modified Cantelli bound) and Sec. 4: v = 1 exactly for d <= mu;
    dv/dmu = -dv/dd = 2 sigma^2 (d - mu) / (sigma^2 + (d - mu)^2)^2 for d > mu,
    0 otherwise; C1 across d = mu."""
    rng = np.random.default_rng(3)
    m1 = torch.as_tensor(rng.uniform(0.2, 0.8, 400))
    var = torch.as_tensor(rng.uniform(1e-4, 1e-2, 400))
    m2 = m1 * m1 + var
    d = (m1 + torch.as_tensor(rng.uniform(-0.1, 0.1, 400))).requires_grad_(True)
    mu = m1.clone().requires_grad_(True)
    v = O.chebyshev(d, mu, mu * mu + var, 0.0)       # sigma^2 held fixed, as in the paper's equation
    lit = (d <= mu).detach()
    assert (v[lit] == 1.0).all()
    gd, gmu = torch.autograd.grad(v.sum(), [d, mu])
    delta = (d - mu).detach()
    paper = torch.where(delta > 0, 2 * var * delta / (var + delta ** 2) ** 2, torch.zeros_like(delta))
    np.testing.assert_allclose(gmu.numpy(), paper.numpy(), rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(gd.numpy(), -paper.numpy(), rtol=1e-8, atol=1e-12)
    # continuity of the derivative at d = mu
    for eps in (1e-3, 1e-5, 1e-7):
        dd = torch.tensor([0.5 + eps, 0.5 - eps], dtype=F64, requires_grad=True)
        vv = O.chebyshev(dd, torch.tensor([0.5, 0.5], dtype=F64), torch.tensor([0.26, 0.26], dtype=F64), 0.0)
        g, = torch.autograd.grad(vv.sum(), [dd])
        assert abs(float(g[0])) <= 2 * eps / 0.01 ** 2 * 1.01 and float(g[1]) == 0.0
    # through m2: sigma^2 = m2 - m1^2 (Sec. 4 product rule) -> dv/dm2 = dv/dsigma^2
    m1t = torch.tensor([0.4], dtype=F64, requires_grad=True)
    m2t = torch.tensor([0.17], dtype=F64, requires_grad=True)
    dt = torch.tensor([0.45], dtype=F64)
    vt = O.chebyshev(dt, m1t, m2t, 0.0)
    g1, g2 = torch.autograd.grad(vt.sum(), [m1t, m2t])
    s2, D = 0.17 - 0.16, 0.05
    dv_ds2 = D * D / (s2 + D * D) ** 2
    dv_dmu = 2 * s2 * D / (s2 + D * D) ** 2
    assert abs(float(g2) - dv_ds2) < 1e-12
    assert abs(float(g1) - (dv_dmu - 2 * 0.4 * dv_ds2)) < 1e-12


# ----------------------------------------------------------------------------- P2/P3: two-depth VSM = PCF, axis-aligned AA
def _two_plane_scene(occluder_px, sigma=1.0, res=48, min_variance=0.0):
    light = _down_light(res=res, half=3.0, sigma=sigma)
    recv = _quad([[-20, 0, -20], [20, 0, -20], [20, 0, 20], [-20, 0, 20]])
    occ = _quad([_light_screen_to_world(light, sx, sy, 1.0) for sx, sy in occluder_px])
    return _scene([(recv[0], recv[1], 0), (occ[0], occ[1], 0)], [light], min_variance=min_variance), light


def test_axis_aligned_antialias_is_exact_box_coverage():
    """Sec. 4 smoothing of f, f^2: for an axis-aligned occluder edge the
    antialiased map equals a*alpha + b*(1 - alpha) with alpha the exact
    pixel-area coverage (box filter), for pixels touched by one edge."""
    xl, xr, yt, yb = 10.375, 29.875, 12.625, 33.125   # world corners exact in float32
    sc, light = _two_plane_scene([(xl, yt), (xr, yt), (xr, yb), (xl, yb)])
    out = O.render(sc)
    L = out["lights"][0]
    ft = L["ftilde"].detach().numpy()
    a = (10.0 - 1.0 - light["near"]) / (light["far"] - light["near"])
    b = (10.0 - 0.0 - light["near"]) / (light["far"] - light["near"])
    alpha = (b - ft[..., 0]) / (b - a)
    R = light["res"]
    i = np.arange(R)
    cx = np.clip(np.minimum(i + 1, xr) - np.maximum(i, xl), 0, 1)
    cy = np.clip(np.minimum(i + 1, yb) - np.maximum(i, yt), 0, 1)
    exact = cy[:, None] * cx[None, :]
    frac_x = (cx > 0) & (cx < 1)
    frac_y = (cy > 0) & (cy < 1)
    single = ~(frac_y[:, None] & frac_x[None, :])
    np.testing.assert_allclose(alpha[single], exact[single], atol=1e-9)
    # the f^2 channel is blended with the same weights: (f^2)~ = a^2 alpha + b^2 (1 - alpha)
    np.testing.assert_allclose(ft[..., 1], a * a * alpha + b * b * (1 - alpha), atol=1e-12)


def test_two_depth_vsm_equals_pcf():
    """Sec. 3: with two depths a < b the Chebyshev bound is tight: with
    p = (b - m1)/(b - a) the filtered fraction of occluder,
    m2 = p a^2 + (1-p) b^2 and v(receiver) = 1 - p exactly."""
    sc, light = _two_plane_scene([(12.2, 9.1), (33.7, 15.4), (29.9, 37.3), (8.8, 30.6)], sigma=1.5)
    out = O.render(sc)
    L = out["lights"][0]
    Q, mom = L["Q"].detach(), L["moments"].detach()
    a = (10.0 - 1.0 - light["near"]) / (light["far"] - light["near"])
    b = (10.0 - 0.0 - light["near"]) / (light["far"] - light["near"])
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(-2.5, 2.5, 3000), np.zeros(3000), rng.uniform(-2.5, 2.5, 3000)], 1)
    xh = torch.as_tensor(np.concatenate([pts, np.ones((3000, 1))], 1))
    v = O.light_visibility(Q, mom, xh, 0.0).numpy()
    R = light["res"]
    cl = xh.numpy() @ Q[:4].numpy().T
    s = (0.5 * cl[:, 0] + 0.5) * R - 0.5
    t = (0.5 - 0.5 * cl[:, 1]) * R - 0.5
    mm = np.stack([ndi.map_coordinates(mom[..., c].numpy(), [t, s], order=1, mode="nearest") for c in range(2)], 1)
    p = (b - mm[:, 0]) / (b - a)
    np.testing.assert_allclose(mm[:, 1], p * a * a + (1 - p) * b * b, atol=1e-12)
    mid = (p > 1e-6) & (p < 1 - 1e-6)
    assert mid.sum() > 200
    np.testing.assert_allclose(v[mid], 1 - p[mid], atol=1e-8)


def test_single_triangle_shadow_outline():
    """Closed form: a triangle parallel above the ground under a
    perpendicular directional light casts its vertical projection: the
    integral of (1 - v) over the ground equals the triangle's area up to the
    smoothing of its perimeter; deep inside v ~ 0, far outside v = 1."""
    light = _down_light(res=64, half=3.0, sigma=1.0)
    tri_px = np.array([(14.3, 12.1), (50.6, 20.7), (24.2, 52.9)])
    tv = np.array([_light_screen_to_world(light, sx, sy, 1.0) for sx, sy in tri_px])
    recv = _quad([[-20, 0, -20], [20, 0, -20], [20, 0, 20], [-20, 0, 20]])
    sc = _scene([(recv[0], recv[1], 0), (tv, np.array([[0, 1, 2]]), 0)], [light], min_variance=1e-7)
    L = O.render(sc)["lights"][0]
    Q, mom = L["Q"].detach(), L["moments"].detach()
    texel = 2 * light["ortho_half"] / light["res"]
    g = np.arange(-2.95, 2.95, texel / 3)
    X, Z = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel(), np.ones(X.size)], 1)
    v = O.light_visibility(Q, mom, torch.as_tensor(pts), 1e-7).numpy()
    area = 0.5 * abs(np.cross(tv[1] - tv[0], tv[2] - tv[0])[1])
    perim = sum(np.linalg.norm(tv[(k + 1) % 3] - tv[k]) for k in range(3))
    shadow = (1 - v).sum() * (texel / 3) ** 2
    assert abs(shadow - area) < 0.25 * perim * texel
    # signed distance to the outline in texels
    p2 = pts[:, [0, 2]]
    sd = np.full(len(p2), np.inf)
    inside = np.ones(len(p2), bool)
    c = tv[:, [0, 2]].mean(0)
    for k in range(3):
        A, B = tv[k][[0, 2]], tv[(k + 1) % 3][[0, 2]]
        nrm = np.array([B[1] - A[1], A[0] - B[0]])
        nrm /= np.linalg.norm(nrm)
        if (c - A) @ nrm > 0:
            nrm = -nrm
        inside &= (p2 - A) @ nrm < 0
        seg = B - A
        tt = np.clip(((p2 - A) @ seg) / (seg @ seg), 0.0, 1.0)
        sd = np.minimum(sd, np.linalg.norm(p2 - (A + tt[:, None] * seg), axis=1))
    sd /= texel
    # footprint of the smoothing: antialiasing 1 texel, filter radius r = 2
    # (sigma 1), bilinear lookup 1 texel, half a texel of pixel box
    reach = 1 + 2 + 1 + 0.5
    assert (v[(~inside) & (sd > reach)] > 1 - 1e-9).all()
    assert (v[inside & (sd > reach)] < 0.02).all()
    half = np.abs(v - 0.5) < 0.1
    assert (sd[half] < 1.5).all()


# ----------------------------------------------------------------------------- AA invariants
def test_antialias_identity_when_ids_equal():
    """Identical ids everywhere -> the antialiasing pass is the identity."""
    light = _down_light(res=24)
    big = np.array([[-20.0, 0.0, -20.0], [-20.0, 0.0, 60.0], [60.0, 0.0, -20.0]])   # covers the whole map
    sc = _scene([(big, np.array([[0, 1, 2]]), 0)], [light])
    L = O.render(sc)["lights"][0]
    assert (L["raster"]["ids"] == 1).all()
    assert torch.equal(L["ftilde"], L["f"])


# ----------------------------------------------------------------------------- P6: Lambert
def test_lambert_closed_form_and_light_gradient():
    """Supplementary Sec. A (Lambert, deferred shading): an unshadowed plane
    gives c = albedo * I * max(0, n . omega); d(sum c)/d dir matches the closed
    form -albedo I (n - (n.f) f) / |dir| per pixel."""
    recv = _quad([[-6, 0, -10], [6, 0, -10], [6, 0, 2.9], [-6, 0, 2.9]])   # in front of the camera, fills it
    d = np.array([0.3, -1.0, 0.2])
    light = scenes.directional_light(d, 32, ortho_half=6.0, dist=20.0, near=1.0, far=40.0, sigma=1.0,
                                     intensity=(0.9, 0.7, 0.5))
    cam = scenes.look_at_perspective((0.0, 3.0, 3.0), (0.0, 0.0, 0.0), 40.0, 20, 20)
    sc = _scene([(recv[0], recv[1], 0)], [light], cam=cam)
    sc["albedo"] = np.array([[0.6, 0.5, 0.4]], np.float32)
    lp = torch.as_tensor(np.concatenate([light["pos"], light["dir"]])[None], dtype=F64).requires_grad_(True)
    out = O.render(sc, light_params=lp)
    img = out["image"]
    n = np.array([0.0, 1.0, 0.0])
    d = light["dir"].astype(np.float64)          # the stored float32 direction
    f = d / np.linalg.norm(d)
    lam = max(0.0, n @ -f)
    expect = sc["albedo"][0].astype(np.float64) * light["intensity"].astype(np.float64) * lam
    np.testing.assert_allclose(img[..., :3].detach().numpy().reshape(-1, 3), np.tile(expect, (400, 1)), atol=1e-12)
    g, = torch.autograd.grad(img[..., :3].sum(), [lp])
    ai = sc["albedo"][0].astype(np.float64) * light["intensity"].astype(np.float64)
    per_pix = -ai.sum() * (n - (n @ f) * f) / np.linalg.norm(d)
    np.testing.assert_allclose(g[0, 3:].numpy(), 400 * per_pix, rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------------------------- P8: central finite differences
def _fd_check(scene, target, seed, h_vert, h_light, n_dirs=3, tol=0.08):
    """Reverse-mode gradient (Sec. 4-5) against central differences of the
    oracle's own loss along random directions."""
    rng = np.random.default_rng(seed)
    res = O.render_and_grad(scene, target)
    gv, gl, ga = res["grad_verts"].numpy(), res["grad_light"].numpy(), res["grad_albedo"].numpy()
    V0 = scene["verts"].astype(np.float64)
    LP0 = np.stack([np.concatenate([l["pos"], l["dir"]]) for l in scene["lights"]]).astype(np.float64)

    def loss(V, LP):
        out = O.render(scene, verts=torch.as_tensor(V), light_params=torch.as_tensor(LP), keep=False)
        return float(O.mse_loss(out["image"], target))

    errs = []
    for k in range(n_dirs):
        dv = rng.standard_normal(V0.shape)
        fd = (loss(V0 + h_vert * dv, LP0) - loss(V0 - h_vert * dv, LP0)) / (2 * h_vert)
        an = float((gv * dv).sum())
        errs.append(abs(fd - an) / max(abs(an), 1e-12))
        dl = rng.standard_normal(LP0.shape)
        if all(l["type"] == 0 for l in scene["lights"]):
            dl[:, :3] = 0
        fd = (loss(V0, LP0 + h_light * dl) - loss(V0, LP0 - h_light * dl)) / (2 * h_light)
        an = float((gl * dl).sum())
        errs.append(abs(fd - an) / max(abs(an), 1e-12))
    assert np.median(errs) < tol, errs
    return errs


@pytest.mark.parametrize("kind,seed", [("directional", 0), ("spot", 1), ("mixed", 2)])
def test_central_fd_tiny(kind, seed):
    sc = scenes.tiny_scene(seed, res=32, img=32, kind=kind, n_lights=2 if kind == "mixed" else 1)
    tgt = O.render(sc, verts=torch.as_tensor(scenes.jitter_vertices(sc, 0.03, seed + 10), dtype=F64),
                   keep=False)["image"].detach()
    # The step sits far below the spacing of the forward events the method does
    # not smooth: the kink of the blend at t = 1/2, a sliver triangle flipping
    # orientation, a sub-pixel triangle starting to own a pixel centre next to
    # a silhouette (Sec. 5: the antialiasing misses primitive boundaries).  In
    # float64 a 1e-6 step still resolves the derivative to ~1e-9.
    _fd_check(sc, tgt, seed, h_vert=1e-6, h_light=1e-6, tol=1e-3)


def test_albedo_gradient_is_exact():
    """The image is linear in the albedo table: the gradient equals the
    difference quotient exactly."""
    sc = scenes.tiny_scene(3)
    tgt = np.zeros((32, 32, 4))
    res = O.render_and_grad(sc, tgt)
    da = np.random.default_rng(0).standard_normal(sc["albedo"].shape)
    h = 1e-3

    def loss(al):
        return float(O.mse_loss(O.render(sc, albedo=torch.as_tensor(al), keep=False)["image"], tgt))
    a0 = sc["albedo"].astype(np.float64)
    fd = (loss(a0 + h * da) - loss(a0 - h * da)) / (2 * h)
    assert abs(fd - float((res["grad_albedo"].numpy() * da).sum())) < 1e-10


# ----------------------------------------------------------------------------- normals, spot-light Lambert, pinned transform
def test_vertex_normals_closed_forms():
    """Supplementary Sec. A shading normals: area-weighted vertex normals are
    the exact face normal on flat regions of a subdivided cube and close to the
    radial direction on a geodesic sphere."""
    v, t = scenes.subdivided_box(4)
    n = O.vertex_normals(torch.as_tensor(v), torch.as_tensor(t)).numpy()
    flat = (np.abs(v) < 1 - 1e-9).sum(1) == 2          # face interiors
    ax = np.abs(v[flat]).argmax(1)
    expect = np.zeros_like(v[flat])
    expect[np.arange(len(ax)), ax] = np.sign(v[flat][np.arange(len(ax)), ax])
    np.testing.assert_allclose(n[flat], expect, atol=1e-12)
    errs = []
    for f in (8, 16):
        v, t = scenes.icosphere(f)
        n = O.vertex_normals(torch.as_tensor(v), torch.as_tensor(t)).numpy()
        np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)
        errs.append(np.abs(n - v).max())
    assert errs[0] < 2e-2 and errs[1] < 0.6 * errs[0]      # converges to the radial normal


def test_vertex_normals_of_zero_area_faces_are_zero_with_finite_derivative():
    """A vertex whose faces all have zero area (collinear or coincident corners)
    keeps the zero normal, and reverse mode through it stays finite: its
    derivative is the identity's, so a zero upstream gradient gives zero.  The
    other vertices keep their unit normals."""
    v = torch.tensor([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0],       # a proper triangle
                      [2.0, 0.0, 0.0], [3.0, 0.0, 0.0], [4.0, 0.0, 0.0],       # collinear corners
                      [5.0, 1.0, 5.0], [5.0, 1.0, 5.0], [6.0, 1.0, 5.0]],      # two coincident corners
                     dtype=F64, requires_grad=True)
    t = torch.tensor([[0, 2, 1], [3, 4, 5], [6, 7, 8]])
    n = O.vertex_normals(v, t)
    assert torch.equal(n[3:].detach(), torch.zeros(6, 3, dtype=F64))
    np.testing.assert_allclose(n[:3].detach().numpy(), [[0.0, 1.0, 0.0]] * 3, atol=1e-15)
    w = torch.zeros(9, 3, dtype=F64)
    w[:3] = torch.randn(3, 3, dtype=F64, generator=torch.Generator().manual_seed(3))
    (n * w).sum().backward()
    g = v.grad.numpy()
    assert np.isfinite(g).all() and np.abs(g[3:]).max() == 0.0
    # an upstream gradient on a zero normal passes through as the identity's
    v.grad = None
    n = O.vertex_normals(v, t)
    n[4].sum().backward()
    assert np.isfinite(v.grad.numpy()).all()


def test_spot_light_lambert_closed_form():
    """Supplementary Sec. A: for a spot light omega = normalize(p - x); on an
    unshadowed plane c = albedo I max(0, n . omega) at the camera ray's hit."""
    recv = _quad([[-6, 0, -10], [6, 0, -10], [6, 0, 2.9], [-6, 0, 2.9]])
    p = np.array([0.4, 3.0, -1.0])
    light = scenes.spot_light(p, -p / np.linalg.norm(p), 16, 120.0, near=0.5, far=20.0, sigma=1.0)
    cam = scenes.look_at_perspective((0.0, 3.0, 3.0), (0.0, 0.0, 0.0), 40.0, 16, 16)
    sc = _scene([(recv[0], recv[1], 0)], [light], cam=cam)
    img = O.render(sc)["image"].detach().numpy()
    Minv = np.linalg.inv(cam["clip"].astype(np.float64))
    H = W = 16
    ii, jj = np.meshgrid(np.arange(W), np.arange(H))
    ndc = np.stack([(2 * ii + 1) / W - 1, 1 - (2 * jj + 1) / H], -1).reshape(-1, 2)
    a = np.concatenate([ndc, -np.ones((len(ndc), 1)), np.ones((len(ndc), 1))], 1) @ Minv.T
    b = np.concatenate([ndc, np.ones((len(ndc), 1)), np.ones((len(ndc), 1))], 1) @ Minv.T
    a, b = a[:, :3] / a[:, 3:], b[:, :3] / b[:, 3:]
    x = a + ((0.0 - a[:, 1]) / (b[:, 1] - a[:, 1]))[:, None] * (b - a)
    pl = light["pos"].astype(np.float64)
    om = pl - x
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    lam = np.maximum(0.0, om[:, 1])
    np.testing.assert_allclose(img[..., 0].reshape(-1), 0.8 * lam, atol=1e-9)


def test_pinned_transform_is_rounded_float64_product():
    """The pinned float32 transform stays within a few ulp of the exact product
    (it is a rounding order, not a different map)."""
    rng = np.random.default_rng(8)
    M = rng.standard_normal((4, 4)).astype(np.float32)
    V = rng.standard_normal((500, 3)).astype(np.float32)
    c32 = O.clip_pinned(M, V).astype(np.float64)
    c64 = np.concatenate([V, np.ones((500, 1), np.float32)], 1).astype(np.float64) @ M.astype(np.float64).T
    scale = np.abs(M).astype(np.float64) @ np.concatenate([np.abs(V), np.ones((500, 1))], 1).T.astype(np.float64)
    assert (np.abs(c32 - c64) <= 4 * np.finfo(np.float32).eps * scale.T).all()


def test_raster_window_matches_full_frame():
    """The windowed raster used for full-size spot checks is the full raster cut
    to the window: same ids and depth keys inside, background outside."""
    import scenes
    sc = scenes.tiny_scene(4, res=70, img=64, freq=3)
    tris = sc["tris"].astype(np.int64)
    L = sc["lights"][0]
    lp = torch.as_tensor(np.concatenate([L["pos"], L["dir"]]), dtype=O.F64)
    Q = O.light_matrix(L, lp[:3], lp[3:]).numpy().astype(np.float32)
    st = O.setup_view(O.clip_pinned(Q[:4], sc["verts"].astype(np.float32)), tris, 70, 70)
    full = O.raster(st, tris)
    for win in ((0, 69, 0, 69), (13, 44, 20, 41), (60, 69, 0, 5), (35, 35, 35, 35)):
        part = O.raster(st, tris, window=win)
        i0, i1, j0, j1 = win
        inside = np.zeros((70, 70), bool)
        inside[j0:j1 + 1, i0:i1 + 1] = True
        assert np.array_equal(part["ids"][inside], full["ids"][inside])
        assert np.array_equal(part["zkey"][inside], full["zkey"][inside])
        assert (part["ids"][~inside] == 0).all()


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step, so each step moves p by lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    p, m, v = p0, np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        p, m, v = O.adam_step(p, g, m, v, t, lr=1e-2)
        np.testing.assert_allclose(p, p0 - t * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-13)


def test_adam_matches_unrolled_moment_sums():
    """m_t and v_t equal the closed sums (1 - b) sum_k b^(t-k) g_k (resp. g_k^2),
    and the parameters move by the sum of the per-step updates."""
    rng = np.random.default_rng(4)
    b1, b2, lr, eps = 0.8, 0.95, 3e-3, 1e-6
    gs = rng.normal(size=(6, 10))
    p, m, v = np.ones(10), np.zeros(10), np.zeros(10)
    moved = np.zeros(10)
    for t in range(1, 7):
        p_prev = p
        p, m, v = O.adam_step(p, gs[t - 1], m, v, t, lr, b1, b2, eps)
        ms = (1 - b1) * sum(b1 ** (t - k) * gs[k - 1] for k in range(1, t + 1))
        vs = (1 - b2) * sum(b2 ** (t - k) * gs[k - 1] ** 2 for k in range(1, t + 1))
        np.testing.assert_allclose(m, ms, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(v, vs, rtol=1e-12, atol=1e-15)
        step = lr * (ms / (1 - b1 ** t)) / (np.sqrt(vs / (1 - b2 ** t)) + eps)
        np.testing.assert_allclose(p_prev - p, step, rtol=1e-9, atol=1e-15)
        moved += step
    np.testing.assert_allclose(1.0 - p, moved, rtol=1e-9, atol=1e-15)


def test_multi_camera_loss_is_sum_of_single_camera_losses():
    """Two cameras: the summed loss and its gradient equal the sum of the
    single-camera results of render_and_grad."""
    sc = scenes.tiny_scene(5, res=16, img=12)
    cam2 = scenes.look_at_perspective((2.5, 2.0, -2.0), (0.0, 0.5, 0.0), 50.0, 10, 14)
    cams = [sc["camera"], cam2]
    rng = np.random.default_rng(8)
    tg = [rng.uniform(0, 1, (c["height"], c["width"], 4)) for c in cams]
    both = O.render_cameras_and_grad(sc, cams, tg)
    singles = [O.render_and_grad(dict(sc, camera=c), t) for c, t in zip(cams, tg)]
    assert abs(float(both["loss"]) - sum(float(s["loss"]) for s in singles)) <= 1e-12
    for k in ("grad_verts", "grad_light", "grad_albedo"):
        exp = sum(s[k] for s in singles)
        assert torch.allclose(both[k], exp, rtol=1e-10, atol=1e-14), k
    for img, s in zip(both["images"], singles):
        assert torch.equal(img, s["image"].detach())


def _minimal_plane_descent(aa: int, steps: int):
    sc = scenes.minimal_plane(res=64, img=32)
    sc["params"]["aa_shadow"] = aa
    tgt = O.render(sc, verts=torch.as_tensor(sc["target_verts"], dtype=F64), keep=False)["image"].detach().numpy()
    k, xz = sc["moved"], [0, 2]
    v = sc["verts"].astype(np.float64).copy()
    p, m, s = v[k, xz].copy(), np.zeros(2), np.zeros(2)
    e0 = np.linalg.norm(p - sc["target_verts"][k, xz])
    g0 = None
    for it in range(1, steps + 1):
        v[k, xz] = p
        g = O.render_and_grad(sc, tgt, verts=v)["grad_verts"][k].numpy()[xz]
        g0 = g if g0 is None else g0
        p, m, s = O.adam_step(p, g, m, s, it, lr=0.01)
    return np.linalg.norm(p - sc["target_verts"][k, xz]) / e0, g0, sc["verts"][k, xz] - sc["target_verts"][k, xz]


def test_minimal_plane_needs_antialiased_shadow_map():
    """Sec. 5 ("optimization without smoothed shadow map") and its figure: with
    the antialiased maps f~, (f^2)~ the displaced occluder vertex is recovered
    from shadow images alone; with the discrete maps the gradient with respect
    to its horizontal position vanishes (the occluder's depth is constant, so
    only the silhouette carries the position) and Adam does not move it."""
    err_aa, g_aa, d = _minimal_plane_descent(1, 60)
    assert err_aa < 0.05
    assert float(g_aa @ d) / (np.linalg.norm(g_aa) * np.linalg.norm(d)) > 0.9   # points back to the target
    err_no, g_no, _ = _minimal_plane_descent(0, 20)
    assert abs(err_no - 1.0) < 1e-9
    assert np.linalg.norm(g_no) < 1e-12 * np.linalg.norm(g_aa)


# ----------------------------------------------------------------------------- point lights (cube maps)
def test_cube_faces_closed_form():
    """Each cube face of a point light at p is the 90-degree perspective view
    along its axis: a point x of the face's region projects inside the face
    (|u|, |v| <= 1, w > 0), the face-centre direction to (0, 0), and its depth
    is (|major component of x - p| - near) / (far - near)."""
    light = scenes.point_light((0.3, 1.1, -0.4), 64, near=0.2, far=9.0, sigma=1.0)
    p = torch.as_tensor(light["pos"], dtype=F64)
    rng = np.random.default_rng(11)
    d = rng.normal(size=(400, 3)) * rng.uniform(0.5, 4.0, (400, 1))
    faces = O.cube_face(d)
    assert set(faces.tolist()) == set(range(6))
    x = torch.as_tensor(d, dtype=F64) + p
    xh = torch.cat([x, torch.ones((400, 1), dtype=F64)], 1)
    near, far = float(np.float32(0.2)), float(np.float32(9.0))
    for k in range(6):
        Q = O.light_matrix(light, p, torch.tensor([0.0, -1.0, 0.0], dtype=F64), face=k)
        sel = faces == k
        cl = xh[sel] @ Q[:4].T
        assert (cl[:, 3] > 0).all()
        assert (cl[:, 0].abs() <= cl[:, 3] * (1 + 1e-12)).all() and (cl[:, 1].abs() <= cl[:, 3] * (1 + 1e-12)).all()
        major = np.abs(d[sel]).max(1)
        np.testing.assert_allclose((xh[sel] @ Q[4]).numpy(), (major - near) / (far - near), rtol=1e-12, atol=1e-12)
        centre = torch.cat([p + torch.tensor(O.CUBE_AXES[k], dtype=F64), torch.ones(1, dtype=F64)])
        cc = Q[:4] @ centre
        assert abs(float(cc[0] / cc[3])) < 1e-12 and abs(float(cc[1] / cc[3])) < 1e-12
        # the direction parameter does not enter a face
        Q2 = O.light_matrix(light, p, torch.tensor([0.3, 0.2, 0.9], dtype=F64), face=k)
        assert torch.equal(Q, Q2)


def test_point_light_over_scene_equals_spot_light():
    """With every shaded point in the -Y face of the cube, a point light is a
    spot light at the same position looking down with a 90-degree field of
    view (same camera up to the rounding of 1 / tan 45 degrees)."""
    sc = scenes.tiny_scene(5, res=40, img=40, kind="point")
    sc["lights"][0]["pos"] = np.array([0.1, 3.5, -0.1], np.float32)
    spot = dict(sc)
    spot["lights"] = [scenes.spot_light(sc["lights"][0]["pos"], (0.0, -1.0, 0.0), 40, 90.0, near=0.3, far=8.0,
                                        sigma=1.0, intensity=(0.8, 0.8, 0.8))]
    tgt = np.zeros((40, 40, 4))
    a = O.render_and_grad(sc, tgt)
    b = O.render_and_grad(spot, tgt)
    assert len([L for L in a["lights"] if (L["raster"]["ids"] > 0).any()]) >= 1
    np.testing.assert_allclose(a["image"].detach().numpy(), b["image"].detach().numpy(), atol=1e-9)
    np.testing.assert_allclose(a["grad_verts"].numpy(), b["grad_verts"].numpy(), atol=1e-9, rtol=1e-6)
    np.testing.assert_allclose(a["grad_light"].numpy()[0, :3], b["grad_light"].numpy()[0, :3], atol=1e-9, rtol=1e-6)
    assert np.all(a["grad_light"].numpy()[0, 3:] == 0.0)


@pytest.mark.parametrize("kind,seed", [("point", 5), ("mixed3", 6)])
def test_central_fd_point_lights(kind, seed):
    """Finite differences through cube maps: the shadow spans three faces of
    the cube (the face choice is a decision, piecewise constant)."""
    sc = scenes.tiny_scene(seed, res=32, img=32, kind=kind, n_lights=3 if kind == "mixed3" else 1)
    tgt = O.render(sc, verts=torch.as_tensor(scenes.jitter_vertices(sc, 0.03, seed + 10), dtype=F64),
                   keep=False)["image"].detach()
    _fd_check(sc, tgt, seed, h_vert=1e-6, h_light=1e-6, tol=1e-3)


# ----------------------------------------------------------------------------- exponential moments (EVSM)
def test_exponential_moments_reduce_light_bleeding():
    """Two occluders at depths z1 < z2 cover a receiver at d > z2 half each
    (the classic bleeding case).  The visibility is the Chebyshev bound on the
    mixture's moments, written out here for the plain and the warped depths;
    the exponential warp lowers the bleeding (the exact visibility is 0)."""
    z1, z2, d, a = 0.2, 0.5, 0.52, 0.5

    def bound(x1, x2, xd):
        mu = a * x1 + (1 - a) * x2
        var = a * (1 - a) * (x2 - x1) ** 2
        return var / (var + (xd - mu) ** 2), mu, a * x1 * x1 + (1 - a) * x2 * x2

    p_vsm, m1, m2 = bound(z1, z2, d)
    got = O.chebyshev(torch.tensor([d], dtype=F64), torch.tensor([m1], dtype=F64), torch.tensor([m2], dtype=F64), 0.0)
    assert abs(float(got[0]) - p_vsm) < 1e-12 and p_vsm > 0.4
    prev = p_vsm
    for c in (10.0, 20.0, 40.0):
        w = np.exp(c * np.array([z1, z2, d]))
        p_exp, m1, m2 = bound(*w)
        enc = O.moment_encode(torch.tensor([z1, z2], dtype=F64), c)
        mom = a * enc[0] + (1 - a) * enc[1]
        assert abs(float(mom[0]) - m1) <= 1e-12 * m1 and abs(float(mom[1]) - m2) <= 1e-12 * m2
        got = O.chebyshev(torch.tensor([w[2]], dtype=F64), mom[0:1], mom[1:2], 0.0)
        assert abs(float(got[0]) - p_exp) < 1e-9
        assert p_exp < prev
        prev = p_exp
    assert prev < 0.1


def test_exponential_moments_constant_map_and_lit_points():
    """With the warp, a receiver at or in front of the occluders is lit
    exactly (v = 1 where exp(c d) <= m1), and a constant map keeps its
    moments under the filter (the warp is applied before filtering)."""
    c = 10.0
    enc = O.moment_encode(torch.full((6, 6), 0.4, dtype=F64), c)
    w = O.filter_weights(1.5, 0)
    filt = O.separable_filter(enc, w, 0)
    assert torch.allclose(filt, enc, rtol=1e-13)
    m1, m2 = filt[..., 0].reshape(-1), filt[..., 1].reshape(-1)
    dw = torch.exp(c * torch.full_like(m1, 0.39))
    assert torch.all(O.chebyshev(dw, m1, m2, 1e-6 * (c * dw) ** 2) == 1.0)


@pytest.mark.parametrize("kind,seed", [("mixed", 7), ("point", 8)])
def test_central_fd_exponential_moments(kind, seed):
    sc = scenes.tiny_scene(seed, res=32, img=32, kind=kind, n_lights=2 if kind == "mixed" else 1)
    sc["params"] = dict(sc["params"], moments=1, exponent=10.0)
    tgt = O.render(sc, verts=torch.as_tensor(scenes.jitter_vertices(sc, 0.03, seed + 10), dtype=F64),
                   keep=False)["image"].detach()
    _fd_check(sc, tgt, seed, h_vert=1e-6, h_light=1e-6, tol=1e-3)


def test_tessellated_occluder_jacobian_is_sparse():
    """Sec. 5: with triangles smaller than a shadow-map texel the antialiasing
    misses primitive boundaries.  The oracle's gradient of a weighted image
    sum with respect to the occluder's translation equals the small-step
    difference quotient (the derivative of the method as implemented) for
    both occluders, but against the one-texel difference quotient (which
    averages over the method's events) it holds for a coarse occluder and is
    far too small for a tessellated one."""
    texel = 3.0 / 64
    ratios = {}
    for n in (4, 64):
        sc = scenes.tessellated_occluder(n=n, res=64, img=32)
        occ = sc["occluder"]
        W = np.random.default_rng(3).normal(size=(32, 32, 4))
        V0 = sc["verts"].astype(np.float64)

        def L(t):
            v = V0.copy()
            v[occ, 0] += t
            return float((O.render(sc, verts=torch.as_tensor(v), keep=False)["image"].detach().numpy() * W).sum())

        v = torch.as_tensor(V0).clone().requires_grad_(True)
        g, = torch.autograd.grad((O.render(sc, verts=v, keep=False)["image"] * torch.as_tensor(W)).sum(), [v])
        ad = float(g[occ, 0].sum())
        fd_small = (L(1e-6) - L(-1e-6)) / 2e-6
        assert abs(fd_small - ad) <= 1e-6 * abs(ad)
        ratios[n] = ad / ((L(texel) - L(-texel)) / (2 * texel))
    assert 0.8 < ratios[4] < 1.3 and ratios[64] < 0.5, ratios
