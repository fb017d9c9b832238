"""CPU oracle for differentiable pre-filtered (variance) shadow mapping.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and never imports it.

What it computes (Worchel & Alexa, "Differentiable Shadow Mapping for Efficient
Inverse Graphics", CVPR 2023), per light l and camera pixel x:

* Sec. 3, Eq. 1: the shadow map f(u) = min d(x) over scene points with
  L(x) = u, obtained by rasterising the mesh from the light (``raster``).
* Sec. 4 and Alg. 1: RenderScene yields the smoothed discrete maps f~ and
  (f^2)~ -- the rasteriser's edge antialiasing applied to f and f (x) f
  (``antialias``) -- which are then filtered: m1 = G f~, m2 = G (f^2)~
  (Eqs. moment1/moment2, ``gaussian_filter``).
* Alg. 2: u = L(x), bilinear lookup of (m1, m2), mu = m1,
  sigma^2 = m2 - m1^2, visibility 1 if d <= mu else
  sigma^2 / (sigma^2 + (d - mu)^2) (Sec. 3, modified Cantelli bound).
* Supplementary Sec. A: deferred Lambert shading summed over lights, and
  light cameras (orthographic for directional lights placed far outside the
  scene facing the origin along the light direction; perspective for spot
  lights at the light position).
* The final image is antialiased with the same edge rule.

Gradients (Sec. 4, Eqs. for dm/dTheta and dv/dmu) are the reverse-mode
derivative of this forward function, taken with torch.autograd in float64 as
the paper does with PyTorch (Sec. 5); IDs, coverage and the fixed-point snap
are constants of the derivative.

Precision: every continuous quantity is float64.  The discrete decisions --
which triangle covers a pixel centre, the fill rule, the nearest-surface key
and every antialiasing test -- are made on the pinned float32 vertex
transform and 24.8 fixed-point coordinates stated below, so that a float32
implementation can reproduce them bit for bit.  Readings of passages the paper
leaves open are marked "reading:".
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64
SUBPIX = 256          # 8 sub-pixel bits (24.8 fixed point)
GUARD = 1 << 28       # |snapped coordinate| limit; beyond it the triangle is culled
W_MIN = np.float32(1e-6)

__all__ = [
    "light_matrix", "light_views", "cube_face", "clip_pinned", "setup_view", "raster", "edge_adjacency", "silhouette_table",
    "silhouette_band",
    "barycentrics", "antialias", "filter_weights", "separable_filter", "bilinear",
    "chebyshev", "moment_encode", "warp_exponent", "light_visibility", "vertex_normals", "render", "mse_loss", "render_and_grad",
    "render_cameras_and_grad", "adam_step",
]


# =============================================================================== a1: light camera
def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return torch.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def _sqrt_rn(x: torch.Tensor) -> torch.Tensor:
    """IEEE 754 square root (rounded to nearest) with torch.sqrt's derivative.

    torch's float64 CPU square root is not correctly rounded on every back end
    (on an AVX-512 host about 0.6 % of inputs come out one ulp off), while
    numpy's is; the value is taken from numpy and the derivative from
    torch.sqrt.  t + (r - t) is exactly r: r and t are within a few ulps, so
    r - t is exact (Sterbenz) and so is the sum."""
    t = torch.sqrt(x)
    r = torch.as_tensor(np.sqrt(x.detach().numpy()), dtype=x.dtype)
    return t + (r - t).detach()


def _normalize(a):
    n = _sqrt_rn(a[0] * a[0] + a[1] * a[1] + a[2] * a[2])
    return torch.stack([a[0] / n, a[1] / n, a[2] / n])


def _f32(x) -> float:
    return float(np.float32(x))


# Cube faces of a point light, in view order: the fixed viewing axis of each.
CUBE_AXES = ((1.0, 0.0, 0.0), (-1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0),
             (0.0, 0.0, -1.0))


def light_views(light: dict) -> list:
    """Shadow-map views of a light: one plane, or for a point light (type 2)
    the six planes of a box around it (Sec. 3: when the rays from the light
    cannot be parameterised over one plane, several planes arranged as a box
    are used).  Returns the cube-face index of each view (None: single view).
    reading: the faces look along +X, -X, +Y, -Y, +Z, -Z with a 90-degree
    field of view; each face map is antialiased and filtered on its own."""
    return list(range(6)) if int(light["type"]) == 2 else [None]


def cube_face(d: np.ndarray) -> np.ndarray:
    """Face of a point light's cube map holding the directions d (n, 3) from
    the light: the axis of largest |component| and its sign, ties to x, then y.
    reading: the paper leaves the face selection open; this is the usual
    major-axis rule."""
    a = np.abs(d)
    fx = (a[:, 0] >= a[:, 1]) & (a[:, 0] >= a[:, 2])
    fy = ~fx & (a[:, 1] >= a[:, 2])
    return np.where(fx, np.where(d[:, 0] >= 0, 0, 1),
                    np.where(fy, np.where(d[:, 1] >= 0, 2, 3), np.where(d[:, 2] >= 0, 4, 5)))


def light_matrix(light: dict, pos: torch.Tensor, direction: torch.Tensor, face=None) -> torch.Tensor:
    """Light camera of Supplementary Sec. A as a 5x4 float64 matrix Q.

    Rows 0-3 map [x, 1] to light clip space; row 4 maps [x, 1] to the
    normalised light depth d(x) of Sec. 3.

    reading: depth d is the view depth along the light's forward axis f,
    normalised as (z_view - near) / (far - near); for a directional light this
    is the distance from a plane outside the scene (Sec. 3).  The eye of a
    directional light is at -dist * f; a spot light looks from ``pos`` along f.
    Up vector +Y, or +Z when |f_y| > 0.99.  Every entry is formed in this exact
    operation order in float64 (``_dot`` left to right, division by the norm)
    and rounded to float32 only by the caller.  A cube face (``face`` of a
    point light) is the perspective camera at ``pos`` looking along the face
    axis with c = 1 (90 degrees); the direction parameter does not enter it.
    """
    if face is not None:
        direction = torch.tensor(CUBE_AXES[face], dtype=F64)
    f = _normalize(direction)
    if abs(float(f[1].detach())) > 0.99:
        up = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    else:
        up = torch.tensor([0.0, 1.0, 0.0], dtype=F64)
    r = _normalize(_cross(f, up))
    u = _cross(r, f)
    # the light's scalar constants are float32 values (as a renderer stores them)
    near, far = _f32(light["near"]), _f32(light["far"])
    if int(light["type"]) == 0:
        dist = _f32(light["dist"])
        e = torch.stack([-dist * f[0], -dist * f[1], -dist * f[2]])
    else:
        e = pos
    fe = _dot(f, e)
    rng = far - near
    depth = torch.stack([f[0] / rng, f[1] / rng, f[2] / rng, (-fe - near) / rng])
    zero = torch.zeros((), dtype=F64)
    one = torch.ones((), dtype=F64)
    if int(light["type"]) == 0:
        h = _f32(light["ortho_half"])
        row0 = torch.stack([r[0] / h, r[1] / h, r[2] / h, -_dot(r, e) / h])
        row1 = torch.stack([u[0] / h, u[1] / h, u[2] / h, -_dot(u, e) / h])
        row2 = depth
        row3 = torch.stack([zero, zero, zero, one])
    else:
        c = 1.0 if int(light["type"]) == 2 else 1.0 / math.tan(_f32(light["fov_y_deg"]) * math.pi / 360.0)
        A = far / rng
        B = -(far * near) / rng
        row0 = torch.stack([c * r[0], c * r[1], c * r[2], -(c * _dot(r, e))])
        row1 = torch.stack([c * u[0], c * u[1], c * u[2], -(c * _dot(u, e))])
        row2 = torch.stack([A * f[0], A * f[1], A * f[2], -(A * fe) + B])
        row3 = torch.stack([f[0], f[1], f[2], -fe])
    return torch.stack([row0, row1, row2, row3, depth])


# =============================================================================== a2: pinned vertex setup
def clip_pinned(M32: np.ndarray, V32: np.ndarray) -> np.ndarray:
    """clip_r = ((M_r0 x + M_r1 y) + M_r2 z) + M_r3, every operation a separately
    rounded float32 multiply or add (no fused multiply-add).  numpy float32
    ufuncs round each operation, which is the pinned rule."""
    M32 = np.asarray(M32, np.float32)
    x, y, z = V32[:, 0], V32[:, 1], V32[:, 2]
    out = np.empty((V32.shape[0], 4), np.float32)
    for r in range(4):
        out[:, r] = ((M32[r, 0] * x + M32[r, 1] * y) + M32[r, 2] * z) + M32[r, 3]
    return out


def setup_view(clip32: np.ndarray, tris: np.ndarray, W: int, H: int) -> dict:
    """Pinned float32 projection and 24.8 fixed-point snap of every vertex, and
    per-triangle signed doubled area / cull flag.

    ndc = clip / w (IEEE float32 division); sx = (0.5 ndc_x + 0.5) W,
    sy = (0.5 - 0.5 ndc_y) H (row 0 at the top); X = rint(256 sx),
    Y = rint(256 sy) (round half to even).  A triangle is culled when a vertex
    has w < 1e-6 (or NaN), a snapped coordinate beyond +-2^28, or zero snapped
    area.  reading: these guard rules are not in the paper; generated scenes do
    not trigger them.
    """
    w = clip32[:, 3]
    with np.errstate(all="ignore"):
        ndc_x = clip32[:, 0] / w
        ndc_y = clip32[:, 1] / w
        ndc_z = clip32[:, 2] / w
        sx = (np.float32(0.5) * ndc_x + np.float32(0.5)) * np.float32(W)
        sy = (np.float32(0.5) - np.float32(0.5) * ndc_y) * np.float32(H)
        fx = sx * np.float32(SUBPIX)
        fy = sy * np.float32(SUBPIX)
    vert_ok = (w >= W_MIN) & (np.abs(fx) <= GUARD) & (np.abs(fy) <= GUARD)
    X = np.where(vert_ok, np.rint(np.where(vert_ok, fx, 0)), 0).astype(np.int64)
    Y = np.where(vert_ok, np.rint(np.where(vert_ok, fy, 0)), 0).astype(np.int64)
    t0, t1, t2 = tris[:, 0], tris[:, 1], tris[:, 2]
    area2 = (X[t1] - X[t0]) * (Y[t2] - Y[t0]) - (Y[t1] - Y[t0]) * (X[t2] - X[t0])
    culled = ~(vert_ok[t0] & vert_ok[t1] & vert_ok[t2]) | (area2 == 0)
    return {"X": X, "Y": Y, "zndc": ndc_z.astype(np.float32), "area2": area2, "culled": culled,
            "orient": np.sign(area2) * (~culled), "W": W, "H": H}


def _order_bits(z32: np.ndarray) -> np.ndarray:
    """Monotone map of float32 values to uint32 (so that -0 < +0)."""
    b = z32.astype(np.float32).view(np.uint32).astype(np.uint64)
    neg = (b & 0x80000000) != 0
    return np.where(neg, (~b) & 0xFFFFFFFF, b | 0x80000000)


# =============================================================================== a3: brute-force raster
def raster(setup: dict, tris: np.ndarray, window=None) -> dict:
    """Eq. 1 on the pixel grid: for every pixel centre the nearest covering
    triangle, by brute force over each triangle's bounding box.

    ``window`` = (i0, i1, j0, j1) (inclusive pixel ranges) restricts the work
    to that window: only triangles whose box meets it are visited, and their
    boxes are cut to it; pixels outside it are left as background.  This is the
    same computation on fewer pixels, for spot checks of full-size frames.

    Coverage: edge functions E_ab(P) = (X_b - X_a)(P_y - Y_a) - (Y_b - Y_a)(P_x - X_a)
    in exact integers at P = (256 i + 128, 256 j + 128); E_0 = E_12,
    E_1 = E_20, E_2 = E_01, multiplied by s = sign(2A) so that inside is
    positive.  A pixel is covered when every E_k > 0, or E_k = 0 on a top-left
    edge: the coefficient a of P_x is positive, or a = 0 and the coefficient b
    of P_y is positive.
    Depth key: z = ((float(E_0) z_0 + float(E_1) z_1) + float(E_2) z_2) / float(2A)
    in float32 (ndc z of each vertex); nearest = smallest (z, triangle id).
    Returns ``ids`` (H, W) int64 with triangle index + 1 (0 = background) and
    ``zkey`` (H, W) float32.
    """
    W, H = setup["W"], setup["H"]
    X, Y, zn = setup["X"], setup["Y"], setup["zndc"]
    best = np.full((H, W), np.iinfo(np.uint64).max, np.uint64)
    zbest = np.zeros((H, W), np.float32)
    wi0, wi1, wj0, wj1 = (0, W - 1, 0, H - 1) if window is None else window
    order = range(tris.shape[0])
    if window is not None:
        # triangles whose pixel box meets the window (the same box as below)
        xs_all, ys_all = X[tris].astype(np.int64), Y[tris].astype(np.int64)
        bi0 = -((128 - xs_all.min(1)) // SUBPIX)
        bi1 = (xs_all.max(1) - 128) // SUBPIX
        bj0 = -((128 - ys_all.min(1)) // SUBPIX)
        bj1 = (ys_all.max(1) - 128) // SUBPIX
        order = np.nonzero((bi1 >= wi0) & (bi0 <= wi1) & (bj1 >= wj0) & (bj0 <= wj1))[0].tolist()
    for t in order:
        if setup["culled"][t]:
            continue
        v = tris[t]
        xs, ys = X[v], Y[v]
        i0 = max(wi0, -((128 - int(xs.min())) // SUBPIX))
        i1 = min(wi1, (int(xs.max()) - 128) // SUBPIX)
        j0 = max(wj0, -((128 - int(ys.min())) // SUBPIX))
        j1 = min(wj1, (int(ys.max()) - 128) // SUBPIX)
        if i0 > i1 or j0 > j1:
            continue
        s = 1 if setup["area2"][t] > 0 else -1
        px = (np.arange(i0, i1 + 1, dtype=np.int64) * SUBPIX + 128)[None, :]
        py = (np.arange(j0, j1 + 1, dtype=np.int64) * SUBPIX + 128)[:, None]
        inside = np.ones((j1 - j0 + 1, i1 - i0 + 1), bool)
        E = []
        for k, (a, b) in enumerate(((1, 2), (2, 0), (0, 1))):
            Xa, Ya, Xb, Yb = xs[a], ys[a], xs[b], ys[b]
            e = s * ((Xb - Xa) * (py - Ya) - (Yb - Ya) * (px - Xa))
            ca, cb = -s * (Yb - Ya), s * (Xb - Xa)
            top_left = (ca > 0) or (ca == 0 and cb > 0)
            inside &= (e > 0) | ((e == 0) & top_left)
            E.append(e)
        if not inside.any():
            continue
        z0, z1, z2 = zn[v[0]], zn[v[1]], zn[v[2]]
        a2f = np.float32(s * setup["area2"][t])
        with np.errstate(all="ignore"):
            z = ((E[0].astype(np.float32) * z0 + E[1].astype(np.float32) * z1)
                 + E[2].astype(np.float32) * z2) / a2f
        z = z.astype(np.float32)
        key = (_order_bits(z) << np.uint64(32)) | np.uint64(t)
        win = inside & (key < best[j0:j1 + 1, i0:i1 + 1])
        best[j0:j1 + 1, i0:i1 + 1] = np.where(win, key, best[j0:j1 + 1, i0:i1 + 1])
        zbest[j0:j1 + 1, i0:i1 + 1] = np.where(win, z, zbest[j0:j1 + 1, i0:i1 + 1])
    covered = best != np.iinfo(np.uint64).max
    ids = np.where(covered, (best & np.uint64(0xFFFFFFFF)).astype(np.int64) + 1, 0)
    return {"ids": ids, "zkey": np.where(covered, zbest, np.float32(0)), "key": best}


# =============================================================================== topology
def edge_adjacency(tris: np.ndarray) -> np.ndarray:
    """For triangle t and its edge e (e = 0: v0v1, 1: v1v2, 2: v2v0) the
    triangle across that edge, -1 for a boundary edge and -2 for an edge shared
    by more than two triangles."""
    owners: dict = {}
    for t, (a, b, c) in enumerate(tris.tolist()):
        for e, (p, q) in enumerate(((a, b), (b, c), (c, a))):
            owners.setdefault((min(p, q), max(p, q)), []).append((t, e))
    adj = np.full((tris.shape[0], 3), -1, np.int64)
    for lst in owners.values():
        if len(lst) == 2:
            (t0, e0), (t1, e1) = lst
            adj[t0, e0], adj[t1, e1] = t1, t0
        elif len(lst) > 2:
            for t, e in lst:
                adj[t, e] = -2
    return adj


def silhouette_table(adj: np.ndarray, setup: dict) -> np.ndarray:
    """Edge e of triangle t is a silhouette edge in this view when it is a mesh
    boundary or non-manifold edge, the triangle across it is culled, or the two
    triangles have opposite screen orientation (sign of the snapped area).

    reading: the paper delegates edge smoothing to its rasteriser's antialias
    primitive (Sec. 5); this is the silhouette rule of that published method,
    stated on exact integer orientation."""
    orient = setup["orient"]
    other = np.where(adj >= 0, adj, 0)
    sil = (adj < 0) | setup["culled"][other] | (orient[other] != orient[:, None])
    return sil


def silhouette_band(ras: dict, sil: np.ndarray) -> np.ndarray:
    """Pixels (H, W) bool in the view's silhouette band: a pixel with a
    4-neighbour of another triangle id such that the nearer surface of the pair
    (key order, as in ``antialias``; the background never is) is a triangle
    with a silhouette edge in this view.  Every antialiasing crossing lies in
    this band, so gradients judged outside it carry no edge-antialiasing term.
    reading: the one-pixel silhouette band of the gradient comparison; a
    4-neighbour of any other id would also take in every boundary between two
    triangles of one smooth surface, most of a dense mesh's pixels."""
    ids, key = ras["ids"], ras["key"]
    has_sil = np.concatenate([[False], sil.any(1)])     # indexed by id (0 = background)
    band = np.zeros(ids.shape, bool)
    for A, B, kA, kB, sa, sb in ((ids[:, :-1], ids[:, 1:], key[:, :-1], key[:, 1:], np.s_[:, :-1], np.s_[:, 1:]),
                                 (ids[:-1, :], ids[1:, :], key[:-1, :], key[1:, :], np.s_[:-1, :], np.s_[1:, :])):
        a_occ = (B == 0) | ((A != 0) & (kA < kB))
        m = (A != B) & has_sil[np.where(a_occ, A, B)]
        band[sa] |= m
        band[sb] |= m
    return band


# =============================================================================== interpolation
def _pixel_ndc(W, H):
    i = torch.arange(W, dtype=F64)
    j = torch.arange(H, dtype=F64)
    return (2.0 * i + 1.0) / W - 1.0, 1.0 - (2.0 * j + 1.0) / H


def barycentrics(clip: torch.Tensor, tris: torch.Tensor, ids: np.ndarray):
    """Perspective-correct barycentrics at covered pixel centres from the
    unsnapped clip coordinates: with a_k = x_k - p_x w_k and c_k = y_k - p_y w_k,
    b is proportional to (a_1 c_2 - a_2 c_1, a_2 c_0 - a_0 c_2, a_0 c_1 - a_1 c_0).
    Returns (pix_j, pix_i, tri index, b (n, 3))."""
    H, W = ids.shape
    jj, ii = np.nonzero(ids)
    tri = torch.as_tensor(ids[jj, ii] - 1)
    pxs, pys = _pixel_ndc(W, H)
    px, py = pxs[torch.as_tensor(ii)], pys[torch.as_tensor(jj)]
    cv = clip[tris[tri]]                       # (n, 3, 4)
    a = cv[:, :, 0] - px[:, None] * cv[:, :, 3]
    c = cv[:, :, 1] - py[:, None] * cv[:, :, 3]
    beta = torch.stack([a[:, 1] * c[:, 2] - a[:, 2] * c[:, 1],
                        a[:, 2] * c[:, 0] - a[:, 0] * c[:, 2],
                        a[:, 0] * c[:, 1] - a[:, 1] * c[:, 0]], dim=1)
    b = beta / beta.sum(1, keepdim=True)
    return jj, ii, tri, b


def screen_coords(clip: torch.Tensor, W: int, H: int):
    """Unsnapped screen position (pixels, y down) of every vertex, float64."""
    sx = (0.5 * clip[:, 0] / clip[:, 3] + 0.5) * W
    sy = (0.5 - 0.5 * clip[:, 1] / clip[:, 3]) * H
    return sx, sy


# =============================================================================== antialiasing
_EDGES = ((0, 1), (1, 2), (2, 0))


def antialias(color: torch.Tensor, ras: dict, setup: dict, sil: np.ndarray, tris: np.ndarray,
              sx: torch.Tensor, sy: torch.Tensor) -> torch.Tensor:
    """Edge antialiasing of the rasteriser (Sec. 4/5: f, f^2 -> f~, (f^2)~, and
    the final image).

    For every horizontally or vertically adjacent pixel pair with different
    triangle ids: the occluder pixel O is the one whose triangle is nearer (key
    order; background never occludes), N the other.  Take the first edge of
    O's triangle, in the order v0v1, v1v2, v2v0, that is a silhouette edge,
    that is handled by this pair's axis (horizontal pairs take edges with
    |dY| > |dX|, vertical pairs edges with |dX| >= |dY|, on the snapped
    deltas) and whose snapped segment crosses the snapped segment between the
    two pixel centres (exact integer test; an endpoint counts as above the line
    when its coordinate is >= the line's).  With t the crossing parameter of the
    unsnapped edge along the centre segment measured from O (clamped to
    [0, 1]): if t > 1/2, N gains (t - 1/2)(c_O - c_N), otherwise O gains
    (1/2 - t)(c_N - c_O).  All gains are computed from the input colours and
    summed.

    reading: this restates the published analytic antialiasing that the paper
    uses through its rasteriser (Sec. 5); exact parameters of that library are
    not given in the paper.
    """
    H, W = ras["ids"].shape
    ids, key = ras["ids"], ras["key"]
    X, Y = setup["X"], setup["Y"]
    delta = torch.zeros_like(color)
    for vertical in (False, True):
        if vertical:
            ja, ia = np.meshgrid(np.arange(H - 1), np.arange(W), indexing="ij")
            jb, ib = ja + 1, ia
        else:
            ja, ia = np.meshgrid(np.arange(H), np.arange(W - 1), indexing="ij")
            jb, ib = ja, ia + 1
        ja, ia, jb, ib = ja.ravel(), ia.ravel(), jb.ravel(), ib.ravel()
        idA, idB = ids[ja, ia], ids[jb, ib]
        m = idA != idB
        ja, ia, jb, ib, idA, idB = ja[m], ia[m], jb[m], ib[m], idA[m], idB[m]
        a_is_occ = (idB == 0) | ((idA != 0) & (key[ja, ia] < key[jb, ib]))
        jo, io = np.where(a_is_occ, ja, jb), np.where(a_is_occ, ia, ib)
        jn, i_n = np.where(a_is_occ, jb, ja), np.where(a_is_occ, ib, ia)
        tri = ids[jo, io] - 1
        chosen = np.full(tri.shape, -1, np.int64)
        for e, (p, q) in enumerate(_EDGES):
            va, vb = tris[tri, p], tris[tri, q]
            if vertical:
                line = ia * SUBPIX + 128
                ua, ub = X[va], X[vb]          # coordinate across the line
                wa, wb = Y[va], Y[vb]          # coordinate along the segment
                lo = ja * SUBPIX + 128
            else:
                line = ja * SUBPIX + 128
                ua, ub = Y[va], Y[vb]
                wa, wb = X[va], X[vb]
                lo = ia * SUBPIX + 128
            hi = lo + SUBPIX
            straddle = (ua >= line) != (ub >= line)
            D = ub - ua
            # each edge is handled along one axis only: by horizontal pairs when
            # it is steeper than 45 degrees, by vertical pairs otherwise
            along = np.abs(wb - wa)
            straddle &= (np.abs(D) >= along) if vertical else (np.abs(D) > along)
            num = wa * D + (line - ua) * (wb - wa)
            pos = D > 0
            inside = np.where(pos, (lo * D <= num) & (num <= hi * D), (lo * D >= num) & (num >= hi * D))
            ok = straddle & inside & sil[tri, e] & (chosen < 0)
            chosen = np.where(ok, e, chosen)
        sel = chosen >= 0
        if not sel.any():
            continue
        jo, io, jn, i_n, tri, chosen = jo[sel], io[sel], jn[sel], i_n[sel], tri[sel], chosen[sel]
        p_idx = np.array([_EDGES[e][0] for e in range(3)])[chosen]
        q_idx = np.array([_EDGES[e][1] for e in range(3)])[chosen]
        va = torch.as_tensor(tris[tri, p_idx])
        vb = torch.as_tensor(tris[tri, q_idx])
        if vertical:
            xa, ya, xb, yb = sx[va], sy[va], sx[vb], sy[vb]
            lc = torch.as_tensor(io, dtype=F64) + 0.5
            cross = ya + (lc - xa) * (yb - ya) / (xb - xa)
            o_pos = torch.as_tensor(jo, dtype=F64) + 0.5
            step = torch.as_tensor(np.sign(jn - jo), dtype=F64)
            degenerate = (xb - xa) == 0
        else:
            xa, ya, xb, yb = sx[va], sy[va], sx[vb], sy[vb]
            lc = torch.as_tensor(jo, dtype=F64) + 0.5
            cross = xa + (lc - ya) * (xb - xa) / (yb - ya)
            o_pos = torch.as_tensor(io, dtype=F64) + 0.5
            step = torch.as_tensor(np.sign(i_n - io), dtype=F64)
            degenerate = (yb - ya) == 0
        t = torch.clamp((cross - o_pos) * step, 0.0, 1.0)
        t = torch.where(degenerate, torch.full_like(t, 0.5), t)
        cO = color[torch.as_tensor(jo), torch.as_tensor(io)]
        cN = color[torch.as_tensor(jn), torch.as_tensor(i_n)]
        far_side = (t > 0.5)[:, None]
        gain_n = torch.where(far_side, (t - 0.5)[:, None] * (cO - cN), torch.zeros_like(cO))
        gain_o = torch.where(far_side, torch.zeros_like(cO), (0.5 - t)[:, None] * (cN - cO))
        flat = delta.view(H * W, -1)
        flat = flat.index_add(0, torch.as_tensor(jn * W + i_n), gain_n)
        flat = flat.index_add(0, torch.as_tensor(jo * W + io), gain_o)
        delta = flat.view(H, W, -1)
    return color + delta


# =============================================================================== a5: filter
def filter_weights(sigma: float, radius: int, kind: int = 0) -> np.ndarray:
    """Gaussian w_i = exp(-i^2 / 2 sigma^2) / sum_j exp(-j^2 / 2 sigma^2), |i| <= r,
    r = ceil(2 sigma) unless given (kernel size k = 2r + 1); kind 1 = box 1/k."""
    r = int(radius) if radius > 0 else int(math.ceil(2.0 * sigma))
    if kind == 1:
        return np.full(2 * r + 1, 1.0 / (2 * r + 1))
    i = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-i * i / (2.0 * sigma * sigma))
    return w / w.sum()


def separable_filter(img: torch.Tensor, w: np.ndarray, boundary: int = 0) -> torch.Tensor:
    """m = G g with G the separable convolution (Eqs. moment1/moment2): first
    along x, then along y.  reading: boundary 0 clamps indices to the edge
    (a constant map stays constant); boundary 1 treats outside texels as 0
    (the literal Toeplitz matrix)."""
    r = (len(w) - 1) // 2
    H, W = img.shape[0], img.shape[1]

    def one_axis(a, axis, n):
        out = torch.zeros_like(a)
        idx = torch.arange(n)
        for k in range(-r, r + 1):
            src = idx + k
            if boundary == 0:
                take = torch.index_select(a, axis, src.clamp(0, n - 1))
                out = out + float(w[k + r]) * take
            else:
                valid = (src >= 0) & (src < n)
                take = torch.index_select(a, axis, src.clamp(0, n - 1))
                shape = [1] * a.dim()
                shape[axis] = n
                out = out + float(w[k + r]) * take * valid.to(F64).view(shape)
        return out

    return one_axis(one_axis(img, 1, W), 0, H)


# =============================================================================== a7/a8: lookup, Chebyshev, Lambert
def bilinear(m: torch.Tensor, s: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """Bilinear sample of map m (R, R, C) at texel coordinates (s, t) (texel
    centres at integers), indices clamped to the map."""
    R = m.shape[0]
    i0 = torch.floor(s).detach()
    j0 = torch.floor(t).detach()
    fs, ft = s - i0, t - j0
    i0l, j0l = i0.long(), j0.long()
    i0c, i1c = i0l.clamp(0, R - 1), (i0l + 1).clamp(0, R - 1)
    j0c, j1c = j0l.clamp(0, R - 1), (j0l + 1).clamp(0, R - 1)
    return (((1 - fs) * (1 - ft))[:, None] * m[j0c, i0c] + (fs * (1 - ft))[:, None] * m[j0c, i1c]
            + ((1 - fs) * ft)[:, None] * m[j1c, i0c] + (fs * ft)[:, None] * m[j1c, i1c])


def chebyshev(d: torch.Tensor, m1: torch.Tensor, m2: torch.Tensor, min_variance) -> torch.Tensor:
    """Modified one-sided Chebyshev (Cantelli) visibility of Sec. 3 / Alg. 2:
    1 if d <= mu, else sigma^2 / (sigma^2 + (d - mu)^2), mu = m1,
    sigma^2 = max(m2 - m1^2, min_variance) (a number, or one per point).
    reading: the variance floor is standard variance-shadow-map practice; the
    paper does not state it."""
    raw = m2 - m1 * m1
    floor = torch.as_tensor(min_variance, dtype=F64).expand_as(raw)
    var = torch.where(raw >= floor, raw, floor)
    delta = d - m1
    lit = delta <= 0
    dpos = torch.where(lit, torch.zeros_like(delta), delta)
    denom = torch.where(lit, torch.ones_like(var), var + dpos * dpos)
    return torch.where(lit, torch.ones_like(var), var / denom)


def moment_encode(f: torch.Tensor, exponent: float = 0.0) -> torch.Tensor:
    """The two moment channels of depth samples f: (w, w^2) with w = f
    (variance shadow maps, Sec. 3) or w = exp(c f) for the exponential warp
    (c = exponent > 0), one of the other pre-filtered families the paper
    suggests against light bleeding (its discussion of limitations).
    reading: exponential variance shadow maps with the positive warp only."""
    w = torch.exp(exponent * f) if exponent > 0 else f
    return torch.stack([w, w * w], -1)


def _stage(value: torch.Tensor, key: str, teach: dict | None, record: dict | None) -> torch.Tensor:
    """Record this stage's own value under `key` (for a stage-wise comparison)
    and return it, or the taught value when `teach` holds one (see
    ``_substitute``)."""
    if record is not None:
        record[key] = value.detach().clone()
    return _substitute(value, None if teach is None else teach.get(key))


def light_visibility(Q: torch.Tensor, mom: torch.Tensor, xh: torch.Tensor, min_variance: float,
                     exponent: float = 0.0, teach: dict | None = None, record: dict | None = None) -> torch.Tensor:
    """Alg. 2 (ComputeVisibility) at homogeneous world points xh (n, 4):
    u = L(x) from the light clip matrix Q[0:4], texel coordinates
    s = (0.5 u_x + 0.5) R - 0.5 and t = (0.5 - 0.5 u_y) R - 0.5, bilinear (m1, m2),
    d = Q[4] . xh, then the Chebyshev visibility.
    reading: points behind the light or outside its window are lit (v = 1).
    With the exponential warp (exponent c > 0) the receiver depth is compared
    as exp(c d) and the floor is min_variance (c exp(c d))^2 (reading: the
    depth-unit floor carried by the warp's slope at the receiver).

    Stage-wise comparison: ``record`` receives each stage's own value and
    ``teach`` may replace it (keeping its derivative): 'uv' (n, 2) light-space
    position, 'st' (n, 2) texel coordinates, 'mm' (n, 2) bilinear moments,
    'dw' (n,) receiver depth in the moments' encoding, 'vis' (n,) Chebyshev
    visibility; NaN entries of a taught array keep the oracle's own value."""
    R = mom.shape[0]
    cl = xh @ Q[:4].T
    d = xh @ Q[4]
    wpos = cl[:, 3] > 0
    wsafe = torch.where(wpos, cl[:, 3], torch.ones_like(cl[:, 3]))
    uv = _stage(torch.stack([cl[:, 0] / wsafe, cl[:, 1] / wsafe], 1), "uv", teach, record)
    u, v = uv[:, 0], uv[:, 1]
    inside = wpos & (u.abs() <= 1) & (v.abs() <= 1)
    st = _stage(torch.stack([(0.5 * u + 0.5) * R - 0.5, (0.5 - 0.5 * v) * R - 0.5], 1), "st", teach, record)
    s, t = st[:, 0], st[:, 1]
    zero = torch.zeros_like(s)
    mm = _stage(bilinear(mom, torch.where(inside, s, zero), torch.where(inside, t, zero)), "mm", teach, record)
    if exponent > 0:
        dw = _stage(torch.exp(exponent * d), "dw", teach, record)
        vis = chebyshev(dw, mm[:, 0], mm[:, 1], min_variance * (exponent * dw) ** 2)
    else:
        dw = _stage(d, "dw", teach, record)
        vis = chebyshev(dw, mm[:, 0], mm[:, 1], min_variance)
    vis = _stage(vis, "vis", teach, record)
    if record is not None:
        record["inside"] = inside.numpy().copy()
        record["front"] = wpos.numpy().copy()
    return torch.where(inside, vis, torch.ones_like(vis))


def vertex_normals(verts: torch.Tensor, tris: torch.Tensor) -> torch.Tensor:
    """Area-weighted sum of face normals cross(v1 - v0, v2 - v0), normalised.

    reading: a vertex whose incident faces all have zero area has no normal
    direction; it keeps the zero vector, and the derivative there is that of
    the identity.  The square root is taken of a stand-in for those vertices,
    so that its infinite slope at 0 never multiplies their zero gradient (a
    NaN in reverse mode)."""
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    fn = torch.cross(v1 - v0, v2 - v0, dim=1)
    n = torch.zeros_like(verts)
    for k in range(3):
        n = n.index_add(0, tris[:, k], fn)
    s = (n * n).sum(1, keepdim=True)
    pos = s > 0
    ln = torch.sqrt(torch.where(pos, s, torch.ones_like(s)))
    return n / torch.where(pos, ln, torch.ones_like(ln))


# =============================================================================== pipeline
def _substitute(value: torch.Tensor, teacher) -> torch.Tensor:
    """Stage-wise comparison: take the given value, keep this stage's
    derivative.  NaN entries of the teacher keep the stage's own value."""
    if teacher is None:
        return value
    tv = torch.as_tensor(np.asarray(teacher), dtype=F64).reshape(value.shape)
    tv = torch.where(torch.isnan(tv), value.detach(), tv)
    return value + (tv - value).detach()


def warp_exponent(params: dict) -> float:
    """Exponent c of the moments' warp: params 'moments' = 1 selects the
    exponential family with c = params 'exponent'; 0 (default) is VSM."""
    return float(np.float32(params.get("exponent", 0.0))) if int(params.get("moments", 0)) == 1 else 0.0


def _teacher_view(teacher: dict, key: str, view: int):
    vals = teacher.get(key)
    return vals[view] if vals is not None and view < len(vals) else None


def _pixel_teacher(teach: dict | None, key: str, jj, ii):
    """The entries of a per-pixel teacher array (H, W, ...) at the given pixels."""
    if teach is None or teach.get(key) is None:
        return None
    return np.asarray(teach[key])[jj, ii]


def shade_pixels(scene: dict, verts: torch.Tensor, light_params: torch.Tensor, albedo: torch.Tensor, maps: list,
                 clipc: torch.Tensor, ids: np.ndarray, teach: dict | None = None, record: dict | None = None):
    """Camera pass of Alg. 2 with Lambert shading (suppl. Sec. A) at the
    covered pixels of ``ids``: world position x and normal n interpolated with
    the perspective-correct barycentrics, visibility of every light from its
    (Q, moment map) in ``maps``, colour = albedo * sum_l I_l v_l max(0, n.omega_l).
    Returns (rows, cols, rgb, per-light visibility).

    Stage-wise comparison: ``record`` receives 'x' and 'n' (n, 3) and, per
    light view in order, a dict of ``light_visibility``'s stage values under
    'lookup'; ``teach`` may give full-image arrays 'x', 'n' (H, W, 3) and
    'lookup', a list per light view of (H, W, 8) arrays (u, v, s, t, dw, m1, m2,
    vis), NaN where a value is not taught."""
    P = scene["params"]
    tris = torch.as_tensor(scene["tris"].astype(np.int64))
    jj, ii, tri, b = barycentrics(clipc, tris, ids)
    tv = tris[tri]
    if record is not None:
        record["pixels"] = (jj, ii)
        record["lookup"] = []
    x = _stage((b[:, :, None] * verts[tv]).sum(1), "x", {"x": _pixel_teacher(teach, "x", jj, ii)}, record)
    vn = vertex_normals(verts, tris)
    n = (b[:, :, None] * vn[tv]).sum(1)
    n = _stage(n / torch.sqrt((n * n).sum(1, keepdim=True)), "n", {"n": _pixel_teacher(teach, "n", jj, ii)}, record)
    xh = torch.cat([x, torch.ones((x.shape[0], 1), dtype=F64)], 1)
    ec = warp_exponent(P)
    radiance = torch.zeros((x.shape[0], 3), dtype=F64)
    vis_all = []
    view = 0

    def visibility(Q, mom):
        nonlocal view
        lt = None
        if teach is not None and teach.get("lookup") is not None and view < len(teach["lookup"]):
            a = np.asarray(teach["lookup"][view])[jj, ii]
            lt = {"uv": a[:, 0:2], "st": a[:, 2:4], "dw": a[:, 4], "mm": a[:, 5:7], "vis": a[:, 7]}
        rec = None
        if record is not None:
            rec = {}
            record["lookup"].append(rec)
        view += 1
        return light_visibility(Q, mom, xh, float(P["min_variance"]), ec, lt, rec)

    for li, light in enumerate(scene["lights"]):
        views = maps[li] if isinstance(maps[li], list) else [maps[li]]
        if int(light["type"]) == 2:
            # the face of the cube map that holds x (a decision, no derivative)
            face = torch.as_tensor(cube_face((x - light_params[li, 0:3][None, :]).detach().numpy()))
            vis = torch.zeros((x.shape[0],), dtype=F64)
            for k, (Q, mom) in enumerate(views):
                vis = torch.where(face == k, visibility(Q, mom), vis)
        else:
            Q, mom = views[0]
            vis = visibility(Q, mom)
        if int(light["type"]) == 0:
            dl = light_params[li, 3:6]
            omega = -(dl / torch.sqrt((dl * dl).sum()))[None, :].expand_as(x)
        else:
            to = light_params[li, 0:3][None, :] - x
            omega = to / torch.sqrt((to * to).sum(1, keepdim=True))
        lam = torch.clamp((n * omega).sum(1), min=0.0)
        I = torch.as_tensor(light["intensity"], dtype=F64)
        radiance = radiance + (vis * lam)[:, None] * I[None, :]
        vis_all.append(vis)
    mat = torch.as_tensor(scene["tri_mat"].astype(np.int64))[tri]
    return jj, ii, albedo[mat] * radiance, vis_all


def _light_params(scene: dict) -> np.ndarray:
    """(L, 6) float64: position and direction of every light (L may be 0)."""
    return np.array([np.concatenate([l["pos"], l["dir"]]) for l in scene["lights"]], np.float64).reshape(-1, 6)


def render(scene: dict, verts: torch.Tensor = None, light_params: torch.Tensor = None,
           albedo: torch.Tensor = None, teacher: dict = None, keep: bool = True,
           grad_mask_sm_band: bool = False) -> dict:
    """Forward pass: Alg. 1 per light view (one per directional or spot light,
    six cube faces per point light), then the camera pass with Alg. 2 and
    Lambert shading, then the final antialiasing.

    ``light_params`` is (L, 6) float64: (pos xyz, dir xyz) per light.
    ``teacher`` optionally replaces stage values ('ftilde', 'moments' lists per
    light view, 'color', and the shading stages 'x', 'n', 'lookup' of
    ``shade_pixels``) by given ones while keeping each stage's derivative.
    With ``grad_mask_sm_band`` the gradient reaching f~ is zeroed at every
    light view's silhouette band (``silhouette_band``); a dict {"on": bool}
    instead of a bool switches that mask per backward pass.
    Returns a dict with the image (H, W, 4: RGB and coverage) and every
    intermediate ('lights' holds one entry per light view; 'shading' the
    shading stages' own values, see ``shade_pixels``)."""
    P = scene["params"]
    tris_np = scene["tris"].astype(np.int64)
    tris = torch.as_tensor(tris_np)
    if verts is None:
        verts = torch.as_tensor(scene["verts"], dtype=F64)
    if light_params is None:
        light_params = torch.as_tensor(_light_params(scene), dtype=F64)
    if albedo is None:
        albedo = torch.as_tensor(scene["albedo"], dtype=F64)
    V32 = verts.detach().numpy().astype(np.float32)
    adj = edge_adjacency(tris_np)
    ones = torch.ones((verts.shape[0], 1), dtype=F64)
    vh = torch.cat([verts, ones], 1)
    out = {"lights": []}
    maps = []
    teach = teacher or {}
    view = 0   # light views in order: a point light's six faces are consecutive
    for li, light in enumerate(scene["lights"]):
        maps.append([])
        for face in light_views(light):
            Q = light_matrix(light, light_params[li, 0:3], light_params[li, 3:6], face)
            Q32 = Q.detach().numpy().astype(np.float32)
            R = int(light["res"])
            st = setup_view(clip_pinned(Q32[:4], V32), tris_np, R, R)
            ras = raster(st, tris_np)
            clip = vh @ Q[:4].T
            depth = vh @ Q[4]
            jj, ii, tri, b = barycentrics(clip, tris, ras["ids"])
            f = (b * depth[tris[tri]]).sum(1)
            ec = warp_exponent(P)
            # background texels hold the encoding of f = 1
            fmap = moment_encode(torch.ones((R, R), dtype=F64), ec)
            fmap = fmap.index_put((torch.as_tensor(jj), torch.as_tensor(ii)), moment_encode(f, ec))
            sil = silhouette_table(adj, st)
            if P.get("aa_shadow", 1):
                sx, sy = screen_coords(clip, R, R)
                ft = antialias(fmap, ras, st, sil, tris_np, sx, sy)
            else:
                ft = fmap
            ft = _substitute(ft, _teacher_view(teach, "ftilde", view))
            if grad_mask_sm_band and P.get("aa_shadow", 1) and ft.requires_grad:
                switch = grad_mask_sm_band if isinstance(grad_mask_sm_band, dict) else {"on": True}
                keep_grad = torch.as_tensor(~silhouette_band(ras, sil), dtype=F64)[:, :, None]
                ft.register_hook(lambda g, k=keep_grad, sw=switch: g * k if sw["on"] else g)
            w = filter_weights(light["sigma"], light["radius"], P.get("filter_kind", 0))
            mom = separable_filter(ft, w, P.get("filter_boundary", 0))
            mom = _substitute(mom, _teacher_view(teach, "moments", view))
            maps[li].append((Q, mom))
            if keep:
                out["lights"].append({"Q": Q, "Q32": Q32, "setup": st, "raster": ras, "f": fmap,
                                      "ftilde": ft, "moments": mom, "weights": w, "light": li, "face": face})
            view += 1
    cam = scene["camera"]
    Wc, Hc = cam["width"], cam["height"]
    M32 = np.asarray(cam["clip"], np.float32)
    stc = setup_view(clip_pinned(M32, V32), tris_np, Wc, Hc)
    rasc = raster(stc, tris_np)
    clipc = vh @ torch.as_tensor(M32, dtype=F64).T
    shading = {}
    jj, ii, rgb, vis_all = shade_pixels(scene, verts, light_params, albedo, maps, clipc, rasc["ids"], teach,
                                        shading if keep else None)
    color = torch.zeros((Hc, Wc, 4), dtype=F64)
    color = color.index_put((torch.as_tensor(jj), torch.as_tensor(ii)),
                            torch.cat([rgb, torch.ones((rgb.shape[0], 1), dtype=F64)], 1))
    color = _substitute(color, (teacher or {}).get("color"))
    silc = silhouette_table(adj, stc)
    if P.get("aa_final", 1):
        sxc, syc = screen_coords(clipc, Wc, Hc)
        image = antialias(color, rasc, stc, silc, tris_np, sxc, syc)
    else:
        image = color
    out.update({"image": image, "color": color, "camera_setup": stc, "camera_raster": rasc,
                "camera_band": silhouette_band(rasc, silc), "visibility": vis_all, "pixels": (jj, ii),
                "shading": shading})
    return out


def mse_loss(image: torch.Tensor, target) -> torch.Tensor:
    """L = mean over all H*W*4 entries of (image - target)^2 (Sec. 4.1 uses a
    mean squared image error)."""
    tgt = torch.as_tensor(np.asarray(target), dtype=F64)
    return ((image - tgt) ** 2).mean()


def render_and_grad(scene: dict, target, teacher: dict = None, verts=None, light_params=None, grad_image=None,
                    grad_mask_sm_band: bool = False, objectives: list = None) -> dict:
    """Forward, loss and reverse-mode gradients with respect to the vertices,
    the light parameters (pos xyz, dir xyz per light) and the albedo table.
    The gradients are those of the mean squared error against ``target``, or,
    when ``grad_image`` (H, W, 4) is given, of sum(image * grad_image): the
    backward of a given dL/dimage (the loss is still reported when a target is
    given).  ``grad_mask_sm_band``: see ``render``.  ``objectives``, a list of
    (grad_image or None for the loss, mask the shadow maps' bands, zero
    grad_image on the camera's silhouette band), adds one backward pass of the
    same forward per entry: 'objective_grads' holds their (verts, light,
    albedo) gradients."""
    v = torch.as_tensor(scene["verts"] if verts is None else verts, dtype=F64).clone().requires_grad_(True)
    if light_params is None:
        light_params = _light_params(scene)
    lp = torch.as_tensor(light_params, dtype=F64).clone().requires_grad_(True)
    al = torch.as_tensor(scene["albedo"], dtype=F64).clone().requires_grad_(True)
    switch = {"on": bool(grad_mask_sm_band)}
    need_mask = bool(grad_mask_sm_band) or any(o[1] for o in (objectives or []))
    out = render(scene, v, lp, al, teacher=teacher, grad_mask_sm_band=switch if need_mask else False)
    loss = mse_loss(out["image"], target) if target is not None else torch.zeros((), dtype=F64)

    def objective(gimg):
        if gimg is None:
            return loss
        return (out["image"] * torch.as_tensor(np.asarray(gimg), dtype=F64)).sum()

    extra = []
    for gimg, masked, cam_band in objectives or []:
        switch["on"] = bool(masked)
        if cam_band and gimg is not None:
            gimg = np.asarray(gimg) * (~out["camera_band"])[:, :, None]
        extra.append(torch.autograd.grad(objective(gimg), [v, lp, al], allow_unused=True, retain_graph=True))
    out["objective_grads"] = extra
    switch["on"] = bool(grad_mask_sm_band)
    if target is None and grad_image is None:
        gv = gl = ga = None            # only the listed objectives were asked for
    else:
        gv, gl, ga = torch.autograd.grad(objective(grad_image), [v, lp, al], allow_unused=True)
    out.update({"loss": loss.detach(), "grad_verts": gv, "grad_light": gl, "grad_albedo": ga})
    return out


def render_cameras_and_grad(scene: dict, cameras: list, targets: list, verts=None, teachers: list = None) -> dict:
    """Several cameras under the same lights: the loss is the sum over the
    cameras of each image's mean squared error; each camera's image is
    ``render`` with that camera (the light maps do not depend on the camera).
    ``teachers`` optionally gives ``render``'s teacher per camera.  Returns
    the images, the summed loss and its gradients."""
    v = torch.as_tensor(scene["verts"] if verts is None else verts, dtype=F64).clone().requires_grad_(True)
    lp = torch.as_tensor(_light_params(scene), dtype=F64).clone().requires_grad_(True)
    al = torch.as_tensor(scene["albedo"], dtype=F64).clone().requires_grad_(True)
    images, loss = [], 0.0
    for c, (cam, tgt) in enumerate(zip(cameras, targets)):
        sc = dict(scene, camera=cam)
        img = render(sc, v, lp, al, teacher=teachers[c] if teachers else None, keep=False)["image"]
        images.append(img.detach())
        loss = loss + mse_loss(img, tgt)
    gv, gl, ga = torch.autograd.grad(loss, [v, lp, al], allow_unused=True)
    return {"images": images, "loss": loss.detach(), "grad_verts": gv, "grad_light": gl, "grad_albedo": ga}


# =============================================================================== optimisation
def adam_step(p, g, m, v, t: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update in float64 (Kingma & Ba 2015, Algorithm 1; the paper
    optimises with Adam, beta1 = 0.9 and beta2 = 0.999, supplementary Sec. B):
    m <- beta1 m + (1 - beta1) g, v <- beta2 v + (1 - beta2) g^2, then
    p <- p - lr m^ / (sqrt(v^) + eps) with m^ = m / (1 - beta1^t),
    v^ = v / (1 - beta2^t).  Returns the new (p, m, v)."""
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
