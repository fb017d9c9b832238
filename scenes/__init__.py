"""Seeded synthetic scenes for differentiable shadow mapping.

This module only *generates inputs*: triangle meshes, light descriptions and
camera matrices.  It holds none of the shadow-mapping arithmetic, so both the
CPU oracle and the CUDA path can read the same bytes from it.

The paper's own test meshes and reference renders are not available, so the
scenes stand in for its workloads (Sec. 6 and the supplementary experiment
details): objects normalised to roughly unit size, placed on a planar
receiver, lit by directional lights (orthographic shadow camera) and spot
lights (perspective shadow camera), Lambertian albedo.

Every scene is a plain dict::

    verts    (V, 3) float32   world-space positions
    tris     (T, 3) int32     vertex indices, counter-clockwise seen from outside
    tri_mat  (T,)   int32     material index per triangle
    albedo   (M, 3) float32   Lambert albedo per material
    lights   list of dicts    see ``directional_light`` / ``spot_light``
    camera   dict             ``clip`` (4, 4) float32 row-major, ``width``, ``height``
    params   dict             filter / variance settings

Randomness comes from ``numpy.random.default_rng(1000 * config + item)``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosphere", "subdivided_box", "ground_quad", "sh_displace", "random_rotation",
    "look_at_perspective", "directional_light", "spot_light", "point_light", "merge_meshes",
    "config1", "config2", "config3", "config4", "config5", "config_by_name",
    "tiny_scene", "jitter_vertices", "displaced_target", "minimal_plane", "tessellated_occluder",
]


# --------------------------------------------------------------------------- geometry
def _orient_outward(verts: np.ndarray, tris: np.ndarray, center: np.ndarray) -> np.ndarray:
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    out = ((a + b + c) / 3.0 - center)
    flip = (n * out).sum(1) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def _dedupe(points: np.ndarray, tris: np.ndarray):
    key = np.round(points, 9)
    _, first, inverse = np.unique(key, axis=0, return_index=True, return_inverse=True)
    return points[first], inverse.reshape(-1)[tris]


def icosphere(freq: int) -> tuple[np.ndarray, np.ndarray]:
    """Geodesic sphere of radius 1: every icosahedron face split into freq**2
    triangles (20 freq**2 triangles, 10 freq**2 + 2 vertices)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    base = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                     [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                     [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    faces = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                      [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                      [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                      [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    pts, tri = [], []
    idx = {}
    n = freq
    for fi, (ia, ib, ic) in enumerate(faces):
        A, B, C = base[ia], base[ib], base[ic]
        local = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                k = n - i - j
                p = (i * A + j * B + k * C) / n
                local[(i, j)] = len(pts)
                pts.append(p)
        for i in range(n):
            for j in range(n - i):
                tri.append([local[(i, j)], local[(i + 1, j)], local[(i, j + 1)]])
                if i + j + 1 < n:
                    tri.append([local[(i + 1, j)], local[(i + 1, j + 1)], local[(i, j + 1)]])
    del idx
    pts = np.array(pts)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    tri = np.array(tri, np.int64)
    pts, tri = _dedupe(pts, tri)
    tri = _orient_outward(pts, tri, np.zeros(3))
    return pts, tri


def subdivided_box(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Axis-aligned cube [-1, 1]^3 with every face split into n x n quads
    (12 n**2 triangles), shared vertices along the cube edges."""
    pts, tri = [], []
    g = np.linspace(-1.0, 1.0, n + 1)
    for axis in range(3):
        for sign in (-1.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            base = len(pts)
            for iu in range(n + 1):
                for iv in range(n + 1):
                    p = np.zeros(3)
                    p[axis] = sign
                    p[u_ax] = g[iu]
                    p[v_ax] = g[iv]
                    pts.append(p)
            for iu in range(n):
                for iv in range(n):
                    a = base + iu * (n + 1) + iv
                    b, c, d = a + (n + 1), a + (n + 1) + 1, a + 1
                    tri.append([a, b, c])
                    tri.append([a, c, d])
    pts, tri = _dedupe(np.array(pts), np.array(tri, np.int64))
    tri = _orient_outward(pts, tri, np.zeros(3))
    return pts, tri


def ground_quad(half: float, y: float) -> tuple[np.ndarray, np.ndarray]:
    """Two-triangle square receiver at height y, normal +Y."""
    v = np.array([[-half, y, -half], [half, y, -half], [half, y, half], [-half, y, half]], np.float64)
    t = np.array([[0, 2, 1], [0, 3, 2]], np.int64)   # normal (0, +1, 0)
    return v, t


def ground_grid(half: float, y: float, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Square receiver at height y split into n x n quads (2 n^2 triangles),
    normal +Y.  Scenes lit by a point light use it: a view drops a triangle
    with a vertex behind its eye plane, so no triangle may be larger than the
    light's near distance (then only points that no cube face shades are lost)."""
    g = np.linspace(-half, half, n + 1)
    X, Z = np.meshgrid(g, g, indexing="xy")
    v = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], 1)
    idx = np.arange((n + 1) ** 2).reshape(n + 1, n + 1)
    a, b, c, d = idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel(), idx[1:, 1:].ravel(), idx[1:, :-1].ravel()
    t = np.concatenate([np.stack([a, c, b], 1), np.stack([a, d, c], 1)])   # normal (0, +1, 0)
    return v, t


def _real_sh_basis(n: np.ndarray) -> np.ndarray:
    """Real spherical-harmonic polynomials of degree 1..3 (15 functions,
    unnormalised) evaluated at unit vectors n (N, 3)."""
    x, y, z = n[:, 0], n[:, 1], n[:, 2]
    return np.stack([
        x, y, z,
        x * y, y * z, 3 * z * z - 1, x * z, x * x - y * y,
        y * (3 * x * x - y * y), x * y * z, y * (5 * z * z - 1), z * (5 * z * z - 3),
        x * (5 * z * z - 1), z * (x * x - y * y), x * (x * x - 3 * y * y)], axis=1)


def sh_displace(verts: np.ndarray, rng: np.random.Generator, amplitude: float = 0.2) -> np.ndarray:
    """Radial displacement r = 1 + A S(n)/max|S| with S a seeded combination
    of real SH of degree 1..3 (low-frequency blob shapes)."""
    n = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    c = rng.standard_normal(15)
    s = _real_sh_basis(n) @ c
    r = 1.0 + amplitude * s / np.abs(s).max()
    return n * r[:, None]


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def merge_meshes(parts):
    """parts: list of (verts, tris, material) -> verts, tris, tri_mat."""
    vs, ts, ms, off = [], [], [], 0
    for v, t, m in parts:
        vs.append(v)
        ts.append(t + off)
        ms.append(np.full(len(t), m, np.int32))
        off += len(v)
    return (np.concatenate(vs).astype(np.float32), np.concatenate(ts).astype(np.int32),
            np.concatenate(ms).astype(np.int32))


# --------------------------------------------------------------------------- cameras / lights
def look_at_perspective(eye, target, fov_y_deg, width, height, near=0.1, far=100.0) -> dict:
    """OpenGL-style camera: clip = P V [x, 1], ndc z in [-1, 1] (near -> -1)."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    if abs(fwd @ up) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = right, upv, -fwd
    V[:3, 3] = -V[:3, :3] @ eye
    f = 1.0 / math.tan(math.radians(fov_y_deg) / 2)
    aspect = width / height
    P = np.zeros((4, 4))
    P[0, 0] = f / aspect
    P[1, 1] = f
    P[2, 2] = (far + near) / (near - far)
    P[2, 3] = 2 * far * near / (near - far)
    P[3, 2] = -1.0
    return {"clip": (P @ V).astype(np.float32), "width": int(width), "height": int(height),
            "eye": eye.astype(np.float32)}


def directional_light(direction, res, ortho_half, dist, near, far, sigma,
                      intensity=(1.0, 1.0, 1.0), radius=0) -> dict:
    """Directional light: orthographic shadow camera placed at -dist * dir,
    looking along dir (the direction light travels)."""
    return {"type": 0, "pos": np.zeros(3, np.float32), "dir": np.asarray(direction, np.float32),
            "res": int(res), "fov_y_deg": 0.0, "ortho_half": float(ortho_half), "dist": float(dist),
            "near": float(near), "far": float(far), "intensity": np.asarray(intensity, np.float32),
            "sigma": float(sigma), "radius": int(radius)}


def spot_light(position, direction, res, fov_y_deg, near, far, sigma,
               intensity=(1.0, 1.0, 1.0), radius=0) -> dict:
    """Spot light: perspective shadow camera at the light position facing dir."""
    return {"type": 1, "pos": np.asarray(position, np.float32), "dir": np.asarray(direction, np.float32),
            "res": int(res), "fov_y_deg": float(fov_y_deg), "ortho_half": 0.0, "dist": 0.0,
            "near": float(near), "far": float(far), "intensity": np.asarray(intensity, np.float32),
            "sigma": float(sigma), "radius": int(radius)}


def point_light(position, res, near, far, sigma, intensity=(1.0, 1.0, 1.0), radius=0) -> dict:
    """Omnidirectional point light: a cube shadow map of six 90-degree
    perspective faces at the light position (res x res texels per face).  The
    direction slot of its parameters is unused."""
    return {"type": 2, "pos": np.asarray(position, np.float32), "dir": np.array([0.0, -1.0, 0.0], np.float32),
            "res": int(res), "fov_y_deg": 90.0, "ortho_half": 0.0, "dist": 0.0,
            "near": float(near), "far": float(far), "intensity": np.asarray(intensity, np.float32),
            "sigma": float(sigma), "radius": int(radius)}


def _default_params(**kw) -> dict:
    p = {"min_variance": 1e-6, "filter_kind": 0, "filter_boundary": 0, "aa_shadow": 1, "aa_final": 1}
    p.update(kw)
    return p


def _upper_hemisphere_dir(rng, el_lo=30.0, el_hi=80.0):
    az = rng.uniform(0, 2 * math.pi)
    s = rng.uniform(math.sin(math.radians(el_lo)), math.sin(math.radians(el_hi)))
    el = math.asin(s)
    to_light = np.array([math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az)])
    return -to_light   # direction light travels (downwards)


# --------------------------------------------------------------------------- configurations
def config1(item: int = 0) -> dict:
    """Icosphere (freq 8, 1280 triangles) 0.5 above a 10x10 quad; one directional
    light (elevation 30-80 deg); 256^2 orthographic map, sigma 1.5 (7 taps);
    256^2 camera with 45 deg FOV."""
    rng = np.random.default_rng(1000 * 1 + item)
    sv, st = icosphere(8)
    sv = sv @ random_rotation(rng).T + np.array([0.0, 1.5, 0.0])
    gv, gt = ground_quad(5.0, 0.0)
    verts, tris, mat = merge_meshes([(sv, st, 0), (gv, gt, 0)])
    light = directional_light(_upper_hemisphere_dir(rng), 256, ortho_half=7.5, dist=20.0,
                              near=1.0, far=40.0, sigma=1.5)
    cam = look_at_perspective((0.0, 3.0, 5.0), (0.0, 0.5, 0.0), 45.0, 256, 256)
    return {"name": "config1", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.full((1, 3), 0.8, np.float32), "lights": [light], "camera": cam,
            "params": _default_params()}


def config2(item: int = 0) -> dict:
    """50k-triangle SH-displaced icosphere (freq 50) with a seeded rigid pose,
    ground 6x6 at y=-1.3, spot light at distance 5 (90 deg), 1024^2 map with
    sigma 2, 1024^2 camera."""
    rng = np.random.default_rng(1000 * 2 + item)
    sv, st = icosphere(50)
    sv = sh_displace(sv, rng, 0.2)
    sv = sv @ random_rotation(rng).T + rng.normal(0.0, 0.3, 3) * np.array([1.0, 0.3, 1.0])
    gv, gt = ground_quad(3.0, -1.3)
    verts, tris, mat = merge_meshes([(sv, st, 0), (gv, gt, 1)])
    lpos = np.array([1.5, 4.6, 1.2])
    lpos = 5.0 * lpos / np.linalg.norm(lpos)
    light = spot_light(lpos, -lpos, 1024, 90.0, near=0.5, far=12.0, sigma=2.0)
    cam = look_at_perspective((0.0, 2.5, 5.5), (0.0, -0.5, 0.0), 45.0, 1024, 1024)
    return {"name": "config2", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.array([[0.8, 0.7, 0.6], [0.7, 0.7, 0.7]], np.float32),
            "lights": [light], "camera": cam, "params": _default_params()}


def _instances(rng, n_inst, total_tris, extent):
    sizes = np.exp(rng.uniform(math.log(1000), math.log(20000), n_inst))
    sizes *= total_tris / sizes.sum()
    parts = []
    for i in range(n_inst):
        if i % 2 == 0:
            f = max(2, int(round(math.sqrt(sizes[i] / 20.0))))
            v, t = icosphere(f)
            v = sh_displace(v, rng, 0.2)
        else:
            n = max(2, int(round(math.sqrt(sizes[i] / 12.0))))
            v, t = subdivided_box(n)
        scale = rng.uniform(0.35, 0.8)
        v = v @ random_rotation(rng).T * scale
        pos = np.array([rng.uniform(-extent, extent), 0.0, rng.uniform(-extent, extent)])
        pos[1] = -v[:, 1].min() + rng.uniform(0.0, 0.6)
        parts.append((v + pos, t, i + 1))
    return parts


def config3(item: int = 0) -> dict:
    """~330k triangles: 64 instances (SH-displaced icospheres and subdivided
    boxes, 1k-20k triangles each) on a 20x20 plane; one directional and one spot
    light (height 10, 90 deg), both 2048^2 with sigma 2; 1920x1080 camera."""
    rng = np.random.default_rng(1000 * 3 + item)
    parts = _instances(rng, 64, 330_000, 8.5)
    gv, gt = ground_quad(10.0, 0.0)
    parts.append((gv, gt, 0))
    verts, tris, mat = merge_meshes(parts)
    albedo = np.concatenate([np.full((1, 3), 0.75), rng.uniform(0.2, 0.9, (64, 3))]).astype(np.float32)
    d0 = _upper_hemisphere_dir(rng, 40.0, 70.0)
    l0 = directional_light(d0, 2048, ortho_half=15.0, dist=30.0, near=1.0, far=60.0, sigma=2.0,
                           intensity=(0.7, 0.7, 0.7))
    l1 = spot_light((0.0, 10.0, 0.0), (0.0, -1.0, 0.0), 2048, 90.0, near=1.0, far=12.0, sigma=2.0,
                    intensity=(0.5, 0.5, 0.5))
    cam = look_at_perspective((0.0, 13.0, 17.0), (0.0, 0.0, 0.5), 50.0, 1920, 1080)
    return {"name": "config3", "verts": verts, "tris": tris, "tri_mat": mat, "albedo": albedo,
            "lights": [l0, l1], "camera": cam, "params": _default_params()}


def config4(item: int = 0, n_scenes: int = 64) -> list:
    """64 independent scenes: one SH-displaced icosphere of 1k-100k triangles on
    a ground quad each; image side in {256,512,768,1024}, shadow-map side in
    {512,1024,2048}, 1-3 directional lights."""
    rng = np.random.default_rng(1000 * 4 + item)
    scenes = []
    for s in range(n_scenes):
        T = rng.uniform(1000, 100_000)
        f = max(2, int(round(math.sqrt(T / 20.0))))
        sv, st = icosphere(f)
        sv = sh_displace(sv, rng, 0.2) @ random_rotation(rng).T + np.array([0.0, 1.3, 0.0])
        gv, gt = ground_quad(4.0, 0.0)
        verts, tris, mat = merge_meshes([(sv, st, 0), (gv, gt, 1)])
        img = int(rng.choice([256, 512, 768, 1024]))
        smr = int(rng.choice([512, 1024, 2048]))
        lights = [directional_light(_upper_hemisphere_dir(rng), smr, ortho_half=6.0, dist=15.0,
                                    near=1.0, far=30.0, sigma=2.0, intensity=(0.6, 0.6, 0.6))
                  for _ in range(int(rng.integers(1, 4)))]
        cam = look_at_perspective((0.0, 3.5, 6.0), (0.0, 0.5, 0.0), 45.0, img, img)
        scenes.append({"name": f"config4_{s}", "verts": verts, "tris": tris, "tri_mat": mat,
                       "albedo": np.array([[0.8, 0.6, 0.5], [0.7, 0.7, 0.7]], np.float32),
                       "lights": lights, "camera": cam, "params": _default_params()})
    return scenes


def config5(item: int = 0) -> dict:
    """1,003,520-triangle SH-displaced icosphere (freq 224) on a ground quad,
    8 cameras (1024^2) on a ring, 4 directional lights with 2048^2 maps."""
    rng = np.random.default_rng(1000 * 5 + item)
    sv, st = icosphere(224)
    sv = sh_displace(sv, rng, 0.2) + np.array([0.0, 1.3, 0.0])
    gv, gt = ground_quad(4.0, 0.0)
    verts, tris, mat = merge_meshes([(sv, st, 0), (gv, gt, 1)])
    lights = [directional_light(_upper_hemisphere_dir(rng), 2048, ortho_half=6.0, dist=15.0,
                                near=1.0, far=30.0, sigma=2.0, intensity=(0.4, 0.4, 0.4))
              for _ in range(4)]
    cams = []
    for k in range(8):
        a = 2 * math.pi * k / 8
        cams.append(look_at_perspective((5.0 * math.cos(a), 3.0, 5.0 * math.sin(a)), (0.0, 1.0, 0.0),
                                        45.0, 1024, 1024))
    return {"name": "config5", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.array([[0.8, 0.7, 0.6], [0.7, 0.7, 0.7]], np.float32),
            "lights": lights, "camera": cams[0], "cameras": cams, "params": _default_params()}


def tiny_scene(seed: int = 0, res: int = 32, img: int = 32, kind: str = "directional",
               n_lights: int = 1, freq: int = 1) -> dict:
    """A few-triangle scene for finite-difference checks: a small icosphere
    (freq 1 = 20 triangles) over a ground quad."""
    rng = np.random.default_rng(77_000 + seed)
    sv, st = icosphere(freq)
    sv = sv @ random_rotation(rng).T * 0.6 + np.array([0.1, 1.0, -0.1])
    gv, gt = ground_grid(2.0, 0.0, 16) if kind in ("point", "mixed3") else ground_quad(2.0, 0.0)
    verts, tris, mat = merge_meshes([(sv, st, 0), (gv, gt, 1)])
    lights = []
    for li in range(n_lights):
        if kind == "point" or (kind == "mixed3" and li == 2):
            p = np.array([1.0, 1.6, 0.8]) + rng.uniform(-0.1, 0.1, 3)   # the shadow spans three cube faces
            lights.append(point_light(p, res, near=0.3, far=8.0, sigma=1.0, intensity=(0.8, 0.8, 0.8)))
        elif kind == "spot" or (kind in ("mixed", "mixed3") and li % 2 == 1):
            p = np.array([0.6, 4.0, 0.5]) + rng.uniform(-0.3, 0.3, 3)
            lights.append(spot_light(p, -p / np.linalg.norm(p), res, 80.0, near=0.5, far=8.0,
                                     sigma=1.0, intensity=(0.8, 0.8, 0.8)))
        else:
            lights.append(directional_light(_upper_hemisphere_dir(rng, 45.0, 75.0), res,
                                            ortho_half=3.0, dist=8.0, near=1.0, far=16.0, sigma=1.0,
                                            intensity=(0.9, 0.9, 0.9)))
    cam = look_at_perspective((0.0, 3.0, 4.0), (0.0, 0.5, 0.0), 45.0, img, img)
    return {"name": f"tiny{seed}", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.array([[0.9, 0.6, 0.4], [0.6, 0.7, 0.8]], np.float32),
            "lights": lights, "camera": cam, "params": _default_params(min_variance=1e-5)}


def minimal_plane(res: int = 256, img: int = 128, sigma: float = 1.0, displace=(0.12, 0.0, 0.08),
                  kind: int = 0) -> dict:
    """The paper's minimal-plane convergence setup (supplementary Sec. B): a
    square occluder (2 triangles, side 1, height 1) parallel to a square
    receiver (side 4, height 0), a directional light orthogonal to both, and a
    camera between them looking down at the receiver (the occluder is behind
    it, so the images show only the shadow).  One occluder corner (vertex
    `moved`) is displaced horizontally by `displace`; "target_verts" holds the
    undisplaced configuration, whose shadow image is the optimisation target."""
    occ = np.array([[-0.5, 1.0, -0.5], [0.5, 1.0, -0.5], [0.5, 1.0, 0.5], [-0.5, 1.0, 0.5]], np.float64)
    occ_t = np.array([[0, 2, 1], [0, 3, 2]], np.int64)          # normal +Y
    gv, gt = ground_quad(2.0, 0.0)
    target, tris, mat = merge_meshes([(occ, occ_t, 0), (gv, gt, 1)])
    moved = 2
    verts = target.copy()
    verts[moved] += np.asarray(displace, np.float32)
    light = directional_light((0.0, -1.0, 0.0), res, ortho_half=1.5, dist=5.0, near=1.0, far=10.0,
                              sigma=sigma, intensity=(1.0, 1.0, 1.0))
    cam = look_at_perspective((0.0, 0.9, 0.0), (0.0, 0.0, 0.0), 90.0, img, img, near=0.05, far=10.0)
    return {"name": "minimal_plane", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.array([[0.8, 0.8, 0.8], [0.8, 0.8, 0.8]], np.float32), "lights": [light],
            "camera": cam, "params": _default_params(min_variance=1e-5, filter_kind=kind),
            "target_verts": target, "moved": moved}


def tessellated_occluder(n: int = 256, angle_deg: float = 7.0, res: int = 256, img: int = 128,
                         sigma: float = 1.0, kind: int = 0) -> dict:
    """The paper's Jacobian setup (supplementary Sec. B): the minimal-plane
    scene with the occluder split into n x n quads (2 n^2 triangles; n = 256
    gives the paper's ~130k faces) and slightly rotated about the vertical
    axis.  "occluder" holds the occluder's vertex indices."""
    ov, ot = ground_grid(0.5, 1.0, n)
    a = math.radians(angle_deg)
    rot = np.array([[math.cos(a), 0.0, math.sin(a)], [0.0, 1.0, 0.0], [-math.sin(a), 0.0, math.cos(a)]])
    ov = (ov - np.array([0.0, 1.0, 0.0])) @ rot.T + np.array([0.0, 1.0, 0.0])
    gv, gt = ground_quad(2.0, 0.0)
    verts, tris, mat = merge_meshes([(ov, ot, 0), (gv, gt, 1)])
    light = directional_light((0.0, -1.0, 0.0), res, ortho_half=1.5, dist=5.0, near=1.0, far=10.0,
                              sigma=sigma, intensity=(1.0, 1.0, 1.0))
    cam = look_at_perspective((0.0, 0.9, 0.0), (0.0, 0.0, 0.0), 90.0, img, img, near=0.05, far=10.0)
    return {"name": "tessellated_occluder", "verts": verts, "tris": tris, "tri_mat": mat,
            "albedo": np.array([[0.8, 0.8, 0.8], [0.8, 0.8, 0.8]], np.float32), "lights": [light],
            "camera": cam, "params": _default_params(min_variance=1e-5, filter_kind=kind),
            "occluder": np.arange(len(ov))}


def with_degenerate_triangles(scene: dict) -> dict:
    """A copy of ``scene`` with triangles the setup must cull or treat as
    edge cases, appended after the original ones (ids unchanged):
    - (a, a, b) on an edge of the first object: zero snapped area in every
      view, and a third triangle on edge (a, b), which makes it non-manifold
      (a silhouette edge of the triangles beside it);
    - a triangle with one corner behind the camera (w < near in the camera
      view, an ordinary triangle for the lights);
    - a triangle far outside every view.
    The degenerate triangle reuses existing vertices, so every vertex still
    has a well-defined area-weighted normal."""
    sc = dict(scene)
    v = np.asarray(scene["verts"], np.float32)
    t = np.asarray(scene["tris"], np.int32)
    m = np.asarray(scene["tri_mat"], np.int32)
    a, b = int(t[0, 0]), int(t[0, 1])
    cam_eye = np.asarray(scene["camera"].get("eye", (0.0, 3.0, 4.0)), np.float32)
    behind = cam_eye + np.float32(1.5) * (cam_eye - np.array([0.0, 0.5, 0.0], np.float32)) / np.linalg.norm(
        cam_eye - np.array([0.0, 0.5, 0.0], np.float32))
    extra_v = np.array([behind, [0.8, 0.05, 0.9], [-0.6, 0.05, 0.7],
                        [60.0, 40.0, 60.0], [61.0, 40.0, 60.0], [60.0, 41.0, 60.0]], np.float32)
    V = len(v)
    extra_t = np.array([[a, a, b], [V, V + 1, V + 2], [V + 3, V + 4, V + 5]], np.int32)
    sc["verts"] = np.concatenate([v, extra_v]).astype(np.float32)
    sc["tris"] = np.concatenate([t, extra_t]).astype(np.int32)
    sc["tri_mat"] = np.concatenate([m, np.zeros(3, np.int32)]).astype(np.int32)
    sc["name"] = scene.get("name", "scene") + "_degenerate"
    return sc


def triangle_soup(seed: int = 0) -> dict:
    """An adversarial triangle soup for the rasteriser's exactness.  A
    directional light looking straight down with ortho_half = 4 maps world x
    and z onto its 64 x 64 map by exact float32 operations, so vertices whose x
    and z are multiples of 1/16 (half a texel) snap exactly onto texel centres
    and edges.  The soup: a 6 x 6 grid of quads split with alternating
    diagonals (shared edges through texel centres), 160 small triangles on the
    same dyadic grid at three heights (coplanar overlaps tie on depth), 40
    slivers (one edge a sixteenth of a texel), four tilted triangles spanning most of
    the map; a second, tilted light on a 48 x 48 map (ragged tiles) and a
    perspective camera."""
    G = 1.0 / 16.0
    rng = np.random.default_rng(40_000 + seed)
    verts, tris = [], []

    def tri(a, b, c):
        base = len(verts)
        verts.extend([a, b, c])
        tris.append([base, base + 1, base + 2])

    def snap(v):
        return np.round(np.asarray(v) / G) * G

    # a 6 x 6 grid of quads of 0.75 x 0.75 at y = 0
    x0, z0, s = -2.25, -2.25, 0.75
    for i in range(6):
        for j in range(6):
            a = (x0 + i * s, 0.0, z0 + j * s)
            b = (x0 + (i + 1) * s, 0.0, z0 + j * s)
            c = (x0 + (i + 1) * s, 0.0, z0 + (j + 1) * s)
            d = (x0 + i * s, 0.0, z0 + (j + 1) * s)
            if (i + j) % 2:
                tri(a, b, c); tri(a, c, d)
            else:
                tri(a, b, d); tri(b, c, d)
    # small dyadic triangles at three heights (coplanar overlaps tie on depth)
    for _ in range(160):
        y = float(rng.choice([0.25, 0.5, 0.75]))
        p = snap(rng.uniform(-3.5, 3.5, 2))
        q = p + snap(rng.uniform(-0.6, 0.6, 2))
        r = p + snap(rng.uniform(-0.6, 0.6, 2))
        tri((p[0], y, p[1]), (q[0], y, q[1]), (r[0], y, r[1]))
    # slivers: one edge a sixteenth of a texel
    for _ in range(40):
        y = float(rng.uniform(0.1, 0.9))
        p = snap(rng.uniform(-3.5, 3.5, 2))
        d = rng.choice([-1.0, 1.0], 2) * G / 8
        q = p + snap(rng.uniform(-1.5, 1.5, 2))
        tri((p[0], y, p[1]), (p[0] + d[0], y, p[1] + d[1]), (q[0], y, q[1]))
    # large triangles over most of the map, tilted (depth varies across them)
    for k in range(4):
        c = rng.uniform(-0.5, 0.5, 2)
        tri((c[0] - 3.6, 0.05 * k, c[1] - 3.4), (c[0] + 3.5, 0.3, c[1] - 3.6), (c[0], 0.9 - 0.1 * k, c[1] + 3.6))
    v = np.asarray(verts, np.float32)
    t = np.asarray(tris, np.int32)
    light = directional_light((0.0, -1.0, 0.0), 64, ortho_half=4.0, dist=8.0, near=1.0, far=16.0, sigma=1.0)
    ragged = directional_light((0.3, -1.0, 0.2), 48, ortho_half=4.0, dist=8.0, near=1.0, far=16.0, sigma=1.0)
    cam = look_at_perspective((0.3, 5.0, 3.0), (0.0, 0.0, 0.0), 50.0, 48, 40)
    return {"name": f"soup{seed}", "verts": v, "tris": t, "tri_mat": np.zeros(len(t), np.int32),
            "albedo": np.array([[0.8, 0.8, 0.8]], np.float32), "lights": [light, ragged], "camera": cam,
            "params": _default_params()}


def jitter_vertices(scene: dict, sigma: float, seed: int) -> np.ndarray:
    """Seeded vertex perturbation used to make a target render."""
    rng = np.random.default_rng(seed)
    return (scene["verts"] + rng.normal(0.0, sigma, scene["verts"].shape)).astype(np.float32)


def displaced_target(scene: dict, amplitude: float = 0.03, seed: int = 0, material: int = 0) -> np.ndarray:
    """Vertices of a seeded smooth displacement of one object (the vertices
    of the triangles with the given material): each moves along its
    direction n from the object's bounding-box centre c,
    x -> c + (x - c) (1 + A S(n) / max|S|), S a seeded combination of real SH
    of degree 1..3.  Used to render reconstruction targets."""
    rng = np.random.default_rng(50_000 + seed)
    verts = scene["verts"].astype(np.float64)
    sel = np.unique(scene["tris"][scene["tri_mat"] == material])
    x = verts[sel]
    c = 0.5 * (x.min(0) + x.max(0))
    d = x - c
    n = d / np.linalg.norm(d, axis=1, keepdims=True)
    s = _real_sh_basis(n) @ rng.standard_normal(15)
    out = verts.copy()
    out[sel] = c + d * (1.0 + amplitude * s / np.abs(s).max())[:, None]
    return out.astype(np.float32)


def config_by_name(name: str):
    return {"config1": config1, "config2": config2, "config3": config3,
            "config4": config4, "config5": config5}[name]()
