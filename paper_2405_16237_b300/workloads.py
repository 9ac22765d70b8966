"""Seeded synthetic workloads: scenes, cameras, rays and parameter initialisation.

This module is shared by the CUDA path (bench, smoke, GPU tests) and by the
oracle tests. It holds none of the method's arithmetic: no slab test, no
hashing, no encoding, no MLP, no ray-triangle test. It only draws the inputs
whose shapes and distributions follow the workloads the paper measures
(complex meshed assets observed by a pinhole camera, Sec. 7 and Table 1), which
are not available here and are replaced by same-shape synthetic stand-ins:

* ``scene_random_tris``   4,096 small triangles (edge ~0.05) in the unit cube.
* ``scene_icosphere``     a subdivided icosphere with fractal radial
                          displacement (level 8 = 1,310,720 triangles).
* ``scene_sphere_clusters`` many displaced UV-spheres of log-uniform size.
* ``camera_rays``         pinhole primary rays from a camera on a sphere.
* ``chord_rays``          rays between uniform points of a bounding sphere.

All generators take an explicit seed and return float32 arrays (triangles as
``[n, 3, 3]``, rays as a dict of structure-of-arrays columns).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 240516237

RAY_KEYS = ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

def scene_random_tris(n_tris: int = 4096, seed: int = SEED_BASE, edge: float = 0.05) -> np.ndarray:
    """Triangles with centroids uniform in [-1/2, 1/2]^3 and vertices on a small
    sphere around the centroid; a sphere of radius 3/4*edge gives a mean
    chord (edge) length of ``edge``."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.5, 0.5, size=(n_tris, 1, 3))
    u = rng.normal(size=(n_tris, 3, 3))
    u /= np.linalg.norm(u, axis=2, keepdims=True)
    r = 0.75 * edge
    return (c + r * u).astype(np.float32)


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v += [(a, b, 0.0), (0.0, a, b), (b, 0.0, a)]
    v = np.array(v, dtype=np.float64)
    # Faces are the vertex triples that are pairwise at the edge length 2.
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    f = [i, j, k]
                    nrm = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(nrm, v[i] + v[j] + v[k]) < 0:
                        f = [i, k, j]
                    faces.append(f)
    assert len(faces) == 20
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, np.array(faces, dtype=np.int64)


def _subdivide(v: np.ndarray, f: np.ndarray):
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    e = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 0)  # [3, F, 2]
    e_sorted = np.sort(e, axis=2)
    key = e_sorted[..., 0] * len(v) + e_sorted[..., 1]
    uniq, inv = np.unique(key.ravel(), return_inverse=True)
    i0 = uniq // len(v)
    i1 = uniq % len(v)
    mid = v[i0] + v[i1]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    m = (inv + len(v)).reshape(3, -1)
    ab, bc, ca = m[0], m[1], m[2]
    nf = np.concatenate([
        np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
        np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)], 0)
    return np.concatenate([v, mid], 0), nf


def _value_noise(p: np.ndarray, perm: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """Seeded lattice value noise with smoothstep blending, in about [-1, 1]."""
    i = np.floor(p).astype(np.int64)
    t = p - i
    s = t * t * (3.0 - 2.0 * t)
    out = np.zeros(len(p))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                h = perm[(perm[(perm[(i[:, 0] + dx) & 255] + i[:, 1] + dy) & 255] + i[:, 2] + dz) & 255]
                w = (np.where(dx, s[:, 0], 1 - s[:, 0]) * np.where(dy, s[:, 1], 1 - s[:, 1])
                     * np.where(dz, s[:, 2], 1 - s[:, 2]))
                out += w * vals[h]
    return out


def fbm(p: np.ndarray, seed: int, octaves: int = 4, lacunarity: float = 2.0, gain: float = 0.5,
        base_freq: float = 4.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    perm = rng.permutation(256)
    vals = rng.uniform(-1.0, 1.0, size=256)
    total = np.zeros(len(p))
    amp, freq, norm = 1.0, base_freq, 0.0
    for _ in range(octaves):
        total += amp * _value_noise(p * freq + 17.0, perm, vals)
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def scene_icosphere(level: int = 8, seed: int = SEED_BASE + 1, radius: float = 0.4,
                    amplitude: float = 0.05) -> np.ndarray:
    """Level-``level`` icosphere (20*4^level triangles), radius ``radius``, with
    a seeded fractal (4-octave fBm of value noise) radial displacement of at
    most ``amplitude``."""
    v, f = _icosahedron()
    for _ in range(level):
        v, f = _subdivide(v, f)
    n = fbm(v, seed)
    n = n / max(1e-12, np.abs(n).max())
    r = radius + amplitude * n
    p = v * r[:, None]
    return p[f].astype(np.float32)


def _uv_sphere(n_tris_target: int, rng) -> np.ndarray:
    """Unit UV-sphere with about ``n_tris_target`` triangles (2*nu*(nv-1))."""
    nv = max(3, int(round(math.sqrt(n_tris_target / 4.0))))
    nu = max(4, int(round(n_tris_target / (2.0 * (nv - 1)))))
    th = np.linspace(0.0, math.pi, nv + 1)
    ph = np.linspace(0.0, 2.0 * math.pi, nu + 1)[:-1]
    T, P = np.meshgrid(th, ph, indexing="ij")
    pts = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], -1)  # [nv+1, nu, 3]
    tris = []
    for i in range(nv):
        a = pts[i]
        b = pts[i + 1]
        a1 = np.roll(a, -1, axis=0)
        b1 = np.roll(b, -1, axis=0)
        if i != 0:
            tris.append(np.stack([a, b, a1], 1))
        if i != nv - 1:
            tris.append(np.stack([a1, b, b1], 1))
    return np.concatenate(tris, 0)


def scene_sphere_clusters(n_clusters: int = 64, seed: int = SEED_BASE + 3, min_tris: int = 1000,
                          max_tris: int = 200000, amplitude: float = 0.15) -> np.ndarray:
    """Displaced UV-spheres: triangle counts log-uniform in [min_tris, max_tris],
    radii U(0.02, 0.12), centres U([-1/2, 1/2]^3), fBm radial displacement of
    relative amplitude ``amplitude``."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_clusters):
        nt = int(round(math.exp(rng.uniform(math.log(min_tris), math.log(max_tris)))))
        s = _uv_sphere(nt, rng)
        flat = s.reshape(-1, 3)
        disp = 1.0 + amplitude * fbm(flat, seed * 131 + c)
        flat = flat * disp[:, None]
        r = rng.uniform(0.02, 0.12)
        ctr = rng.uniform(-0.5, 0.5, size=3)
        out.append((flat * r + ctr).reshape(-1, 3, 3))
    return np.concatenate(out, 0).astype(np.float32)


# ----------------------------------------------------------------------------
# Rays
# ----------------------------------------------------------------------------

def _pack(o: np.ndarray, d: np.ndarray, tmin, tmax) -> dict:
    n = len(o)
    return {
        "ox": np.ascontiguousarray(o[:, 0], np.float32),
        "oy": np.ascontiguousarray(o[:, 1], np.float32),
        "oz": np.ascontiguousarray(o[:, 2], np.float32),
        "dx": np.ascontiguousarray(d[:, 0], np.float32),
        "dy": np.ascontiguousarray(d[:, 1], np.float32),
        "dz": np.ascontiguousarray(d[:, 2], np.float32),
        "tmin": np.broadcast_to(np.asarray(tmin, np.float32), (n,)).copy(),
        "tmax": np.broadcast_to(np.asarray(tmax, np.float32), (n,)).copy(),
    }


def look_at_rays(width: int, height: int, eye, target=(0.0, 0.0, 0.0), fov_deg: float = 40.0) -> dict:
    """Pinhole primary rays, one per pixel centre, row-major, from ``eye``
    towards ``target``; up is +y (+x if colinear); vertical field of view
    ``fov_deg``."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    if abs(np.dot(up, fwd)) > 0.999:
        up = np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = math.tan(math.radians(fov_deg) / 2.0)
    aspect = width / height
    jj, ii = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    x = ((ii + 0.5) / width * 2.0 - 1.0) * th * aspect
    y = (1.0 - (jj + 0.5) / height * 2.0) * th
    d = fwd[None, :] + x.reshape(-1, 1) * right[None, :] + y.reshape(-1, 1) * upv[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(eye, d.shape)
    return _pack(o, d, 0.0, np.inf)


def camera_rays(width: int, height: int, seed: int = SEED_BASE + 7, radius: float = 2.0,
                fov_deg: float = 40.0) -> dict:
    """Pinhole primary rays, one per pixel centre, row-major. The camera sits at
    a seeded point of the sphere of radius ``radius`` and looks at the origin;
    up is +y (+x if colinear); vertical field of view ``fov_deg``."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    return look_at_rays(width, height, radius * u, (0.0, 0.0, 0.0), fov_deg)


def _sphere_dir(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], 1)


def chord_rays(n: int, seed: int, centre=(0.0, 0.0, 0.0), radius: float = 0.9) -> dict:
    """Rays from a uniform point of a sphere towards another uniform point of it;
    unit directions, tmax = chord length."""
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, np.float64)
    a = c + radius * _sphere_dir(rng, n)
    b = c + radius * _sphere_dir(rng, n)
    d = b - a
    ln = np.linalg.norm(d, axis=1)
    ln = np.where(ln > 0, ln, 1.0)
    d /= ln[:, None]
    return _pack(a, d, 0.0, ln)


def mixed_rays(n: int, seed: int, camera_fraction: float = 0.6, radius: float = 0.9) -> dict:
    """``camera_fraction`` of the rays from a seeded camera (radius 2, looking at
    the origin, directions uniform in a 40 degree cone), the rest as chords of
    the sphere of radius ``radius``."""
    rng = np.random.default_rng(seed)
    nc = int(round(n * camera_fraction))
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    eye = 2.0 * u
    fwd = -u
    cos_max = math.cos(math.radians(20.0))
    z = rng.uniform(cos_max, 1.0, nc)
    ph = rng.uniform(0.0, 2.0 * math.pi, nc)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    t1 = np.cross(fwd, [0.0, 1.0, 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(fwd, t1)
    dc = (z[:, None] * fwd + (s * np.cos(ph))[:, None] * t1 + (s * np.sin(ph))[:, None] * t2)
    cam = _pack(np.broadcast_to(eye, dc.shape), dc, 0.0, np.inf)
    ch = chord_rays(n - nc, seed + 1, radius=radius)
    return {k: np.concatenate([cam[k], ch[k]]) for k in RAY_KEYS}


def subset(rays: dict, idx: np.ndarray) -> dict:
    return {k: np.ascontiguousarray(rays[k][idx]) for k in RAY_KEYS}


# ----------------------------------------------------------------------------
# Parameters (random initialisation, Sec. 6 "Neural model & training")
# ----------------------------------------------------------------------------

def init_table(n_entries: int, n_features: int, seed: int, scale: float = 1e-4) -> np.ndarray:
    """Hash-table entries ~U(-scale, scale), float32 ``[n_entries, n_features]``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(n_entries, n_features)).astype(np.float32)


def init_mlp(dims, seed: int, gain: float = 1.0):
    """Dense layers ``dims[i] -> dims[i+1]``: weights ~N(0, gain/fan_in) stored
    ``[out, in]`` row-major, biases 0. Returns a list of (W, b) float32."""
    rng = np.random.default_rng(seed)
    layers = []
    for i in range(len(dims) - 1):
        w = rng.normal(0.0, math.sqrt(gain / dims[i]), size=(dims[i + 1], dims[i]))
        layers.append((w.astype(np.float32), np.zeros(dims[i + 1], np.float32)))
    return layers


def random_labels(n: int, seed: int, hit_fraction: float = 0.6, albedo: bool = False) -> dict:
    """Synthetic training labels: hit bit, local depth in [0, 1], unit normal,
    and with albedo=True an RGB albedo in [0, 1] (ar, ag, ab)."""
    rng = np.random.default_rng(seed)
    hit = (rng.uniform(size=n) < hit_fraction).astype(np.uint8)
    depth = rng.uniform(0.0, 1.0, n).astype(np.float32)
    nrm = _sphere_dir(rng, n).astype(np.float32)
    out = {"hit": hit, "depth": depth, "nx": nrm[:, 0].copy(), "ny": nrm[:, 1].copy(),
           "nz": nrm[:, 2].copy()}
    if albedo:
        a = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
        out.update(ar=a[:, 0].copy(), ag=a[:, 1].copy(), ab=a[:, 2].copy())
    return out


def tri_albedo(tris: np.ndarray, seed: int = SEED_BASE + 11) -> np.ndarray:
    """Per-triangle RGB albedo [n_tris][3] float32 in [0.05, 0.95]: fBm of the
    triangle's centroid, one seed per channel, so that nearby triangles have
    similar colours (a texture-like signal the albedo head can learn)."""
    c = np.asarray(tris, np.float64).reshape(-1, 3, 3).mean(axis=1)
    rgb = np.stack([fbm(c, seed + k, base_freq=3.0) for k in range(3)], axis=1)
    return (0.5 + 0.45 * np.clip(rgb * 1.6, -1.0, 1.0)).astype(np.float32)


# ----------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------

@dataclass
class ModelConfig:
    n_levels: int
    n_features: int
    log2_table: int
    base_res: int
    growth: float
    n_samples: int
    n_hidden: int
    width: int
    n_out: int = 5

    @property
    def n_inputs(self) -> int:
        return self.n_samples * self.n_levels * self.n_features

    def mlp_dims(self):
        return [self.n_inputs] + [self.width] * self.n_hidden + [self.n_out]


@dataclass
class Workload:
    name: str
    model: ModelConfig
    n_leaves: int
    table_dtype: str          # "f32" | "f16" | "bf16"
    inflate_rel: float = 1e-4
    extra: dict = field(default_factory=dict)


C0 = Workload(
    name="random-tris-4096_leaves-64_L4F2T12_N8_mlp2x32_rays-64x64",
    model=ModelConfig(n_levels=4, n_features=2, log2_table=12, base_res=16, growth=1.5,
                      n_samples=8, n_hidden=2, width=32),
    n_leaves=64, table_dtype="f32")

C1 = Workload(
    name="icosphere-l8-1310720tris_leaves-2048_L16F2T20-fp16_N16_mlp3x64_1920x1080+bounce",
    model=ModelConfig(n_levels=16, n_features=2, log2_table=20, base_res=16, growth=1.5,
                      n_samples=16, n_hidden=3, width=64),
    n_leaves=2048, table_dtype="f16")


# ----------------------------------------------------------------------------
# Hybrid scene: neural assets next to classical triangles (Sec. 7, Table 1:
# scenes mixing large assets, stored as N-BVHs, with ordinary geometry)
# ----------------------------------------------------------------------------

def ground_heightfield(n_cells: int = 500, half: float = 1.5, y0: float = -0.35, amplitude: float = 0.03,
                       seed: int = SEED_BASE + 5) -> np.ndarray:
    """A displaced ground grid over [-half, half]^2 (xz) at height ``y0``:
    (n_cells + 1)^2 vertices, 2 n_cells^2 triangles (500 cells: 500,000)."""
    g = np.linspace(-half, half, n_cells + 1)
    X, Z = np.meshgrid(g, g, indexing="ij")
    p = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], 1)
    h = fbm(p * 0.5, seed)
    P = np.stack([X.ravel(), y0 + amplitude * h, Z.ravel()], 1).reshape(n_cells + 1, n_cells + 1, 3)
    a, b = P[:-1, :-1], P[1:, :-1]
    c, d = P[:-1, 1:], P[1:, 1:]
    t1 = np.stack([a, c, b], 2).reshape(-1, 3, 3)
    t2 = np.stack([b, c, d], 2).reshape(-1, 3, 3)
    return np.concatenate([t1, t2], 0).astype(np.float32)


@dataclass
class HybridAsset:
    tris: np.ndarray
    model: "ModelConfig"
    n_leaves: int


def scene_hybrid(n_assets: int = 16, seed: int = SEED_BASE + 4, asset_level: int = 5, ground_cells: int = 500,
                 n_leaves: int = 128):
    """Neural assets on a classical ground. Each asset is a displaced icosphere
    (20 * 4^asset_level triangles, radius U(0.10, 0.18)) standing on the
    ground at a jittered 4x4 grid position; its model is the icosphere
    workload's (16 levels, base resolution 16, growth 1.5, 16 samples, a 3x64
    MLP) with F drawn from {2, 4, 8} and log2 T from {16, ..., 22} (seeded):
    N * L * F = 512, 1024 or 2048 first-layer inputs.
    Returns (ground triangles, [HybridAsset])."""
    rng = np.random.default_rng(seed)
    ground = ground_heightfield(ground_cells)
    assets = []
    side = int(math.ceil(math.sqrt(n_assets)))
    for k in range(n_assets):
        gx, gz = k % side, k // side
        r = rng.uniform(0.10, 0.18)
        cx = -1.05 + 2.1 * (gx + 0.5) / side + rng.uniform(-0.08, 0.08)
        cz = -1.05 + 2.1 * (gz + 0.5) / side + rng.uniform(-0.08, 0.08)
        tris = scene_icosphere(level=asset_level, seed=seed * 7 + k, radius=r, amplitude=0.2 * r)
        tris = tris + np.array([cx, -0.35 + r, cz], np.float32)
        F = int(rng.choice([2, 4, 8]))
        lt = int(rng.integers(16, 23))
        model = ModelConfig(n_levels=16, n_features=F, log2_table=lt, base_res=16, growth=1.5, n_samples=16,
                            n_hidden=3, width=64)
        assets.append(HybridAsset(tris.astype(np.float32), model, n_leaves))
    return ground, assets


def hybrid_camera_rays(width: int, height: int) -> dict:
    """The hybrid scene's camera: radius 3.2 at 35 degrees elevation, looking
    at (0, -0.2, 0), 40 degree vertical field of view."""
    el = math.radians(35.0)
    az = math.radians(30.0)
    eye = (3.2 * math.cos(el) * math.sin(az), 3.2 * math.sin(el), 3.2 * math.cos(el) * math.cos(az))
    return look_at_rays(width, height, eye, (0.0, -0.2, 0.0), 40.0)


C3 = Workload(
    name="sphere-clusters-64_leaves-8192_L16F2T20-fp16_N16_mlp3x64_4M-mixed-rays",
    model=ModelConfig(n_levels=16, n_features=2, log2_table=20, base_res=16, growth=1.5,
                      n_samples=16, n_hidden=3, width=64),
    n_leaves=8192, table_dtype="f16",
    extra={"n_clusters": 64, "min_tris": 1000, "max_tris": 200000, "n_rays": 4194304, "camera_fraction": 0.6})
