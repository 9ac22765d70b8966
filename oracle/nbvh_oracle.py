"""FP64 CPU oracle of the N-BVH neural ray query and its training step.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it. It shares no code with
the CUDA library (no kernels, headers, helpers or constant tables) and is a
plain, slow, step-by-step restatement of what the paper defines, in float64
(inputs stored in float32/float16 are upcast exactly).

Paper: Weier et al., "N-BVH: Neural ray queries with bounding volume
hierarchies", SIGGRAPH 2024. Sections cited below are that paper's.

Pipeline (Sec. 4 "Neural ray query", Fig. 3; Sec. 5; Sec. 6 "Implementation"):
  S0 ``build_leaves``      leaf boxes of a median-split BVH over triangle
                           centroids, slightly inflated (Sec. 5, Sec. 6).
  S1 ``ray_segments``      every leaf box a ray crosses, clipped to the ray's
                           [tmin, tmax], ordered front to back (Sec. 3, Sec. 5).
  S2 ``sample_points``     stratified points along each segment (Sec. 4).
  S3 ``encode``            multi-resolution hash-grid features of each point,
                           concatenated in ray order (Sec. 4, Fig. 3).
  S4 ``mlp_forward``       ReLU MLP decoding visibility, distance, normal
                           and, with 8 outputs, albedo (Sec. 5.2, Sec. 6).
  S5 ``decode``/``resolve``  per-segment hit and depth, closest predicted hit
                           per ray (Sec. 5: queries until an intersection).
  S7 ``train_rays``/``labels``  training rays and brute-force Moller-Trumbore
                           ground truth of the trained leaf (Sec. 4, Sec. 5.2).
  S8 ``loss``/``backward``/``adam``  combined loss and its analytic gradient
                           into MLP and hash table; Adam (Sec. 5.2, Sec. 6).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_*.py) against closed forms, brute force, invariants or
published test vectors; none is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np

F64 = np.float64

# Spatial-hash primes of the multi-resolution hash encoding (Mueller et al.
# 2022, the encoding Sec. 3 and Sec. 4 build on).
HASH_PRIMES = (1, 2654435761, 805459861)


# ============================================================================
# Level layout and grid frame (Sec. 3, Sec. 6 "Neural model & training")
# ============================================================================

def level_layout(n_levels: int, base_res: int, growth: float, log2_table: int):
    """Per level l: resolution N_l = floor(base_res * growth^l); the level is
    dense (direct indexing of the (N_l+1)^3 grid vertices) when that fits the
    table size T = 2^log2_table, hashed otherwise. Returns dict with int64
    arrays ``res``, ``dense``, ``size``, ``offset`` and ``total`` entries."""
    T = 1 << log2_table
    res, dense, size = [], [], []
    for l in range(n_levels):
        n = int(math.floor(base_res * growth ** l))
        res.append(n)
        verts = (n + 1) ** 3
        dense.append(verts <= T)
        size.append(verts if verts <= T else T)
    offset = np.concatenate([[0], np.cumsum(size)[:-1]]).astype(np.int64)
    return {"res": np.array(res, np.int64), "dense": np.array(dense, bool),
            "size": np.array(size, np.int64), "offset": offset,
            "total": int(np.sum(size)), "T": T}


def scene_frame(tris: np.ndarray):
    """Grid frame: the model is contained in the scene bounds (Sec. 5). Points
    map to the unit cube isotropically: xhat = (p - c)/E + 1/2 with c the centre
    and E the largest extent of the triangles' AABB. Also returns the bounding
    sphere used for chord training rays (centre c, radius 1.01 * half diagonal).
    The frame is a parameter of the model and is stored in float32
    (``model_centre``, ``model_extent``: the float64 values rounded to
    nearest float32); the encoding uses those stored values.
    """
    v = tris.reshape(-1, 3).astype(F64)
    lo = v.min(0)
    hi = v.max(0)
    c = (lo + hi) / 2.0
    E = float(np.max(hi - lo))
    R = 1.01 * float(np.linalg.norm(hi - lo)) / 2.0
    return {"lo": lo, "hi": hi, "centre": c, "extent": E, "sphere_radius": R,
            "model_centre": c.astype(np.float32).astype(F64),
            "model_extent": float(np.float32(E))}


# ============================================================================
# S0: leaf boxes (Sec. 5 leaves are hollow boxes over geometric clusters;
# Sec. 6 nodes are inflated slightly)
# ============================================================================

def _round_down_f32(x: np.ndarray) -> np.ndarray:
    f = x.astype(np.float32)
    bad = f.astype(F64) > x
    f[bad] = np.nextafter(f[bad], np.float32(-np.inf))
    return f


def _round_up_f32(x: np.ndarray) -> np.ndarray:
    f = x.astype(np.float32)
    bad = f.astype(F64) < x
    f[bad] = np.nextafter(f[bad], np.float32(np.inf))
    return f


def build_leaves(tris: np.ndarray, n_leaves: int, inflate_rel: float = 1e-4):
    """Median-split leaf clusters.

    Reading (the paper builds a SAH base BVH and cuts it; the configured
    workloads ask for a plain median split): starting from one leaf holding all
    triangles, repeatedly split the leaf with the most triangles (ties: lowest
    node id) until ``n_leaves`` leaves exist. A split sorts the leaf's
    triangles by their centroid coordinate on the axis of largest centroid
    extent (ties x < y < z; equal coordinates by triangle index) and gives the
    first floor(n/2) to the left child (node id next) and the rest to the right
    child (node id next + 1). Centroid = ((v0 + v1) + v2)/3 in float64.

    Leaves are numbered left to right (in-order over the split tree); each
    leaf's triangles are listed by ascending original index. Leaf boxes are
    the triangles' AABB moved out by ``inflate_rel * E`` on every face and
    rounded outward to float32.
    """
    t = tris.astype(F64)
    cent = ((t[:, 0] + t[:, 1]) + t[:, 2]) / 3.0
    n = len(tris)
    if n_leaves < 1 or n_leaves > n:
        raise ValueError("n_leaves must be in [1, n_tris]")
    # node: id -> (tri index array, left, right)
    tri_of = {0: np.arange(n)}
    children = {}
    leaves = {0}
    next_id = 1
    while len(leaves) < n_leaves:
        best = min(leaves, key=lambda i: (-len(tri_of[i]), i))
        idx = tri_of[best]
        if len(idx) < 2:
            raise ValueError("cannot split a leaf with fewer than two triangles")
        c = cent[idx]
        ext = c.max(0) - c.min(0)
        axis = int(np.argmax(ext))  # first maximum: ties x < y < z
        order = np.lexsort((idx, c[:, axis]))
        idx_sorted = idx[order]
        h = len(idx) // 2
        l_id, r_id = next_id, next_id + 1
        next_id += 2
        tri_of[l_id] = idx_sorted[:h]
        tri_of[r_id] = idx_sorted[h:]
        children[best] = (l_id, r_id)
        leaves.remove(best)
        leaves.update((l_id, r_id))

    order_leaves = []

    def walk(i):
        if i in children:
            walk(children[i][0])
            walk(children[i][1])
        else:
            order_leaves.append(i)

    walk(0)
    frame = scene_frame(tris)
    pad = inflate_rel * frame["extent"]
    perm, ranges, lo, hi = [], [], [], []
    start = 0
    v32 = tris.astype(F64)
    for i in order_leaves:
        idx = np.sort(tri_of[i])
        perm.append(idx)
        ranges.append((start, start + len(idx)))
        start += len(idx)
        pts = v32[idx].reshape(-1, 3)
        lo.append(pts.min(0) - pad)
        hi.append(pts.max(0) + pad)
    return {
        "tri_perm": np.concatenate(perm).astype(np.int32),
        "leaf_range": np.array(ranges, np.int32),
        "leaf_lo": _round_down_f32(np.array(lo)),
        "leaf_hi": _round_up_f32(np.array(hi)),
        "node_of_leaf": np.array(order_leaves, np.int64),
        "frame": frame,
    }


# ============================================================================
# S1: ray-box clip and segment lists (Sec. 3: probe only within ray-box
# intervals; Sec. 5: traverse, query each leaf reached)
# ============================================================================

def clip_ray_box(o, d, tmin, tmax, lo, hi):
    """Slab test of rays against boxes, broadcast over leading dims.

    o, d: [..., 3]; tmin, tmax: [...]; lo, hi: [..., 3]. For each axis with
    d_i != 0 the slab gives [min(a, b), max(a, b)] with a = (lo_i - o_i)/d_i,
    b = (hi_i - o_i)/d_i; with d_i == 0 the slab is all of R if
    lo_i <= o_i <= hi_i and empty otherwise. Entry/exit are the max/min over
    axes; the segment is [max(entry, tmin), min(exit, tmax)], kept iff
    t0 <= t1.

    Precision reading: ray-box clipping is float32 arithmetic in this method
    (inputs, boxes and segment endpoints are float32 data), so every slab
    value is the float32 value nearest the exact quotient (computed in
    float64, rounded once to float32); entry, exit, t0, t1 and the keep
    decision follow from those rounded values. Returns (keep, t0, t1, entry,
    exit) as float64 arrays holding float32 values."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    lo = np.asarray(lo, F64)
    hi = np.asarray(hi, F64)
    shape = np.broadcast_shapes(o.shape, lo.shape)[:-1]
    entry = np.full(shape, -np.inf)
    exit_ = np.full(shape, np.inf)
    empty = np.zeros(shape, bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for i in range(3):
            oi, di = o[..., i], d[..., i]
            a = ((lo[..., i] - oi) / di).astype(np.float32).astype(F64)
            b = ((hi[..., i] - oi) / di).astype(np.float32).astype(F64)
            near = np.minimum(a, b)
            far = np.maximum(a, b)
            zero = np.broadcast_to(di == 0, shape)
            inside = (lo[..., i] <= oi) & (oi <= hi[..., i])
            near = np.where(zero, -np.inf, near)
            far = np.where(zero, np.inf, far)
            empty = empty | (zero & ~np.broadcast_to(inside, shape))
            entry = np.maximum(entry, near)
            exit_ = np.minimum(exit_, far)
    t0 = np.maximum(entry, np.asarray(tmin, F64).astype(np.float32).astype(F64))
    t1 = np.minimum(exit_, np.asarray(tmax, F64).astype(np.float32).astype(F64))
    keep = (~empty) & (t0 <= t1)
    return keep, t0, t1, entry, exit_


def rays_od(rays: dict, idx=None):
    o = np.stack([rays["ox"], rays["oy"], rays["oz"]], -1).astype(F64)
    d = np.stack([rays["dx"], rays["dy"], rays["dz"]], -1).astype(F64)
    tmin = rays["tmin"].astype(F64)
    tmax = rays["tmax"].astype(F64)
    if idx is not None:
        return o[idx], d[idx], tmin[idx], tmax[idx]
    return o, d, tmin, tmax


def ray_segments(rays: dict, leaf_lo, leaf_hi, chunk: int = 1024, reverse_inside: bool = False):
    """All (ray, leaf) pairs whose clip is non-empty, sorted per ray by
    (t0, leaf id). With ``reverse_inside`` (the Sec. 6 reading of depth from
    within a node) a pair whose box entry lies below tmin (the origin is
    inside the box) is listed over the box's whole chord with swapped
    endpoints, t0 = exit > t1 = entry, and sorted by its entry.
    Returns CSR dict: ``offsets`` [R+1], ``ray``, ``leaf``,
    ``t0``, ``t1``, ``entry``, ``exit`` (float64) and per-pair ``grazing``
    pairs ``grazing_pairs`` [G, 2] = (ray, leaf) with |exit - entry| <= 1e-6,
    |entry - tmax| <= 1e-6 or |exit - tmin| <= 1e-6: touching or nearly
    touching pairs, whose membership another precision may decide either
    way."""
    o, d, tmin, tmax = rays_od(rays)
    R = len(o)
    out = {k: [] for k in ("ray", "leaf", "t0", "t1", "entry", "exit")}
    graz_pairs = []
    lo = np.asarray(leaf_lo, F64)[None]
    hi = np.asarray(leaf_hi, F64)[None]
    for s in range(0, R, chunk):
        e = min(R, s + chunk)
        keep, t0, t1, en, ex = clip_ray_box(o[s:e, None, :], d[s:e, None, :], tmin[s:e, None],
                                            tmax[s:e, None], lo, hi)
        tm = np.broadcast_to(tmax[s:e, None], en.shape)
        tn = np.broadcast_to(tmin[s:e, None], en.shape)
        graz = (np.abs(ex - en) <= 1e-6) | (np.abs(en - tm) <= 1e-6) | (np.abs(ex - tn) <= 1e-6)
        gr, gl = np.nonzero(graz)
        graz_pairs.append(np.stack([gr + s, gl], 1))
        r, l = np.nonzero(keep)
        out["ray"].append(r + s)
        out["leaf"].append(l)
        out["t0"].append(t0[r, l])
        out["t1"].append(t1[r, l])
        out["entry"].append(en[r, l])
        out["exit"].append(ex[r, l])
    seg = {k: np.concatenate(v) for k, v in out.items()}
    if reverse_inside:
        inside = (seg["entry"] < tmin[seg["ray"]]) & np.isfinite(seg["entry"]) & np.isfinite(seg["exit"])
        seg["t0"] = np.where(inside, seg["exit"], seg["t0"])
        seg["t1"] = np.where(inside, seg["entry"], seg["t1"])
    key = np.minimum(seg["t0"], seg["t1"])
    order = np.lexsort((seg["leaf"], key, seg["ray"]))
    seg = {k: v[order] for k, v in seg.items()}
    seg["offsets"] = np.concatenate([[0], np.cumsum(np.bincount(seg["ray"], minlength=R))]).astype(np.int64)
    seg["grazing_pairs"] = np.concatenate(graz_pairs, 0) if graz_pairs else np.zeros((0, 2), np.int64)
    return seg


# ============================================================================
# S2: stratified samples (Sec. 4 "Sampling & reconstruction quality")
# ============================================================================

def sample_points(o, d, t0, t1, n_samples: int):
    """Points p_k = o + t_k d with t_k = t0 + (k + 1/2)/N (t1 - t0), k in
    increasing order along the ray (stratum midpoints). Shapes: o, d [S, 3];
    t0, t1 [S] -> [S, N, 3]."""
    k = (np.arange(n_samples, dtype=F64) + 0.5) / n_samples
    t = np.asarray(t0, F64)[:, None] + k[None, :] * (np.asarray(t1, F64) - np.asarray(t0, F64))[:, None]
    return np.asarray(o, F64)[:, None, :] + t[..., None] * np.asarray(d, F64)[:, None, :]


def normalize_points(p, centre, extent):
    """Grid coordinates xhat = (p - c)/E + 1/2, clamped to [0, 1]^3."""
    x = (np.asarray(p, F64) - np.asarray(centre, F64)) / float(extent) + 0.5
    return np.clip(x, 0.0, 1.0)


def _fma32(a, b, c):
    """float32 fused multiply-add: the product of two float32 values is exact
    in float64, so one rounding of the float64 sum to float32 is the fused
    result (up to a double rounding of probability ~2^-29)."""
    return (np.asarray(a, np.float32).astype(F64) * np.asarray(b, np.float32).astype(F64)
            + np.asarray(c, np.float32).astype(F64)).astype(np.float32)


def sample_grid_f32(o, d, t0, t1, n_samples: int, centre, extent):
    """Grid coordinates of the stratified samples as the reduced-precision
    (FP16/BF16 tensor-core) form computes them: float32 throughout, one
    rounding per fused step. u_k = (k + 1/2)/N, t_k = fma(u_k, t1 - t0, t0),
    xhat = clamp(fma(fma(t_k, d, o) - c, 1/E, 1/2), 0, 1), 1/E rounded to
    float32. (Reading: the paper runs its model in half precision, Sec. 6; a
    half-precision oracle that models those operands also takes the form's
    float32 positions, since at the finest levels, resolution ~7,000, a float32
    position error is of the order of a 16-bit feature's rounding.) Shapes as
    sample_points; returns float64 arrays of float32 values."""
    f32 = np.float32
    o = np.asarray(o, f32)
    d = np.asarray(d, f32)
    t0 = np.asarray(t0, f32)
    t1 = np.asarray(t1, f32)
    u = (np.arange(n_samples, dtype=f32) + f32(0.5)) / f32(n_samples)
    dt = (t1 - t0).astype(f32)
    t = _fma32(u[None, :], dt[:, None], t0[:, None])
    p = _fma32(t[..., None], d[:, None, :], o[:, None, :])
    q = (p - np.asarray(centre, f32)).astype(f32)
    inv = f32(1.0) / f32(extent)
    x = _fma32(q, inv, f32(0.5))
    return np.clip(x, f32(0.0), f32(1.0)).astype(F64)


# ============================================================================
# S3: multi-resolution hash-grid encoding (Sec. 3, Sec. 4, Fig. 3)
# ============================================================================

def grid_index(c, res: int, dense: bool, T: int):
    """Table index of integer grid vertices c [..., 3] (each in 0..res)."""
    c = np.asarray(c, np.int64)
    if dense:
        n1 = res + 1
        return c[..., 0] + c[..., 1] * n1 + c[..., 2] * n1 * n1
    h = (c[..., 0].astype(np.uint64) * np.uint64(HASH_PRIMES[0])) & np.uint64(0xFFFFFFFF)
    h ^= (c[..., 1].astype(np.uint64) * np.uint64(HASH_PRIMES[1])) & np.uint64(0xFFFFFFFF)
    h ^= (c[..., 2].astype(np.uint64) * np.uint64(HASH_PRIMES[2])) & np.uint64(0xFFFFFFFF)
    return (h & np.uint64(T - 1)).astype(np.int64)


def level_corners(x, res: int, f32: bool = False):
    """Cell and trilinear corner weights of points x [..., 3] in [0,1] at
    resolution ``res``: cell = min(floor(x*res), res - 1), frac = x*res - cell.
    Returns (corners [..., 8, 3] int64, weights [..., 8]); corner bit b of the
    corner number selects +1 along axis b.

    ``f32``: the reduced-precision form's grid coordinates: x (float32) * res
    rounded once to float32, then cell and frac from that value (frac exact).
    (Reading, as for sample_grid_f32: at resolution ~7,000 the float32
    rounding of x * res moves frac by up to ~2e-4, of the order of a 16-bit
    feature's rounding, so a half-precision oracle takes the form's value.)"""
    if f32:
        pos = (np.asarray(x, np.float32) * np.float32(res)).astype(np.float32).astype(F64)
    else:
        pos = np.asarray(x, F64) * res
    cell = np.minimum(np.floor(pos), res - 1).astype(np.int64)
    frac = pos - cell
    corners, weights = [], []
    for c in range(8):
        delta = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1], np.int64)
        corners.append(cell + delta)
        w = np.ones(pos.shape[:-1])
        for a in range(3):
            w = w * (frac[..., a] if delta[a] else 1.0 - frac[..., a])
        weights.append(w)
    return np.stack(corners, -2), np.stack(weights, -1)


def encode(x, table, layout, f32: bool = False):
    """Features of points x [S, N, 3] (grid coords): for each sample k, level l
    and feature f, the trilinear interpolation of the 8 surrounding vertices'
    table entries. Concatenation order index = k*L*F + l*F + f, i.e. samples in
    ray order (Sec. 4: the order encodes the ray's direction).
    ``table`` [total, F] (any float dtype; the gathered entries are upcast
    exactly). ``f32``: float32 grid coordinates (level_corners). Returns
    [S, N*L*F]."""
    tab = np.asarray(table)
    S, N, _ = x.shape
    L = len(layout["res"])
    F = tab.shape[1]
    out = np.zeros((S, N, L, F))
    for l in range(L):
        corners, w = level_corners(x, int(layout["res"][l]), f32)
        idx = grid_index(corners, int(layout["res"][l]), bool(layout["dense"][l]), layout["T"])
        vals = tab[layout["offset"][l] + idx].astype(F64)  # [S, N, 8, F]
        out[:, :, l, :] = np.sum(w[..., None] * vals, axis=2)
    return out.reshape(S, N * L * F)


# ============================================================================
# S4: MLP (Sec. 6: ReLU hidden layers; sigmoid on distance, linear normal)
# ============================================================================

def _same(a):
    return a


def mlp_forward(feat, layers, rnd=None):
    """ReLU hidden layers, linear last layer. ``layers`` = [(W [out,in], b)].
    Returns raw outputs [S, n_out] and the list of layer inputs (activations)
    and pre-activations for the backward pass.

    ``rnd``: optional rounding of the multiplication operands to a
    half-precision type (Sec. 6 trains and infers in half precision): each
    layer's input and weight matrix are rounded, products and sums stay exact
    and the bias is added unrounded. The layer inputs returned are the rounded
    ones."""
    r = rnd or _same
    h = r(np.asarray(feat, F64))
    acts, pre = [h], []
    for i, (W, b) in enumerate(layers):
        z = h @ r(np.asarray(W, F64)).T + np.asarray(b, F64)
        pre.append(z)
        if i < len(layers) - 1:
            h = r(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = z
    return h, acts, pre


def sigmoid(x):
    x = np.asarray(x, F64)
    e = np.exp(-np.abs(x))
    return np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


# ============================================================================
# S5: decode and resolve (Sec. 5.2 visibility / local distance / normal;
# Sec. 5: the first intersection along the ray)
# ============================================================================

def decode(raw, t0, t1):
    """Per segment: hit iff hit logit > 0 (sigmoid > 1/2, Sec. 5.2
    "Visibility"); t = t0 + sigmoid(o_d) (t1 - t0) (distance local to the
    segment, Sec. 5.2 "Intersection point"); normal = o_n/|o_n| (linear head,
    Sec. 6), (0, 0, 1) for a zero vector."""
    raw = np.asarray(raw, F64)
    hit = raw[:, 0] > 0.0
    t = np.asarray(t0, F64) + sigmoid(raw[:, 1]) * (np.asarray(t1, F64) - np.asarray(t0, F64))
    n = raw[:, 2:5]
    ln = np.linalg.norm(n, axis=1)
    nrm = np.where(ln[:, None] > 0, n / np.where(ln > 0, ln, 1.0)[:, None], np.array([0.0, 0.0, 1.0]))
    return hit, t, nrm


def decode_albedo(raw):
    """Albedo of each segment from a model with an albedo head (outputs 5-7):
    sigmoid of the three logits, so that it lies in [0, 1] like the signal it
    learns (Sec. 5.2 "Auxiliary intersection data"); None without the head."""
    raw = np.asarray(raw, F64)
    return sigmoid(raw[:, 5:8]) if raw.shape[1] >= 8 else None


def resolve(n_rays: int, seg, hit, t, nrm, albedo=None):
    """Closest predicted hit per ray over all its segments; equal t goes to the
    segment first in (t0, leaf) order. Rays without a predicted hit get
    hit = 0, t = +inf, leaf = -1, normal = 0 (and albedo 0 when given)."""
    out_hit = np.zeros(n_rays, np.uint8)
    out_t = np.full(n_rays, np.inf)
    out_n = np.zeros((n_rays, 3))
    out_a = np.zeros((n_rays, 3))
    out_leaf = np.full(n_rays, -1, np.int64)
    off = seg["offsets"]
    for r in range(n_rays):
        best = None
        for j in range(off[r], off[r + 1]):
            if hit[j] and (best is None or t[j] < t[best]):
                best = j
        if best is not None:
            out_hit[r] = 1
            out_t[r] = t[best]
            out_n[r] = nrm[best]
            out_leaf[r] = seg["leaf"][best]
            if albedo is not None:
                out_a[r] = albedo[best]
    res = {"hit": out_hit, "t": out_t, "normal": out_n, "leaf": out_leaf}
    if albedo is not None:
        res["albedo"] = out_a
    return res


def eval_segments(o, d, t0, t1, table, layers, layout, centre, extent, n_samples: int):
    """S2 -> S4 for a list of segments: features, raw MLP outputs."""
    p = sample_points(o, d, t0, t1, n_samples)
    x = normalize_points(p, centre, extent)
    feat = encode(x, table, layout)
    raw, _, _ = mlp_forward(feat, layers)
    return feat, raw


def query(rays: dict, leaves: dict, table, layers, layout, n_samples: int, chunk: int = 4096,
          reverse_inside: bool = False):
    """The full neural ray query: S1 -> S5 over every segment of every ray.
    With ``reverse_inside`` a chord listed reversed (t0 > t1, see
    ray_segments) is sampled from its exit back to its entry, its hit lies at
    t = exit - sigmoid(o_d) (exit - entry) and counts only if tmin < t <= tmax."""
    seg = ray_segments(rays, leaves["leaf_lo"], leaves["leaf_hi"], reverse_inside=reverse_inside)
    o, d, _, _ = rays_od(rays)
    fr = leaves["frame"]
    S = len(seg["ray"])
    raws, feats = [], []
    for s in range(0, S, chunk):
        e = min(S, s + chunk)
        rr = seg["ray"][s:e]
        f, r = eval_segments(o[rr], d[rr], seg["t0"][s:e], seg["t1"][s:e], table, layers, layout,
                             fr["model_centre"], fr["model_extent"], n_samples)
        raws.append(r)
        feats.append(f)
    raw = np.concatenate(raws) if raws else np.zeros((0, layers[-1][0].shape[0]))
    hit, t, nrm = decode(raw, seg["t0"], seg["t1"])
    if reverse_inside:
        rev = seg["t0"] > seg["t1"]
        _, _, tmin, tmax = rays_od(rays)
        rr = seg["ray"]
        hit = hit & (~rev | ((t > tmin[rr]) & (t <= tmax[rr])))
    res = resolve(len(o), seg, hit, t, nrm, decode_albedo(raw))
    res["segments"] = seg
    res["raw"] = raw
    res["seg_hit"] = hit
    res["seg_t"] = t
    return res


# ============================================================================
# Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC 2011)
# ============================================================================

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(ctr, key):
    """ctr: 4 uint32 arrays (broadcastable), key: 2 uint32 values/arrays.
    Ten rounds; the key is bumped by the Weyl constants between rounds.
    Returns 4 uint32 arrays."""
    M = np.uint64(0xFFFFFFFF)
    x = [np.asarray(c, np.uint64) & M for c in ctr]
    k0 = np.asarray(key[0], np.uint64) & M
    k1 = np.asarray(key[1], np.uint64) & M
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & M
            k1 = (k1 + np.uint64(PHILOX_W1)) & M
        p0 = np.uint64(PHILOX_M0) * x[0]
        p1 = np.uint64(PHILOX_M1) * x[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & M
        hi1, lo1 = p1 >> np.uint64(32), p1 & M
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return [v.astype(np.uint32) for v in x]


def u24(x):
    """Uniform in [0, 1): the top 24 bits of a uint32 times 2^-24 (exact)."""
    return (np.asarray(x, np.uint32) >> np.uint32(8)).astype(F64) * (1.0 / 16777216.0)


def sphere_dir(u1, u2):
    """Uniform direction on S^2: z = 1 - 2 u1, phi = 2 pi u2."""
    z = 1.0 - 2.0 * u1
    phi = 2.0 * math.pi * u2
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], -1)


def _keys(seed: int):
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


# ============================================================================
# S7: training rays and labels (Sec. 4 "Encoding, inference & training";
# Sec. 5.2 "Ray distribution": each ray trains the first leaf it meets)
# ============================================================================

TRAIN_MODE_PROBED_MIX = 0   # even index: BVH-probed ray through a random leaf; odd: sphere chord
TRAIN_MODE_PAPER = 1        # origin uniform in the 1.5x scene box, uniform direction


def first_leaf(o, d, tmin, tmax, leaf_lo, leaf_hi):
    """First leaf a ray meets: minimum (t0, leaf id). Returns (leaf or -1, t0, t1)."""
    keep, t0, t1, _, _ = clip_ray_box(o[:, None, :], d[:, None, :], tmin[:, None], tmax[:, None],
                                      np.asarray(leaf_lo, F64)[None], np.asarray(leaf_hi, F64)[None])
    key = np.where(keep, t0, np.inf)
    leaf = np.argmin(key, axis=1)  # first minimum: lowest leaf id among equal t0
    ok = keep[np.arange(len(o)), leaf]
    r = np.arange(len(o))
    return np.where(ok, leaf, -1), np.where(ok, t0[r, leaf], 0.0), np.where(ok, t1[r, leaf], 0.0)


def train_rays(mode: int, seed: int, step: int, n: int, leaves: dict):
    """Training rays of one step, from Philox keyed by ``seed`` with counter
    (ray index, step lo, step hi, draw block). Returns dict with o, d, tmin,
    tmax (float64) and the trained leaf with its segment [t0, t1]; leaf = -1
    marks a ray that meets no leaf (it does not train).

    * probed mix (even ray index): leaf = floor(r0 * n_leaves / 2^32), a point
      uniform in that leaf's box, a uniform direction, origin moved back along
      -d to the bounding sphere; the ray trains that leaf.
    * probed mix (odd index): chord between two uniform points of the
      bounding sphere; trains the first leaf it meets.
    * paper mode: origin uniform in the scene box inflated by 50%, uniform
      direction; trains the first leaf it meets.
    """
    i = np.arange(n, dtype=np.uint64)
    key = _keys(seed)
    s_lo, s_hi = step & 0xFFFFFFFF, (step >> 32) & 0xFFFFFFFF
    r = philox4x32_10([i, s_lo, s_hi, 0], key)
    q = philox4x32_10([i, s_lo, s_hi, 1], key)
    fr = leaves["frame"]
    C = fr["centre"]
    R = fr["sphere_radius"]
    lo = leaves["leaf_lo"].astype(F64)
    hi = leaves["leaf_hi"].astype(F64)
    L = len(lo)
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    tmin = np.zeros(n)
    tmax = np.full(n, np.inf)
    leaf = np.full(n, -1, np.int64)
    t0 = np.zeros(n)
    t1 = np.zeros(n)
    if mode == TRAIN_MODE_PROBED_MIX:
        pr = (np.arange(n) % 2) == 0
        # probed rays
        lf = ((r[0].astype(np.uint64) * np.uint64(L)) >> np.uint64(32)).astype(np.int64)
        u = np.stack([u24(r[1]), u24(r[2]), u24(r[3])], -1)
        p = lo[lf] + u * (hi[lf] - lo[lf])
        dd = sphere_dir(u24(q[0]), u24(q[1]))
        w = p - C
        b = np.sum(w * dd, -1)
        c = np.sum(w * w, -1) - R * R
        tb = b + np.sqrt(np.maximum(0.0, b * b - c))
        op = p - tb[:, None] * dd
        # chords
        a = C + R * sphere_dir(u24(r[0]), u24(r[1]))
        e = C + R * sphere_dir(u24(r[2]), u24(r[3]))
        v = e - a
        ln = np.linalg.norm(v, axis=1)
        dc = np.where(ln[:, None] > 0, v / np.where(ln > 0, ln, 1.0)[:, None], np.array([0.0, 0.0, 1.0]))
        o = np.where(pr[:, None], op, a)
        d = np.where(pr[:, None], dd, dc)
        tmax = np.where(pr, np.inf, ln)
        # segments
        keep, s0, s1, _, _ = clip_ray_box(o, d, tmin, tmax, lo[lf], hi[lf])
        fl, f0, f1 = first_leaf(o, d, tmin, tmax, lo, hi)
        leaf = np.where(pr, np.where(keep, lf, -1), fl)
        t0 = np.where(pr, s0, f0)
        t1 = np.where(pr, s1, f1)
    elif mode == TRAIN_MODE_PAPER:
        ext = fr["hi"] - fr["lo"]
        u = np.stack([u24(r[0]), u24(r[1]), u24(r[2])], -1)
        o = C + (u - 0.5) * (1.5 * ext)
        d = sphere_dir(u24(r[3]), u24(q[0]))
        leaf, t0, t1 = first_leaf(o, d, tmin, tmax, lo, hi)
    else:
        raise ValueError("unknown training ray mode")
    t0 = np.where(leaf >= 0, t0, 0.0)
    t1 = np.where(leaf >= 0, t1, 0.0)
    return {"o": o, "d": d, "tmin": tmin, "tmax": tmax, "leaf": leaf, "t0": t0, "t1": t1}


def moller_trumbore(o, d, v0, v1, v2):
    """Moller & Trumbore (1997) ray-triangle test, broadcast over leading dims.
    Edges inclusive (u >= 0, v >= 0, u + v <= 1); det == 0 is a miss.
    Returns (hit, t, u, v)."""
    e1 = v1 - v0
    e2 = v2 - v0
    p = np.cross(d, e2)
    det = np.sum(e1 * p, -1)
    ok = det != 0.0
    inv = 1.0 / np.where(ok, det, 1.0)
    s = o - v0
    u = np.sum(s * p, -1) * inv
    q = np.cross(s, e1)
    v = np.sum(d * q, -1) * inv
    t = np.sum(e2 * q, -1) * inv
    hit = ok & (u >= 0.0) & (v >= 0.0) & (u + v <= 1.0)
    return hit, t, u, v


def labels(o, d, leaf, t0, t1, tris, tri_perm, leaf_range, tri_albedo=None):
    """Ground truth of the trained segment: the closest intersection among the
    leaf's own triangles with t in [t0, t1] (Sec. 4: obtained by intersecting
    the actual geometry). Equal t: the lowest position in the leaf's list.
    Returns hit (uint8), local depth (t - t0)/(t1 - t0) (0 for t1 == t0), the
    geometric normal flipped to face -d (Sec. 5.2), the hit t and margins
    describing how close each decision was (for rounding exceptions); with
    ``tri_albedo`` ([n_tris][3]) also the hit triangle's albedo (0 on a miss)."""
    n = len(o)
    tv = tris.astype(F64)
    hit = np.zeros(n, np.uint8)
    depth = np.zeros(n)
    nrm = np.zeros((n, 3))
    alb = np.zeros((n, 3))
    thit = np.full(n, np.inf)
    margin = np.full(n, np.inf)
    for i in range(n):
        if leaf[i] < 0:
            continue
        a, b = leaf_range[leaf[i]]
        T = tv[tri_perm[a:b]]
        h, t, u, v = moller_trumbore(o[i][None], d[i][None], T[:, 0], T[:, 1], T[:, 2])
        inside = h & (t >= t0[i]) & (t <= t1[i])
        # closeness of every triangle's decision to its boundary
        m = np.minimum.reduce([np.abs(u), np.abs(v), np.abs(1.0 - u - v),
                               np.abs(t - t0[i]), np.abs(t - t1[i])])
        margin[i] = np.min(np.where(np.isfinite(m), m, np.inf)) if len(m) else np.inf
        if not np.any(inside):
            continue
        tt = np.where(inside, t, np.inf)
        j = int(np.argmin(tt))
        srt = np.sort(tt[np.isfinite(tt)])
        if len(srt) > 1:
            margin[i] = min(margin[i], srt[1] - srt[0])
        hit[i] = 1
        thit[i] = t[j]
        span = t1[i] - t0[i]
        depth[i] = (t[j] - t0[i]) / span if span > 0 else 0.0
        g = np.cross(T[j, 1] - T[j, 0], T[j, 2] - T[j, 0])
        g = g / np.linalg.norm(g)
        if np.dot(g, d[i]) > 0:
            g = -g
        nrm[i] = g
        if tri_albedo is not None:
            alb[i] = np.asarray(tri_albedo, F64)[tri_perm[a + j]]
    out = {"hit": hit, "depth": depth, "normal": nrm, "t": thit, "margin": margin}
    if tri_albedo is not None:
        out["albedo"] = alb
    return out


# ============================================================================
# S8: loss, analytic gradient, Adam (Sec. 5.2 losses and "Combined loss";
# Sec. 6 "Neural model & training")
# ============================================================================

W_VIS, W_DIST, W_NORMAL, W_ALBEDO = 2.0, 2.0, 1.0, 1.0
# Relative L2 (Sec. 5.2 "Auxiliary intersection data"): the squared error over
# the prediction's own square plus this constant, the denominator held fixed.
ALBEDO_EPS = 0.01


def softplus(x):
    x = np.asarray(x, F64)
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def loss(raw, y_hit, y_depth, y_normal, valid, y_albedo=None):
    """L = (1/n_valid) sum over valid rays of
         2 BCE(sigmoid(o_hit), y) + y (2 |sigmoid(o_d) - d| + (1/3) sum_j |o_nj - n_j|)
    (Sec. 5.2: BCE for visibility, L1 on local distance, L1 on the normal, the
    other losses zeroed without an intersection; combined weights 2, 2, 1).
    BCE from the logit: softplus(o) - y o. With an albedo head (8 outputs) and
    albedo labels the term adds, weight 1, y times the relative L2 of the
    albedo averaged over RGB: (1/3) sum_c (s_c - a_c)^2 / (s_c^2 + 0.01),
    s_c = sigmoid(o_{5+c}). Returns (L, per-ray terms)."""
    raw = np.asarray(raw, F64)
    y = np.asarray(y_hit, F64)
    v = np.asarray(valid, bool)
    nv = max(1, int(v.sum()))
    bce = softplus(raw[:, 0]) - y * raw[:, 0]
    dist = np.abs(sigmoid(raw[:, 1]) - np.asarray(y_depth, F64))
    nl1 = np.sum(np.abs(raw[:, 2:5] - np.asarray(y_normal, F64)), 1) / 3.0
    per = W_VIS * bce + y * (W_DIST * dist + W_NORMAL * nl1)
    if y_albedo is not None and raw.shape[1] >= 8:
        s = sigmoid(raw[:, 5:8])
        rel = np.sum((s - np.asarray(y_albedo, F64)) ** 2 / (s * s + ALBEDO_EPS), 1) / 3.0
        per = per + y * W_ALBEDO * rel
    per = np.where(v, per, 0.0)
    return float(per.sum() / nv), per


def loss_grad(raw, y_hit, y_depth, y_normal, valid, y_albedo=None):
    """dL/d(raw outputs) of ``loss`` (sign(0) = 0 at the L1 kinks; the
    relative L2's denominator is a constant, so its gradient is
    2 (s - a) / (s^2 + 0.01) times sigmoid's derivative)."""
    raw = np.asarray(raw, F64)
    y = np.asarray(y_hit, F64)
    v = np.asarray(valid, bool).astype(F64)
    nv = max(1.0, float(v.sum()))
    g = np.zeros_like(raw)
    s0 = sigmoid(raw[:, 0])
    g[:, 0] = W_VIS * (s0 - y)
    s1 = sigmoid(raw[:, 1])
    g[:, 1] = y * W_DIST * np.sign(s1 - np.asarray(y_depth, F64)) * s1 * (1.0 - s1)
    g[:, 2:5] = y[:, None] * (W_NORMAL / 3.0) * np.sign(raw[:, 2:5] - np.asarray(y_normal, F64))
    if y_albedo is not None and raw.shape[1] >= 8:
        s = sigmoid(raw[:, 5:8])
        g[:, 5:8] = (y[:, None] * (W_ALBEDO / 3.0) * 2.0 * (s - np.asarray(y_albedo, F64)) / (s * s + ALBEDO_EPS)
                     * s * (1.0 - s))
    return g * (v / nv)[:, None]


def mlp_backward(g_out, acts, pre, layers, rnd=None, scale: float = 1.0):
    """Backward of ``mlp_forward``: returns (dfeatures, [(dW, db)]).

    ``rnd`` (half-precision operands, as in ``mlp_forward``): the gradient that
    enters each product with a weight matrix is rounded, dL/d(raw) after
    multiplication by the loss scale ``scale`` (a power of two) so that small
    values keep their precision; the weights are rounded; the hidden layers'
    weight gradients take the rounded dZ and the output layer's the unrounded
    dL/d(raw). The ReLU mask is the stored activation's sign."""
    r = rnd or _same
    grads = [None] * len(layers)
    g = np.asarray(g_out, F64)
    last = len(layers) - 1
    for i in range(last, -1, -1):
        W = r(np.asarray(layers[i][0], F64))
        gq = g if rnd is None else r(g * scale) / scale
        gw = g if i == last else gq
        grads[i] = (gw.T @ acts[i], gw.sum(0))
        g = gq @ W
        if i > 0:
            g = g * (acts[i] > 0.0)
    return g, grads


def encode_backward(x, g_feat, n_entries: int, n_features: int, layout, f32: bool = False):
    """Adjoint of ``encode``: every (sample, level, corner) adds
    weight * dL/dfeature into its table entry (collisions accumulate)."""
    S, N, _ = x.shape
    L = len(layout["res"])
    F = n_features
    g = np.asarray(g_feat, F64).reshape(S, N, L, F)
    out = np.zeros((n_entries, F))
    for l in range(L):
        corners, w = level_corners(x, int(layout["res"][l]), f32)
        idx = grid_index(corners, int(layout["res"][l]), bool(layout["dense"][l]), layout["T"])
        rows = (layout["offset"][l] + idx).reshape(-1)
        contrib = (w[..., None] * g[:, :, l, None, :]).reshape(-1, F)
        np.add.at(out, rows, contrib)
    return out


def forward_backward(o, d, t0, t1, valid, y_hit, y_depth, y_normal, table, layers, layout,
                     centre, extent, n_samples: int, rnd=None, scale: float = 1.0, y_albedo=None,
                     positions: str = "f64"):
    """Loss of a batch of segments and its exact gradient with respect to every
    table entry and MLP weight/bias. Returns (L, dtable, [(dW, db)], raw).
    ``rnd``/``scale``: half-precision MLP operands (``mlp_forward``,
    ``mlp_backward``); the encoding and the table gradient stay exact.
    ``positions``: "f64" (exact sample points) or "f32" (the reduced-precision
    form's float32 positions, sample_grid_f32, and grid coordinates,
    level_corners(f32=True))."""
    f32 = positions == "f32"
    if f32:
        x = sample_grid_f32(o, d, t0, t1, n_samples, centre, extent)
    else:
        p = sample_points(o, d, t0, t1, n_samples)
        x = normalize_points(p, centre, extent)
    feat = encode(x, table, layout, f32)
    raw, acts, pre = mlp_forward(feat, layers, rnd)
    L, _ = loss(raw, y_hit, y_depth, y_normal, valid, y_albedo)
    g = loss_grad(raw, y_hit, y_depth, y_normal, valid, y_albedo)
    g_feat, g_layers = mlp_backward(g, acts, pre, layers, rnd, scale)
    tab = np.asarray(table)
    g_tab = encode_backward(x, g_feat, tab.shape[0], tab.shape[1], layout, f32)
    return L, g_tab, g_layers, raw


def adam(param, grad, m, v, step: int, lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """Adam (Kingma & Ba 2015) with bias correction; ``step`` counts from 1.
    Returns (param, m, v) new arrays."""
    p = np.asarray(param, F64)
    g = np.asarray(grad, F64)
    m = beta1 * np.asarray(m, F64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, F64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ============================================================================
# Secondary bounce (Sec. 7: the path tracer samples the next direction at the
# returned intersection); cosine-weighted about the predicted normal
# ============================================================================

def onb(n):
    """Orthonormal basis (t, b) completing unit n (Duff et al., "Building an
    Orthonormal Basis, Revisited", JCGT 2017)."""
    n = np.asarray(n, F64)
    sgn = np.where(n[..., 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sgn + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t = np.stack([1.0 + sgn * n[..., 0] ** 2 * a, sgn * b, -sgn * n[..., 0]], -1)
    bt = np.stack([b, sgn + n[..., 1] ** 2 * a, -n[..., 1]], -1)
    return t, bt


BOUNCE_OFFSET = 1e-4


def bounce_rays(o, d, t, nrm, ray_index, seed: int):
    """For hits: origin = o + t d + 1e-4 n' with n' the predicted normal turned
    to face -d; direction cosine-weighted about n' from Philox counter
    (ray index low word, ray index high word, 0, 2) keyed by the seed's two
    words: r = sqrt(u1), phi = 2 pi u2."""
    n = np.asarray(nrm, F64).copy()
    flip = np.sum(n * d, -1) > 0
    n[flip] = -n[flip]
    p = o + t[:, None] * d + BOUNCE_OFFSET * n
    ri = np.asarray(ray_index, np.uint64)
    r = philox4x32_10([ri & np.uint64(0xFFFFFFFF), ri >> np.uint64(32), 0, 2], _keys(seed))
    u1, u2 = u24(r[0]), u24(r[1])
    rad = np.sqrt(u1)
    phi = 2.0 * math.pi * u2
    x, y, z = rad * np.cos(phi), rad * np.sin(phi), np.sqrt(np.maximum(0.0, 1.0 - u1))
    tt, bb = onb(n)
    dirs = x[:, None] * tt + y[:, None] * bb + z[:, None] * n
    return p, dirs


# ============================================================================
# S9: the hybrid two-level hierarchy (Sec. 7 "Application: Hybrid path
# tracing"): each bottom-level structure is a classical triangle BVH or an
# N-BVH, both answer with the same intersection record, and the ray keeps the
# closest answer over all of them
# ============================================================================

def closest_triangle_hit(o, d, tmin, tmax, tris, eps: float = 1e-5):
    """Brute force over every triangle (Moller-Trumbore, edges inclusive,
    det == 0 a miss): the closest t in [tmin, tmax], equal t to the lowest
    triangle index; normal = geometric normal turned to face -d.
    ``margin`` is how close the answer is to flipping: the smallest distance
    of a candidate's barycentrics to the triangle's edges among triangles
    within eps of being a hit no farther than the answer, the gap to the next
    candidate's t, and the answer's distance to tmin / tmax."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    tv = np.asarray(tris, F64)
    v0, v1, v2 = tv[:, 0], tv[:, 1], tv[:, 2]
    n = len(o)
    hit = np.zeros(n, np.uint8)
    t_out = np.full(n, np.inf)
    nrm = np.zeros((n, 3))
    idx = np.full(n, -1, np.int64)
    margin = np.full(n, np.inf)
    for i in range(n):
        h, t, u, v = moller_trumbore(o[i][None], d[i][None], v0, v1, v2)
        inside = h & (t >= tmin[i]) & (t <= tmax[i])
        best = np.inf
        if np.any(inside):
            tt = np.where(inside, t, np.inf)
            best = float(np.min(tt))
            j = int(np.flatnonzero(tt == best)[0])   # lowest index among equal t
            hit[i] = 1
            t_out[i] = best
            idx[i] = j
            g = np.cross(v1[j] - v0[j], v2[j] - v0[j])
            g = g / np.linalg.norm(g)
            if np.dot(g, d[i]) > 0:
                g = -g
            nrm[i] = g
            srt = np.sort(tt[np.isfinite(tt)])
            if len(srt) > 1:
                margin[i] = min(margin[i], srt[1] - srt[0])
            margin[i] = min(margin[i], best - tmin[i], tmax[i] - best)
        lim = min(best, tmax[i]) + eps
        near = (np.isfinite(t) & (u >= -eps) & (v >= -eps) & (u + v <= 1.0 + eps) & (t >= tmin[i] - eps)
                & (t <= lim))
        if np.any(near):
            m = np.minimum.reduce([np.abs(u[near]), np.abs(v[near]), np.abs(1.0 - u[near] - v[near])])
            margin[i] = min(margin[i], float(np.min(m)))
    return {"hit": hit, "t": t_out, "normal": nrm, "index": idx, "margin": margin}


def hybrid_trace(rays: dict, instances):
    """Closest hit over the instances, taken in index order: an instance's
    answer replaces the record only when it is a hit strictly closer than the
    record (equal t stays with the lower instance index). Instances are dicts:
    {"kind": "triangles", "tris": [n, 3, 3], optional "albedo": [n, 3]} or
    {"kind": "neural", "leaves", "table", "layers", "layout", "n_samples"}
    (each neural instance answers with ``query`` over the ray's full
    [tmin, tmax]). Returns the record (hit, t, normal, leaf = triangle index
    or N-BVH leaf, inst, albedo: the triangle's, the albedo head's, or 0 where
    the answering instance has none) and every instance's own answer."""
    o, d, tmin, tmax = rays_od(rays)
    n = len(o)
    out = {"hit": np.zeros(n, np.uint8), "t": np.full(n, np.inf), "normal": np.zeros((n, 3)),
           "leaf": np.full(n, -1, np.int64), "inst": np.full(n, -1, np.int64), "albedo": np.zeros((n, 3))}
    answers = []
    for k, x in enumerate(instances):
        if x["kind"] == "triangles":
            a = closest_triangle_hit(o, d, tmin, tmax, x["tris"])
            ans = {"hit": a["hit"], "t": a["t"], "normal": a["normal"], "leaf": a["index"], "margin": a["margin"]}
            alb = np.zeros((n, 3))
            if x.get("albedo") is not None:
                h = a["index"] >= 0
                alb[h] = np.asarray(x["albedo"], F64)[a["index"][h]]
            ans["albedo"] = alb
        else:
            q = query(rays, x["leaves"], x["table"], x["layers"], x["layout"], x["n_samples"])
            ans = {"hit": q["hit"], "t": q["t"], "normal": q["normal"], "leaf": q["leaf"], "query": q,
                   "albedo": q.get("albedo", np.zeros((n, 3)))}
        answers.append(ans)
        better = ans["hit"].astype(bool) & (ans["t"] < out["t"])
        out["hit"][better] = 1
        out["t"][better] = ans["t"][better]
        out["normal"][better] = ans["normal"][better]
        out["leaf"][better] = ans["leaf"][better]
        out["inst"][better] = k
        out["albedo"][better] = ans["albedo"][better]
    out["answers"] = answers
    return out


# ============================================================================
# Error-driven construction (Sec. 5.1 "Base-BVH cut optimization", "Node
# error"; Sec. 5.2 "Ray distribution")
# ============================================================================

def training_selection(leaf, prob, seed: int, step: int):
    """Which rays train their first leaf: ray i with first leaf l >= 0 trains
    iff u < prob[l], u = top 24 bits of the first word of Philox4x32-10 with
    counter (i, step low, step high, 3) keyed by the seed's words, * 2^-24."""
    leaf = np.asarray(leaf, np.int64)
    i = np.arange(len(leaf), dtype=np.uint64)
    st = np.uint64(step)
    r = philox4x32_10([i & np.uint64(0xFFFFFFFF), np.full_like(i, st & np.uint64(0xFFFFFFFF)),
                       np.full_like(i, st >> np.uint64(32)), np.full_like(i, 3)], _keys(seed))
    u = u24(r[0])
    p = np.asarray(prob, np.float32).astype(F64)
    keep = leaf >= 0
    keep[keep] = u[keep] < p[leaf[keep]]
    return keep


def leaf_statistics(first_leaf, trains, loss_terms, n_leaves: int):
    """Per leaf: rays whose first leaf it is, the rays among them that train
    it, and the sum of their loss terms (Sec. 5.1: error = loss q x hit
    probability p, p estimated from the training rays)."""
    first_leaf = np.asarray(first_leaf, np.int64)
    hits = np.zeros(n_leaves, np.int64)
    trained = np.zeros(n_leaves, np.int64)
    loss = np.zeros(n_leaves)
    for i, l in enumerate(first_leaf):
        if l < 0:
            continue
        hits[l] += 1
        if trains[i]:
            trained[l] += 1
            loss[l] += float(loss_terms[i])
    return hits, trained, loss


def node_rank(hits, trained, loss, n_rays: int):
    """q = mean loss of a leaf's trained rays, p = hits / n_rays, ranking
    r = 2 ln q + ln p (Sec. 5.1); training probability max(exp(r - r_max),
    0.005) (Sec. 5.2, read in the linear domain of the ranking). A leaf with
    no hit ranks -inf; a hit leaf without trained rays takes the mean q of
    the trained leaves."""
    n = len(hits)
    q = np.zeros(n)
    have = [i for i in range(n) if trained[i] > 0]
    qm = sum(loss[i] / trained[i] for i in have) / len(have) if have else 1.0
    for i in range(n):
        q[i] = loss[i] / trained[i] if trained[i] > 0 else qm
    p = np.array([hits[i] / max(1, n_rays) for i in range(n)], F64)
    r = np.array([2.0 * math.log(q[i]) + math.log(p[i]) if hits[i] > 0 and q[i] > 0 else -math.inf
                  for i in range(n)])
    finite = [x for x in r if math.isfinite(x)]
    rmax = max(finite) if finite else 0.0
    prob = np.array([max(math.exp(x - rmax), 0.005) if math.isfinite(x) else 0.005 for x in r])
    return q, p, r, prob


def split_cut(refs, r, k: int, children):
    """Replace the k splittable leaves of largest r (ties: lower leaf index)
    by their children; children(ref) lists a reference's children, empty for
    a base leaf. Leaf order is kept, children in their order."""
    cand = sorted([i for i in range(len(refs)) if children(refs[i]) and math.isfinite(r[i])],
                  key=lambda i: (-r[i], i))[:k]
    out = []
    for i, ref in enumerate(refs):
        out += list(children(ref)) if i in cand else [ref]
    return out


def cut_leaves(tris, base_nodes, base_leaf_range, base_tri_perm, cut, inflate_rel: float, extent: float):
    """Leaves of the N-BVH of a cut, by brute force over the base tree: walk
    from the root (first child first); a cut reference becomes a leaf whose
    triangles are those of every base leaf below it and whose box is their
    AABB pushed out by inflate_rel * extent (FP64) and rounded outward to
    float32. base_nodes: records with child0, child1 (leaf = ~index, none =
    0x7fffffff). Returns (refs in leaf order, triangle index sets, lo, hi)."""
    cut = set(int(c) for c in cut)

    def leaves_below(ref):
        if ref < 0:
            return [~ref]
        nd = base_nodes[ref]
        out = []
        for c in (int(nd["child0"]), int(nd["child1"])):
            if c != 0x7fffffff:
                out += leaves_below(c)
        return out

    refs, sets, lo, hi = [], [], [], []
    pad = inflate_rel * float(extent)

    def walk(ref):
        if ref in cut:
            bl = leaves_below(ref)
            idx = np.concatenate([base_tri_perm[base_leaf_range[b][0]:base_leaf_range[b][1]] for b in bl])
            v = np.asarray(tris, F64)[idx].reshape(-1, 3)
            refs.append(ref)
            sets.append(np.sort(idx))
            lo.append(_round_down_f32(v.min(0) - pad))
            hi.append(_round_up_f32(v.max(0) + pad))
            return
        if ref < 0:
            raise ValueError("a base leaf below no cut reference")
        nd = base_nodes[ref]
        for c in (int(nd["child0"]), int(nd["child1"])):
            if c != 0x7fffffff:
                walk(c)

    walk(0)
    return refs, sets, np.array(lo), np.array(hi)
