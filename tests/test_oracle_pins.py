"""Pins of the FP64 oracle against facts that do not come from the oracle:
published test vectors, hand-derived values, closed forms, brute force on tiny
inputs, invariants and finite differences. CPU only."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import workloads as W


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10([np.uint64(x) for x in v[0:4]], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform24_exact_and_range():
    x = np.array([0, 255, 256, 0xFFFFFFFF], np.uint32)
    u = O.u24(x)
    assert u[0] == 0.0 and u[1] == 0.0 and u[2] == 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24


# ---------------------------------------------------------------- layout / hash
def test_level_layout_hand_derived():
    rows = read_golden("level_layout_L16_N16_b1.5_T2p20.txt")
    lay = O.level_layout(16, 16, 1.5, 20)
    for r in rows[:-1]:
        l, n, dense, size = map(int, r)
        assert lay["res"][l] == n and bool(lay["dense"][l]) == bool(dense) and lay["size"][l] == size
    assert lay["total"] == int(rows[-1][1])
    assert lay["offset"][0] == 0 and lay["offset"][5] == 4913 + 15625 + 50653 + 166375 + 551368


def test_hash_hand_values():
    for r in read_golden("hash_index_T2p20.txt"):
        x, y, z, h = map(int, r)
        assert O.grid_index(np.array([x, y, z]), 7006, False, 1 << 20) == h


def test_dense_index_is_bijective():
    n = 6
    g = np.stack(np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij"), -1)
    idx = O.grid_index(g.reshape(-1, 3), n, True, 1 << 20)
    assert sorted(idx.tolist()) == list(range((n + 1) ** 3))
    # x is the fastest-varying coordinate
    assert O.grid_index(np.array([1, 0, 0]), n, True, 0) == 1
    assert O.grid_index(np.array([0, 1, 0]), n, True, 0) == n + 1


def test_hash_buckets_roughly_uniform():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 4000, size=(200000, 3))
    T = 1 << 10
    h = O.grid_index(c, 4000, False, T)
    counts = np.bincount(h, minlength=T)
    exp = len(c) / T
    chi2 = np.sum((counts - exp) ** 2 / exp)
    # chi-square with T-1 dof: mean 1023, sd ~45
    assert chi2 < 1023 + 8 * 45


# ---------------------------------------------------------------- encoding
def _linear_table(layout, F, a, b):
    """Table whose entry for every dense-level vertex i/N holds a.x + b."""
    tab = np.zeros((layout["total"], F))
    for l, n in enumerate(layout["res"]):
        assert layout["dense"][l]
        g = np.stack(np.meshgrid(*(np.arange(n + 1),) * 3, indexing="ij"), -1).reshape(-1, 3)
        idx = O.grid_index(g, int(n), True, layout["T"])
        for f in range(F):
            tab[layout["offset"][l] + idx, f] = (g / n) @ a[f] + b[f]
    return tab


def test_trilinear_reproduces_linear_field_on_dense_levels():
    lay = O.level_layout(3, 4, 2.0, 16)   # N = 4, 8, 16: all dense
    assert lay["dense"].all()
    rng = np.random.default_rng(2)
    F = 2
    a = rng.normal(size=(F, 3))
    b = rng.normal(size=F)
    tab = _linear_table(lay, F, a, b)
    x = rng.uniform(0, 1, size=(50, 3, 3))
    x[0, 0] = [1.0, 1.0, 1.0]   # upper corner: clamped cell, frac = 1
    x[0, 1] = [0.0, 0.5, 1.0]
    feat = O.encode(x, tab, lay).reshape(50, 3, 3, F)
    expect = np.einsum("snd,fd->snf", x, a) + b
    for l in range(3):
        assert np.max(np.abs(feat[:, :, l, :] - expect)) <= 1e-12


def test_trilinear_on_hashed_level_without_collisions():
    # One hashed level ((128+1)^3 > 2^20); points in a tiny region so the
    # used vertices do not collide; entries there hold a linear field.
    lay = O.level_layout(1, 128, 2.0, 20)
    assert not lay["dense"][0]
    rng = np.random.default_rng(3)
    x = 0.3 + 0.03 * rng.uniform(size=(40, 2, 3))
    cells = np.floor(x * 128).astype(int)
    verts = np.unique((cells[..., None, :] + np.array(
        [[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])).reshape(-1, 3), axis=0)
    h = O.grid_index(verts, 64, False, lay["T"])
    assert len(np.unique(h)) == len(verts), "choose a region without collisions"
    a = np.array([[0.3, -1.2, 2.0]])
    tab = np.zeros((lay["total"], 1))
    tab[h, 0] = (verts / 128.0) @ a[0] + 0.25
    feat = O.encode(x, tab, lay).reshape(40, 2)
    assert np.max(np.abs(feat - (x @ a[0] + 0.25))) <= 1e-12


def test_encoding_order_is_sample_level_feature():
    lay = O.level_layout(2, 2, 2.0, 12)
    # table entry value encodes (level, feature): level 0 -> 10+f, level 1 -> 20+f
    tab = np.zeros((lay["total"], 2))
    for l in range(2):
        tab[lay["offset"][l]:lay["offset"][l] + lay["size"][l]] = [10 * (l + 1), 10 * (l + 1) + 1]
    x = np.full((1, 3, 3), 0.4)
    feat = O.encode(x, tab, lay)[0]
    assert feat.tolist() == [10, 11, 20, 21] * 3


# ---------------------------------------------------------------- slab test / segments
def test_clip_axis_aligned_closed_form():
    lo, hi = np.array([1.0, -1.0, -1.0]), np.array([3.0, 1.0, 1.0])
    keep, t0, t1, _, _ = O.clip_ray_box(np.array([0.0, 0.2, 0.3]), np.array([2.0, 0.0, 0.0]), 0.0,
                                        np.inf, lo, hi)
    assert keep and t0 == 0.5 and t1 == 1.5
    # origin inside the slab of a zero direction component, outside of another
    keep, _, _, _, _ = O.clip_ray_box(np.array([0.0, 1.5, 0.0]), np.array([1.0, 0.0, 0.0]), 0.0,
                                      np.inf, lo, hi)
    assert not keep
    # ray starting inside the box: t0 = tmin
    keep, t0, t1, _, _ = O.clip_ray_box(np.array([2.0, 0.0, 0.0]), np.array([-1.0, 0.0, 0.0]), 0.25,
                                        0.75, lo, hi)
    assert keep and t0 == 0.25 and t1 == 0.75
    # interval beyond tmax
    keep, _, _, _, _ = O.clip_ray_box(np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), 0.0, 0.9,
                                      lo, hi)
    assert not keep


def test_clip_matches_pointwise_membership():
    rng = np.random.default_rng(4)
    n = 3000
    o = rng.uniform(-2, 2, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d[::7, 1] = 0.0
    lo = rng.uniform(-1, 0.5, size=(n, 3))
    hi = lo + rng.uniform(0.05, 1.0, size=(n, 3))
    tmin = rng.uniform(0, 0.5, n)
    tmax = rng.uniform(0.5, 6, n)
    keep, t0, t1, _, _ = O.clip_ray_box(o, d, tmin, tmax, lo, hi)
    ts = np.linspace(0, 1, 257)
    for i in range(n):
        t = tmin[i] + ts * (tmax[i] - tmin[i])
        p = o[i] + t[:, None] * d[i]
        inside = np.all((p >= lo[i] - 1e-9) & (p <= hi[i] + 1e-9), axis=1)
        # endpoints are float32 values: within one float32 ulp of the exact ones
        eps = 2.0 ** -23 * max(1.0, abs(t0[i]), abs(t1[i]))
        if keep[i]:
            pm = o[i] + 0.5 * (t0[i] + t1[i]) * d[i]
            tol = eps * np.abs(d[i]) + 1e-9
            assert np.all(pm >= lo[i] - tol) and np.all(pm <= hi[i] + tol)
            # brute-force samples inside the box lie within [t0, t1]
            assert np.all((t[inside] >= t0[i] - eps) & (t[inside] <= t1[i] + eps))
        else:
            strict = np.all((p > lo[i] + 1e-7) & (p < hi[i] - 1e-7), axis=1)
            assert not strict.any()


def test_clip_endpoints_are_nearest_float32_of_exact_quotients():
    from fractions import Fraction
    rng = np.random.default_rng(21)
    for _ in range(300):
        o = rng.uniform(-2, 2, 3).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        lo = rng.uniform(-1, 0.5, 3).astype(np.float32)
        hi = (lo + rng.uniform(0.05, 1.0, 3)).astype(np.float32)
        keep, t0, t1, en, ex = O.clip_ray_box(o.astype(np.float64), d.astype(np.float64), 0.0, np.inf,
                                              lo.astype(np.float64), hi.astype(np.float64))
        near, far = [], []
        for i in range(3):
            qa = (Fraction(float(lo[i])) - Fraction(float(o[i]))) / Fraction(float(d[i]))
            qb = (Fraction(float(hi[i])) - Fraction(float(o[i]))) / Fraction(float(d[i]))
            near.append(min(qa, qb))
            far.append(max(qa, qb))

        def nearest_f32(q):
            f = np.float32(float(q))
            cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
            return min(cands, key=lambda c: abs(Fraction(float(c)) - q))

        assert en == float(nearest_f32(max(near))) and ex == float(nearest_f32(min(far)))
        assert bool(keep) == (max(float(en), 0.0) <= float(ex))


def test_segments_sorted_and_complete():
    tris = W.scene_random_tris(512, seed=5)
    lv = O.build_leaves(tris, 16)
    rays = W.camera_rays(24, 24, seed=6)
    seg = O.ray_segments(rays, lv["leaf_lo"], lv["leaf_hi"])
    off = seg["offsets"]
    lo, hi = lv["leaf_lo"].astype(np.float64), lv["leaf_hi"].astype(np.float64)
    # brute force by pointwise membership: dense points along each ray (the
    # camera sits at radius 2 and every box lies inside [-1, 1]^3)
    ts = np.linspace(0.0, 4.0, 8001)
    n_listed = 0
    for r in range(len(rays["ox"])):
        t0 = seg["t0"][off[r]:off[r + 1]]
        t1 = seg["t1"][off[r]:off[r + 1]]
        lf = seg["leaf"][off[r]:off[r + 1]]
        keys = list(zip(t0, lf))
        assert keys == sorted(keys)
        o, d, tmin, tmax = O.rays_od(rays, r)
        t = ts[(ts >= tmin) & (ts <= tmax)]
        p = o[None, :] + t[:, None] * d[None, :]
        for leaf in range(16):
            strictly = np.all((p > lo[leaf] + 1e-7) & (p < hi[leaf] - 1e-7), axis=1)
            listed = np.flatnonzero(lf == leaf)
            if strictly.any():
                # a point strictly inside the box: the leaf is listed once, and
                # its interval covers every such point
                assert len(listed) == 1, (r, leaf)
                j = listed[0]
                eps = 2.0 ** -22 * max(1.0, abs(t0[j]), abs(t1[j]))
                assert t[strictly].min() >= t0[j] - eps and t[strictly].max() <= t1[j] + eps
            for j in listed:
                # a listed interval lies in the box: its midpoint is inside
                pm = o + 0.5 * (t0[j] + t1[j]) * d
                assert np.all(pm >= lo[leaf] - 1e-6) and np.all(pm <= hi[leaf] + 1e-6), (r, leaf)
                n_listed += 1
    assert n_listed > 100


def test_scene_frame_hand_made():
    # the AABB spans x in [-1, 3], y in [0, 1], z in [2, 2.5]; most vertices
    # sit near one corner, so the vertex mean is far from the box centre
    tris = np.array([[[-1.0, 0.0, 2.0], [-0.9, 0.0, 2.0], [-1.0, 0.1, 2.0]],
                     [[-1.0, 0.0, 2.1], [-0.9, 0.1, 2.0], [-1.0, 0.1, 2.1]],
                     [[3.0, 1.0, 2.5], [-1.0, 0.0, 2.0], [-0.95, 0.05, 2.0]]], np.float32)
    fr = O.scene_frame(tris)
    assert fr["lo"].tolist() == [-1.0, 0.0, 2.0] and fr["hi"].tolist() == [3.0, 1.0, 2.5]
    assert fr["centre"].tolist() == [1.0, 0.5, 2.25]
    assert fr["extent"] == 4.0
    assert fr["sphere_radius"] == pytest.approx(1.01 * math.sqrt(16.0 + 1.0 + 0.25) / 2.0, rel=1e-15)
    # stored frame: nearest float32 of the centre and extent
    tri2 = tris + np.float32(0.1)
    fr2 = O.scene_frame(tri2)
    c = (tri2.reshape(-1, 3).astype(np.float64).min(0) + tri2.reshape(-1, 3).astype(np.float64).max(0)) / 2
    assert fr2["model_centre"].tolist() == c.astype(np.float32).astype(np.float64).tolist()
    assert np.abs(fr2["model_centre"] - fr2["centre"]).max() <= 2.0 ** -24 * 3


def test_normalize_points_clamp_and_centre():
    c = np.array([1.0, -2.0, 0.5])
    E = 4.0
    p = np.array([c, c + E / 2, c - E / 2, c + E, c - E, c + 0.25 * E, c + [-E, 0.0, 3 * E]])
    x = O.normalize_points(p, c, E)
    assert x[0].tolist() == [0.5, 0.5, 0.5]
    assert x[1].tolist() == [1.0, 1.0, 1.0] and x[2].tolist() == [0.0, 0.0, 0.0]
    assert x[3].tolist() == [1.0, 1.0, 1.0] and x[4].tolist() == [0.0, 0.0, 0.0]   # clamped
    assert x[5].tolist() == [0.75, 0.75, 0.75]
    assert x[6].tolist() == [0.0, 0.5, 1.0]
    # isotropic: one scale for every axis
    q = O.normalize_points(np.array([[2.0, -1.0, 1.5]]), c, E)
    assert q[0].tolist() == [0.75, 0.75, 0.75]


# ---------------------------------------------------------------- leaf build
def test_median_split_tiny_known_partition():
    # 8 triangles centred at x = 0..7 (y, z spread smaller): 4 leaves of 2 in x order
    base = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0]], np.float64)
    perm = [3, 0, 6, 1, 7, 2, 5, 4]
    tris = np.stack([base + [perm[i], 0, 0] for i in range(8)]).astype(np.float32)
    lv = O.build_leaves(tris, 4, inflate_rel=0.0)
    xs = [sorted(perm[i] for i in lv["tri_perm"][a:b]) for a, b in lv["leaf_range"]]
    assert xs == [[0, 1], [2, 3], [4, 5], [6, 7]]
    assert np.allclose(lv["leaf_lo"][0], [0, 0, 0]) and np.allclose(lv["leaf_hi"][3], [7.1, 0.1, 0])


def test_leaf_build_invariants():
    tris = W.scene_random_tris(4096, seed=7)
    lv = O.build_leaves(tris, 64)
    assert sorted(lv["tri_perm"].tolist()) == list(range(4096))
    sizes = lv["leaf_range"][:, 1] - lv["leaf_range"][:, 0]
    assert (sizes == 64).all()
    E = lv["frame"]["extent"]
    for i, (a, b) in enumerate(lv["leaf_range"]):
        pts = tris[lv["tri_perm"][a:b]].reshape(-1, 3).astype(np.float64)
        assert (lv["leaf_lo"][i] <= pts.min(0) - 1e-4 * E).all()
        assert (lv["leaf_hi"][i] >= pts.max(0) + 1e-4 * E).all()
        # outward rounding is tight: within one float32 ulp of the exact bound
        ex_lo = pts.min(0) - 1e-4 * E
        ex_hi = pts.max(0) + 1e-4 * E
        assert (lv["leaf_lo"][i] >= ex_lo - np.abs(np.spacing(lv["leaf_lo"][i])).astype(np.float64)).all()
        assert (lv["leaf_hi"][i] <= ex_hi + np.abs(np.spacing(lv["leaf_hi"][i])).astype(np.float64)).all()
        assert np.all(np.diff(lv["tri_perm"][a:b]) > 0)


# ---------------------------------------------------------------- sampling, MLP
def test_sample_points_closed_form():
    o = np.array([[0.0, 0.0, 0.0]])
    d = np.array([[1.0, 2.0, 0.0]])
    p = O.sample_points(o, d, np.array([1.0]), np.array([3.0]), 4)
    assert np.allclose(p[0, :, 0], [1.25, 1.75, 2.25, 2.75], atol=0, rtol=0)
    p1 = O.sample_points(o, d, np.array([1.0]), np.array([3.0]), 1)
    assert p1[0, 0, 0] == 2.0 and p1[0, 0, 1] == 4.0


def test_mlp_forward_against_loops():
    rng = np.random.default_rng(8)
    dims = [5, 4, 3, 2]
    layers = [(rng.normal(size=(dims[i + 1], dims[i])), rng.normal(size=dims[i + 1])) for i in range(3)]
    x = rng.normal(size=(6, 5))
    raw, _, _ = O.mlp_forward(x, layers)
    for s in range(6):
        h = list(x[s])
        for li, (Wm, b) in enumerate(layers):
            z = [sum(Wm[j][k] * h[k] for k in range(len(h))) + b[j] for j in range(len(b))]
            h = [max(0.0, v) for v in z] if li < 2 else z
        assert np.allclose(raw[s], h, rtol=1e-14, atol=1e-14)


def test_mlp_half_precision_operands_worked_example():
    """Operand rounding of the half-precision MLP (Sec. 6), with rounding to
    integers so every step can be followed by hand. Inputs x = (0.4, 1.6);
    W0 rows (1.4, 0.6), (-0.7, 2.2), (0.2, -1.4), (0.1, 0.1), b0 = (0.25,
    -0.3, 0.5, 0.3); Wo = (0.7, -1.2, 0.9, 2.6), bo = 0.1.
    Forward: x -> (0, 2); W0 -> rows (1, 1), (-1, 2), (0, -1), (0, 0);
    z0 = (2.25, 3.7, -1.5, 0.3); h0 = relu -> rounded (2, 4, 0, 0);
    Wo -> (1, -1, 1, 3); raw = 2 - 4 + 0.1 = -1.9.
    Backward with dL/d(raw) = 0.3 and loss scale 4: the output layer's
    weight gradient takes the unrounded 0.3: dWo = 0.3 h0 = (0.6, 1.2, 0, 0),
    dbo = 0.3; the product operand is round(0.3 * 4) / 4 = 0.25, so
    dH0 = 0.25 (1, -1, 1, 3), masked by the stored activations' sign (the
    fourth unit had z0 > 0 but rounded to 0): dZ0 = (0.25, -0.25, 0, 0),
    exact under rounding of dZ0 * 4; dW0 = dZ0 x0^T with x0 = (0, 2);
    dfeatures = dZ0 W0 = (0.5, -0.25)."""
    feat = np.array([[0.4, 1.6]])
    layers = [(np.array([[1.4, 0.6], [-0.7, 2.2], [0.2, -1.4], [0.1, 0.1]]), np.array([0.25, -0.3, 0.5, 0.3])),
              (np.array([[0.7, -1.2, 0.9, 2.6]]), np.array([0.1]))]
    raw, acts, pre = O.mlp_forward(feat, layers, rnd=np.round)
    assert np.allclose(raw, [[-1.9]], rtol=0, atol=1e-15)
    assert np.array_equal(acts[0], [[0.0, 2.0]]) and np.array_equal(acts[1], [[2.0, 4.0, 0.0, 0.0]])
    g_feat, grads = O.mlp_backward(np.array([[0.3]]), acts, pre, layers, rnd=np.round, scale=4.0)
    (dW0, db0), (dWo, dbo) = grads
    assert np.allclose(dWo, [[0.6, 1.2, 0.0, 0.0]], rtol=0, atol=1e-15) and np.allclose(dbo, [0.3], rtol=0, atol=1e-15)
    assert np.array_equal(dW0, [[0.0, 0.5], [0.0, -0.5], [0.0, 0.0], [0.0, 0.0]])
    assert np.array_equal(db0, [0.25, -0.25, 0.0, 0.0])
    assert np.array_equal(g_feat, [[0.5, -0.25]])
    # without rounding the same call is the exact backward (mask = pre-activation sign)
    raw1, acts1, pre1 = O.mlp_forward(feat, layers)
    g1, _ = O.mlp_backward(np.array([[0.3]]), acts1, pre1, layers)
    W0, Wo = layers[0][0], layers[1][0]
    z0 = W0 @ feat[0] + layers[0][1]
    assert np.allclose(g1[0], ((0.3 * Wo[0]) * (z0 > 0)) @ W0, rtol=1e-15, atol=1e-15)


def test_sigmoid_softplus_closed_forms():
    assert O.sigmoid(0.0) == 0.5
    assert abs(O.sigmoid(np.log(3.0)) - 0.75) < 1e-15
    assert abs(O.softplus(0.0) - math.log(2.0)) < 1e-15
    assert O.sigmoid(-800.0) == 0.0 and O.sigmoid(800.0) == 1.0


# ---------------------------------------------------------------- decode / resolve
def test_resolve_early_out_equals_all_segments():
    rng = np.random.default_rng(9)
    tris = W.scene_random_tris(1024, seed=10)
    lv = O.build_leaves(tris, 32)
    rays = W.camera_rays(20, 20, seed=11)
    seg = O.ray_segments(rays, lv["leaf_lo"], lv["leaf_hi"])
    S = len(seg["ray"])
    raw = rng.normal(size=(S, 5))
    hit, t, nrm = O.decode(raw, seg["t0"], seg["t1"])
    res = O.resolve(len(rays["ox"]), seg, hit, t, nrm)
    off = seg["offsets"]
    for r in range(len(rays["ox"])):
        best_t, best_leaf = np.inf, -1
        for j in range(off[r], off[r + 1]):
            if seg["t0"][j] >= best_t:
                break       # early out: later segments cannot be closer
            if hit[j] and t[j] < best_t:
                best_t, best_leaf = t[j], seg["leaf"][j]
        assert res["t"][r] == best_t and res["leaf"][r] == best_leaf


def test_decode_closed_form():
    raw = np.array([[0.0, 0.0, 0.0, 0.0, 0.0], [1.0, np.log(3.0), 3.0, 0.0, 4.0]])
    hit, t, n = O.decode(raw, np.array([1.0, 2.0]), np.array([3.0, 6.0]))
    assert hit.tolist() == [False, True]
    assert t[0] == 2.0 and abs(t[1] - 5.0) < 1e-14
    assert n[0].tolist() == [0, 0, 1] and np.allclose(n[1], [0.6, 0, 0.8], atol=1e-15)


# ---------------------------------------------------------------- Moller-Trumbore / labels
def test_moller_trumbore_plane_closed_form():
    v0, v1, v2 = np.array([-1.0, -1.0, 0.5]), np.array([3.0, -1.0, 0.5]), np.array([-1.0, 3.0, 0.5])
    rng = np.random.default_rng(12)
    o = rng.uniform(-0.5, 0.5, size=(100, 3))
    o[:, 2] = -1.0
    d = np.array([0.1, 0.05, 1.0])
    hit, t, _, _ = O.moller_trumbore(o, d, v0, v1, v2)
    assert hit.all()
    assert np.allclose(t, (0.5 - o[:, 2]) / d[2], rtol=1e-14)


def test_moller_trumbore_icosphere_vs_analytic_sphere():
    tris = W.scene_icosphere(level=4, radius=0.4, amplitude=0.0).astype(np.float64)
    rng = np.random.default_rng(13)
    o = np.array([0.0, 0.0, -2.0])
    n = 200
    d = np.stack([rng.uniform(-0.12, 0.12, n), rng.uniform(-0.12, 0.12, n), np.ones(n)], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    hit, t, _, _ = O.moller_trumbore(o[None, None], d[:, None], tris[None, :, 0], tris[None, :, 1],
                                     tris[None, :, 2])
    tt = np.where(hit & (t > 0), t, np.inf).min(1)
    b = d @ o
    disc = b * b - (o @ o - 0.16)
    t_sphere = -b - np.sqrt(disc)
    # the polyhedron is inscribed: its faces lie inside the sphere, at most
    # the largest face-plane depth ``sag`` below it
    e1 = tris[:, 1] - tris[:, 0]
    e2 = tris[:, 2] - tris[:, 0]
    nf = np.cross(e1, e2)
    nf /= np.linalg.norm(nf, axis=1, keepdims=True)
    sag = 0.4 - np.min(np.abs(np.sum(nf * tris[:, 0], 1)))
    assert 0 < sag < 2e-3
    assert np.all(tt >= t_sphere - 1e-12)
    cos_inc = np.abs(np.sum(d * (o + t_sphere[:, None] * d), 1)) / 0.4
    assert np.all(tt - t_sphere <= sag / cos_inc + 1e-12)


def test_labels_min_over_leaves_equals_global_closest_hit():
    tris = W.scene_random_tris(600, seed=14)
    lv = O.build_leaves(tris, 12)
    rays = W.camera_rays(14, 14, seed=15)
    seg = O.ray_segments(rays, lv["leaf_lo"], lv["leaf_hi"])
    o, d, tmin, tmax = O.rays_od(rays)
    rr = seg["ray"]
    lab = O.labels(o[rr], d[rr], seg["leaf"], seg["t0"], seg["t1"], tris, lv["tri_perm"], lv["leaf_range"])
    tv = tris.astype(np.float64)
    for r in range(len(o)):
        hit, t, _, _ = O.moller_trumbore(o[r][None], d[r][None], tv[:, 0], tv[:, 1], tv[:, 2])
        glob = np.where(hit & (t >= tmin[r]) & (t <= tmax[r]), t, np.inf).min()
        sel = rr == r
        per_leaf = np.where(lab["hit"][sel] == 1, lab["t"][sel], np.inf)
        best = per_leaf.min() if per_leaf.size else np.inf
        assert best == glob
    # depths lie in [0, 1], normals face the ray
    h = lab["hit"] == 1
    assert np.all((lab["depth"][h] >= 0) & (lab["depth"][h] <= 1))
    assert np.all(np.sum(lab["normal"][h] * d[rr][h], 1) <= 0)


# ---------------------------------------------------------------- loss / gradients / Adam
def _tiny_problem(seed=16):
    rng = np.random.default_rng(seed)
    lay = O.level_layout(3, 4, 2.0, 8)    # mixed dense and hashed levels
    assert lay["dense"][0] and not lay["dense"][2]
    F, N = 2, 3
    tab = rng.uniform(-0.5, 0.5, size=(lay["total"], F))
    dims = [N * 3 * F, 8, 8, 5]
    layers = [(rng.normal(0, 1 / math.sqrt(dims[i]), size=(dims[i + 1], dims[i])),
               rng.normal(0, 0.1, size=dims[i + 1])) for i in range(3)]
    S = 12
    o = rng.uniform(-0.3, 0.3, size=(S, 3))
    d = rng.normal(size=(S, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t0 = rng.uniform(0, 0.2, S)
    t1 = t0 + rng.uniform(0.1, 0.4, S)
    valid = np.ones(S, bool)
    valid[3] = False
    yh = (rng.uniform(size=S) < 0.6).astype(float)
    yd = rng.uniform(size=S)
    yn = rng.normal(size=(S, 3))
    return dict(o=o, d=d, t0=t0, t1=t1, valid=valid, yh=yh, yd=yd, yn=yn, tab=tab, layers=layers,
                lay=lay, N=N)


def _loss_of(P, tab=None, layers=None):
    p = O.sample_points(P["o"], P["d"], P["t0"], P["t1"], P["N"])
    x = O.normalize_points(p, np.zeros(3), 1.0)
    feat = O.encode(x, P["tab"] if tab is None else tab, P["lay"])
    raw, _, _ = O.mlp_forward(feat, P["layers"] if layers is None else layers)
    return O.loss(raw, P["yh"], P["yd"], P["yn"], P["valid"])[0]


def test_loss_special_case_closed_form():
    raw = np.zeros((2, 5))
    L, _ = O.loss(raw, [1, 0], [0.25, 0.9], np.array([[0.0, 0.0, 1.0], [1, 1, 1]]), [True, True])
    expect = (2 * math.log(2) + 2 * 0.25 + 1.0 / 3.0 + 2 * math.log(2)) / 2
    assert abs(L - expect) < 1e-15


def test_gradients_match_central_differences():
    P = _tiny_problem()
    L, g_tab, g_layers, raw = O.forward_backward(P["o"], P["d"], P["t0"], P["t1"], P["valid"], P["yh"],
                                                  P["yd"], P["yn"], P["tab"], P["layers"], P["lay"],
                                                  np.zeros(3), 1.0, P["N"])
    # keep away from the L1 kinks so central differences are exact to O(h^2)
    s1 = O.sigmoid(raw[:, 1])
    assert np.min(np.abs(s1 - P["yd"])) > 1e-4 and np.min(np.abs(raw[:, 2:5] - P["yn"])) > 1e-4
    h = 1e-6
    used = np.nonzero(np.abs(g_tab).sum(1) > 0)[0]
    rng = np.random.default_rng(17)
    for e in rng.choice(used, size=12, replace=False):
        for f in range(2):
            tp = P["tab"].copy(); tp[e, f] += h
            tm = P["tab"].copy(); tm[e, f] -= h
            fd = (_loss_of(P, tab=tp) - _loss_of(P, tab=tm)) / (2 * h)
            assert abs(fd - g_tab[e, f]) <= 1e-6 * max(1e-3, abs(g_tab[e, f])) + 1e-9
    for li in range(3):
        Wm, b = P["layers"][li]
        for (j, k) in [(0, 0), (1, 2), (Wm.shape[0] - 1, Wm.shape[1] - 1)]:
            lp = [(w.copy(), bb.copy()) for w, bb in P["layers"]]
            lm = [(w.copy(), bb.copy()) for w, bb in P["layers"]]
            lp[li][0][j, k] += h
            lm[li][0][j, k] -= h
            fd = (_loss_of(P, layers=lp) - _loss_of(P, layers=lm)) / (2 * h)
            assert abs(fd - g_layers[li][0][j, k]) <= 1e-6 * max(1e-3, abs(g_layers[li][0][j, k])) + 1e-9
        lp = [(w.copy(), bb.copy()) for w, bb in P["layers"]]
        lm = [(w.copy(), bb.copy()) for w, bb in P["layers"]]
        lp[li][1][0] += h
        lm[li][1][0] -= h
        fd = (_loss_of(P, layers=lp) - _loss_of(P, layers=lm)) / (2 * h)
        assert abs(fd - g_layers[li][1][0]) <= 1e-6 * max(1e-3, abs(g_layers[li][1][0])) + 1e-9


def test_invalid_rays_do_not_contribute():
    P = _tiny_problem()
    _, g_tab, g_layers, _ = O.forward_backward(P["o"], P["d"], P["t0"], P["t1"], P["valid"], P["yh"],
                                                P["yd"], P["yn"], P["tab"], P["layers"], P["lay"],
                                                np.zeros(3), 1.0, P["N"])
    Q = dict(P)
    Q["o"] = P["o"].copy(); Q["o"][3] += 0.1   # the invalid ray changes
    _, g_tab2, _, _ = O.forward_backward(Q["o"], Q["d"], Q["t0"], Q["t1"], Q["valid"], Q["yh"],
                                          Q["yd"], Q["yn"], Q["tab"], Q["layers"], Q["lay"],
                                          np.zeros(3), 1.0, Q["N"])
    assert np.array_equal(g_tab, g_tab2)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(18)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = O.adam(p, g, np.zeros(100), np.zeros(100), 1, lr=1e-2)
    assert np.allclose(p1, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# ---------------------------------------------------------------- training rays / bounce
def test_train_rays_probed_cross_their_leaf_and_chords_on_sphere():
    tris = W.scene_random_tris(2048, seed=19)
    lv = O.build_leaves(tris, 32)
    R = O.train_rays(O.TRAIN_MODE_PROBED_MIX, seed=123, step=7, n=2000, leaves=lv)
    fr = lv["frame"]
    assert np.allclose(np.linalg.norm(R["d"], axis=1), 1.0, atol=1e-12)
    even = np.arange(2000) % 2 == 0
    assert (R["leaf"][even] >= 0).all()
    # probed origins lie on the bounding sphere, as do chord origins
    dist = np.linalg.norm(R["o"] - fr["centre"], axis=1)
    assert np.allclose(dist, fr["sphere_radius"], rtol=1e-12)
    # the probed leaf's segment is non-empty and inside the ray
    assert np.all(R["t1"][even] >= R["t0"][even])
    # leaf choice uniform-ish over 32 leaves
    cnt = np.bincount(R["leaf"][even], minlength=32)
    assert cnt.min() > 10
    # directions uniform: mean ~ 0, mean z^2 ~ 1/3
    assert np.all(np.abs(R["d"].mean(0)) < 0.06) and abs((R["d"][:, 2] ** 2).mean() - 1 / 3) < 0.03
    # chords: the trained leaf is the first one met
    odd = np.nonzero(~even & (R["leaf"] >= 0))[0][:50]
    for i in odd:
        k, t0, _, _, _ = O.clip_ray_box(R["o"][i], R["d"][i], 0.0, R["tmax"][i], lv["leaf_lo"], lv["leaf_hi"])
        assert R["t0"][i] == np.min(t0[k])


def test_bounce_rays_cosine_hemisphere():
    rng = np.random.default_rng(20)
    n = 20000
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    d = -nrm + 0.1 * rng.normal(size=(n, 3))
    o = np.zeros((n, 3))
    p, dirs = O.bounce_rays(o, d, np.ones(n), nrm, np.arange(n), seed=5)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-12)
    flip = np.sum(nrm * d, 1) > 0
    nn = np.where(flip[:, None], -nrm, nrm)
    cos = np.sum(dirs * nn, 1)
    assert np.all(cos >= -1e-12)
    # cosine-weighted: E[cos] = 2/3
    assert abs(cos.mean() - 2 / 3) < 0.01
    t, b = O.onb(nn)
    assert np.allclose(np.sum(t * nn, 1), 0, atol=1e-12) and np.allclose(np.sum(t * b, 1), 0, atol=1e-12)
    assert np.allclose(p, d + 1e-4 * nn)


# ---------------------------------------------------------------- S9 hybrid hierarchy
def _flat_grid_case(n_cells=20, half=1.0, y0=-0.25, n_rays=400, seed=3):
    tris = W.ground_heightfield(n_cells, half=half, y0=y0, amplitude=0.0)
    rng = np.random.default_rng(seed)
    h = 2 * half / n_cells
    # targets away from cell edges and diagonals
    # one cell clear of the border: rays cross a grid raised by 0.2 inside it
    i = rng.integers(1, n_cells - 1, n_rays)
    j = rng.integers(1, n_cells - 1, n_rays)
    fx = rng.uniform(0.1, 0.9, n_rays)
    fz = rng.uniform(0.1, 0.9, n_rays)
    keep = np.abs(fx + fz - 1.0) > 0.05
    i, j, fx, fz = i[keep], j[keep], fx[keep], fz[keep]
    target = np.stack([-half + (i + fx) * h, np.full(len(i), y0), -half + (j + fz) * h], 1)
    o = target + np.array([0.0, 1.0, 0.0]) + rng.uniform(-0.3, 0.3, (len(i), 3)) * np.array([1.0, 0.0, 1.0])
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return tris, i, j, fx, fz, o, d, target


def test_closest_triangle_hit_flat_grid_closed_form():
    """A flat grid: t = (y0 - o_y) / d_y, the triangle is the grid cell's
    lower or upper half (fx + fz < 1 or > 1), the normal is +y (facing -d)."""
    tris, i, j, fx, fz, o, d, target = _flat_grid_case()
    n_cells = 20
    n = len(o)
    res = O.closest_triangle_hit(o, d, np.zeros(n), np.full(n, np.inf), tris)
    assert np.all(res["hit"] == 1)
    t_exact = (-0.25 - o[:, 1]) / d[:, 1]
    assert np.allclose(res["t"], t_exact, rtol=1e-12, atol=0)
    idx = np.where(fx + fz < 1.0, i * n_cells + j, n_cells * n_cells + i * n_cells + j)
    assert np.array_equal(res["index"], idx)
    assert np.allclose(res["normal"], [0.0, 1.0, 0.0], atol=1e-12)
    # the interval decides: tmax below the plane's t misses, tmin beyond it misses
    r2 = O.closest_triangle_hit(o, d, np.zeros(n), t_exact * 0.999, tris)
    r3 = O.closest_triangle_hit(o, d, t_exact * 1.001, np.full(n, np.inf), tris)
    assert not r2["hit"].any() and not r3["hit"].any()


def test_closest_triangle_hit_nearest_and_lowest_index_on_ties():
    """Two parallel grids: rays from above take the upper one, from below the
    lower one; a duplicated triangle set resolves ties to the first copy."""
    tris, i, j, fx, fz, o, d, target = _flat_grid_case(n_rays=100)
    upper = tris + np.array([0.0, 0.2, 0.0], np.float32)
    both = np.concatenate([tris, upper])
    n = len(o)
    a = O.closest_triangle_hit(o, d, np.zeros(n), np.full(n, np.inf), both)
    assert np.all(a["index"] >= len(tris))
    assert np.allclose(a["t"], (-0.05 - o[:, 1]) / d[:, 1], rtol=1e-12)
    ob = o * np.array([1.0, -1.0, 1.0]) + np.array([0.0, -0.5, 0.0])
    db = d * np.array([1.0, -1.0, 1.0])
    b = O.closest_triangle_hit(ob, db, np.zeros(n), np.full(n, np.inf), both)
    assert np.all(b["index"] < len(tris))
    assert np.allclose(b["normal"], [0.0, -1.0, 0.0], atol=1e-12)
    dup = np.concatenate([tris, tris])
    c = O.closest_triangle_hit(o, d, np.zeros(n), np.full(n, np.inf), dup)
    assert np.all(c["index"] < len(tris)) and np.all(c["margin"] == 0.0)


def test_hybrid_trace_split_instances_equal_their_union():
    """Splitting a triangle set into two instances gives the closest hit over
    the union: same t, and the instance/index that hold the union's answer."""
    g = W.ground_heightfield(12, half=1.0, y0=-0.3, amplitude=0.05)
    s = W.scene_icosphere(level=2, radius=0.3) + np.array([0.0, 0.0, 0.0], np.float32)
    rays = W.chord_rays(300, seed=5, radius=1.2)
    o, d, tmin, tmax = O.rays_od(rays)
    union = np.concatenate([g, s])
    u = O.closest_triangle_hit(o, d, tmin, tmax, union)
    h = O.hybrid_trace(rays, [{"kind": "triangles", "tris": g}, {"kind": "triangles", "tris": s}])
    assert np.array_equal(h["hit"], u["hit"])
    assert np.array_equal(h["t"], u["t"])
    hit = u["hit"].astype(bool)
    assert hit.sum() > 50
    glob = np.where(h["inst"] == 0, h["leaf"], h["leaf"] + len(g))
    assert np.array_equal(glob[hit], u["index"][hit])
    assert np.all(h["inst"][~hit] == -1)
    # reversed order: the same record wherever no two instances tie
    h2 = O.hybrid_trace(rays, [{"kind": "triangles", "tris": s}, {"kind": "triangles", "tris": g}])
    assert np.array_equal(h2["t"], h["t"])
    assert np.array_equal(np.where(hit, 1 - h2["inst"], -1), h["inst"])


def test_hybrid_trace_neural_instance_alone_is_its_query():
    """A single neural instance: the hybrid record is the neural query's."""
    tris = W.scene_icosphere(level=2, radius=0.35)
    cfg = W.ModelConfig(n_levels=4, n_features=2, log2_table=10, base_res=4, growth=1.5, n_samples=4,
                        n_hidden=1, width=16)
    leaves = O.build_leaves(tris, 8, 1e-4)
    lay = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
    tab = W.init_table(lay["total"], cfg.n_features, 3, 1.0).astype(np.float64)
    layers = W.init_mlp(cfg.mlp_dims(), 4, gain=2.0)
    rays = W.chord_rays(200, seed=6, radius=0.6)
    q = O.query(rays, leaves, tab, layers, lay, cfg.n_samples)
    h = O.hybrid_trace(rays, [{"kind": "neural", "leaves": leaves, "table": tab, "layers": layers, "layout": lay,
                               "n_samples": cfg.n_samples}])
    assert q["hit"].sum() > 10
    assert np.array_equal(h["hit"], q["hit"]) and np.array_equal(h["t"], q["t"])
    assert np.array_equal(h["leaf"], q["leaf"])
    assert np.array_equal(h["inst"], np.where(q["hit"] > 0, 0, -1))


# ---------------------------------------------------------------- error-driven construction
def test_node_rank_worked_example():
    """q, p, r = 2 ln q + ln p and the training probability
    max(q^2 p / max q^2 p, 0.005), values derived by hand."""
    hits = [10, 0, 5, 20]
    trained = [5, 0, 5, 10]
    loss = [1.0, 0.0, 2.0, 0.5]
    q, p, r, prob = O.node_rank(hits, trained, loss, 100)
    qm = (0.2 + 0.4 + 0.05) / 3.0
    assert np.allclose(q, [0.2, qm, 0.4, 0.05], rtol=1e-15)
    assert np.allclose(p, [0.1, 0.0, 0.05, 0.2], rtol=1e-15)
    assert np.isinf(r[1]) and r[1] < 0
    assert math.isclose(r[0], 2 * math.log(0.2) + math.log(0.1), rel_tol=1e-14)
    # q^2 p: 0.004, -, 0.008, 0.0005 -> ratios 0.5, floor, 1, 0.0625
    assert np.allclose(prob, [0.5, 0.005, 1.0, 0.0625], rtol=1e-12)


def test_split_cut_replaces_highest_ranked_splittable_leaves():
    kids = {0: [1, 2], 1: [3, -1], 2: [-2, -3], 3: [-4, -5]}
    children = lambda ref: kids.get(ref, [])
    # leaves: 1 (r=5), 2 (r=7), ~0 (r=9, a base leaf: not splittable)
    assert O.split_cut([1, 2, -1], [5.0, 7.0, 9.0], 1, children) == [1, -2, -3, -1]
    assert O.split_cut([1, 2, -1], [5.0, 7.0, 9.0], 2, children) == [3, -1, -2, -3, -1]
    # ties go to the lower leaf index
    assert O.split_cut([1, 2], [4.0, 4.0], 1, children) == [3, -1, 2]


def test_training_selection_rates_and_extremes():
    n = 200000
    leaf = np.arange(n) % 4
    leaf[::7] = -1
    prob = np.array([0.0, 1.0, 0.25, 0.6], np.float32)
    keep = O.training_selection(leaf, prob, seed=11, step=3)
    assert not keep[leaf < 0].any()
    assert not keep[leaf == 0].any() and keep[leaf == 1].all()
    for l, pr in ((2, 0.25), (3, 0.6)):
        frac = keep[leaf == l].mean()
        assert abs(frac - pr) < 4 * math.sqrt(pr * (1 - pr) / np.sum(leaf == l))
    # the selection is a function of (ray, step, seed)
    assert np.array_equal(keep, O.training_selection(leaf, prob, seed=11, step=3))
    assert not np.array_equal(keep, O.training_selection(leaf, prob, seed=11, step=4))


def test_leaf_statistics_counts_by_hand():
    hits, trained, loss = O.leaf_statistics([0, 1, 1, -1, 2, 1], [True, False, True, False, True, True],
                                            [1.0, 9.0, 2.0, 5.0, 0.5, 3.0], 3)
    assert list(hits) == [1, 3, 1] and list(trained) == [1, 2, 1]
    assert np.allclose(loss, [1.0, 5.0, 0.5])


def test_reverse_inside_chord_listing():
    """Reading of depth from within a node: a ray starting inside a box lists
    that box over its whole chord with swapped endpoints (exit, entry) and
    first in order; boxes ahead of it are listed as usual; without the flag
    nothing changes."""
    lo = np.array([[-1.0, -1.0, -1.0], [2.0, -1.0, -1.0]])
    hi = np.array([[1.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    rays = {k: np.zeros(2, np.float32) for k in W.RAY_KEYS}
    rays["ox"][:] = [0.5, -3.0]
    rays["dx"][:] = [1.0, 1.0]
    rays["tmax"][:] = np.inf
    seg = O.ray_segments(rays, lo, hi, reverse_inside=True)
    # ray 0 starts at x = 0.5 inside box 0: chord entry -1.5, exit 0.5; box 1 at [1.5, 2.5]
    assert list(seg["leaf"][:2]) == [0, 1]
    assert seg["t0"][0] == 0.5 and seg["t1"][0] == -1.5
    assert seg["t0"][1] == 1.5 and seg["t1"][1] == 2.5
    # ray 1 starts outside both: plain segments
    assert list(seg["t0"][2:]) == [2.0, 5.0] and list(seg["t1"][2:]) == [4.0, 6.0]
    plain = O.ray_segments(rays, lo, hi)
    assert plain["t0"][0] == 0.0 and plain["t1"][0] == 0.5


def test_reverse_inside_decode_window():
    """A reversed chord [exit 0.5 .. entry -1.5] of a ray starting at t = 0:
    the sample order runs from the exit back, and a predicted depth fraction
    s puts the hit at 0.5 - 2 s, kept only for 0 < t <= tmax."""
    p = O.sample_points(np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]), np.array([0.5]), np.array([-1.5]), 4)
    assert np.allclose(p[0, :, 0], [0.25, -0.25, -0.75, -1.25])
    hit, t, _ = O.decode(np.array([[3.0, 0.0, 0, 0, 1]]), np.array([0.5]), np.array([-1.5]))
    assert hit[0] and t[0] == 0.5 - 2.0 * 0.5  # sigmoid(0) = 1/2: t = -0.5, behind the origin


# ---------------------------------------------------------------- albedo head (Sec. 5.2 auxiliary data)
def _logit(p):
    return math.log(p / (1.0 - p))


def test_albedo_relative_l2_closed_form():
    """Predicted albedo (0.2, 0.5, 0.8) against labels (0.1, 0.5, 1.0) on a
    hit ray: (0.01/0.05 + 0 + 0.04/0.65)/3 by hand; a missed ray adds nothing;
    a five-output model ignores albedo labels."""
    raw = np.zeros((2, 8))
    raw[:, 5:8] = [_logit(0.2), 0.0, _logit(0.8)]
    yn = np.array([[0.0, 0.0, 1.0], [1, 1, 1]])
    ya = np.array([[0.1, 0.5, 1.0], [0.9, 0.9, 0.9]])
    L8, per8 = O.loss(raw, [1, 0], [0.25, 0.9], yn, [True, True], ya)
    L5, per5 = O.loss(raw[:, :5], [1, 0], [0.25, 0.9], yn, [True, True], ya)
    rel = (0.01 / 0.05 + 0.0 + 0.04 / 0.65) / 3.0
    assert abs((per8[0] - per5[0]) - rel) < 1e-14
    assert per8[1] == per5[1]
    assert abs((L8 - L5) - rel / 2) < 1e-14
    assert np.all(O.loss_grad(raw[:, :5], [1, 0], [0.25, 0.9], yn, [True, True], ya)
                  == O.loss_grad(raw[:, :5], [1, 0], [0.25, 0.9], yn, [True, True]))


def test_albedo_gradient_near_the_target_matches_differences():
    """The relative L2 holds its denominator constant. Near s = a the constant
    and the differentiated denominator agree to first order (their ratio is
    1 - 2 s (s - a) / (s^2 + 0.01)), so central differences of the full loss
    pin the gradient's factor 2, sign, 1/3 mean, 1/(s^2 + 0.01) scale and
    sigmoid derivative there; away from it they differ by that known term. The
    gradient vanishes at s = a and for rays without a hit."""
    rng = np.random.default_rng(90)
    S = 20
    raw = rng.normal(0, 1.5, (S, 8))
    y = (rng.uniform(size=S) < 0.7).astype(float)
    y[0], y[1] = 1.0, 0.0
    yd = rng.uniform(size=S)
    yn = rng.normal(size=(S, 3))
    valid = np.ones(S, bool)
    s = O.sigmoid(raw[:, 5:8])
    delta = rng.choice([-1.0, 1.0], (S, 3)) * rng.uniform(5e-5, 2e-4, (S, 3))
    ya = s + delta
    g = O.loss_grad(raw, y, yd, yn, valid, ya)
    h = 1e-6
    for i in range(S):
        for c in range(3):
            rp, rm = raw.copy(), raw.copy()
            rp[i, 5 + c] += h
            rm[i, 5 + c] -= h
            fd = (O.loss(rp, y, yd, yn, valid, ya)[0] - O.loss(rm, y, yd, yn, valid, ya)[0]) / (2 * h)
            if y[i] == 0:
                assert g[i, 5 + c] == 0.0
            else:
                assert abs(fd - g[i, 5 + c]) <= 2e-3 * abs(g[i, 5 + c]) + 1e-12, (i, c, fd, g[i, 5 + c])
    # far from the target: the finite difference also sees the denominator
    ya2 = np.clip(s + 0.3, 0, 1)
    g2 = O.loss_grad(raw, y, yd, yn, valid, ya2)
    i, c = 0, 0
    rp, rm = raw.copy(), raw.copy()
    rp[i, 5 + c] += h
    rm[i, 5 + c] -= h
    fd = (O.loss(rp, y, yd, yn, valid, ya2)[0] - O.loss(rm, y, yd, yn, valid, ya2)[0]) / (2 * h)
    sc, ac = s[i, c], ya2[i, c]
    den = sc * sc + O.ALBEDO_EPS
    denom_term = -(sc - ac) ** 2 * 2 * sc / den ** 2 * sc * (1 - sc) / 3.0 / S
    assert abs(fd - (g2[i, 5 + c] + denom_term)) <= 1e-7 * abs(fd) + 1e-12
    # stationary at the target
    g3 = O.loss_grad(raw, y, yd, yn, valid, s)
    assert np.all(g3[:, 5:8] == 0.0)


def test_labels_albedo_is_the_hit_triangles():
    """Label albedo encodes the triangle index; decoding it gives a triangle of
    the trained leaf whose own Moller-Trumbore t is the label's t, and misses
    carry 0 (brute force per segment)."""
    tris = W.scene_random_tris(600, seed=14)
    lv = O.build_leaves(tris, 12)
    rays = W.camera_rays(14, 14, seed=15)
    seg = O.ray_segments(rays, lv["leaf_lo"], lv["leaf_hi"])
    o, d, _, _ = O.rays_od(rays)
    rr = seg["ray"]
    n = len(tris)
    alb = np.stack([(np.arange(n) + 1) / (n + 1), np.full(n, 0.25), np.full(n, 0.75)], 1)
    lab = O.labels(o[rr], d[rr], seg["leaf"], seg["t0"], seg["t1"], tris, lv["tri_perm"], lv["leaf_range"], alb)
    h = lab["hit"] == 1
    assert h.sum() > 15 and np.all(lab["albedo"][~h] == 0.0)
    tv = tris.astype(np.float64)
    for k in np.nonzero(h)[0]:
        j = int(round(lab["albedo"][k, 0] * (n + 1))) - 1
        a, b = lv["leaf_range"][seg["leaf"][k]]
        assert j in set(lv["tri_perm"][a:b].tolist())
        hit, t, _, _ = O.moller_trumbore(o[rr[k]][None], d[rr[k]][None], tv[j:j + 1, 0], tv[j:j + 1, 1],
                                         tv[j:j + 1, 2])
        assert hit[0] and t[0] == lab["t"][k]
        assert np.all(lab["albedo"][k, 1:] == [0.25, 0.75])


def test_albedo_head_leaves_geometry_and_resolves_with_the_hit():
    """Adding three albedo outputs leaves hit, t, normal and leaf unchanged.
    With the albedo rows of the output layer zero and biases b, every hit ray
    reads sigmoid(b) and every miss 0 (closed form); with random rows the
    albedo is that of the segment whose t the ray reports."""
    tris = W.scene_random_tris(400, seed=21)
    lv = O.build_leaves(tris, 8)
    rays = W.camera_rays(12, 12, seed=22)
    lay = O.level_layout(4, 4, 2.0, 10)
    rng = np.random.default_rng(23)
    tab = rng.uniform(-1, 1, (lay["total"], 2))
    layers5 = W.init_mlp([4 * 4 * 2, 16, 5], 24, gain=2.0)
    layers5[-1][1][0] += 0.3      # more predicted hits
    W8 = np.concatenate([layers5[-1][0], np.zeros((3, 16))], 0)
    b8 = np.concatenate([layers5[-1][1], [-1.0, 0.0, 2.0]])
    q5 = O.query(rays, lv, tab, layers5, lay, 4)
    q8 = O.query(rays, lv, tab, layers5[:-1] + [(W8, b8)], lay, 4)
    for k in ("hit", "t", "normal", "leaf"):
        assert np.array_equal(q5[k], q8[k]), k
    h = q8["hit"] == 1
    assert 10 < h.sum() < len(h)
    expect = 1.0 / (1.0 + np.exp(-np.array([-1.0, 0.0, 2.0])))
    assert np.allclose(q8["albedo"][h], expect, rtol=0, atol=1e-15)
    assert np.all(q8["albedo"][~h] == 0.0)
    Wr = np.concatenate([layers5[-1][0], rng.normal(0, 1, (3, 16))], 0)
    qr = O.query(rays, lv, tab, layers5[:-1] + [(Wr, b8)], lay, 4)
    seg = qr["segments"]
    for r in np.nonzero(qr["hit"] == 1)[0]:
        js = [j for j in range(seg["offsets"][r], seg["offsets"][r + 1])
              if qr["seg_hit"][j] and qr["seg_t"][j] == qr["t"][r]]
        assert np.array_equal(qr["albedo"][r], O.sigmoid(qr["raw"][js[0], 5:8]))


def test_hybrid_albedo_follows_the_answering_instance():
    """In the two-level trace the record's albedo is the triangle's where a
    triangle instance answers and 0 where an instance without albedo does."""
    tris = W.scene_random_tris(300, seed=31, edge=0.25)
    a = tris[:150]
    b = tris[150:]
    alb = np.random.default_rng(32).uniform(0, 1, (150, 3))
    rays = W.camera_rays(16, 16, seed=33)
    out = O.hybrid_trace(rays, [{"kind": "triangles", "tris": a, "albedo": alb}, {"kind": "triangles", "tris": b}])
    ia = out["inst"] == 0
    ib = out["inst"] == 1
    assert ia.sum() > 5 and ib.sum() > 5
    assert np.array_equal(out["albedo"][ia], alb[out["leaf"][ia]])
    assert np.all(out["albedo"][ib] == 0.0) and np.all(out["albedo"][out["inst"] < 0] == 0.0)


# ---------------------------------------------------------------- cut leaves (Sec. 5.1)
def _hand_base():
    """A hand-built base tree: node 0 -> (node 2, node 1) (second child first,
    so depth-first order differs from node order), node 1 -> (leaf 0, leaf 1),
    node 2 -> (leaf 2, leaf 3). Triangle i spans x in [i, i + 0.5], y in
    [0, 1], z in [0, 2]; a permuted triangle order catches index mix-ups."""
    dt = np.dtype([("child0", "<i4"), ("child1", "<i4")])
    nodes = np.array([(2, 1), (~0, ~1), (~2, ~3)], dt)
    tri_perm = np.array([3, 1, 0, 2, 7, 5, 6, 4], np.int32)
    leaf_range = np.array([[0, 2], [2, 4], [4, 6], [6, 8]], np.int32)
    tris = np.array([[[i, 0.0, 0.0], [i + 0.5, 1.0, 0.0], [i, 0.0, 2.0]] for i in range(8)], np.float32)
    return tris, nodes, leaf_range, tri_perm


def _is_outward_f32(lo, exact_lo, hi, exact_hi):
    """lo is the largest float32 <= exact_lo, hi the smallest float32 >= exact_hi."""
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    up = np.nextafter(lo, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(hi, np.float32(-np.inf)).astype(np.float64)
    return (np.all(lo.astype(np.float64) <= exact_lo) and np.all(up > exact_lo)
            and np.all(hi.astype(np.float64) >= exact_hi) and np.all(dn < exact_hi))


def test_cut_leaves_root_only_is_one_leaf_of_everything():
    tris, nodes, rng, perm = _hand_base()
    refs, sets, lo, hi = O.cut_leaves(tris, nodes, rng, perm, [0], 0.01, 10.0)
    assert refs == [0]
    assert sets[0].tolist() == list(range(8))
    # AABB x [0, 7.5], y [0, 1], z [0, 2], pushed out by 0.01 * 10 = 0.1
    assert _is_outward_f32(lo[0], np.array([-0.1, -0.1, -0.1]), hi[0], np.array([7.6, 1.1, 2.1]))


def test_cut_leaves_all_base_leaves_in_depth_first_order():
    tris, nodes, rng, perm = _hand_base()
    cut = [~0, ~1, ~2, ~3]
    refs, sets, lo, hi = O.cut_leaves(tris, nodes, rng, perm, cut, 0.01, 10.0)
    # node 0 visits node 2 first: base leaves 2, 3, then 0, 1
    assert refs == [~2, ~3, ~0, ~1]
    assert [s.tolist() for s in sets] == [[5, 7], [4, 6], [1, 3], [0, 2]]
    xs = [(5, 7.5), (4, 6.5), (1, 3.5), (0, 2.5)]
    for i, (a, b) in enumerate(xs):
        assert _is_outward_f32(lo[i], np.array([a - 0.1, -0.1, -0.1]), hi[i], np.array([b + 0.1, 1.1, 2.1]))


def test_cut_leaves_mixed_cut_unions_the_base_leaves_below():
    tris, nodes, rng, perm = _hand_base()
    refs, sets, lo, hi = O.cut_leaves(tris, nodes, rng, perm, [1, ~2, ~3], 0.0, 10.0)
    assert refs == [~2, ~3, 1]
    assert [s.tolist() for s in sets] == [[5, 7], [4, 6], [0, 1, 2, 3]]
    # no inflation: the exact AABB (representable values)
    assert lo[2].tolist() == [0.0, 0.0, 0.0] and hi[2].tolist() == [3.5, 1.0, 2.0]
    refs2, sets2, _, _ = O.cut_leaves(tris, nodes, rng, perm, [2, ~0, ~1], 0.0, 10.0)
    assert refs2 == [2, ~0, ~1]
    assert [s.tolist() for s in sets2] == [[4, 5, 6, 7], [1, 3], [0, 2]]


def test_cut_leaves_rejects_an_incomplete_cut():
    tris, nodes, rng, perm = _hand_base()
    with pytest.raises(ValueError):
        O.cut_leaves(tris, nodes, rng, perm, [2, ~0], 0.0, 10.0)   # base leaf 1 below no reference


def test_sample_grid_f32_hand_example_and_rounding_bound():
    """sample_grid_f32: a hand example whose every step is exact in float32
    (t_k = 1.25, 1.75, 2.25, 2.75; x = t/8 + 1/2, y = 2t/8 + 1/2 clamped), and
    on random inputs every coordinate within 3 float32 ulps of the exact
    float64 value of the same formula (a dropped term or a wrong operand
    would be far off)."""
    o = np.array([[0.0, 0.0, 0.0]])
    d = np.array([[1.0, 2.0, 0.0]])
    x = O.sample_grid_f32(o, d, np.array([1.0]), np.array([3.0]), 4, np.zeros(3), 8.0)
    assert x[0, :, 0].tolist() == [0.65625, 0.71875, 0.78125, 0.84375]
    assert x[0, :, 1].tolist() == [0.8125, 0.9375, 1.0, 1.0]
    assert x[0, :, 2].tolist() == [0.5, 0.5, 0.5, 0.5]
    rng = np.random.default_rng(3)
    n = 2000
    o = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    t0 = rng.uniform(0, 1, n).astype(np.float32)
    t1 = (t0 + rng.uniform(0, 1, n)).astype(np.float32)
    c = np.array([0.1, -0.2, 0.05], np.float32)
    E = np.float32(3.0)
    g32 = O.sample_grid_f32(o, d, t0, t1, 16, c, E)
    ref = O.normalize_points(O.sample_points(o, d, t0, t1, 16), c, E)
    inside = (ref > 1e-3) & (ref < 1 - 1e-3)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(g32 - ref)[inside] <= 3 * ulp[inside] + 2e-7)


def _round_f32(v: float) -> float:
    """Round a Python float to the nearest float32 (ties to even) through the
    IEEE single format of the struct module."""
    import struct
    return struct.unpack("<f", struct.pack("<f", v))[0]


def test_level_corners_f32_grid_coordinates():
    """level_corners(f32=True): p = x * res rounded once to float32 (the exact
    double product of two float32 values, rounded through struct), cell =
    min(floor(p), res - 1), frac = p - cell. Hand values: x = 0.1 (float32)
    at res 7006 gives p = 700.6000366..., x = 0.5 at res 7006 is exact (3503),
    and x = 1 clamps to the last cell with frac 1. Random points: frac within
    half a float32 ulp of p of the float64 form, and weights summing to 1."""
    x32 = np.float32(0.1)
    p = _round_f32(float(x32) * 7006.0)
    assert p != float(x32) * 7006.0 and abs(p - float(x32) * 7006.0) <= 2.0 ** -15
    pts = np.array([[float(x32), 0.5, 1.0]])
    c32, w32 = O.level_corners(pts, 7006, f32=True)
    c64, w64 = O.level_corners(pts, 7006)
    assert c32[0, 0].tolist() == [700, 3503, 7005] == c64[0, 0].tolist()
    fx = p - 700.0
    # corner 1 (+x): weight fx * (1 - 0) * (1 - 1) = 0; corner 7 (+x,+y,+z): fx * 0 * 1
    # corner 5 (+x, +z): fx * (1 - fy) * fz with fy = 0, fz = 1
    assert w32[0, 5] == fx and w32[0, 4] == 1.0 - fx
    assert abs(w64[0, 5] - (float(x32) * 7006.0 - 700.0)) < 1e-12 and w64[0, 5] != w32[0, 5]
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (3000, 3)).astype(np.float32).astype(np.float64)
    for res in (16, 81, 1383, 7006):
        c32, w32 = O.level_corners(x, res, f32=True)
        c64, w64 = O.level_corners(x, res)
        pos = x * res
        half_ulp = 0.5 * np.spacing(pos.astype(np.float32)).astype(np.float64)
        same = np.all(c32 == c64, axis=(-1, -2))
        assert same.mean() > 0.99
        f32 = (np.asarray(x, np.float32) * np.float32(res)).astype(np.float64) - c32[:, 0, :]
        assert np.all(np.abs(f32 - (pos - c64[:, 0, :]))[same] <= half_ulp[same] + 1e-12)
        assert np.allclose(w32.sum(-1), 1.0, atol=1e-12)
