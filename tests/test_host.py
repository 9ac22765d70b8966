"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
function the headers declare, and its host computations (level layout, MLP
parameter count, S0 leaf build) agree exactly with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(nbvh_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function():
    L = B.lib()
    names = declared_functions()
    assert "nbvh_query_rays" in names and "nbvh_build_leaves" in names
    for n in names:
        assert hasattr(L, n), n
    assert L.nbvh_built_arch() == 1030


def test_binding_covers_declared_functions():
    assert set(declared_functions()) <= set(B.EXPORTED) | {"nbvh_status_string"}


def test_status_strings():
    for code in range(8):
        assert B.lib().nbvh_status_string(code)


def _desc(cfg, tp=B.FP16, mp=B.FP32):
    return B.model_desc(cfg, tp, mp, (0.0, 0.0, 0.0), 1.0)


@pytest.mark.parametrize("cfg", [W.C0.model, W.C1.model])
def test_level_layout_matches_oracle(cfg):
    got = B.level_layout(_desc(cfg))
    ref = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
    for k in ("res", "dense", "size", "offset"):
        assert np.array_equal(got[k], ref[k]), k
    assert got["total"] == ref["total"]


def test_mlp_param_count():
    cfg = W.C1.model
    n = B.mlp_param_count(_desc(cfg))
    dims = cfg.mlp_dims()
    assert n == sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
    assert len(B.pack_mlp(W.init_mlp(dims, 1))) == n


def test_invalid_descriptors_rejected():
    cfg = W.C0.model
    d = _desc(cfg)
    d.n_features = 3
    with pytest.raises(B.NBVHError):
        B.level_layout(d)
    d = _desc(cfg)
    d.frame_extent = 0.0
    with pytest.raises(B.NBVHError):
        B.mlp_param_count(d)


@pytest.mark.parametrize("n_tris,n_leaves,seed", [(4096, 64, 1), (3000, 37, 2), (500, 1, 3), (777, 200, 4)])
def test_leaf_build_matches_oracle_exactly(n_tris, n_leaves, seed):
    tris = W.scene_random_tris(n_tris, seed=seed)
    got = B.build_leaves(tris, n_leaves, 1e-4)
    ref = O.build_leaves(tris, n_leaves, 1e-4)
    assert np.array_equal(got["tri_perm"], ref["tri_perm"])
    assert np.array_equal(got["leaf_range"], ref["leaf_range"])
    assert np.array_equal(got["leaf_lo"], ref["leaf_lo"])
    assert np.array_equal(got["leaf_hi"], ref["leaf_hi"])
    fr = ref["frame"]
    assert np.array_equal(got["info"]["centre"], fr["centre"].astype(np.float32))
    assert got["info"]["extent"] == np.float32(fr["extent"])
    assert got["info"]["sphere_radius"] == np.float32(fr["sphere_radius"])


def test_leaf_build_icosphere_matches_oracle():
    tris = W.scene_icosphere(level=5)
    got = B.build_leaves(tris, 256, 1e-4)
    ref = O.build_leaves(tris, 256, 1e-4)
    assert np.array_equal(got["tri_perm"], ref["tri_perm"])
    assert np.array_equal(got["leaf_lo"], ref["leaf_lo"]) and np.array_equal(got["leaf_hi"], ref["leaf_hi"])


def test_node_tree_is_consistent():
    tris = W.scene_random_tris(2000, seed=5)
    lv = B.build_leaves(tris, 50)
    nodes = B.node_array(lv)
    assert len(nodes) == lv["n_nodes"] == 49
    seen = []

    def walk(i, lo, hi):
        nd = nodes[i]
        for c, l, h in ((nd["child0"], nd["lo0"], nd["hi0"]), (nd["child1"], nd["lo1"], nd["hi1"])):
            assert np.all(l >= lo) and np.all(h <= hi)       # children nest in the parent
            if c < 0:
                leaf = ~c
                seen.append(leaf)
                assert np.array_equal(l, lv["leaf_lo"][leaf]) and np.array_equal(h, lv["leaf_hi"][leaf])
            else:
                walk(c, l, h)

    walk(0, np.full(3, -np.inf), np.full(3, np.inf))
    assert sorted(seen) == list(range(50))


def test_build_leaves_rejects_bad_arguments():
    tris = W.scene_random_tris(10, seed=6)
    with pytest.raises(B.NBVHError):
        B.build_leaves(tris, 11)
    with pytest.raises(B.NBVHError):
        B.build_leaves(tris, 0)


@pytest.mark.parametrize("max_leaf", [1, 4, 16])
def test_tri_blas_build_invariants(max_leaf):
    """Triangle BLAS (host SAH build): every triangle in exactly one leaf of
    at most max_leaf triangles, each child box the exact AABB of its
    subtree's triangles and nested in its parent, a binary tree of
    n_leaves - 1 internal nodes."""
    ground = W.ground_heightfield(16, amplitude=0.05)
    sph = W.scene_icosphere(level=2, radius=0.3)
    tris = np.concatenate([ground, sph]).astype(np.float32)
    blas = B.build_tri_blas(tris, max_leaf)
    nl = blas["n_leaves"]
    assert blas["n_nodes"] == max(1, nl - 1)
    assert sorted(blas["tri_perm"].tolist()) == list(range(len(tris)))
    rng = blas["leaf_range"]
    assert rng[0, 0] == 0 and rng[-1, 1] == len(tris) and np.all(rng[1:, 0] == rng[:-1, 1])
    assert np.all(rng[:, 1] - rng[:, 0] >= 1) and np.all(rng[:, 1] - rng[:, 0] <= max_leaf)
    nodes = B.node_array({"nodes": blas["nodes"]})
    seen = []

    def walk(i, lo, hi):
        nd = nodes[i]
        tri_sets = []
        for c, l, h in ((nd["child0"], nd["lo0"], nd["hi0"]), (nd["child1"], nd["lo1"], nd["hi1"])):
            assert np.all(l >= lo) and np.all(h <= hi)
            if c < 0:
                seen.append(~c)
                a, b = rng[~c]
                ids = blas["tri_perm"][a:b]
            else:
                ids = walk(c, l, h)
            v = tris[ids].reshape(-1, 3)
            assert np.array_equal(v.min(0), l) and np.array_equal(v.max(0), h)
            tri_sets.append(ids)
        return np.concatenate(tri_sets)

    walk(0, np.full(3, -np.inf), np.full(3, np.inf))
    assert sorted(seen) == list(range(nl))


def test_tri_blas_single_leaf_and_bad_arguments():
    # three copies of one triangle: no split separates them, so one leaf
    tris = np.repeat(W.scene_random_tris(1, seed=8), 3, axis=0)
    blas = B.build_tri_blas(tris, 4)
    assert blas["n_leaves"] == 1 and blas["n_nodes"] == 1
    nd = B.node_array({"nodes": blas["nodes"]})[0]
    assert nd["child0"] == ~0 and nd["child1"] == 0x7fffffff
    with pytest.raises(B.NBVHError):
        B.build_tri_blas(tris, 0)
    bad = tris.copy()
    bad[1, 1, 1] = np.nan
    with pytest.raises(B.NBVHError):
        B.build_tri_blas(bad, 4)


def test_query_options_checked_on_host():
    """nbvh_query_options_default gives the documented defaults; invalid
    options and autotuner arguments are rejected before any device work (no
    GPU needed: zero rays return before the first CUDA call)."""
    L = B.lib()
    o = B.query_options()
    assert (o.schedule, o.patience_cycles, o.traverse_block, o.eval_threads, o.w1_mode) == (1, 4000, 128, 0, 0)
    desc = _desc(W.C1.model, B.FP16, B.FP16)
    fake = ctypes.c_void_p(1 << 20)
    rays = B.Rays()
    rays.n = 0
    hits = B.Hits()
    for bad in (dict(schedule=7), dict(patience_cycles=-5), dict(traverse_block=100), dict(eval_threads=384),
                dict(w1_mode=3)):
        assert L.nbvh_query_rays_opt(ctypes.byref(desc), fake, fake, fake, 1, rays, 8, hits, fake, 1 << 30,
                                     ctypes.byref(B.query_options(**bad)), None) == 1, bad
    assert L.nbvh_query_rays_opt(ctypes.byref(desc), fake, fake, fake, 1, rays, 8, hits, fake, 1 << 30,
                                 ctypes.byref(B.query_options()), None) == 0
    best = B.TuneResult()
    n_all = ctypes.c_int32()
    assert L.nbvh_autotune_query(None, None, None, None, 0, B.Rays(), 8, B.Hits(), None, 0, 1, ctypes.byref(best),
                                 None, 0, ctypes.byref(n_all), None) == 1


def test_unsupported_query_enqueues_nothing():
    """A valid descriptor with options the kernels cannot run (256-thread
    evaluation CTAs at width 128) returns NBVH_ERR_UNSUPPORTED from the host
    check, before any launch: the library's launch count does not move and no
    CUDA call is made (this runs without a GPU)."""
    L = B.lib()
    from dataclasses import replace
    desc = _desc(replace(W.C1.model, width=128), B.FP16, B.FP16)
    fake = ctypes.c_void_p(1 << 20)
    rays = B.Rays()
    for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax"):
        setattr(rays, k, 1 << 20)
    rays.n = 1000
    hits = B.Hits()
    for k in B.HIT_KEYS:
        setattr(hits, k, 1 << 20)
    n0 = B.launch_count()
    st = L.nbvh_query_rays_opt(ctypes.byref(desc), fake, fake, fake, 1, rays, 8, hits, ctypes.c_void_p(1 << 20),
                               1 << 40, ctypes.byref(B.query_options(eval_threads=256)), None)
    assert st == 7 and B.launch_count() == n0


def test_rank_leaves_matches_oracle():
    """nbvh_rank_leaves (Sec. 5.1 node error, Sec. 5.2 training probability)
    against the oracle's node_rank on random statistics with unhit and
    untrained leaves."""
    rng = np.random.default_rng(17)
    n = 300
    hits = rng.integers(0, 500, n).astype(np.uint32)
    hits[rng.choice(n, 30, replace=False)] = 0
    trained = np.minimum(hits, rng.integers(0, 400, n)).astype(np.uint32)
    trained[rng.choice(n, 20, replace=False)] = 0
    loss = (trained * rng.uniform(0.01, 2.0, n)).astype(np.float32)
    n_rays = int(hits.sum()) + 1000
    q, p, r, prob = B.node_rank(hits, trained, loss, n_rays)
    oq, op, orr, oprob = O.node_rank(hits.astype(np.int64), trained.astype(np.int64), loss.astype(np.float64), n_rays)
    assert np.allclose(q, oq, rtol=1e-14, atol=0) and np.allclose(p, op, rtol=1e-15, atol=0)
    fin = np.isfinite(orr)
    assert np.array_equal(np.isfinite(r), fin) and np.allclose(r[fin], orr[fin], rtol=1e-13, atol=1e-13)
    assert np.array_equal(prob, oprob.astype(np.float32))
    assert (prob[~fin] == np.float32(0.005)).all() and prob.max() == 1.0


def test_refine_cut_matches_oracle_split():
    """nbvh_refine_cut against the oracle's split_cut on a real SAH base BVH:
    the k best-ranked splittable leaves become their children (ties to the
    lower index), new leaves train with probability 1, others keep theirs."""
    tris = np.concatenate([W.ground_heightfield(10, amplitude=0.05), W.scene_icosphere(level=2, radius=0.3)])
    base = _base(tris)
    nodes = B.node_array({"nodes": base["nodes"]})

    def children(ref):
        if ref < 0:
            return []
        nd = nodes[ref]
        return [int(nd["child0"])] + ([int(nd["child1"])] if int(nd["child1"]) != 0x7fffffff else [])

    rng = np.random.default_rng(5)
    cut = [0]
    for _ in range(6):
        r = rng.normal(size=len(cut))
        r[rng.uniform(size=len(cut)) < 0.2] = -np.inf
        r[rng.integers(0, len(cut))] = r.max() if np.isfinite(r).any() else 0.0  # a tie
        prob = rng.uniform(0.005, 1.0, len(cut)).astype(np.float32)
        k = int(rng.integers(1, 4))
        new_cut, new_prob = B.refine_cut(base, cut, r, prob, k)
        assert new_cut == O.split_cut(cut, r, k, children)
        kept = {c: float(p) for c, p in zip(cut, prob)}
        for c, p in zip(new_cut, new_prob):
            assert p == (kept[c] if c in kept else 1.0)
        cut = new_cut


def test_train_workspace_budget_picks_recompute_below_the_stored_size():
    """nbvh_train_workspace_budget: the stored size when it fits (chunk = n),
    else the largest 128-ray multiple whose activation chunk fits (recompute
    mode, smaller than stored), else NBVH_ERR_WORKSPACE_TOO_SMALL."""
    for mp in (B.FP32, B.FP16):
        desc = _desc(W.C1.model, B.FP16, mp)
        n = 1 << 18
        stored = B.train_workspace_size(desc, n, 2048)
        b, c = B.train_workspace_budget(desc, n, 2048, stored)
        assert (b, c) == (stored, n)
        b2, c2 = B.train_workspace_budget(desc, n, 2048, stored // 3)
        assert c2 < n and c2 % 128 == 0 and b2 <= stored // 3
        b3, c3 = B.train_workspace_budget(desc, n, 2048, b2 + 1)
        assert c3 == c2  # the largest chunk that fits
        with pytest.raises(B.NBVHError):
            B.train_workspace_budget(desc, n, 2048, 1 << 20)


def _base(tris, max_leaf=8):
    return B.build_tri_blas(tris, max_leaf)


@pytest.mark.parametrize("depths", ["root", "leaves", "mixed"])
def test_build_cut_matches_oracle(depths):
    """nbvh_build_cut: leaves in depth-first order, each with the triangles of
    every base leaf below its reference and their AABB pushed out and rounded
    outward, exactly as the oracle's brute-force walk gives; the node tree's
    child boxes nest their descendants' leaf boxes."""
    tris = np.concatenate([W.ground_heightfield(10, amplitude=0.05), W.scene_icosphere(level=2, radius=0.3)])
    base = _base(tris)
    nodes = B.node_array({"nodes": base["nodes"]})
    info = B.build_leaves(tris, 1)["info"]
    if depths == "root":
        cut = [0]
    elif depths == "leaves":
        cut = [~i for i in range(base["n_leaves"])]
    else:
        rng = np.random.default_rng(4)
        cut, stack = [], [0]
        while stack:  # random cut: stop or descend at each internal reference
            ref = stack.pop()
            if ref < 0 or rng.uniform() < 0.3:
                cut.append(ref)
                continue
            nd = nodes[ref]
            kids = [int(nd["child0"])] + ([int(nd["child1"])] if int(nd["child1"]) != 0x7fffffff else [])
            stack += kids[::-1]
    lv = B.build_cut(base, cut, 1e-4, info)
    refs, sets, lo, hi = O.cut_leaves(tris, nodes, base["leaf_range"], base["tri_perm"], cut, 1e-4, info["extent"])
    assert list(lv["leaf_ref"]) == refs
    for i, st in enumerate(sets):
        a, b = lv["leaf_range"][i]
        assert np.array_equal(np.sort(base["tri_perm"][a:b]), st)
    assert np.array_equal(lv["leaf_lo"], lo) and np.array_equal(lv["leaf_hi"], hi)
    assert sum(len(st) for st in sets) == len(tris)
    # tree consistency
    nn = B.node_array(lv)
    seen = []

    def walk(i):
        nd = nn[i]
        boxes = []
        for c, l, h in ((nd["child0"], nd["lo0"], nd["hi0"]), (nd["child1"], nd["lo1"], nd["hi1"])):
            if c == 0x7fffffff:
                continue
            if c < 0:
                seen.append(~c)
                assert np.array_equal(l, lv["leaf_lo"][~c]) and np.array_equal(h, lv["leaf_hi"][~c])
            else:
                clo, chi = walk(c)
                assert np.array_equal(l, clo) and np.array_equal(h, chi)
            boxes.append((l, h))
        return np.min([b[0] for b in boxes], 0), np.max([b[1] for b in boxes], 0)

    walk(0)
    assert sorted(seen) == list(range(len(cut)))


def test_build_cut_rejects_invalid_cuts():
    tris = W.ground_heightfield(6, amplitude=0.05)
    base = _base(tris, 4)
    info = B.build_leaves(tris, 1)["info"]
    nd = B.node_array({"nodes": base["nodes"]})[0]
    with pytest.raises(B.NBVHError):   # overlapping: the root and one of its children
        B.build_cut(base, [0, int(nd["child0"])], 1e-4, info)
    with pytest.raises(B.NBVHError):   # incomplete: one child only
        B.build_cut(base, [int(nd["child0"])], 1e-4, info)
    with pytest.raises(B.NBVHError):   # out of range
        B.build_cut(base, [base["n_nodes"] + 5], 1e-4, info)
