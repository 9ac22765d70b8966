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


def test_schedule_and_tuner_arguments_checked_on_host():
    """Invalid schedule settings and autotuner arguments are rejected before
    any device work (no GPU needed)."""
    L = B.lib()
    assert L.nbvh_set_query_schedule(7, 0) == 1
    assert L.nbvh_set_query_schedule(1, -5) == 1
    assert L.nbvh_set_traverse_block(100) == 1
    best = B.TuneResult()
    n_all = ctypes.c_int32()
    assert L.nbvh_autotune_query(None, None, None, None, 0, B.Rays(), 8, B.Hits(), None, 0, 1, ctypes.byref(best),
                                 None, 0, ctypes.byref(n_all), None) == 1
    s, p = B.get_query_schedule()
    assert s in (0, 1) and p >= 0


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
