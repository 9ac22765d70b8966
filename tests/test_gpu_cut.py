"""GPU parity of the error-driven construction (Sec. 5.1 "Base-BVH cut
optimization", "Node error"; Sec. 5.2 "Ray distribution") through the C ABI:
the weighted training step's ray selection and per-leaf statistics against the
FP64 oracle, and the cut optimizer's result against the oracle's cut walk."""
import numpy as np
import pytest

from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _setup(mlp_prec=B.FP32, n_leaves=32, seed=5):
    torch = _torch()
    tris = W.scene_icosphere(level=4, radius=0.35)
    leaves = B.build_leaves(tris, n_leaves)
    oleaves = O.build_leaves(tris, n_leaves)
    cfg = W.ModelConfig(n_levels=8, n_features=2, log2_table=14, base_res=8, growth=1.5, n_samples=8, n_hidden=2,
                        width=32)
    info = leaves["info"]
    desc = B.model_desc(cfg, B.FP32, mlp_prec, info["centre"], info["extent"])
    lay = B.level_layout(desc)
    tab = W.init_table(lay["total"], cfg.n_features, seed, 0.5)
    layers = W.init_mlp(cfg.mlp_dims(), seed + 1, gain=2.0)
    opt = B.Optimizer(desc, torch.as_tensor(tab).cuda(), torch.as_tensor(B.pack_mlp(layers)).cuda())
    scene = B.DeviceScene(tris, leaves)
    return tris, leaves, oleaves, cfg, desc, tab, layers, opt, scene


def test_weighted_step_selection_and_leaf_statistics():
    """One weighted FP32 step: per-leaf first-leaf hits and trained counts equal
    the oracle's (same Philox rays and selection), loss sums within 1e-4."""
    torch = _torch()
    tris, leaves, oleaves, cfg, desc, tab, layers, opt, scene = _setup()
    n_leaves = len(leaves["leaf_lo"])
    n, seed, step = 3000, 77, 3
    prob = np.random.default_rng(1).uniform(0.05, 1.0, n_leaves).astype(np.float32)
    prob[3] = 0.0
    prob[4] = 1.0
    stats = {"hits": torch.zeros(n_leaves, dtype=torch.int32, device="cuda"),
             "trained": torch.zeros(n_leaves, dtype=torch.int32, device="cuda"),
             "loss": torch.zeros(n_leaves, dtype=torch.float32, device="cuda")}
    ws = B.new_workspace(B.train_workspace_size(desc, n, n_leaves))
    B.train_step_weighted(desc, opt, scene, B.TRAIN_PROBED_MIX, n, seed, step, 1e-2, ws,
                          leaf_prob=torch.as_tensor(prob).cuda(), stats=stats)
    assert B.device_status() == 0
    # oracle: the same rays, labels, selection and per-ray loss terms
    R = O.train_rays(O.TRAIN_MODE_PROBED_MIX, seed, step - 1, n, oleaves)
    keep = O.training_selection(R["leaf"], prob, seed, step - 1)
    lab = O.labels(R["o"], R["d"], R["leaf"], R["t0"], R["t1"], tris, oleaves["tri_perm"], oleaves["leaf_range"])
    lay = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
    fr = oleaves["frame"]
    valid = R["leaf"] >= 0
    _, raw = O.eval_segments(R["o"], R["d"], R["t0"], R["t1"], tab.astype(np.float64), layers, lay,
                             fr["model_centre"], fr["model_extent"], cfg.n_samples)
    _, per = O.loss(raw, lab["hit"], lab["depth"], lab["normal"], valid)
    hits, trained, loss = O.leaf_statistics(R["leaf"], keep, per, n_leaves)
    assert np.array_equal(stats["hits"].cpu().numpy(), hits)
    assert np.array_equal(stats["trained"].cpu().numpy(), trained)
    assert trained[3] == 0 and trained[4] == hits[4] and hits.sum() > 2000
    got = stats["loss"].cpu().numpy()
    assert np.all(np.abs(got - loss) <= 1e-4 * np.maximum(np.abs(loss), 1.0))


def test_unweighted_step_equals_plain_step():
    """Without probabilities and statistics the weighted step is nbvh_train_step:
    the same loss (FP64 reduction) and the same parameters after one step,
    except where Adam's first step (lr * g / (|g| + eps)) turns the sign of a
    gradient that float atomics leave at rounding level."""
    torch = _torch()
    _, leaves, _, _, desc, _, _, opt_a, scene = _setup()
    _, _, _, _, _, _, _, opt_b, _ = _setup()
    n = 2048
    ws = B.new_workspace(B.train_workspace_size(desc, n, len(leaves["leaf_lo"])))
    la = torch.zeros(1, dtype=torch.float32, device="cuda")
    lb = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.train_step(desc, opt_a, scene, B.TRAIN_PROBED_MIX, n, 9, 1, 1e-2, ws, loss_out=la)
    B.train_step_weighted(desc, opt_b, scene, B.TRAIN_PROBED_MIX, n, 9, 1, 1e-2, ws, loss_out=lb)
    assert B.device_status() == 0
    assert abs(la.item() - lb.item()) <= 1e-12 * abs(la.item()) and la.item() > 0
    for a, b in ((opt_a.table_master, opt_b.table_master), (opt_a.mlp, opt_b.mlp)):
        off = (a - b).abs() > 1e-5
        assert off.float().mean().item() <= 1e-3
    assert not torch.equal(opt_a.mlp, _setup()[7].mlp)  # the step did change the parameters


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_cut_optimizer_reaches_target_with_a_valid_cut(mp):
    """optimize_cut from the root to 24 leaves: the final cut covers every
    triangle once (oracle walk of the base tree), its N-BVH has the target leaf
    count, every round trains, and the loss stays finite."""
    _torch()
    tris, _, _, cfg, desc, _, _, opt, _ = _setup(mlp_prec=mp)
    lv, scene, hist, step = B.optimize_cut(tris, desc, opt, 24, base_max_leaf=8, iters=3, splits=2, factor=1.5,
                                           final_iters=4, batch=4096, seed=3)
    assert B.device_status() == 0
    assert len(lv["leaf_ref"]) == 24 and scene.n_leaves == 24
    base = B.build_tri_blas(tris, 8)
    nodes = B.node_array({"nodes": base["nodes"]})
    refs, sets, lo, hi = O.cut_leaves(tris, nodes, base["leaf_range"], base["tri_perm"], list(lv["leaf_ref"]), 1e-4,
                                      lv["info"]["extent"])
    assert refs == list(lv["leaf_ref"])
    assert np.array_equal(np.sort(np.concatenate(sets)), np.arange(len(tris)))
    assert np.array_equal(lv["leaf_lo"], lo) and np.array_equal(lv["leaf_hi"], hi)
    assert hist[0]["leaves"] == 1 and hist[-1].get("final") and len(hist) >= 4
    assert all(np.isfinite(h["loss"]) and h["mean_q"] > 0 for h in hist)
    assert step == 1 + sum(h["iters"] for h in hist)


def test_levels_of_detail():
    """optimize_cut with LoDs registered every 8 training steps: the LoDs are
    valid cuts of increasing size ending with the final cut; every step trains
    one of them; a query on each LoD runs, and a coarser LoD evaluates fewer
    segments for the same rays."""
    torch = _torch()
    tris, _, _, cfg, desc, _, _, opt, _ = _setup(mlp_prec=B.FP16)
    lods = []
    lv, scene, hist, step = B.optimize_cut(tris, desc, opt, 32, base_max_leaf=8, iters=4, splits=2, factor=1.5,
                                           final_iters=6, batch=4096, seed=3, lod_every=8, lods_out=lods)
    assert B.device_status() == 0
    sizes = [len(x[0]["leaf_ref"]) for x in lods]
    assert len(lods) >= 3 and sizes == sorted(sizes) and sizes[-1] == 32 and sizes[0] < 32
    assert lods[-1][0] is lv
    base = B.build_tri_blas(tris, 8)
    nodes = B.node_array({"nodes": base["nodes"]})
    for leaves, _ in lods:
        _, sets, _, _ = O.cut_leaves(tris, nodes, base["leaf_range"], base["tri_perm"], list(leaves["leaf_ref"]),
                                     1e-4, leaves["info"]["extent"])
        assert np.array_equal(np.sort(np.concatenate(sets)), np.arange(len(tris)))
    rays = B.to_device_rays(W.chord_rays(4000, seed=8, radius=0.6))
    segs = []
    for leaves, _ in (lods[0], lods[-1]):
        ws = B.new_workspace(B.query_workspace_size(desc, 4000, 40))
        # one launch per segment slot: the count is the early-out's, free of
        # the persistent schedule's lookahead evaluations
        B.query_rays(desc, opt.table, opt.mlp, torch.as_tensor(leaves["nodes"]).cuda(), leaves["n_nodes"], rays, 40,
                     workspace=ws, options=B.query_options(schedule=B.SCHEDULE_WAVES))
        segs.append(B.query_stats(ws, 4000, 40)[0])
    assert B.device_status() == 0
    assert segs[0] < segs[1]
