"""GPU parity of the albedo head (Sec. 5.2 "Auxiliary intersection data": the
model also learns the surface albedo, with a relative L2 loss of weight 1 in
the combined loss) against the FP64 oracle, through the C ABI: albedo labels,
the loss and its gradients on both MLP paths, the query's albedo, the hybrid
record's albedo, and a learning test against brute-force ground truth."""
from dataclasses import replace

import numpy as np
import pytest

from gpu_cases import Built, HybridBuilt, ambiguous_rays, hybrid_ambiguous, hybrid_rays, make_case, \
    small_hybrid_scene
from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


_CACHE = {}


def built8(scale=0.5, gain=2.0):
    """The 4,096-triangle case with an 8-output MLP and per-triangle albedo."""
    key = (scale, gain)
    if key not in _CACHE:
        _torch()
        case = make_case("random_tris_c0", scale, gain)
        b = Built(replace(case, model=replace(case.model, n_out=8)))
        b.albedo = W.tri_albedo(b.case.tris)
        b.scene = B.DeviceScene(b.case.tris, b.leaves, albedo=b.albedo)
        _CACHE[key] = b
    return _CACHE[key]


def _dev(torch, *arrs):
    return [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in arrs]


def _alb(h):
    return np.stack([h["ar"], h["ag"], h["ab"]], 1)


def test_albedo_labels_parity():
    """Label albedo is the hit triangle's, bit for bit, wherever the hit
    decision is not within rounding; misses and untrained rays carry 0."""
    torch = _torch()
    b = built8()
    rays = W.mixed_rays(3000, seed=141, radius=0.8)
    o, d, tmin, tmax = O.rays_od(rays)
    leaf, t0, t1 = O.first_leaf(o, d, tmin, tmax, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    leaf, t0, t1 = leaf.astype(np.int32), t0.astype(np.float32), t1.astype(np.float32)
    dl, dt0, dt1 = _dev(torch, leaf, t0, t1)
    lab = B.train_labels(B.to_device_rays(rays), dl, dt0, dt1, b.scene)
    assert "ar" in lab
    got = {k: v.cpu().numpy() for k, v in lab.items()}
    ref = O.labels(o, d, leaf, t0.astype(np.float64), t1.astype(np.float64), b.case.tris, b.oleaves["tri_perm"],
                   b.oleaves["leaf_range"], b.albedo)
    ok = ref["margin"] > 1e-5
    h = ok & (ref["hit"] == 1)
    assert h.sum() > 50
    assert np.array_equal(got["hit"][ok], ref["hit"][ok])
    assert np.array_equal(_alb(got)[h], ref["albedo"][h].astype(np.float32))
    m = got["hit"] == 0
    assert np.all(_alb(got)[m] == 0.0)


def _batch8(b, n=2000, seed=143):
    torch = _torch()
    rays = W.mixed_rays(n, seed=seed, radius=0.8)
    o, d, tmin, tmax = O.rays_od(rays)
    leaf, t0, t1 = O.first_leaf(o, d, tmin, tmax, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    leaf, t0, t1 = leaf.astype(np.int32), t0.astype(np.float32), t1.astype(np.float32)
    lab = W.random_labels(n, seed=seed + 1, hit_fraction=0.6, albedo=True)
    valid = leaf >= 0
    dev = dict(rays=B.to_device_rays(rays), leaf=_dev(torch, leaf)[0], t0=_dev(torch, t0)[0],
               t1=_dev(torch, t1)[0], lab={k: _dev(torch, v)[0] for k, v in lab.items()},
               n_valid=torch.tensor([int(valid.sum())], dtype=torch.int32, device="cuda"))
    host = dict(o=o, d=d, leaf=leaf, t0=t0.astype(np.float64), t1=t1.astype(np.float64), valid=valid,
                yh=lab["hit"].astype(np.float64), yd=lab["depth"].astype(np.float64),
                yn=np.stack([lab["nx"], lab["ny"], lab["nz"]], 1).astype(np.float64),
                ya=np.stack([lab["ar"], lab["ag"], lab["ab"]], 1).astype(np.float64))
    return dev, host


def _oracle_fb(b, h, rnd=None, scale=1.0):
    fr = b.oleaves["frame"]
    return O.forward_backward(h["o"], h["d"], h["t0"], h["t1"], h["valid"], h["yh"], h["yd"], h["yn"],
                              b.table_host, b.layers, b.olayout, fr["model_centre"], fr["model_extent"],
                              b.case.model.n_samples, rnd=rnd, scale=scale, y_albedo=h["ya"])


def test_albedo_forward_loss_and_gradients_fp32():
    """FP32 MLP, eight outputs, albedo labels: raw outputs, loss (with the
    relative L2 term), table and MLP gradients within 1e-5 of the oracle; the
    albedo term is present (the loss differs from the five-term loss)."""
    torch = _torch()
    b = built8()
    dv, h = _batch8(b)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(b.desc, n))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    raw = B.forward_train(b.desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws,
                          labels=dv["lab"], n_valid=dv["n_valid"], loss_out=loss)
    g_tab = torch.zeros((b.layout["total"], b.case.model.n_features), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(b.desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    L, ref_tab, ref_layers, ref_raw = _oracle_fb(b, h)
    v = h["valid"]
    r = raw.cpu().numpy()[v]
    assert r.shape[1] == 8
    scale_j = np.sqrt(np.mean(ref_raw[v] ** 2, axis=0))
    assert np.max(np.abs(r - ref_raw[v]) / (np.abs(ref_raw[v]) + scale_j)) <= 1e-5
    assert abs(float(loss.item()) - L) <= 1e-5 * abs(L)
    L5, _ = O.loss(ref_raw, h["yh"], h["yd"], h["yn"], v)
    assert L - L5 > 1e-3 * L
    gt = g_tab.cpu().numpy()
    assert np.max(np.abs(gt - ref_tab)) <= 1e-5 * np.max(np.abs(ref_tab))
    gm = g_mlp.cpu().numpy()
    ref_m = B.pack_mlp([(dw, db) for dw, db in ref_layers])
    assert np.max(np.abs(gm - ref_m)) <= 1e-5 * np.max(np.abs(ref_m))
    # the albedo rows of the output layer get their gradient
    K = b.case.model.n_inputs
    Wd = b.case.model.width
    off = Wd * K + Wd + (b.case.model.n_hidden - 1) * (Wd * Wd + Wd)
    wo = gm[off:off + 8 * Wd].reshape(8, Wd)
    assert np.abs(wo[5:]).max() > 0


def _half_round(prec):
    import torch
    dt = torch.float16 if prec == B.FP16 else torch.bfloat16
    return lambda a: torch.as_tensor(np.asarray(a, np.float64)).to(dt).double().numpy()


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
def test_albedo_tensor_core_gradients_match_half_precision_oracle(mp):
    """Tensor-core forward and backward with the albedo head against the
    oracle run with the same 16-bit operand rounding: loss within 1e-4
    relative, table and MLP gradients within 1e-2 relative L2."""
    torch = _torch()
    b = built8()
    desc = b.with_prec(mp)
    dv, h = _batch8(b, n=1500, seed=147)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(desc, n))
    scale = 1024.0
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws,
                    labels=dv["lab"], n_valid=dv["n_valid"], loss_scale=scale, loss_out=loss)
    g_tab = torch.zeros((b.layout["total"], b.case.model.n_features), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    L, ref_tab, ref_layers, _ = _oracle_fb(b, h, rnd=_half_round(mp), scale=scale)
    assert abs(float(loss.item()) - L) <= 1e-4 * abs(L)
    gt, rt = g_tab.cpu().numpy().ravel() / scale, ref_tab.ravel()
    gm, rm = g_mlp.cpu().numpy() / scale, B.pack_mlp(ref_layers).astype(np.float64)
    l2t = np.linalg.norm(gt - rt) / np.linalg.norm(rt)
    l2m = np.linalg.norm(gm - rm) / np.linalg.norm(rm)
    assert l2t <= 1e-2 and l2m <= 1e-2, (l2t, l2m)


@pytest.mark.parametrize("schedule", [B.SCHEDULE_WAVES, B.SCHEDULE_PERSISTENT])
@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_albedo_query_parity(mp, schedule):
    """The query's albedo is sigmoid of the winning segment's outputs 5-7:
    FP32 within 1e-5 of the oracle on every unambiguous hit, FP16 within 2e-2
    where both sides pick the same leaf; misses read 0. Hit, t and leaf are
    those of the five-output query."""
    _torch()
    b = built8()
    desc = b.with_prec(mp)
    opt = B.query_options(schedule=schedule, patience_cycles=0)
    h = {k: v.cpu().numpy() for k, v in
         B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, 24, options=opt).items()}
    assert B.device_status() == 0 and "ar" in h
    res = b.oracle_query()
    n = len(h["hit"])
    hit = h["hit"].astype(bool)
    assert np.all(_alb(h)[~hit] == 0.0)
    if mp == B.FP32:
        ok = ~ambiguous_rays(res, n) & res["hit"].astype(bool)
        assert ok.sum() > 200
        assert np.array_equal(hit[ok], np.ones(ok.sum(), bool))
        assert np.max(np.abs(_alb(h)[ok] - res["albedo"][ok])) <= 1e-5
    else:
        same = hit & res["hit"].astype(bool) & (h["leaf"] == res["leaf"])
        assert same.sum() > 200
        assert np.max(np.abs(_alb(h)[same] - res["albedo"][same])) <= 2e-2
    a = _alb(h)[hit]
    assert np.all((a >= 0.0) & (a <= 1.0))


def test_hybrid_albedo_matches_oracle():
    """A triangle BLAS with albedo and FP32 neural instances with albedo
    heads: the record's albedo follows the answering instance (the
    triangle's, bit for bit, or the head's within 1e-5), then the same
    hierarchy without the triangle albedo reads 0 on triangle answers."""
    _torch()
    ground, assets = small_hybrid_scene(3)
    for a in assets:
        a.model = replace(a.model, n_out=8)
    hb = HybridBuilt(ground, assets, B.FP32, table_prec=B.FP32)
    alb = W.tri_albedo(ground, seed=W.SEED_BASE + 50)
    blas_a = B.DeviceTriBlas(ground, hb.blas, albedo=alb)
    inst = [B.tri_instance(blas_a)] + hb.instances[1:]
    oinst = [dict(hb.oinstances[0], albedo=alb)] + hb.oinstances[1:]
    rays = hybrid_rays(40, 800)
    h, ins = B.hybrid_trace(inst, B.to_device_rays(rays))
    assert B.device_status() == 0 and "ar" in h
    h = {k: v.cpu().numpy() for k, v in h.items()}
    ins = ins.cpu().numpy()
    ref = O.hybrid_trace(rays, oinst)
    n = len(rays["ox"])
    ok = ~hybrid_ambiguous(ref, n) & (ins == ref["inst"])
    tri = ok & (ref["inst"] == 0)
    neu = ok & (ref["inst"] > 0)
    assert tri.sum() > 100 and neu.sum() > 50
    assert np.array_equal(_alb(h)[tri], ref["albedo"][tri].astype(np.float32))
    assert np.max(np.abs(_alb(h)[neu] - ref["albedo"][neu])) <= 1e-5
    assert np.all(_alb(h)[ins < 0] == 0.0)
    h0, ins0 = B.hybrid_trace(hb.instances, B.to_device_rays(rays), out=B.new_hits(n, albedo=True))
    h0 = {k: v.cpu().numpy() for k, v in h0.items()}
    t0 = ins0.cpu().numpy() == 0
    assert t0.sum() > 100 and np.all(_alb(h0)[t0] == 0.0)


def test_albedo_training_learns():
    """Train an FP16 model with the albedo head (8 levels, 2^16 entries, 2x64
    MLP) on a 5,120-triangle sphere whose albedo is a smooth fBm texture: on
    rays that hit in both the query and brute force, the predicted albedo's
    mean error ends well below the untrained network's and below the best
    constant colour's."""
    torch = _torch()
    tris = W.scene_icosphere(level=4, radius=0.35)
    albedo = W.tri_albedo(tris)
    case = make_case("random_tris_c0")
    model = W.ModelConfig(n_levels=8, n_features=2, log2_table=16, base_res=16, growth=1.5, n_samples=8,
                          n_hidden=2, width=64, n_out=8)
    b = Built(replace(case, tris=tris, n_leaves=64, model=model))
    scene = B.DeviceScene(tris, b.leaves, albedo=albedo)
    desc = b.with_prec(B.FP16)
    opt = B.Optimizer(desc, b.table.clone(), b.mlp.clone(), loss_scale=32768.0)
    batch = 1 << 14
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    rays = W.camera_rays(48, 48, seed=W.SEED_BASE + 78)
    drays = B.to_device_rays(rays)
    o, d, tmin, tmax = O.rays_od(rays)
    gt = O.closest_triangle_hit(o, d, tmin, tmax, tris)
    gt_hit = gt["hit"].astype(bool)
    gt_alb = np.zeros((len(o), 3))
    gt_alb[gt_hit] = albedo[gt["index"][gt_hit]]

    def albedo_error():
        hh = B.query_rays(desc, opt.table, opt.mlp, b.nodes, b.leaves["n_nodes"], drays, 32)
        hit = hh["hit"].cpu().numpy().astype(bool)
        a = np.stack([hh[k].cpu().numpy() for k in ("ar", "ag", "ab")], 1)
        both = hit & gt_hit
        return float(np.mean(np.abs(a[both] - gt_alb[both]))), int(both.sum())

    before, _ = albedo_error()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(1, 1201):
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, 7, step, 1e-2, ws, loss_out=loss)
    assert B.device_status() == 0 and np.isfinite(float(loss.item()))
    after, n_both = albedo_error()
    const = float(np.mean(np.abs(gt_alb[gt_hit] - np.median(gt_alb[gt_hit], axis=0))))
    assert n_both > 300, n_both
    assert after < 0.6 * before and after < 0.6 * const, (before, after, const)
