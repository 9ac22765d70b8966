"""GPU parity of the training path (S7, S8) against the FP64 oracle through the
C ABI: training rays, labels, loss, analytic gradients (table and MLP), the
autograd.Function, Adam, a finite-difference check with FP64 reductions on the
GPU, and a learning test against brute-force ground truth."""
import math

import numpy as np
import pytest

from gpu_cases import Built, make_case
from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


_CACHE = {}


def built(scale=0.5, gain=2.0):
    key = (scale, gain)
    if key not in _CACHE:
        _torch()
        b = Built(make_case("random_tris_c0", scale, gain))
        b.scene = B.DeviceScene(b.case.tris, b.leaves)
        _CACHE[key] = b
    return _CACHE[key]


# ---------------------------------------------------------------- S7 rays
@pytest.mark.parametrize("mode", [B.TRAIN_PROBED_MIX, B.TRAIN_PAPER])
def test_train_rays_parity(mode):
    b = built()
    n, seed, step = 4096, (3 << 32) | 977, 5
    rays, leaf, t0, t1, nv = B.train_rays(mode, seed, step, b.scene, n)
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in rays.items()}
    gl = leaf.cpu().numpy()
    ref = O.train_rays(mode, seed, step, n, b.oleaves)
    go = np.stack([g["ox"], g["oy"], g["oz"]], 1)
    gd = np.stack([g["dx"], g["dy"], g["dz"]], 1)
    assert np.max(np.abs(gd - ref["d"])) <= 2e-6
    assert np.max(np.abs(go - ref["o"])) <= 5e-6
    assert int(nv.item()) == int((gl >= 0).sum())
    same = gl == ref["leaf"]
    assert same.mean() >= 0.998
    # the rest are near ties of the first leaf (t0 within 1e-5) or marginal clips
    for i in np.nonzero(~same)[0]:
        k, a0, _, _, _ = O.clip_ray_box(ref["o"][i], ref["d"][i], 0.0, ref["tmax"][i], b.oleaves["leaf_lo"],
                                        b.oleaves["leaf_hi"])
        if gl[i] >= 0 and ref["leaf"][i] >= 0:
            assert abs(a0[gl[i]] - ref["t0"][i]) <= 1e-5
    ok = same & (gl >= 0)
    assert np.max(np.abs(t0.cpu().numpy()[ok] - ref["t0"][ok])) <= 1e-5
    assert np.max(np.abs(t1.cpu().numpy()[ok] - ref["t1"][ok])) <= 1e-5


def _segments(b, n=3000, seed=41):
    """Input rays (workloads module) with the oracle's first-leaf segments."""
    rays = W.mixed_rays(n, seed=seed, radius=0.8)
    o, d, tmin, tmax = O.rays_od(rays)
    leaf, t0, t1 = O.first_leaf(o, d, tmin, tmax, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    return rays, o, d, leaf.astype(np.int32), t0.astype(np.float32), t1.astype(np.float32)


def _dev(torch, *arrs):
    return [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in arrs]


# ---------------------------------------------------------------- S7 labels
def test_labels_parity():
    torch = _torch()
    b = built()
    rays, o, d, leaf, t0, t1 = _segments(b)
    dl, dt0, dt1 = _dev(torch, leaf, t0, t1)
    lab = B.train_labels(B.to_device_rays(rays), dl, dt0, dt1, b.scene)
    got = {k: v.cpu().numpy() for k, v in lab.items()}
    ref = O.labels(o, d, leaf, t0.astype(np.float64), t1.astype(np.float64), b.case.tris, b.oleaves["tri_perm"],
                   b.oleaves["leaf_range"])
    ok = ref["margin"] > 1e-5
    assert ok.mean() > 0.97 and (ref["hit"][ok] == 1).sum() > 50
    assert np.array_equal(got["hit"][ok], ref["hit"][ok])
    h = ok & (ref["hit"] == 1)
    assert np.max(np.abs(got["depth"][h] - ref["depth"][h])) <= 1e-4
    gn = np.stack([got["nx"], got["ny"], got["nz"]], 1)
    assert np.max(np.abs(gn[h] - ref["normal"][h])) <= 1e-5
    assert np.all(got["hit"][leaf < 0] == 0)


# ---------------------------------------------------------------- S8 forward, loss, gradients
def _batch(b, n=2000, seed=43, hit_fraction=0.6):
    torch = _torch()
    rays, o, d, leaf, t0, t1 = _segments(b, n, seed)
    lab = W.random_labels(n, seed=seed + 1, hit_fraction=hit_fraction)
    valid = leaf >= 0
    dev = dict(rays=B.to_device_rays(rays), leaf=_dev(torch, leaf)[0], t0=_dev(torch, t0)[0],
               t1=_dev(torch, t1)[0], lab={k: _dev(torch, v)[0] for k, v in lab.items()},
               n_valid=torch.tensor([int(valid.sum())], dtype=torch.int32, device="cuda"))
    host = dict(o=o, d=d, leaf=leaf, t0=t0.astype(np.float64), t1=t1.astype(np.float64), valid=valid,
                yh=lab["hit"].astype(np.float64), yd=lab["depth"].astype(np.float64),
                yn=np.stack([lab["nx"], lab["ny"], lab["nz"]], 1).astype(np.float64))
    return dev, host


def _oracle_fb(b, h):
    fr = b.oleaves["frame"]
    return O.forward_backward(h["o"], h["d"], h["t0"], h["t1"], h["valid"], h["yh"], h["yd"], h["yn"],
                              b.table_host, b.layers, b.olayout, fr["model_centre"], fr["model_extent"],
                              b.case.model.n_samples)


def test_forward_loss_and_gradients_fp32():
    torch = _torch()
    b = built()
    dv, h = _batch(b)
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
    scale_j = np.sqrt(np.mean(ref_raw[v] ** 2, axis=0))
    assert np.max(np.abs(r - ref_raw[v]) / (np.abs(ref_raw[v]) + scale_j)) <= 1e-5
    assert abs(float(loss.item()) - L) <= 1e-5 * abs(L)
    gt = g_tab.cpu().numpy()
    assert np.max(np.abs(gt - ref_tab)) <= 1e-5 * np.max(np.abs(ref_tab))
    gm = g_mlp.cpu().numpy()
    ref_m = B.pack_mlp([(dw, db) for dw, db in ref_layers])
    assert np.max(np.abs(gm - ref_m)) <= 1e-5 * np.max(np.abs(ref_m))


def test_autograd_function_matches_oracle_adjoint():
    torch = _torch()
    from paper_2405_16237_b300.autograd import NBVHQueryFn
    b = built()
    dv, h = _batch(b, n=1200, seed=51)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(b.desc, n))
    table = b.table.clone().requires_grad_(True)
    mlp = b.mlp.clone().requires_grad_(True)
    raw = NBVHQueryFn.apply(table, mlp, b.desc, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws)
    R = torch.as_tensor(np.random.default_rng(52).normal(size=(n, 5)).astype(np.float32)).cuda()
    valid = torch.as_tensor(h["valid"]).cuda()
    (raw * R * valid[:, None]).sum().backward()
    fr = b.oleaves["frame"]
    p = O.sample_points(h["o"], h["d"], h["t0"], h["t1"], b.case.model.n_samples)
    x = O.normalize_points(p, fr["model_centre"], fr["model_extent"])
    feat = O.encode(x, b.table_host, b.olayout)
    _, acts, pre = O.mlp_forward(feat, b.layers)
    Rv = R.cpu().numpy().astype(np.float64) * h["valid"][:, None]
    g_feat, g_layers = O.mlp_backward(Rv, acts, pre, b.layers)
    g_tab = O.encode_backward(x, g_feat, b.table_host.shape[0], b.table_host.shape[1], b.olayout)
    assert np.max(np.abs(table.grad.cpu().numpy() - g_tab)) <= 1e-5 * np.max(np.abs(g_tab))
    ref_m = B.pack_mlp(g_layers)
    assert np.max(np.abs(mlp.grad.cpu().numpy() - ref_m)) <= 1e-5 * np.max(np.abs(ref_m))


def test_fd_gradient_check_fp64_reduction():
    """Central differences of the GPU loss (per-segment FP32 terms, FP64
    reduction) on a 256-ray batch against the GPU's analytic gradient."""
    torch = _torch()
    b = built()
    dv, h = _batch(b, n=256, seed=61)
    n = 256
    ws = B.new_workspace(B.train_workspace_size(b.desc, n))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def L_of(table, mlp):
        B.forward_train(b.desc, table, mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, labels=dv["lab"],
                        n_valid=dv["n_valid"])
        B.loss_fp64(b.desc, n, dv["n_valid"], ws, loss)  # the check's FP64 reduction
        return float(loss.item())

    L_of(b.table, b.mlp)
    g_tab = torch.zeros((b.layout["total"], 2), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(b.desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    gt = g_tab.cpu().numpy().ravel()
    gm = g_mlp.cpu().numpy()
    checked = 0
    for idx in np.argsort(-np.abs(gm))[:6]:
        hstep = 1e-3
        mp, mm = b.mlp.clone(), b.mlp.clone()
        mp[idx] += hstep
        mm[idx] -= hstep
        fd = (L_of(b.table, mp) - L_of(b.table, mm)) / (2 * hstep)
        assert abs(fd - gm[idx]) <= 3e-2 * abs(gm[idx]) + 1e-6, (idx, fd, gm[idx])
        checked += 1
    # Table: the largest-gradient entries one at a time (h = 1e-3; an entry
    # next to a ReLU or L1 kink can still be off, so the median is held to 1%
    # and every entry to 10%), then one unit-norm direction over every entry
    # the batch touches (a +-1 direction over thousands of entries would be a
    # large move that crosses kinks).
    rel = []
    for idx in np.argsort(-np.abs(gt))[:6]:
        hstep = 1e-3
        tp, tm = b.table.clone().view(-1), b.table.clone().view(-1)
        tp[idx] += hstep
        tm[idx] -= hstep
        fd = (L_of(tp.view_as(b.table), b.mlp) - L_of(tm.view_as(b.table), b.mlp)) / (2 * hstep)
        rel.append(abs(fd - gt[idx]) / abs(gt[idx]))
        checked += 1
    assert np.median(rel) <= 1e-2 and max(rel) <= 0.1, rel
    rng = np.random.default_rng(62)
    used = np.abs(gt) > 0
    delta = np.where(used, rng.choice([-1.0, 1.0], size=gt.shape), 0.0) / math.sqrt(used.sum())
    dv_ = torch.as_tensor(delta.astype(np.float32)).cuda().view_as(b.table)
    hstep = 2e-3
    fd = (L_of(b.table + hstep * dv_, b.mlp) - L_of(b.table - hstep * dv_, b.mlp)) / (2 * hstep)
    an = float(np.dot(gt.astype(np.float64), delta))
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)
    checked += 1
    assert checked == 13


# ---------------------------------------------------------------- Adam
def test_adam_step_matches_oracle_and_skips_nonfinite():
    torch = _torch()
    b = built()
    rng = np.random.default_rng(71)
    master = torch.as_tensor(b.table_host.astype(np.float32)).cuda()
    opt = B.Optimizer(b.desc, master.clone(), b.mlp.clone(), loss_scale=4.0)
    gt = rng.normal(size=opt.grad_table.shape).astype(np.float32)
    gm = rng.normal(size=opt.grad_mlp.shape).astype(np.float32)
    opt.grad_table.copy_(torch.as_tensor(gt))
    opt.grad_mlp.copy_(torch.as_tensor(gm))
    p0t, p0m = opt.table_master.cpu().numpy(), opt.mlp.cpu().numpy()
    opt.adam(1, lr=1e-2)
    ref_t, _, _ = O.adam(p0t, gt / 4.0, np.zeros_like(p0t), np.zeros_like(p0t), 1, lr=1e-2)
    ref_m, _, _ = O.adam(p0m, gm / 4.0, np.zeros_like(p0m), np.zeros_like(p0m), 1, lr=1e-2)
    assert np.max(np.abs(opt.table_master.cpu().numpy() - ref_t)) <= 1e-6
    assert np.max(np.abs(opt.mlp.cpu().numpy() - ref_m)) <= 1e-6
    assert float(opt.grad_table.abs().max()) == 0.0 and float(opt.grad_mlp.abs().max()) == 0.0
    # a non-finite gradient skips the step and halves a dynamic scale
    before = opt.mlp.clone()
    opt.grad_mlp[3] = float("inf")
    opt.adam(2, lr=1e-2, dynamic_scale=True)
    assert torch.equal(before, opt.mlp) and float(opt.loss_scale.item()) == 2.0
    assert int(opt.counters[2].item()) == 0


# ---------------------------------------------------------------- learning
def _gt_hits(tris, rays):
    """Closest hit of every ray against every triangle (oracle brute force)."""
    o, d, tmin, tmax = O.rays_od(rays)
    tv = tris.astype(np.float64)
    best = np.full(len(o), np.inf)
    for s in range(0, len(tv), 512):
        T = tv[s:s + 512]
        hit, t, _, _ = O.moller_trumbore(o[:, None], d[:, None], T[None, :, 0], T[None, :, 1], T[None, :, 2])
        t = np.where(hit & (t >= tmin[:, None]) & (t <= tmax[:, None]), t, np.inf)
        best = np.minimum(best, t.min(1))
    return best


def test_training_gains_over_untrained_and_box_proxy():
    """Train on the 4,096-triangle scene and compare hit agreement and depth
    error against brute-force ground truth: the trained network must beat the
    untrained one and the box-only proxy (hit = any leaf box hit, t = its t0)."""
    torch = _torch()
    b = Built(make_case("random_tris_c0"))
    scene = B.DeviceScene(b.case.tris, b.leaves)
    desc = b.desc
    opt = B.Optimizer(desc, b.table.clone(), b.mlp.clone())
    batch = 1 << 14
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    rays = W.camera_rays(64, 64, seed=W.SEED_BASE + 77)
    drays = B.to_device_rays(rays)
    gt = _gt_hits(b.case.tris, rays)
    gt_hit = np.isfinite(gt)

    def evaluate(table, mlp):
        h = B.query_rays(desc, table, mlp, b.nodes, b.leaves["n_nodes"], drays, 32)
        hit = h["hit"].cpu().numpy().astype(bool)
        t = h["t"].cpu().numpy()
        both = hit & gt_hit
        return np.mean(hit == gt_hit), (np.median(np.abs(t[both] - gt[both])) if both.any() else np.inf)

    untrained = evaluate(b.table, b.mlp)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(1, 401):
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, 1234, step, 1e-2, ws, loss_out=loss)
    assert B.device_status() == 0
    trained = evaluate(opt.table, opt.mlp)
    seg = O.ray_segments(rays, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    first = np.full(len(gt), np.inf)
    off = seg["offsets"]
    for r in range(len(gt)):
        if off[r + 1] > off[r]:
            first[r] = seg["t0"][off[r]]
    proxy_hit = np.isfinite(first)
    both = proxy_hit & gt_hit
    proxy = (np.mean(proxy_hit == gt_hit), np.median(np.abs(first[both] - gt[both])))
    assert np.isfinite(float(loss.item()))
    assert trained[0] > untrained[0] + 0.05 and trained[0] > proxy[0] + 0.02, (trained, untrained, proxy)
    assert trained[1] < proxy[1], (trained, proxy)


# ---------------------------------------------------------------- tensor-core training path
@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
def test_tensor_core_gradients_match_oracle(mp):
    """FP16/BF16 operands with FP32 accumulation and a static loss scale of
    1024: gradients (divided by the scale) against the oracle's exact ones.
    16-bit rounding of features, weights, activations and dZ bounds the
    agreement: relative L2 error <= 2e-2 for FP16; BF16's unit roundoff
    (2^-8) is 8x FP16's (2^-11), its bound is 1e-1; cosine >= 0.999 (FP16) /
    0.995 (BF16)."""
    torch = _torch()
    b = built()
    desc = b.with_prec(mp)
    dv, h = _batch(b, n=2000, seed=81)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(desc, n))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scale = 1024.0
    raw = B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws,
                          labels=dv["lab"], n_valid=dv["n_valid"], loss_scale=scale, loss_out=loss)
    g_tab = torch.zeros((b.layout["total"], 2), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    L, ref_tab, ref_layers, ref_raw = _oracle_fb(b, h)
    v = h["valid"]
    assert abs(float(loss.item()) - L) <= 2e-2 * abs(L)
    tol_rel, tol_cos = (2e-2, 0.999) if mp == B.FP16 else (1e-1, 0.995)
    for got, ref in ((g_tab.cpu().numpy().ravel() / scale, ref_tab.ravel()),
                     (g_mlp.cpu().numpy() / scale, B.pack_mlp(ref_layers).astype(np.float64))):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        cos = float(np.dot(got, ref) / (np.linalg.norm(got) * np.linalg.norm(ref)))
        assert rel <= tol_rel and cos >= tol_cos, (rel, cos)
    r = raw.cpu().numpy()[v]
    assert np.mean((r[:, 0] > 0) == (ref_raw[v][:, 0] > 0)) >= 0.99


def _half_round(prec):
    """Round-to-nearest-even to the 16-bit operand type (torch conversion)."""
    import torch
    dt = torch.float16 if prec == B.FP16 else torch.bfloat16
    return lambda a: torch.as_tensor(np.asarray(a, np.float64)).to(dt).double().numpy()


def _entry_err(got, ref):
    """Per-entry error |got - ref| / (|ref| + 1e-3 rms(ref)) over the entries
    either side touches."""
    nz = (np.abs(ref) > 0) | (np.abs(got) > 0)
    rms = np.sqrt(np.mean(ref[np.abs(ref) > 0] ** 2))
    return (np.abs(got - ref) / (np.abs(ref) + 1e-3 * rms))[nz]


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
@pytest.mark.parametrize("n_samples,n_features", [(8, 2), (16, 1), (12, 2), (8, 4)])
def test_tensor_core_backward_matches_half_precision_oracle(n_samples, n_features, mp):
    """The tensor-core forward and backward against the oracle run with the
    same half-precision operand rounding (features, weights, activations,
    dL/d(raw) times the loss scale, dZ), so that only FP32-versus-FP64
    accumulation separates them. Both forms of the table-gradient scatter:
    walking each ray through one level (N*F = 16 or 32 features per level:
    (8, 2), (16, 1)) and per sample ((12, 2): N*F = 24; (8, 4): four features).
    Accumulation differences are ~1e-6 relative, but now and then one moves an
    operand across a 16-bit rounding boundary or a pre-activation across zero,
    which changes that ray's whole contribution; such events touch few
    entries. Bounds: table gradient median per-entry error <= 1e-4 and 90th
    percentile <= 1e-3 (a wrong corner, weight or level moves whole levels or
    corner classes), relative L2 error <= 1e-2 for table and MLP, MLP median
    <= 1e-3."""
    from dataclasses import replace
    torch = _torch()
    base = make_case("random_tris_c0", 0.5, 2.0)
    model = replace(base.model, n_samples=n_samples, n_features=n_features)
    b = Built(replace(base, model=model))
    desc = b.with_prec(mp)
    dv, h = _batch(b, n=1500, seed=83)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(desc, n))
    scale = 1024.0
    B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws,
                    labels=dv["lab"], n_valid=dv["n_valid"], loss_scale=scale)
    g_tab = torch.zeros((b.layout["total"], n_features), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    fr = b.oleaves["frame"]
    _, ref_tab, ref_layers, _ = O.forward_backward(h["o"], h["d"], h["t0"], h["t1"], h["valid"], h["yh"], h["yd"],
                                                   h["yn"], b.table_host, b.layers, b.olayout, fr["model_centre"],
                                                   fr["model_extent"], n_samples, rnd=_half_round(mp), scale=scale)
    gt, rt = g_tab.cpu().numpy().ravel() / scale, ref_tab.ravel()
    gm, rm = g_mlp.cpu().numpy() / scale, B.pack_mlp(ref_layers).astype(np.float64)
    et, em = _entry_err(gt, rt), _entry_err(gm, rm)
    l2t = np.linalg.norm(gt - rt) / np.linalg.norm(rt)
    l2m = np.linalg.norm(gm - rm) / np.linalg.norm(rm)
    stats = (np.median(et), np.percentile(et, 90), l2t, np.median(em), l2m)
    assert np.median(et) <= 1e-4 and np.percentile(et, 90) <= 1e-3 and l2t <= 1e-2, stats
    assert np.median(em) <= 1e-3 and l2m <= 1e-2, stats


def test_tensor_core_training_learns():
    """The whole FP16 training step (dynamic loss scaling) on the 4,096-triangle
    scene: the trained FP16 network beats the untrained network."""
    torch = _torch()
    b = Built(make_case("random_tris_c0"))
    scene = B.DeviceScene(b.case.tris, b.leaves)
    desc = b.with_prec(B.FP16)
    opt = B.Optimizer(desc, b.table.clone(), b.mlp.clone(), loss_scale=32768.0)
    batch = 1 << 14
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    rays = W.camera_rays(64, 64, seed=W.SEED_BASE + 77)
    drays = B.to_device_rays(rays)
    gt = _gt_hits(b.case.tris, rays)
    gt_hit = np.isfinite(gt)

    def agreement():
        hh = B.query_rays(desc, opt.table, opt.mlp, b.nodes, b.leaves["n_nodes"], drays, 32)
        return np.mean(hh["hit"].cpu().numpy().astype(bool) == gt_hit)

    before = agreement()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(1, 401):
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, 99, step, 1e-2, ws, loss_out=loss)
    assert B.device_status() == 0
    after = agreement()
    assert np.isfinite(float(loss.item())) and after > before + 0.05, (before, after)


# ---------------------------------------------------------------- the benchmarked model (C1/C2)
def c1_built(scale=0.5, gain=2.0):
    """The model of the full-size icosphere workload and its training step
    (16 levels, F = 2, 2^20-entry hashed levels, 16 samples: N * F = 32,
    three 64-wide hidden layers) on a level-6 icosphere."""
    key = ("c1", scale, gain)
    if key not in _CACHE:
        _torch()
        b = Built(make_case("icosphere_l6", scale, gain))
        b.scene = B.DeviceScene(b.case.tris, b.leaves)
        _CACHE[key] = b
    return _CACHE[key]


def _decided_rays(b, h, mp, tau=1e-3):
    """Rays whose gradient no rounding-level difference can change by a
    discrete step: every hidden pre-activation of the oracle's reduced-
    precision model (16-bit operands, float32 positions and grid
    coordinates) lies more than tau
    times its layer's RMS from zero (a ReLU mask flip moves the ray's whole
    contribution) and the depth and normal L1 terms lie more than tau from
    their kinks."""
    fr = b.oleaves["frame"]
    x = O.sample_grid_f32(h["o"], h["d"], h["t0"], h["t1"], b.case.model.n_samples, fr["model_centre"],
                          fr["model_extent"])
    raw, _, pre = O.mlp_forward(O.encode(x, b.table_host, b.olayout, f32=True), b.layers, _half_round(mp))
    v = h["valid"].copy()
    for z in pre[:-1]:
        rms = np.sqrt(np.mean(z[v] ** 2))
        v &= np.min(np.abs(z), axis=1) > tau * rms
    v &= np.abs(O.sigmoid(raw[:, 1]) - h["yd"]) > tau
    v &= np.min(np.abs(raw[:, 2:5] - h["yn"]), axis=1) > tau
    return v


@pytest.mark.parametrize("mp", [B.FP32, B.FP16, B.BF16])
def test_benchmarked_model_forward_and_gradients_match_oracle(mp):
    """Forward, loss and gradients of the benchmarked training model through
    the kernels the training bench runs (FP16/BF16: the tensor-core forward
    at width 64, train_backward_tc<2, 64> with level-major scatter (N * F =
    32) and the tensor-core first-layer weight gradient; FP32: the CUDA-core
    forward and backward). FP32 against the exact oracle: raw outputs and the
    loss <= 1e-5 relative, gradients <= 1e-5 of the largest entry. FP16/BF16
    against the oracle run with the same 16-bit operand rounding, loss scale
    and float32 sample positions (sample_grid_f32), on the rays whose
    gradient is decided (_decided_rays: ~85 %; the others are dropped on both
    sides). A ReLU mask flipped by a rounding-level difference moves a whole
    ray's contribution: with every ray kept, a handful of flips among the
    288,000 hidden units changes the MLP gradients by 1-4 %. Bounds: table
    gradient median per-entry error <= 1e-4, 90th percentile <= 1e-3,
    relative L2 <= 1e-2 for table and MLP, MLP median <= 1e-3."""
    torch = _torch()
    b = c1_built()
    desc = b.with_prec(mp)
    dv, h = _batch(b, n=2500, seed=91)
    if mp != B.FP32:
        dv, h = _keep_decided(torch, b, dv, h, mp)
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(desc, n))
    scale = 1.0 if mp == B.FP32 else 1024.0
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    raw = B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, labels=dv["lab"],
                          n_valid=dv["n_valid"], loss_scale=scale, loss_out=loss)
    g_tab = torch.zeros((b.layout["total"], b.case.model.n_features), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    v = h["valid"]
    assert v.sum() > 500
    if mp == B.FP32:
        L, ref_tab, ref_layers, ref_raw = _oracle_fb(b, h)
        r = raw.cpu().numpy()[v]
        scale_j = np.sqrt(np.mean(ref_raw[v] ** 2, axis=0))
        assert np.max(np.abs(r - ref_raw[v]) / (np.abs(ref_raw[v]) + scale_j)) <= 1e-5
        assert abs(float(loss.item()) - L) <= 1e-5 * abs(L)
        gt = g_tab.cpu().numpy()
        assert np.max(np.abs(gt - ref_tab)) <= 1e-5 * np.max(np.abs(ref_tab))
        ref_m = B.pack_mlp([(dw, db) for dw, db in ref_layers])
        assert np.max(np.abs(g_mlp.cpu().numpy() - ref_m)) <= 1e-5 * np.max(np.abs(ref_m))
        return
    _check_half_grads(b, mp, h, g_tab, g_mlp, scale)


def _check_half_grads(b, mp, h, g_tab, g_mlp, scale):
    """Table and MLP gradients against the oracle run with the same 16-bit
    operand rounding, loss scale and float32 sample positions, on the rays
    h["valid"] keeps."""
    fr = b.oleaves["frame"]
    _, ref_tab, ref_layers, _ = O.forward_backward(h["o"], h["d"], h["t0"], h["t1"], h["valid"], h["yh"], h["yd"],
                                                   h["yn"], b.table_host, b.layers, b.olayout, fr["model_centre"],
                                                   fr["model_extent"], b.case.model.n_samples,
                                                   rnd=_half_round(mp), scale=scale, positions="f32")
    gt, rt = g_tab.cpu().numpy().ravel() / scale, ref_tab.ravel()
    gm, rm = g_mlp.cpu().numpy() / scale, B.pack_mlp(ref_layers).astype(np.float64)
    et, em = _entry_err(gt, rt), _entry_err(gm, rm)
    l2t = np.linalg.norm(gt - rt) / np.linalg.norm(rt)
    l2m = np.linalg.norm(gm - rm) / np.linalg.norm(rm)
    stats = (np.median(et), np.percentile(et, 90), l2t, np.median(em), l2m)
    assert np.median(et) <= 1e-4 and np.percentile(et, 90) <= 1e-3 and l2t <= 1e-2, stats
    assert np.median(em) <= 1e-3 and l2m <= 1e-2, stats


def _keep_decided(torch, b, dv, h, mp):
    keep = _decided_rays(b, h, mp)
    assert keep.sum() > 0.7 * h["valid"].sum()
    leaf = np.where(keep, h["leaf"], -1).astype(np.int32)
    return (dict(dv, leaf=torch.as_tensor(leaf).cuda(),
                 n_valid=torch.tensor([int(keep.sum())], dtype=torch.int32, device="cuda")),
            dict(h, leaf=leaf, valid=keep))


_WIDE = {}


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
@pytest.mark.parametrize("n_features", [4, 8])
def test_wide_first_layer_training_matches_half_precision_oracle(n_features, mp):
    """16 levels x 16 samples x F = 4 or 8 features (K = 1024 or 2048 inputs,
    the wide assets of the hybrid scene) at width 64: the tensor-core forward
    (first layer in K chunks) and backward (K = 2048: W0^T does not fit
    shared memory whole and is copied in 128-feature chunks from a global
    image; K = 1024: staged whole) against the oracle run with the same
    16-bit rounding, on the rays whose gradient is decided. Same bounds as
    the benchmarked-model test."""
    from dataclasses import replace
    torch = _torch()
    if n_features not in _WIDE:
        base = make_case("icosphere_l6", 0.5, 2.0)
        _WIDE[n_features] = Built(replace(base, model=replace(base.model, n_features=n_features, log2_table=15)))
    b = _WIDE[n_features]
    desc = b.with_prec(mp)
    dv, h = _batch(b, n=2500, seed=97)
    dv, h = _keep_decided(torch, b, dv, h, mp)
    assert h["valid"].sum() > 500
    n = len(h["leaf"])
    ws = B.new_workspace(B.train_workspace_size(desc, n))
    scale = 1024.0
    B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, labels=dv["lab"],
                    n_valid=dv["n_valid"], loss_scale=scale)
    g_tab = torch.zeros((b.layout["total"], n_features), dtype=torch.float32, device="cuda")
    g_mlp = torch.zeros_like(b.mlp)
    B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
    assert B.device_status() == 0
    _check_half_grads(b, mp, h, g_tab, g_mlp, scale)


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_recompute_mode_equals_stored_mode(mp):
    """A workspace a third of the stored size selects recompute mode (the
    activations of one chunk of rays at a time, rebuilt in the backward). Raw
    outputs and the loss are the same bits (every row is evaluated the same
    way wherever it sits); the gradients differ only by FP32 summation order
    (float atomics and split-K sums): relative L2 <= 1e-6 and every entry
    within 1e-6 of the largest."""
    torch = _torch()
    b = c1_built()
    desc = b.with_prec(mp)
    dv, h = _batch(b, n=3000, seed=93)
    n = len(h["leaf"])
    stored = B.train_workspace_size(desc, n)
    small, chunk = B.train_workspace_budget(desc, n, 0, stored // 3)
    assert chunk < n and small < stored

    def run(nbytes):
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if ws.data_ptr() % 256:
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        raw = B.forward_train(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws,
                              labels=dv["lab"], n_valid=dv["n_valid"], loss_scale=1024.0, loss_out=loss)
        g_tab = torch.zeros((b.layout["total"], b.case.model.n_features), dtype=torch.float32, device="cuda")
        g_mlp = torch.zeros_like(b.mlp)
        B.backward(desc, b.table, b.mlp, dv["rays"], dv["leaf"], dv["t0"], dv["t1"], ws, g_tab, g_mlp)
        assert B.workspace_bytes(ws) < stored or nbytes >= stored
        return raw, loss, g_tab, g_mlp

    ra, la, ta, ma = run(stored)
    rb, lb, tb, mb = run(small)
    assert B.device_status() == 0
    assert torch.equal(ra, rb) and torch.equal(la, lb)
    for x, y in ((ta, tb), (ma, mb)):
        x, y = x.double(), y.double()
        assert float((x - y).norm() / x.norm()) <= 1e-6
        assert float((x - y).abs().max()) <= 1e-6 * float(x.abs().max())


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
def test_pipelined_weight_gradients_equal_sum_of_pieces(mp):
    """The weight-gradient kernels with several chunks per CTA (37,925 rays:
    593 chunks of 64 for the 512-feature first layer on 148 CTAs, so every
    CTA cycles its three copy stages and the last chunk is ragged) against
    the same rays in pieces of 9,024 (one chunk per CTA). Gradients are
    linear in the rays and each piece is normalised by the whole batch's
    valid count, so the sums agree up to FP32 summation order: relative L2
    and every entry within 1e-5 of the largest. Raw outputs are the same
    bits (each row is evaluated the same way wherever it sits)."""
    torch = _torch()
    b = c1_built()
    desc = b.with_prec(mp)
    n = 4 * 148 * 64 + 37
    rays, leaf, t0, t1, n_valid = B.train_rays(B.TRAIN_PROBED_MIX, 2024, 1, b.scene, n)
    lab = B.train_labels(rays, leaf, t0, t1, b.scene)
    assert int(n_valid.item()) > n // 2

    def run(bounds):
        g_tab = torch.zeros((b.layout["total"], b.case.model.n_features), dtype=torch.float32, device="cuda")
        g_mlp = torch.zeros_like(b.mlp)
        raws = []
        for lo, hi in bounds:  # lo a multiple of 64: every slice stays 256-byte aligned
            r = {k: v[lo:hi] for k, v in rays.items()}
            lb = {k: v[lo:hi] for k, v in lab.items()}
            ws = B.new_workspace(B.train_workspace_size(desc, hi - lo))
            raws.append(B.forward_train(desc, b.table, b.mlp, r, leaf[lo:hi], t0[lo:hi], t1[lo:hi], ws, labels=lb,
                                        n_valid=n_valid, loss_scale=1024.0))
            B.backward(desc, b.table, b.mlp, r, leaf[lo:hi], t0[lo:hi], t1[lo:hi], ws, g_tab, g_mlp)
        return torch.cat(raws), g_tab, g_mlp

    piece = 141 * 64
    ra, ta, ma = run([(0, n)])
    rb, tb, mb = run([(lo, min(n, lo + piece)) for lo in range(0, n, piece)])
    assert B.device_status() == 0
    assert torch.equal(ra, rb)
    for x, y in ((ta, tb), (ma, mb)):
        x, y = x.double(), y.double()
        assert float(x.abs().max()) > 0
        assert float((x - y).norm() / x.norm()) <= 1e-5
        assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max())
