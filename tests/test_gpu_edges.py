"""Edge cases of the GPU path through the C ABI against the FP64 oracle: empty
and ragged ray sets under both evaluation schedules, degenerate intervals
(tmin > tmax, zero-length segments), a query capped at one segment slot, a
hybrid trace of triangles alone, and a one-ray training step."""
import numpy as np
import pytest

from gpu_cases import Built, ambiguous_rays, make_case, small_hybrid_scene
from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


_B = {}


def built():
    if "c0" not in _B:
        _torch()
        _B["c0"] = Built(make_case("random_tris_c0", 1.0, 2.0))
    return _B["c0"]


def _sub(rays, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in rays.items()}


def _np(h):
    return {k: v.cpu().numpy() for k, v in h.items()}


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
@pytest.mark.parametrize("schedule", [B.SCHEDULE_WAVES, B.SCHEDULE_PERSISTENT])
def test_empty_and_ragged_ray_sets(mp, schedule):
    """0, 1, 127, 129 and 1000 rays (tiles of 128 rows, partial and single):
    FP32 exact and FP16 within tolerance against the oracle; an empty set
    launches nothing and succeeds."""
    torch = _torch()
    b = built()
    desc = b.with_prec(mp)
    old = B.get_query_schedule()
    B.set_query_schedule(schedule, 0)
    try:
        empty = {k: v[:0] for k, v in B.to_device_rays(b.case.rays).items()}
        out = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], empty, 8)
        assert out["hit"].numel() == 0
        rng = np.random.default_rng(3)
        n_all = len(b.case.rays["ox"])
        for n in (1, 127, 129, 1000):
            idx = np.sort(rng.choice(n_all, n, replace=False))
            rays = _sub(b.case.rays, idx)
            res = O.query(rays, b.oleaves, b.table_host, b.layers, b.olayout, b.case.model.n_samples)
            h = _np(B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], B.to_device_rays(rays), 24))
            ok = ~ambiguous_rays(res, n)
            if mp == B.FP32:
                assert np.array_equal(h["hit"][ok].astype(bool), res["hit"][ok].astype(bool))
                hh = ok & res["hit"].astype(bool)
                assert np.all(np.abs(h["t"][hh] - res["t"][hh]) <= 1e-5 * np.abs(res["t"][hh]))
            else:
                assert np.mean(h["hit"][ok].astype(bool) == res["hit"][ok].astype(bool)) >= (0.99 if n > 100 else 0.0)
    finally:
        B.set_query_schedule(*old)
    assert B.device_status() == 0


def test_degenerate_intervals():
    """Rays whose [tmin, tmax] is empty (tmin > tmax) have no segment and miss;
    a ray whose interval is a single point inside a leaf box gives a
    zero-length segment that decodes to t = t0 (FP32 against the oracle)."""
    _torch()
    b = built()
    rays = _sub(b.case.rays, np.arange(400))
    rays["tmin"][:200] = 5.0
    rays["tmax"][:200] = 1.0
    # rays 200..399: a point interval at the middle of their first leaf segment, if any
    seg = O.ray_segments(rays, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    off = seg["offsets"]
    for r in range(200, 400):
        if off[r + 1] > off[r]:
            tm = np.float32(0.5 * (seg["t0"][off[r]] + seg["t1"][off[r]]))
            rays["tmin"][r] = tm
            rays["tmax"][r] = tm
    res = O.query(rays, b.oleaves, b.table_host, b.layers, b.olayout, b.case.model.n_samples)
    h = _np(B.query_rays(b.with_prec(B.FP32), b.table, b.mlp, b.nodes, b.leaves["n_nodes"],
                         B.to_device_rays(rays), 16))
    assert B.device_status() == 0
    assert not h["hit"][:200].any() and np.all(np.isinf(h["t"][:200])) and np.all(h["leaf"][:200] == -1)
    ok = ~ambiguous_rays(res, 400)
    assert np.array_equal(h["hit"][ok].astype(bool), res["hit"][ok].astype(bool))
    hh = ok & res["hit"].astype(bool)
    assert hh[200:].sum() > 5
    assert np.array_equal(h["t"][hh], rays["tmin"][hh])  # t = t0 = t1 exactly


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_one_segment_slot(mp):
    """max_segs = 1: every ray keeps only its first segment (the device status
    reports the overflow) and the result is the oracle's resolve over that
    segment alone."""
    _torch()
    b = built()
    rays = b.case.rays
    n = len(rays["ox"])
    res = O.query(rays, b.oleaves, b.table_host, b.layers, b.olayout, b.case.model.n_samples)
    seg = res["segments"]
    first = seg["offsets"][:-1][np.diff(seg["offsets"]) > 0]
    h = _np(B.query_rays(b.with_prec(mp), b.table, b.mlp, b.nodes, b.leaves["n_nodes"], B.to_device_rays(rays), 1))
    assert B.device_status() == 5  # NBVH_ERR_SEGMENT_OVERFLOW
    ref_hit = np.zeros(n, bool)
    ref_t = np.full(n, np.inf)
    ref_hit[seg["ray"][first]] = res["seg_hit"][first]
    ref_t[seg["ray"][first]] = np.where(res["seg_hit"][first], res["seg_t"][first], np.inf)
    amb = ambiguous_rays(res, n)
    if mp == B.FP32:
        assert np.array_equal(h["hit"][~amb].astype(bool), ref_hit[~amb])
        hh = ~amb & ref_hit
        assert np.all(np.abs(h["t"][hh] - ref_t[hh]) <= 1e-5 * np.abs(ref_t[hh]))
    else:
        assert np.mean(h["hit"].astype(bool) == ref_hit) >= 0.99
    assert h["hit"].sum() > 20


def test_hybrid_triangles_only_is_trace_triangles():
    """A hierarchy with one triangle instance answers exactly as
    nbvh_trace_triangles, instance 0 on hits and -1 on misses."""
    torch = _torch()
    ground, _ = small_hybrid_scene(1)
    blas = B.DeviceTriBlas(ground, B.build_tri_blas(ground, 4))
    rays = B.to_device_rays(W.hybrid_camera_rays(48, 48))
    h, inst = B.hybrid_trace([B.tri_instance(blas)], rays)
    t = B.trace_triangles(blas, rays)
    assert B.device_status() == 0
    for k in h:
        assert torch.equal(h[k], t[k]), k
    assert torch.equal(inst, torch.where(t["hit"] > 0, 0, -1).to(torch.int32))
    assert int(t["hit"].sum()) > 100


def test_one_ray_training_step():
    """A batch of one ray trains (or skips, when it meets no leaf) without
    error; the loss stays finite."""
    torch = _torch()
    b = built()
    scene = B.DeviceScene(b.case.tris, b.leaves)
    opt = B.Optimizer(b.with_prec(B.FP32), b.table.clone(), b.mlp.clone())
    ws = B.new_workspace(B.train_workspace_size(b.with_prec(B.FP32), 1, scene.n_leaves))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for step in range(1, 6):
        B.train_step(b.with_prec(B.FP32), opt, scene, B.TRAIN_PROBED_MIX, 1, 21, step, 1e-2, ws, loss_out=loss)
        assert np.isfinite(loss.item())
    assert B.device_status() == 0


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_inputs_beyond_the_kernels_report_unsupported(mp):
    """N * L * F = 1024 is a valid descriptor (<= NBVH_MAX_INPUTS) that neither
    MLP kernel stages (the first layer's weights or features exceed shared
    memory or TMEM): the query returns NBVH_ERR_UNSUPPORTED and the device
    status stays clean."""
    from dataclasses import replace
    torch = _torch()
    case = make_case("random_tris_c0", 1.0, 2.0)
    model = replace(case.model, n_samples=32, n_levels=16, n_features=2, log2_table=12, width=64)
    b = Built(replace(case, model=model))
    desc = b.with_prec(mp)
    B.device_status()  # clear the status word
    with pytest.raises(B.NBVHError) as err:
        B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, 64)
    assert err.value.code == 7  # NBVH_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert B.device_status() == 0
