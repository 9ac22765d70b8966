"""GPU parity of the neural ray query path (S1..S5) against the FP64 oracle,
through the C ABI. FP32 path: <= 1e-5 relative on MLP outputs; FP16/BF16
tensor-core path: <= 2e-3 absolute depth, <= 1 degree mean normal error,
>= 99.9% hit agreement; segment lists exact (grazing pairs excepted)."""
import numpy as np
import pytest

from gpu_cases import Built, Trained, ambiguous_rays, compare_segment_lists, make_case
from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


_BUILT = {}


def built(name, scale=1e-4, gain=1.0):
    key = (name, scale, gain)
    if key not in _BUILT:
        _torch()
        _BUILT[key] = Built(make_case(name, scale, gain))
    return _BUILT[key]


def _oracle_segments(b):
    return O.ray_segments(b.case.rays, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])


# ---------------------------------------------------------------- S1
@pytest.mark.parametrize("name", ["random_tris_c0", "icosphere_l6", "clusters_small"])
def test_traverse_segment_lists_exact(name):
    b = built(name)
    seg = _oracle_segments(b)
    n = len(b.case.rays["ox"])
    max_segs = int(np.max(np.diff(seg["offsets"]))) + 2
    out = B.traverse(b.nodes, b.leaves["n_nodes"], b.rays, max_segs)
    assert B.device_status() == 0
    cnt = out["count"].cpu().numpy()
    checked, exc = compare_segment_lists(cnt, out["leaf"].cpu().numpy(), out["t0"].cpu().numpy(),
                                         out["t1"].cpu().numpy(), n, seg)
    assert checked > 0.99 * len(seg["ray"]) and exc <= 0.01 * max(1, len(seg["ray"]))


def test_traverse_edge_rays():
    """Zero direction components, origins inside boxes, finite [tmin, tmax],
    rays missing everything, an empty ray set."""
    torch = _torch()
    b = built("random_tris_c0")
    rng = np.random.default_rng(5)
    n = 1000
    o = rng.uniform(-0.6, 0.6, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d[0::3, 0] = 0.0
    d[1::5, 1] = 0.0
    d[2::7, :2] = 0.0
    d[3] = [0.0, 0.0, 0.0]
    tmin = rng.uniform(0.0, 0.3, n)
    tmax = tmin + rng.uniform(0.0, 1.0, n)
    tmax[::11] = np.inf
    rays = {"ox": o[:, 0], "oy": o[:, 1], "oz": o[:, 2], "dx": d[:, 0], "dy": d[:, 1], "dz": d[:, 2],
            "tmin": tmin, "tmax": tmax}
    rays = {k: np.asarray(v, np.float32) for k, v in rays.items()}
    seg = O.ray_segments(rays, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    dr = B.to_device_rays(rays)
    max_segs = int(np.max(np.diff(seg["offsets"]))) + 1
    out = B.traverse(b.nodes, b.leaves["n_nodes"], dr, max_segs)
    assert B.device_status() == 0
    compare_segment_lists(out["count"].cpu().numpy(), out["leaf"].cpu().numpy(), out["t0"].cpu().numpy(),
                          out["t1"].cpu().numpy(), n, seg)
    empty = {k: v[:0] for k, v in dr.items()}
    B.traverse(b.nodes, b.leaves["n_nodes"], empty, 4)
    torch.cuda.synchronize()


def test_traverse_overflow_status():
    b = built("icosphere_l6")
    seg = _oracle_segments(b)
    n = len(b.case.rays["ox"])
    counts = np.diff(seg["offsets"])
    assert counts.max() > 2
    out = B.traverse(b.nodes, b.leaves["n_nodes"], b.rays, 2)
    assert B.device_status() == 5  # NBVH_ERR_SEGMENT_OVERFLOW
    cnt = out["count"].cpu().numpy()
    assert np.array_equal(cnt, np.minimum(counts, 2))
    assert B.device_status() == 0  # cleared by the read


# ---------------------------------------------------------------- S2 + S3
@pytest.mark.parametrize("name,prec", [("random_tris_c0", B.FP32), ("icosphere_l6", B.FP16),
                                       ("icosphere_l6", B.BF16)])
def test_encode_parity(name, prec):
    torch = _torch()
    case = make_case(name, table_scale=1.0)
    case.table_prec = prec
    b = Built(case)
    seg = _oracle_segments(b)
    S = min(len(seg["ray"]), 3000)
    sr = torch.as_tensor(seg["ray"][:S].astype(np.int32)).cuda()
    t0 = seg["t0"][:S].astype(np.float32)
    t1 = seg["t1"][:S].astype(np.float32)
    feat = B.encode(b.desc, b.table, b.rays, sr, torch.as_tensor(t0).cuda(), torch.as_tensor(t1).cuda())
    got = feat.cpu().numpy()
    o, d, _, _ = O.rays_od(b.case.rays)
    rr = seg["ray"][:S]
    p = O.sample_points(o[rr], d[rr], t0.astype(np.float64), t1.astype(np.float64), case.model.n_samples)
    x = O.normalize_points(p, b.oleaves["frame"]["model_centre"], b.oleaves["frame"]["model_extent"])
    ref = O.encode(x, b.table_host, b.olayout)
    # Positions are carried in float-float, so what remains is FP32 rounding
    # of the weights and the 8-term sums on entries of magnitude <= 1.
    assert np.max(np.abs(got - ref)) <= 2e-6


# ---------------------------------------------------------------- S4 (FP32)
@pytest.mark.parametrize("name,scale", [("random_tris_c0", 1e-4), ("random_tris_c0", 1.0),
                                        ("icosphere_l6", 1.0)])
def test_eval_segments_fp32_parity(name, scale):
    torch = _torch()
    b = built(name, scale)
    seg = _oracle_segments(b)
    S = min(len(seg["ray"]), 4000)
    t0 = seg["t0"][:S].astype(np.float32)
    t1 = seg["t1"][:S].astype(np.float32)
    out = B.eval_segments(b.with_prec(B.FP32), b.table, b.mlp, b.rays,
                          torch.as_tensor(seg["ray"][:S].astype(np.int32)).cuda(), torch.as_tensor(t0).cuda(),
                          torch.as_tensor(t1).cuda())
    assert B.device_status() == 0
    got = out.cpu().numpy()
    o, d, _, _ = O.rays_od(b.case.rays)
    rr = seg["ray"][:S]
    _, ref = O.eval_segments(o[rr], d[rr], t0.astype(np.float64), t1.astype(np.float64), b.table_host,
                             b.layers, b.olayout, b.oleaves["frame"]["model_centre"], b.oleaves["frame"]["model_extent"],
                             b.case.model.n_samples)
    # <= 1e-5 relative, with each output's RMS over the batch as the floor
    scale_j = np.sqrt(np.mean(ref ** 2, axis=0))
    err = np.abs(got - ref) / (np.abs(ref) + scale_j)
    assert err.max() <= 1e-5, err.max()


# ---------------------------------------------------------------- S1..S5 (FP32)
@pytest.mark.parametrize("name,scale,gain", [("random_tris_c0", 1e-4, 1.0), ("random_tris_c0", 1.0, 1.0),
                                             ("icosphere_l6", 1.0, 2.0), ("clusters_small", 1.0, 1.0)])
def test_query_fp32_parity(name, scale, gain):
    b = built(name, scale, gain)
    res = b.oracle_query()
    n = len(b.case.rays["ox"])
    max_segs = int(np.max(np.diff(res["segments"]["offsets"]))) + 1
    h = B.query_rays(b.with_prec(B.FP32), b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, max_segs)
    assert B.device_status() == 0
    amb = ambiguous_rays(res, n)
    ok = ~amb
    assert ok.mean() > 0.97
    hit = h["hit"].cpu().numpy().astype(bool)
    assert np.array_equal(hit[ok], res["hit"][ok].astype(bool))
    assert np.array_equal(h["leaf"].cpu().numpy()[ok], res["leaf"][ok])
    hh = ok & hit
    t = h["t"].cpu().numpy()
    assert np.all(np.abs(t[hh] - res["t"][hh]) <= 1e-5 * np.abs(res["t"][hh]))
    nrm = np.stack([h["nx"].cpu().numpy(), h["ny"].cpu().numpy(), h["nz"].cpu().numpy()], 1)
    # The raw normal head is held to 1e-5 relative (RMS floor); normalising a
    # raw vector of length l divides that error by l: tol = 2e-5 (l + rms) / l.
    raw_n = winning_raw_normals(res, n)
    ln = np.linalg.norm(raw_n, axis=1)
    rms = float(np.sqrt(np.mean(np.sum(res["raw"][:, 2:5] ** 2, 1))))
    tol = 2e-5 * (ln + rms) / np.maximum(ln, 1e-30)
    assert np.all(np.max(np.abs(nrm[hh] - res["normal"][hh]), 1) <= tol[hh])
    assert np.all(np.isinf(t[~hit])) and np.all(h["leaf"].cpu().numpy()[~hit] == -1)
    assert hh.sum() > 0


def winning_raw_normals(res, n):
    """Raw normal-head output of each ray's winning segment (zeros for misses)."""
    out = np.zeros((n, 3))
    seg = res["segments"]
    off = seg["offsets"]
    for r in range(n):
        if not res["hit"][r]:
            continue
        for j in range(off[r], off[r + 1]):
            if res["seg_hit"][j] and res["seg_t"][j] == res["t"][r]:
                out[r] = res["raw"][j, 2:5]
                break
    return out


# ---------------------------------------------------------------- tensor-core path
# Unit roundoff of the operand formats: FP16 has an 11-bit significand, BF16 8.
UNIT_ROUNDOFF = {B.FP16: 2.0 ** -11, B.BF16: 2.0 ** -8}
# Hit agreement: >= 99.9 % for both formats. Random-init networks centre their
# logits on 0, where BF16's rounding flips ~0.15 % of segments, so the raw
# bound applies to trained networks (Trained: logits far from zero, as a
# query meets them in use); with random weights only the segments the format
# resolves (|oracle logit| > 4 u RMS(logit)) are held to it.
RAW_AGREEMENT = {B.FP16: 0.999, B.BF16: 0.999}


def hit_agreement(got_logit, ref_logit, mp):
    raw = np.mean((got_logit > 0) == (ref_logit > 0))
    rms = float(np.sqrt(np.mean(ref_logit ** 2)))
    res = np.abs(ref_logit) > 4 * UNIT_ROUNDOFF[mp] * rms
    resolved = np.mean((got_logit[res] > 0) == (ref_logit[res] > 0))
    return raw, resolved


def _angle_deg(a, b):
    c = np.clip(np.sum(a * b, 1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1)), -1.0, 1.0)
    return np.degrees(np.arccos(c))


_TRAINED = {}


def trained(name):
    if name not in _TRAINED:
        _TRAINED[name] = Trained(built(name, 1e-4, 1.0))
    return _TRAINED[name]


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
@pytest.mark.parametrize("name,scale,gain", [("random_tris_c0", 1.0, 2.0), ("icosphere_l6", 1.0, 2.0)])
def test_eval_segments_tensor_core_parity(name, scale, gain, mp):
    """Random weights with O(1) logits: >= 99.9 % hit agreement on the
    segments the format resolves, depth <= 2e-3, mean normal <= 1 degree."""
    torch = _torch()
    b = built(name, scale, gain)
    seg = _oracle_segments(b)
    t0 = seg["t0"].astype(np.float32)
    t1 = seg["t1"].astype(np.float32)
    out = B.eval_segments(b.with_prec(mp), b.table, b.mlp, b.rays, torch.as_tensor(seg["ray"].astype(np.int32)).cuda(),
                          torch.as_tensor(t0).cuda(), torch.as_tensor(t1).cuda())
    assert B.device_status() == 0
    got = out.cpu().numpy()
    o, d, _, _ = O.rays_od(b.case.rays)
    rr = seg["ray"]
    _, ref = O.eval_segments(o[rr], d[rr], t0.astype(np.float64), t1.astype(np.float64), b.table_host,
                             b.layers, b.olayout, b.oleaves["frame"]["model_centre"], b.oleaves["frame"]["model_extent"],
                             b.case.model.n_samples)
    raw_agree, resolved_agree = hit_agreement(got[:, 0], ref[:, 0], mp)
    assert resolved_agree >= 0.999, (raw_agree, resolved_agree)
    if mp == B.FP16:
        assert raw_agree >= 0.999, raw_agree
    dg = t0 + O.sigmoid(got[:, 1]) * (t1 - t0)
    dr = t0 + O.sigmoid(ref[:, 1]) * (t1 - t0)
    assert np.max(np.abs(dg - dr)) <= 2e-3
    assert np.mean(_angle_deg(got[:, 2:5], ref[:, 2:5])) <= 1.0


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
def test_query_tensor_core_parity(mp):
    """The whole query with a trained network (the library's own training,
    300 FP16 steps): >= 99.9 % hit agreement with the oracle over the
    non-grazing rays for FP16 and BF16, depth <= 2e-3 and mean normal error
    <= 1 degree where both pick the same leaf."""
    b = built("icosphere_l6", 1e-4, 1.0)
    tr = trained("icosphere_l6")
    res = tr.oracle_query()
    n = len(b.case.rays["ox"])
    max_segs = int(np.max(np.diff(res["segments"]["offsets"]))) + 1
    h = B.query_rays(b.with_prec(mp), tr.table, tr.mlp, b.nodes, b.leaves["n_nodes"], b.rays, max_segs)
    assert B.device_status() == 0
    graz = np.zeros(n, bool)
    graz[res["segments"]["grazing_pairs"][:, 0].astype(int)] = True
    hit = h["hit"].cpu().numpy().astype(bool)
    assert res["hit"].sum() > 500
    agree = np.mean(hit[~graz] == res["hit"][~graz].astype(bool))
    assert agree >= RAW_AGREEMENT[mp], agree
    both = hit & res["hit"].astype(bool) & ~graz & (h["leaf"].cpu().numpy() == res["leaf"])
    t = h["t"].cpu().numpy()
    assert np.max(np.abs(t[both] - res["t"][both])) <= 2e-3
    nrm = np.stack([h["nx"].cpu().numpy(), h["ny"].cpu().numpy(), h["nz"].cpu().numpy()], 1)
    assert np.mean(_angle_deg(nrm[both], res["normal"][both])) <= 1.0


def test_full_size_persistent_equals_waves():
    """The full-size primary query (1920 x 1080 rays on the level-8 displaced
    icosphere, 2,048 leaves, the 16-level model in FP16 with O(1) logits):
    the persistent queue, where ring wrap-around and back-pressure occur, gives
    the same records as one launch per segment slot, bit for bit."""
    torch = _torch()
    spec = W.C1
    tris = W.scene_icosphere(level=8)
    leaves = B.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
    info = leaves["info"]
    desc = B.model_desc(spec.model, B.FP16, B.FP16, info["centre"], info["extent"])
    lay = B.level_layout(desc)
    table = torch.as_tensor(W.init_table(lay["total"], spec.model.n_features, 3, 1.0)).cuda().half()
    mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(spec.model.mlp_dims(), 4, gain=2.0))).cuda()
    nodes = torch.as_tensor(leaves["nodes"]).cuda()
    rays = B.to_device_rays(W.camera_rays(1920, 1080))
    n = rays["ox"].numel()
    ws = B.new_workspace(B.query_workspace_size(desc, n, 48))
    hw = B.query_rays(desc, table, mlp, nodes, leaves["n_nodes"], rays, 48, workspace=ws,
                      options=B.query_options(schedule=B.SCHEDULE_WAVES))
    segs_w, waves = B.query_stats(ws, n, 48)
    for pipe in (B.PIPELINE_PHASES, B.PIPELINE_WARP_SPECIALISED):
        hp = B.query_rays(desc, table, mlp, nodes, leaves["n_nodes"], rays, 48, workspace=ws,
                          options=B.query_options(schedule=B.SCHEDULE_PERSISTENT, eval_pipeline=pipe))
        segs_p, launches = B.query_stats(ws, n, 48)
        assert B.device_status() == 0
        assert n == 2073600 and launches == 1 and waves > 3 and segs_w > n // 8
        # lookahead rows evaluate a ray's later segments before its earlier
        # ones resolve, so the persistent schedule may evaluate segments that
        # the waves skip, never fewer
        assert segs_p >= segs_w
        assert int(hw["hit"].sum()) > 100000
        for k in hw:
            assert torch.equal(hw[k], hp[k]), (pipe, k)


def test_query_workspace_too_small():
    b = built("random_tris_c0")
    torch = _torch()
    n = len(b.case.rays["ox"])
    need = B.query_workspace_size(b.desc, n, 8)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.NBVHError) as e:
        B.query_rays(b.desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, 8, workspace=ws)
    assert e.value.code == 4


def test_bounce_rays_parity():
    torch = _torch()
    rng = np.random.default_rng(31)
    n = 5000
    rays = W.mixed_rays(n, seed=32)
    lab = W.random_labels(n, seed=33, hit_fraction=0.7)
    t = rng.uniform(0.1, 3.0, n).astype(np.float32)
    nrm = np.stack([lab["nx"], lab["ny"], lab["nz"]], 1).astype(np.float32)
    hits = {"hit": torch.as_tensor(lab["hit"]).cuda(), "t": torch.as_tensor(t).cuda(),
            "nx": torch.as_tensor(nrm[:, 0].copy()).cuda(), "ny": torch.as_tensor(nrm[:, 1].copy()).cuda(),
            "nz": torch.as_tensor(nrm[:, 2].copy()).cuda(), "leaf": torch.zeros(n, dtype=torch.int32).cuda()}
    seed = (7 << 32) | 12345
    out = B.bounce_rays(B.to_device_rays(rays), hits, seed)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    h = lab["hit"].astype(bool)
    o, d, _, _ = O.rays_od(rays)
    p, dirs = O.bounce_rays(o[h], d[h], t[h].astype(np.float64), nrm[h].astype(np.float64), np.nonzero(h)[0], seed)
    gp = np.stack([got["ox"], got["oy"], got["oz"]], 1)[h]
    gd = np.stack([got["dx"], got["dy"], got["dz"]], 1)[h]
    assert np.max(np.abs(gp - p)) <= 2e-6 * max(1.0, float(np.abs(p).max()))
    assert np.max(np.abs(gd - dirs)) <= 2e-6
    assert np.all(got["tmin"][h] == 0) and np.all(np.isinf(got["tmax"][h]))
    assert np.all(got["tmax"][~h] == -1.0)


def test_kernel_class_timing():
    """While timing is on, each eager query records one traversal and one
    evaluation group (the persistent schedule: the queue set-up and the one
    evaluation launch) and each bounce one group, all with positive device
    time; a graph recording records nothing; with timing off nothing is
    recorded."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    desc = b.with_prec(B.FP16)
    n = b.rays["ox"].numel()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ws = B.new_workspace(B.query_workspace_size(desc, n, 16))
        out = B.new_hits(n)
        rays2 = B.new_rays(n)

        def step():
            B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, 16, out=out, workspace=ws)
            B.bounce_rays(b.rays, out, 5, out=rays2)

        B.get_kernel_times()
        B.set_timing(True)
        try:
            for _ in range(3):
                step()
            t = B.get_kernel_times()
            g = B.Graph.record(step)
            g.launch()
            s.synchronize()
            g.destroy()
            t_graph = B.get_kernel_times()
        finally:
            B.set_timing(False)
        step()
        t_off = B.get_kernel_times()
    assert B.device_status() == 0
    for k in ("traverse", "eval", "bounce"):
        assert t[k]["groups"] == 3 and t[k]["ms"] > 0.0, (k, t[k])
    assert t["traverse"]["launches"] == 3 and t["bounce"]["launches"] == 3
    assert t["eval"]["launches"] >= 6  # per query: queue set-up + the persistent evaluation (+ W1 image)
    assert all(v["groups"] == 0 for v in t_graph.values()) and all(v["groups"] == 0 for v in t_off.values())


def test_graph_replay_equals_eager_query():
    """A query step recorded as a CUDA graph (nbvh_graph_*) and replayed twice
    gives bit-identical results to the eager call."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    desc = b.with_prec(B.FP16)
    n = b.rays["ox"].numel()
    ms = 16
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ws_e = B.new_workspace(B.query_workspace_size(desc, n, ms))
        ws_g = B.new_workspace(B.query_workspace_size(desc, n, ms))
        out_e = B.new_hits(n)
        out_g = B.new_hits(n)
        rays2 = B.new_rays(n)
        out_e2 = B.new_hits(n)
        out_g2 = B.new_hits(n)

        def step(out, out2, ws):
            B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, ms, out=out, workspace=ws)
            B.bounce_rays(b.rays, out, 5, out=rays2)
            B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays2, ms, out=out2, workspace=ws)

        step(out_e, out_e2, ws_e)
        g = B.Graph.record(lambda: step(out_g, out_g2, ws_g))
        for _ in range(2):
            for v in list(out_g.values()) + list(out_g2.values()):
                v.fill_(7)
            g.launch()
        s.synchronize()
        g.destroy()
    assert B.device_status() == 0
    for a, c in ((out_e, out_g), (out_e2, out_g2)):
        for k in a:
            assert torch.equal(a[k], c[k]), k


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
@pytest.mark.parametrize("patience", [0, 4000, 1 << 30])
@pytest.mark.parametrize("pipeline,partial", [(B.PIPELINE_PHASES, 0), (B.PIPELINE_PHASES, 1),
                                              (B.PIPELINE_PHASES, 128), (B.PIPELINE_WARP_SPECIALISED, 0)])
def test_persistent_schedule_equals_waves(mp, patience, pipeline, partial):
    """The persistent queue (one launch, tiles claimed as resolves refill the
    queue; patience from eager partial tiles, which take lookahead rows, to
    waiting until drained), in the phase kernel and in the warp-specialised
    pipeline, gives bit-identical hit records to one launch per segment
    slot. Partial tiles claim at most `partial` items (0: the default)."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    rays = B.to_device_rays(W.mixed_rays(6000, seed=W.SEED_BASE + 31, radius=0.6))
    desc = b.with_prec(mp)
    hw = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays, 24,
                      options=B.query_options(schedule=B.SCHEDULE_WAVES))
    ws = B.new_workspace(B.query_workspace_size(desc, rays["ox"].numel(), 24))
    hp = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays, 24, workspace=ws,
                      options=B.query_options(schedule=B.SCHEDULE_PERSISTENT, patience_cycles=patience,
                                              eval_pipeline=pipeline, partial_items=partial))
    segs, launches = B.query_stats(ws, rays["ox"].numel(), 24)
    assert B.device_status() == 0
    for k in hw:
        assert torch.equal(hw[k], hp[k]), k
    assert launches == 1 and segs > rays["ox"].numel() // 4
    assert int(hw["hit"].sum()) > 100


@pytest.mark.parametrize("mp", [B.FP16, B.FP32])
def test_autotuner_times_candidates_and_keeps_results(mp):
    """nbvh_autotune_query: the schedules (and for FP16/BF16 the evaluation
    CTA shapes and first-layer placements, the partial-tile sizes, then
    traversal CTA sizes) are each
    timed; the fastest is returned, nothing is kept in the library, and every
    candidate's options give hit records equal to the default query's bit for
    bit (the options change only the order and shape of evaluation)."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    desc = b.with_prec(mp)
    rays = B.to_device_rays(W.mixed_rays(5000, seed=W.SEED_BASE + 32, radius=0.6))
    ref = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays, 24)
    best, cands = B.autotune_query(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays, 24, reps=2)
    assert B.device_status() == 0
    n_sched = 6 if mp != B.FP32 else 1
    assert {c["schedule"] for c in cands} == ({"waves", "persistent"} if mp != B.FP32 else {"waves"})
    if mp == B.FP32:
        assert len(cands) == n_sched + 2
    else:
        # stage 1 runs the automatic pipeline and shape; stage 2 the phase
        # kernel's CTA shapes and weight placements it did not already time
        # (and the warp-specialised pipeline if stage 1 did not run it)
        shapes = {(c["eval_pipeline"], c["eval_threads"], c["w1_mode"]) for c in cands}
        phase_shapes = {("phases", t, w) for t in (256, 512) for w in ("resident", "streamed")}
        assert len(phase_shapes - shapes) <= 1 and ("auto", 0, "auto") in shapes
        # stage 3 (partial-tile sizes 4, 8, 32, 128) starts from the fastest
        # persistent phase-kernel candidate
        partials = {c["partial_items"] for c in cands}
        stage3 = 4
        assert partials in ({0, 4, 8, 32, 128}, {4, 8, 32, 128}), partials
        assert n_sched + 3 + 2 + stage3 <= len(cands) <= n_sched + 5 + 2 + stage3
    assert all(c["ms"] > 0 for c in cands)
    assert best["ms"] == min(c["ms"] for c in cands)
    for c in cands:
        got = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], rays, 24,
                           options=B.options_from_dict(c))
        for k in ref:
            assert torch.equal(ref[k], got[k]), (c, k)
    assert B.device_status() == 0


def _surface_rays(tris, n, seed):
    """Rays starting on the mesh (a uniform point of a random triangle) in a
    uniform direction: their origins lie inside leaf boxes."""
    rng = np.random.default_rng(seed)
    t = tris[rng.integers(0, len(tris), n)].astype(np.float64)
    u, v = rng.uniform(size=(2, n))
    flip = u + v > 1
    u[flip], v[flip] = 1 - u[flip], 1 - v[flip]
    o = t[:, 0] + u[:, None] * (t[:, 1] - t[:, 0]) + v[:, None] * (t[:, 2] - t[:, 0])
    z = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - z * z)
    d = np.stack([s * np.cos(ph), s * np.sin(ph), z], 1)
    keys = ("ox", "oy", "oz", "dx", "dy", "dz")
    vals = (o[:, 0], o[:, 1], o[:, 2], d[:, 0], d[:, 1], d[:, 2])
    rays = {k: np.asarray(x, np.float32) for k, x in zip(keys, vals)}
    rays["tmin"] = np.full(n, 1e-4, np.float32)
    rays["tmax"] = np.full(n, np.inf, np.float32)
    return rays


@pytest.mark.parametrize("mp", [B.FP32, B.FP16])
def test_reverse_inside_query_matches_oracle(mp):
    """NBVH_FLAG_REVERSE_INSIDE on rays that start on the surface: segment
    lists with the reversed chords first (endpoints exact), FP32 results equal
    to the oracle's on unambiguous rays, FP16 hit agreement >= 99.9 % there."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    rays = _surface_rays(b.case.tris, 3000, 12)
    res = O.query(rays, b.oleaves, b.table_host, b.layers, b.olayout, b.case.model.n_samples, reverse_inside=True)
    seg = res["segments"]
    n = len(rays["ox"])
    rev = seg["t0"] > seg["t1"]
    assert rev.sum() > 1000
    desc = B.with_flags(b.with_prec(mp), B.FLAG_REVERSE_INSIDE)
    ms = int(np.max(np.diff(seg["offsets"]))) + 1
    dr = B.to_device_rays(rays)
    h = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], dr, ms)
    assert B.device_status() == 0
    h = {k: v.cpu().numpy() for k, v in h.items()}
    amb = ambiguous_rays(res, n)
    # a reversed chord's hit counts only inside (tmin, tmax]: decisions within
    # rounding of the window's ends are ambiguous too
    raw_hit = res["raw"][:, 0] > 0
    near_end = rev & raw_hit & ((np.abs(res["seg_t"] - rays["tmin"][seg["ray"]]) <= 1e-5 * np.maximum(
        1.0, np.abs(res["seg_t"]))) | (np.abs(res["seg_t"] - rays["tmax"][seg["ray"]]) <= 1e-5))
    amb[seg["ray"][near_end]] = True
    if mp == B.FP32:
        ok = ~amb
        assert ok.mean() > 0.95
        bad = np.flatnonzero(ok & (h["hit"].astype(bool) != res["hit"].astype(bool)))
        assert len(bad) == 0, [(int(r), float(h["t"][r]), float(res["t"][r]), float(rays["tmin"][r])) for r in bad[:5]]
        assert np.array_equal(h["leaf"][ok], res["leaf"][ok])
        hh = ok & res["hit"].astype(bool)
        assert hh.sum() > 100
        assert np.all(np.abs(h["t"][hh] - res["t"][hh]) <= 1e-5 * np.maximum(np.abs(res["t"][hh]), 1e-3))
    else:  # >= 99.9 % on the rays whose answer is not within rounding of a flip
        assert np.mean((h["hit"].astype(bool) == res["hit"].astype(bool))[~amb]) >= 0.999
    # the chords themselves: the traversal step of the query lists the same swapped segments
    plain = O.ray_segments(rays, b.oleaves["leaf_lo"], b.oleaves["leaf_hi"])
    assert not np.array_equal(plain["t0"], seg["t0"])
    # the flag off gives the plain query
    h0 = B.query_rays(b.with_prec(mp), b.table, b.mlp, b.nodes, b.leaves["n_nodes"], dr, ms)
    r0 = O.query(rays, b.oleaves, b.table_host, b.layers, b.olayout, b.case.model.n_samples)
    if mp == B.FP32:
        ok0 = ~ambiguous_rays(r0, n)
        assert np.array_equal(h0["hit"].cpu().numpy()[ok0].astype(bool), r0["hit"][ok0].astype(bool))


@pytest.mark.parametrize("table_prec", [B.FP16, B.BF16])
@pytest.mark.parametrize("n_levels", [6, 8, 12, 16])
def test_tensor_core_gather_paths_by_level_count(n_levels, table_prec):
    """Every form of the tensor-core gather against the oracle on the same
    segments: 16 levels (unrolled level loop), 8 and 12 (four-level chunks in
    a loop) and 6 (levels one by one), with FP16 and BF16 tables."""
    from dataclasses import replace
    torch = _torch()
    base = make_case("random_tris_c0", 1.0, 2.0)
    model = replace(base.model, n_levels=n_levels, growth=1.3)
    b = Built(replace(base, model=model, table_prec=table_prec))
    seg = _oracle_segments(b)
    t0 = seg["t0"].astype(np.float32)
    t1 = seg["t1"].astype(np.float32)
    out = B.eval_segments(b.with_prec(B.FP16), b.table, b.mlp, b.rays,
                          torch.as_tensor(seg["ray"].astype(np.int32)).cuda(), torch.as_tensor(t0).cuda(),
                          torch.as_tensor(t1).cuda())
    assert B.device_status() == 0
    got = out.cpu().numpy()
    o, d, _, _ = O.rays_od(b.case.rays)
    rr = seg["ray"]
    _, ref = O.eval_segments(o[rr], d[rr], t0.astype(np.float64), t1.astype(np.float64), b.table_host,
                             b.layers, b.olayout, b.oleaves["frame"]["model_centre"], b.oleaves["frame"]["model_extent"],
                             b.case.model.n_samples)
    raw_agree, resolved_agree = hit_agreement(got[:, 0], ref[:, 0], B.FP16)
    assert raw_agree >= RAW_AGREEMENT[B.FP16] and resolved_agree >= 0.999, (raw_agree, resolved_agree)
    dg = t0 + O.sigmoid(got[:, 1]) * (t1 - t0)
    dr = t0 + O.sigmoid(ref[:, 1]) * (t1 - t0)
    assert np.max(np.abs(dg - dr)) <= 2e-3
    assert np.mean(_angle_deg(got[:, 2:5], ref[:, 2:5])) <= 1.0


@pytest.mark.parametrize("mp", [B.FP16, B.BF16])
def test_query_independent_of_ray_order(mp):
    """A ray's result does not depend on where in a tile (or in which lane
    pair of the gather) it is evaluated: the query of a permuted ray set,
    mapped back, equals the query of the original order bit for bit."""
    torch = _torch()
    b = built("icosphere_l6", 1.0, 2.0)
    rays = b.case.rays
    n = len(rays["ox"])
    perm = np.random.default_rng(5).permutation(n)
    prays = {k: np.ascontiguousarray(v[perm]) for k, v in rays.items()}
    h = B.query_rays(b.with_prec(mp), b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, 24)
    hp = B.query_rays(b.with_prec(mp), b.table, b.mlp, b.nodes, b.leaves["n_nodes"], B.to_device_rays(prays), 24)
    assert B.device_status() == 0
    inv = torch.as_tensor(np.argsort(perm)).cuda()
    for k in h:
        assert torch.equal(h[k], hp[k][inv]), k
    assert int(h["hit"].sum()) > 1000
