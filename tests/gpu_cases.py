"""Shared set-up of the GPU parity tests: seeded scenes, models and the
comparison helpers. Inputs come from the workloads module only; expected
values come from the oracle only."""
from dataclasses import dataclass, replace

import numpy as np

from oracle import nbvh_oracle as O
from paper_2405_16237_b300 import nbvh as B
from paper_2405_16237_b300 import workloads as W


@dataclass
class Case:
    name: str
    tris: np.ndarray
    n_leaves: int
    model: W.ModelConfig
    table_prec: int
    rays: dict
    table_scale: float = 1e-4
    mlp_gain: float = 1.0
    seed: int = 0


def small_icosphere_model():
    # The 16-level, F=2, 2^20-entry, 16-sample, 3x64 model of the full-size
    # icosphere workload, on a smaller mesh.
    return replace(W.C1.model)


def make_case(name: str, table_scale: float = 1e-4, mlp_gain: float = 1.0) -> Case:
    if name == "random_tris_c0":
        return Case(name, W.scene_random_tris(4096, seed=W.SEED_BASE), 64, W.C0.model, B.FP32,
                    W.camera_rays(64, 64, seed=W.SEED_BASE + 7), table_scale, mlp_gain, 11)
    if name == "icosphere_l6":
        return Case(name, W.scene_icosphere(level=6), 256, small_icosphere_model(), B.FP16,
                    W.camera_rays(96, 96, seed=W.SEED_BASE + 8), table_scale, mlp_gain, 12)
    if name == "clusters_small":
        tris = W.scene_sphere_clusters(n_clusters=12, min_tris=200, max_tris=4000, seed=W.SEED_BASE + 5)
        return Case(name, tris, 512, W.C0.model, B.FP32, W.mixed_rays(3000, seed=W.SEED_BASE + 9),
                    table_scale, mlp_gain, 13)
    raise KeyError(name)


class Built:
    """Device copies of one case plus the oracle's own leaf build."""

    def __init__(self, case: Case, mlp_prec: int = B.FP32):
        import torch
        self.case = case
        self.leaves = B.build_leaves(case.tris, case.n_leaves, 1e-4)
        self.oleaves = O.build_leaves(case.tris, case.n_leaves, 1e-4)
        info = self.leaves["info"]
        self.desc = B.model_desc(case.model, case.table_prec, mlp_prec, info["centre"], info["extent"])
        self.layout = B.level_layout(self.desc)
        self.olayout = O.level_layout(case.model.n_levels, case.model.base_res, case.model.growth,
                                      case.model.log2_table)
        tab = W.init_table(self.layout["total"], case.model.n_features, case.seed, case.table_scale)
        tdt = {B.FP32: np.float32, B.FP16: np.float16, B.BF16: None}[case.table_prec]
        if case.table_prec == B.BF16:
            t = torch.as_tensor(tab).to(torch.bfloat16)
            self.table_host = t.float().numpy()
            self.table = t.cuda()
        else:
            self.table_host = tab.astype(tdt)
            self.table = torch.as_tensor(self.table_host).cuda()
        self.layers = W.init_mlp(case.model.mlp_dims(), case.seed + 1, gain=case.mlp_gain)
        self.mlp = torch.as_tensor(B.pack_mlp(self.layers)).cuda()
        self.nodes = torch.as_tensor(self.leaves["nodes"]).cuda()
        self.rays = B.to_device_rays(case.rays)

    def with_prec(self, mlp_prec: int):
        return B.with_mlp_prec(self.desc, mlp_prec)

    def oracle_query(self):
        return O.query(self.case.rays, self.oleaves, self.table_host, self.layers, self.olayout,
                       self.case.model.n_samples)


def segments_by_ray(seg, n_rays):
    off = seg["offsets"]
    return [(seg["leaf"][off[r]:off[r + 1]], seg["t0"][off[r]:off[r + 1]], seg["t1"][off[r]:off[r + 1]])
            for r in range(n_rays)]


def compare_segment_lists(count, leaf, t0, t1, n, seg):
    """GPU slot-major lists vs the oracle's CSR lists. Exact leaf sequence,
    except (a) grazing (ray, leaf) pairs, dropped on both sides, and (b)
    neighbours whose oracle t0 differ by <= 1e-6, which may swap. Returns
    (n_pairs_checked, n_excepted)."""
    graz = {(int(r), int(l)) for r, l in seg["grazing_pairs"]}
    ref = segments_by_ray(seg, n)
    checked = excepted = exact = 0
    for r in range(n):
        c = int(count[r])
        g_leaf = [int(leaf[s * n + r]) for s in range(c)]
        g_t = {int(leaf[s * n + r]): (float(t0[s * n + r]), float(t1[s * n + r])) for s in range(c)}
        o_leaf, o_t0, o_t1 = ref[r]
        o_map = {int(l): (a, b) for l, a, b in zip(o_leaf, o_t0, o_t1)}
        gl = [l for l in g_leaf if (r, l) not in graz]
        ol = [int(l) for l in o_leaf if (r, int(l)) not in graz]
        excepted += (len(g_leaf) - len(gl)) + (len(o_leaf) - len(ol))
        assert sorted(gl) == sorted(ol), f"ray {r}: leaf sets differ {gl} vs {ol}"
        keys = [o_map[l][0] for l in gl]
        for i in range(len(keys) - 1):
            if keys[i + 1] < keys[i]:
                assert keys[i] - keys[i + 1] <= 1e-6, f"ray {r}: order {gl}"
                excepted += 1
        for l in gl:
            a, b = o_map[l]
            ga, gb = g_t[l]
            assert abs(ga - a) <= 1e-6 * max(1.0, abs(a)) and abs(gb - b) <= 1e-6 * max(1.0, abs(b)), (r, l)
            exact += int(ga == a) + int(gb == b)
        checked += len(gl)
    # both sides round each slab value once to float32: endpoints agree bit for bit
    assert exact >= 2 * checked - max(2, checked // 1000), (exact, 2 * checked)
    return checked, excepted


def ambiguous_rays(res, n_rays, rel=1e-5):
    """Rays whose resolved result depends on rounding: a segment's hit logit
    within rel * RMS(logits) of 0, or two hit candidates within rel * |t|."""
    seg = res["segments"]
    raw = res["raw"]
    scale = float(np.sqrt(np.mean(raw[:, 0] ** 2))) if len(raw) else 1.0
    amb = np.zeros(n_rays, bool)
    near0 = np.abs(raw[:, 0]) <= rel * scale
    amb[seg["ray"][near0]] = True
    off = seg["offsets"]
    for r in range(n_rays):
        t = res["seg_t"][off[r]:off[r + 1]][res["seg_hit"][off[r]:off[r + 1]]]
        if len(t) > 1:
            ts = np.sort(t)
            if ts[1] - ts[0] <= rel * max(1.0, abs(ts[0])):
                amb[r] = True
    for r, _ in seg["grazing_pairs"]:
        amb[int(r)] = True
    return amb


# ---------------------------------------------------------------- hybrid hierarchy (S9)
def small_hybrid_scene(n_assets: int = 3, seed: int = W.SEED_BASE + 40):
    """A small version of the hybrid scene: a 40x40-cell ground (3,200
    triangles) and level-3 icosphere assets (1,280 triangles, 16 leaves) with
    hashed levels of 2^12..2^14 entries."""
    ground, assets = W.scene_hybrid(n_assets=n_assets, seed=seed, asset_level=3, ground_cells=40, n_leaves=16)
    rng = np.random.default_rng(seed + 1)
    for a in assets:
        a.model = replace(a.model, log2_table=int(rng.integers(12, 15)))
    return ground, assets


def hybrid_rays(n_side: int = 40, n_chords: int = 800, seed: int = W.SEED_BASE + 41):
    cam = W.hybrid_camera_rays(n_side, n_side)
    ch = W.chord_rays(n_chords, seed, centre=(0.0, -0.2, 0.0), radius=1.6)
    return {k: np.concatenate([cam[k], ch[k]]) for k in W.RAY_KEYS}


class HybridBuilt:
    """Device instances (triangle BLAS first, then the neural assets) and the
    oracle's description of the same instances."""

    def __init__(self, ground, assets, mlp_prec: int, table_prec: int = B.BF16, table_scale: float = 1.0,
                 gain: float = 2.0, max_segs: int = 16, train_steps: int = 0):
        """train_steps > 0: each asset's model is first trained on its own
        triangles with the library's FP16 training step (2^13 rays a step)."""
        import torch
        self.ground = ground
        self.blas = B.build_tri_blas(ground, 4)
        self.dev_blas = B.DeviceTriBlas(ground, self.blas)
        self.instances = [B.tri_instance(self.dev_blas)]
        self.oinstances = [{"kind": "triangles", "tris": ground}]
        self.keep = []
        for k, a in enumerate(assets):
            lv = B.build_leaves(a.tris, a.n_leaves, 1e-4)
            info = lv["info"]
            desc = B.model_desc(a.model, table_prec, mlp_prec, info["centre"], info["extent"])
            lay = B.level_layout(desc)
            tab = W.init_table(lay["total"], a.model.n_features, 500 + k, table_scale)
            t = torch.as_tensor(tab)
            t = t.to(torch.bfloat16) if table_prec == B.BF16 else (t.half() if table_prec == B.FP16 else t)
            table = t.cuda()
            layers = W.init_mlp(a.model.mlp_dims(), 600 + k, gain=gain)
            mlp = torch.as_tensor(B.pack_mlp(layers)).cuda()
            nodes = torch.as_tensor(lv["nodes"]).cuda()
            if train_steps > 0:
                d16 = B.model_desc(a.model, table_prec, B.FP16, info["centre"], info["extent"])
                scene = B.DeviceScene(a.tris, lv)
                opt = B.Optimizer(d16, table.float().clone(), mlp.clone(), loss_scale=32768.0)
                ws = B.new_workspace(B.train_workspace_size(d16, 1 << 13, scene.n_leaves))
                for step in range(1, train_steps + 1):
                    B.train_step(d16, opt, scene, B.TRAIN_PROBED_MIX, 1 << 13, 900 + k, step, 1e-2, ws)
                table = opt.table.clone()
                mlp = opt.mlp.clone()
                layers = unpack_mlp(mlp.cpu().numpy(), a.model.mlp_dims())
            table_host = table.float().cpu().numpy().astype(np.float64)
            self.keep += [table, mlp, nodes]
            self.instances.append(B.neural_instance(desc, table, mlp, nodes, lv["n_nodes"], max_segs))
            self.oinstances.append({"kind": "neural", "leaves": O.build_leaves(a.tris, a.n_leaves, 1e-4),
                                    "table": table_host, "layers": layers,
                                    "layout": O.level_layout(a.model.n_levels, a.model.base_res, a.model.growth,
                                                             a.model.log2_table),
                                    "n_samples": a.model.n_samples})


def hybrid_ambiguous(ref, n_rays, rel=1e-5):
    """Rays whose hybrid answer depends on rounding: the triangle answer's
    margin, an ambiguous neural answer, or two instances' hits within
    rel * |t| of each other."""
    amb = np.zeros(n_rays, bool)
    ts = []
    for ans in ref["answers"]:
        if "margin" in ans:
            amb |= ans["margin"] <= rel
        else:
            amb |= ambiguous_rays(ans["query"], n_rays, rel)
        ts.append(np.where(ans["hit"].astype(bool), ans["t"], np.inf))
    T = np.sort(np.stack(ts, 1), 1)
    if T.shape[1] > 1:
        with np.errstate(invalid="ignore"):
            close = np.isfinite(T[:, 1]) & (T[:, 1] - T[:, 0] <= rel * np.maximum(1.0, np.abs(T[:, 0])))
        amb |= close
    return amb


# ---------------------------------------------------------------- trained weights
def unpack_mlp(flat, dims):
    """The library's flat MLP parameters as [(W [out, in], b [out])]."""
    flat = np.asarray(flat, np.float32)
    layers, off = [], 0
    for i in range(len(dims) - 1):
        w = flat[off:off + dims[i + 1] * dims[i]].reshape(dims[i + 1], dims[i])
        off += dims[i + 1] * dims[i]
        bias = flat[off:off + dims[i + 1]]
        off += dims[i + 1]
        layers.append((w.copy(), bias.copy()))
    return layers


class Trained:
    """A case's model after `steps` of the library's own FP16 training step
    (probed-mix rays of its scene, 2^14 per step, lr 1e-2, dynamic loss
    scale). Trained networks put most logits far from zero, as a query meets
    them in use; the table stays in the case's storage precision."""

    def __init__(self, b: Built, steps: int = 300, batch: int = 1 << 14, seed: int = 7):
        import torch
        desc = b.with_prec(B.FP16)
        scene = B.DeviceScene(b.case.tris, b.leaves)
        opt = B.Optimizer(desc, b.table.float().clone(), b.mlp.clone(), loss_scale=32768.0)
        ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
        for step in range(1, steps + 1):
            B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, seed, step, 1e-2, ws)
        torch.cuda.synchronize()
        assert B.device_status() == 0
        self.b = b
        self.table = opt.table.clone()
        self.table_host = self.table.float().cpu().numpy().astype(np.float64)
        self.mlp = opt.mlp.clone()
        self.layers = unpack_mlp(self.mlp.cpu().numpy(), b.case.model.mlp_dims())

    def oracle_query(self, rays=None):
        b = self.b
        return O.query(b.case.rays if rays is None else rays, b.oleaves, self.table_host, self.layers, b.olayout,
                       b.case.model.n_samples)
