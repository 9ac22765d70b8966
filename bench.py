#!/usr/bin/env python
"""Neural ray query benchmark on one or more B300s (one process per GPU).

Workload (the full-size configuration): a level-8 displaced icosphere
(1,310,720 triangles) split into 2,048 median-split leaf boxes; a 16-level
hash grid (F = 2, 2^20 entries per hashed level, FP16 entries), 16 samples per
segment, a 3x64 MLP; 1920x1080 pinhole primary rays plus one cosine-weighted
secondary bounce per predicted hit. One step = primary query -> bounce rays ->
secondary query, all in the library's kernels. The metric counts primary and
secondary rays per second.

Printed as one JSON line by rank 0. ``--impl reference`` times the FP64 CPU
oracle instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

# The CPU baseline (the FP64 oracle) runs single-threaded: pin numpy's BLAS
# before numpy loads. The GPU path does not use numpy arithmetic.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neural ray queries Mrays/s (fp16 TC vs fp32 plain, same GPU, same err); train rays/s"
SEED = 240516237


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-rays", type=int, default=24576, help="oracle sample size (primary rays)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--max-segs", type=int, default=48)
    p.add_argument("--train-steps", type=int, default=20, help="timed training steps (2^18 rays each)")
    p.add_argument("--hybrid-frames", type=int, default=5,
                   help="timed frames of the hybrid-scene workload (0: skip it)")
    p.add_argument("--hybrid-size", default="3840x2160")
    p.add_argument("--hybrid-cpu-rays", type=int, default=128, help="oracle sample of the hybrid workload")
    p.add_argument("--uneven-steps", type=int, default=5,
                   help="timed queries of the uneven-segment workload (0: skip it)")
    p.add_argument("--cut-steps", type=int, default=1700,
                   help="training-step budget of the error-driven-cut comparison (0: skip it)")
    p.add_argument("--lod-steps", type=int, default=1200,
                   help="training steps of the level-of-detail measurement (0: skip it)")
    p.add_argument("--no-albedo", action="store_true", help="skip the albedo-head measurement")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the library's default query schedule (no autotuning before the timed region)")
    p.add_argument("--primary", default="1920x1080",
                   help="primary image of the icosphere workload (smaller only for profiling captures)")
    p.add_argument("--quick", action="store_true",
                   help="time the FP16 tensor-core form only (no other forms, no e2e, no CPU baseline)")
    return p.parse_args()


# ---------------------------------------------------------------------------- distributed
def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def _reduce_device() -> str:
    """Where the process group reduces: the GPU under NCCL, the host under gloo."""
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def dist_max(x: float, world: int) -> float:
    """The largest value over the ranks (a time: the slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_max_rate(rate: float, world: int) -> float:
    """Whole-job rate of per-rank rates: world x the slowest rank's rate."""
    if world == 1:
        return rate
    import torch
    import torch.distributed as dist
    t = torch.tensor([-rate], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return world * float(-t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------- workload
def make_scene(primary="1920x1080"):
    from paper_2405_16237_b300 import workloads as W
    tris = W.scene_icosphere(level=8)
    w, h = (int(x) for x in primary.split("x"))
    return W.C1, tris, W.camera_rays(w, h)


class GpuWorkload:
    def __init__(self, spec, tris, rays_np, max_segs):
        import torch
        from paper_2405_16237_b300 import nbvh as B
        from paper_2405_16237_b300 import workloads as W
        self.B = B
        self.spec = spec
        self.max_segs = max_segs
        self.leaves = B.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
        info = self.leaves["info"]
        cfg = spec.model
        self.desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
        lay = B.level_layout(self.desc)
        self.table_np = W.init_table(lay["total"], cfg.n_features, SEED + 21, 1e-4).astype(np.float16)
        self.layers = W.init_mlp(cfg.mlp_dims(), SEED + 22)
        self.table = torch.as_tensor(self.table_np).cuda()
        self.mlp = torch.as_tensor(B.pack_mlp(self.layers)).cuda()
        self.nodes = torch.as_tensor(self.leaves["nodes"]).cuda()
        self.n = len(rays_np["ox"])
        self.rays_host = {k: torch.as_tensor(np.ascontiguousarray(rays_np[k])).pin_memory() for k in B.RAY_KEYS}
        self.rays = {k: v.cuda() for k, v in self.rays_host.items()}
        self.rays2 = B.new_rays(self.n)
        self.h1 = B.new_hits(self.n)
        self.h2 = B.new_hits(self.n)
        ws = B.query_workspace_size(self.desc, self.n, max_segs)
        self.ws1 = B.new_workspace(ws)
        self.ws2 = B.new_workspace(ws)
        self.h1_host = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in self.h1.items()}
        self.h2_host = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in self.h2.items()}
        # a buffer larger than L2 (126 MB), rewritten between timed steps
        self.flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        self.graphs = {}
        self.launches_per_step = {}
        self.options = None  # query options (None: the library's defaults), set from the autotuner

    def step(self, desc):
        B = self.B
        B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], self.rays, self.max_segs,
                     out=self.h1, workspace=self.ws1, options=self.options)
        B.bounce_rays(self.rays, self.h1, SEED + 3, out=self.rays2)
        B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], self.rays2, self.max_segs,
                     out=self.h2, workspace=self.ws2, options=self.options)

    def graph_step(self, desc):
        """The step replayed from a CUDA graph recorded on first use."""
        key = (desc.mlp_prec, desc.table_prec)
        if key not in self.graphs:
            n0 = self.B.launch_count()
            self.graphs[key] = self.B.Graph.record(lambda: self.step(desc))
            self.launches_per_step[key] = self.B.launch_count() - n0
        self.graphs[key].launch()

    def step_e2e(self, desc):
        for k in self.B.RAY_KEYS:
            self.rays[k].copy_(self.rays_host[k], non_blocking=True)
        self.graph_step(desc)
        for k in self.h1:
            self.h1_host[k].copy_(self.h1[k], non_blocking=True)
            self.h2_host[k].copy_(self.h2[k], non_blocking=True)

    def e2e_pipelined(self, desc, steps):
        """End to end with host buffers: every step copies its rays in from
        pinned host memory, runs the graph-captured step and reads both hit
        records back. Two device buffer sets and separate copy streams let step
        s+1's copy-in and step s-1's read-back run under step s's compute.
        Returns the device time of `steps` steps (events on the compute stream,
        which waits for the last read-back)."""
        import torch
        B = self.B
        if not hasattr(self, "_sets"):
            second = {"rays": {k: torch.empty_like(v) for k, v in self.rays.items()}, "rays2": B.new_rays(self.n),
                      "h1": B.new_hits(self.n), "h2": B.new_hits(self.n),
                      "ws1": B.new_workspace(self.ws1.numel()), "ws2": B.new_workspace(self.ws2.numel())}
            first = {"rays": self.rays, "rays2": self.rays2, "h1": self.h1, "h2": self.h2, "ws1": self.ws1,
                     "ws2": self.ws2}
            self._sets = [first, second]
            for st in self._sets:
                st["h1_host"] = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in st["h1"].items()}
                st["h2_host"] = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in st["h2"].items()}
                st["graph"] = None
            self._s_in = torch.cuda.Stream()
            self._s_out = torch.cuda.Stream()
        comp = torch.cuda.current_stream()
        for st in self._sets:
            if st["graph"] is None:
                def run(st=st):
                    B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], st["rays"],
                                 self.max_segs, out=st["h1"], workspace=st["ws1"], options=self.options)
                    B.bounce_rays(st["rays"], st["h1"], SEED + 3, out=st["rays2"])
                    B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], st["rays2"],
                                 self.max_segs, out=st["h2"], workspace=st["ws2"], options=self.options)
                st["graph"] = B.Graph.record(run)
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(comp)
        self._s_in.wait_event(start)
        self._s_out.wait_event(start)
        done_out = [None, None]
        done_comp = [None, None]
        for i in range(steps):
            st = self._sets[i % 2]
            with torch.cuda.stream(self._s_in):
                if done_comp[i % 2] is not None:
                    self._s_in.wait_event(done_comp[i % 2])  # rays of this set no longer read
                for k in B.RAY_KEYS:
                    st["rays"][k].copy_(self.rays_host[k], non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(self._s_in)
            comp.wait_event(ev_in)
            if done_out[i % 2] is not None:
                comp.wait_event(done_out[i % 2])  # hit records of this set already read back
            st["graph"].launch()
            ev_c = torch.cuda.Event()
            ev_c.record(comp)
            done_comp[i % 2] = ev_c
            with torch.cuda.stream(self._s_out):
                self._s_out.wait_event(ev_c)
                for k in st["h1"]:
                    st["h1_host"][k].copy_(st["h1"][k], non_blocking=True)
                    st["h2_host"][k].copy_(st["h2"][k], non_blocking=True)
                ev_o = torch.cuda.Event()
                ev_o.record(self._s_out)
            done_out[i % 2] = ev_o
        for ev in done_out:
            if ev is not None:
                comp.wait_event(ev)
        end.record(comp)
        end.synchronize()
        return start.elapsed_time(end)

    def rays_per_step(self):
        return self.n + int(self.h1["hit"].sum().item())

    def flush(self):
        self.flush_buf.fill_(1)


def time_training(spec, tris, wl, steps, warmup, batch=1 << 18, desc=None, mlp=None, scene=None):
    """Training steps (2^18 rays each) on the same scene and model, FP16
    tensor-core compute on FP32 masters, Adam lr 1e-2, dynamic loss scale.
    desc/mlp/scene replace the workload's model and the plain scene."""
    import torch
    from paper_2405_16237_b300 import nbvh as B
    scene = scene if scene is not None else B.DeviceScene(tris, wl.leaves)
    desc = B.with_mlp_prec(desc if desc is not None else wl.desc, B.FP16)
    opt = B.Optimizer(desc, torch.as_tensor(wl.table_np.astype(np.float32)).cuda(),
                      (mlp if mlp is not None else wl.mlp).clone(), loss_scale=32768.0)
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    step = 0
    for _ in range(warmup):
        step += 1
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, SEED + 9, step, 1e-2, ws, loss_out=loss)
    torch.cuda.synchronize()
    first = float(loss.item())
    total = 0.0
    for _ in range(steps):
        step += 1
        wl.flush()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, SEED + 9, step, 1e-2, ws, loss_out=loss)
        e.record()
        e.synchronize()
        total += s.elapsed_time(e)
    if B.device_status() != 0:
        raise RuntimeError("device status after training steps")
    ms = total / steps
    return {"value": batch / (ms * 1e-3), "unit": "rays/s", "batch": batch, "ms_per_step": ms, "steps": steps,
            "dtype": "f16 compute, f32 masters", "loss_after_warmup": first, "loss_last": float(loss.item()),
            "loss_scale": float(opt.loss_scale.item())}


def time_albedo(args, world, spec, tris, wl):
    """The icosphere step with the albedo head (8 outputs, FP16 tensor cores):
    both queries write albedo into their hit records; and training steps with
    per-triangle albedo labels (smooth fBm colours) and the relative L2 term."""
    import torch
    from dataclasses import replace
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    cfg = replace(spec.model, n_out=8)
    info = wl.leaves["info"]
    desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
    mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 22))).cuda()
    h1 = B.new_hits(wl.n, albedo=True)
    h2 = B.new_hits(wl.n, albedo=True)

    def step():
        B.query_rays(desc, wl.table, mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays, wl.max_segs, out=h1,
                     workspace=wl.ws1)
        B.bounce_rays(wl.rays, h1, SEED + 3, out=wl.rays2)
        B.query_rays(desc, wl.table, mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays2, wl.max_segs, out=h2,
                     workspace=wl.ws2)

    step()
    torch.cuda.synchronize()
    g = B.Graph.record(step)
    for _ in range(args.warmup):
        g.launch()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(args.steps):
        wl.flush()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        g.launch()
        e.record()
        e.synchronize()
        total += s.elapsed_time(e)
    if B.device_status() != 0:
        raise RuntimeError("device status after the albedo query")
    ms = dist_max(total, world) / args.steps
    rays = wl.n + int(h1["hit"].sum().item())
    a = torch.stack([h1["ar"], h1["ag"], h1["ab"]], 1)[h1["hit"] > 0]
    out = {"query": {"value": world * rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms,
                     "rays_per_step": rays, "albedo_mean_on_hits": a.float().mean(0).tolist()}}
    if args.train_steps > 0:
        scene = B.DeviceScene(tris, wl.leaves, albedo=W.tri_albedo(tris))
        tr = time_training(spec, tris, wl, args.train_steps, 3, desc=desc, mlp=mlp, scene=scene)
        tr["value"] = dist_max_rate(tr["value"], world)
        out["train"] = tr
    return out


def oracle_train_sample(spec, tris, n=256):
    """One FP64 oracle training step (rays, labels, loss, gradient, Adam) on n
    rays of the same scene and model. Returns rays/s and seconds."""
    import contextlib
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import workloads as W
    cfg = spec.model
    leaves = O.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
    lay = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
    tab = W.init_table(lay["total"], cfg.n_features, SEED + 21, 1e-4).astype(np.float64)
    layers = W.init_mlp(cfg.mlp_dims(), SEED + 22)
    fr = leaves["frame"]
    t0 = time.perf_counter()
    R = O.train_rays(O.TRAIN_MODE_PROBED_MIX, SEED + 9, 0, n, leaves)
    valid = R["leaf"] >= 0
    lab = O.labels(R["o"], R["d"], R["leaf"], R["t0"], R["t1"], tris, leaves["tri_perm"], leaves["leaf_range"])
    L, g_tab, g_layers, _ = O.forward_backward(R["o"], R["d"], R["t0"], R["t1"], valid, lab["hit"], lab["depth"],
                                               lab["normal"], tab, layers, lay, fr["model_centre"],
                                               fr["model_extent"], cfg.n_samples)
    O.adam(tab, g_tab, np.zeros_like(tab), np.zeros_like(tab), 1)
    for (w_, b_), (gw, gb) in zip(layers, g_layers):
        O.adam(w_, gw, np.zeros_like(gw), np.zeros_like(gw), 1)
        O.adam(b_, gb, np.zeros_like(gb), np.zeros_like(gb), 1)
    dt = time.perf_counter() - t0
    return n / dt, dt


def time_steps(wl, desc, steps, warmup, e2e=False, graph=True):
    import torch
    fn = wl.step_e2e if e2e else (wl.graph_step if graph else wl.step)
    for _ in range(warmup):
        fn(desc)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        wl.flush()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn(desc)
        e.record()
        e.synchronize()
        total += s.elapsed_time(e)
    torch.cuda.synchronize()
    return total


class ClockSampler:
    def __init__(self):
        self.path = os.path.join(tempfile.gettempdir(), f"nbvh_clocks_{os.getpid()}.csv")
        self.proc = None

    def start(self):
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            dev = os.environ.get("LOCAL_RANK", "0")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (bounded) for its first sample
        # so that the timed region that follows is sampled from its start
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources of the dominant kernel (eval_tc_kernel, its argument struct and device helpers)
KERNEL_SOURCES = ("eval_tc.cuh", "eval_plain.cuh", "nbvh_internal.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2405_16237_b300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        t = json.load(open(p))
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    return t


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ---------------------------------------------------------------------------- oracle sample
def oracle_sample(spec, tris, rays_np, n_sample):
    """Time the FP64 oracle on a seeded subset of the primary rays plus their
    bounce rays. Returns (Mrays/s, seconds, sample description, results)."""
    import contextlib
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # BLAS threads are pinned through the environment above
        def threadpool_limits(limits):
            return contextlib.nullcontext()
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import workloads as W
    rng = np.random.default_rng(SEED + 5)
    idx = np.sort(rng.choice(len(rays_np["ox"]), size=n_sample, replace=False))
    sub = W.subset(rays_np, idx)
    cfg = spec.model
    with threadpool_limits(limits=1):
        leaves = O.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
        lay = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
        tab = W.init_table(lay["total"], cfg.n_features, SEED + 21, 1e-4).astype(np.float16)
        layers = W.init_mlp(cfg.mlp_dims(), SEED + 22)
        t0 = time.perf_counter()
        res = O.query(sub, leaves, tab, layers, lay, cfg.n_samples)
        o, d, _, _ = O.rays_od(sub)
        hit = res["hit"].astype(bool)
        p, dirs = O.bounce_rays(o[hit], d[hit], res["t"][hit], res["normal"][hit], idx[hit], SEED + 3)
        n2 = int(hit.sum())
        sec = {"ox": p[:, 0], "oy": p[:, 1], "oz": p[:, 2], "dx": dirs[:, 0], "dy": dirs[:, 1], "dz": dirs[:, 2],
               "tmin": np.zeros(n2), "tmax": np.full(n2, np.inf)}
        sec = {k: np.asarray(v, np.float32) for k, v in sec.items()}
        res2 = O.query(sec, leaves, tab, layers, lay, cfg.n_samples)
        dt = time.perf_counter() - t0
    n_rays = n_sample + n2
    return n_rays / dt / 1e6, dt, n_rays, idx, res


def accuracy(wl, idx, res):
    """Hit agreement, depth and normal error of the GPU's primary hits against
    the oracle's on the sampled rays."""
    h = {k: v.cpu().numpy() for k, v in wl.h1.items()}
    g_hit = h["hit"][idx].astype(bool)
    o_hit = res["hit"].astype(bool)
    both = g_hit & o_hit & (h["leaf"][idx] == res["leaf"])
    out = {"rays": int(len(idx)), "hit_agreement": float(np.mean(g_hit == o_hit))}
    if both.any():
        out["depth_max_abs"] = float(np.max(np.abs(h["t"][idx][both] - res["t"][both])))
        gn = np.stack([h["nx"][idx], h["ny"][idx], h["nz"][idx]], 1)[both]
        c = np.clip(np.sum(gn * res["normal"][both], 1), -1, 1)
        out["normal_mean_deg"] = float(np.degrees(np.arccos(c)).mean())
    return out


# ---------------------------------------------------------------------------- uneven segments (S6)
def time_uneven(args, world):
    """64 displaced sphere clusters (1k-200k triangles each) in one 8,192-leaf
    N-BVH; 4,194,304 rays (60% from a camera, 40% sphere chords) with 1-40
    segments each; the icosphere model in FP16. The autotuner picks the
    schedule on this workload; each timed step is one graph-captured query."""
    import torch
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    spec = W.C3
    ex = spec.extra
    t0 = time.perf_counter()
    tris = W.scene_sphere_clusters(n_clusters=ex["n_clusters"], min_tris=ex["min_tris"], max_tris=ex["max_tris"])
    rays_np = W.mixed_rays(ex["n_rays"], seed=SEED + 40, camera_fraction=ex["camera_fraction"])
    leaves = B.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
    info = leaves["info"]
    cfg = spec.model
    desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
    lay = B.level_layout(desc)
    table = torch.as_tensor(W.init_table(lay["total"], cfg.n_features, SEED + 41, 1e-4)).cuda().half()
    mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 42))).cuda()
    nodes = torch.as_tensor(leaves["nodes"]).cuda()
    rays = B.to_device_rays(rays_np)
    n = rays["ox"].numel()
    # segments per ray (traversal only, untimed) with room to spare; the
    # query then gets exactly the slots the deepest ray needs
    tr = B.traverse(nodes, leaves["n_nodes"], rays, 160)
    cnt = tr["count"].cpu().numpy()
    del tr
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the uneven-segment traversal")
    ms_max = int(cnt.max())
    out = B.new_hits(n)
    ws = B.new_workspace(B.query_workspace_size(desc, n, ms_max))
    setup_s = time.perf_counter() - t0
    best, table_all = B.autotune_query(desc, table, mlp, nodes, leaves["n_nodes"], rays, ms_max, out=out,
                                       workspace=ws, reps=3)
    opts = B.options_from_dict(best)
    g = B.Graph.record(lambda: B.query_rays(desc, table, mlp, nodes, leaves["n_nodes"], rays, ms_max, out=out,
                                            workspace=ws, options=opts))
    launches = 0
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    total = 0.0
    for _ in range(args.uneven_steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.launch()
        e1.record()
        e1.synchronize()
        total += e0.elapsed_time(e1)
    g.destroy()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the uneven-segment queries")
    segs, _ = B.query_stats(ws, n, ms_max)
    ms = dist_max(total, world) / args.uneven_steps
    hit = cnt > 0
    return {"workload": spec.name, "value": world * n / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_query": ms,
            "rays": n, "triangles": int(len(tris)), "segments_per_ray": {
                "max": int(cnt.max()), "mean_of_rays_with_segments": float(cnt[hit].mean()),
                "rays_with_segments": int(hit.sum()), "p99": float(np.percentile(cnt[hit], 99))},
            "segments_evaluated": int(segs), "autotuner": {"best": best, "candidates": table_all},
            "setup_s": setup_s, "l2": "flushed (256 MB write) between timed queries"}


# ---------------------------------------------------------------------------- error-driven cut (NEXT-1)
def time_cut(args, world):
    """Error-driven cut optimization (Sec. 5.1) against the median-split N-BVH
    with the same leaf count (2,048) and the same training budget (steps of
    2^16 rays, the paper's ray distribution, FP16 tensor cores), on the
    displaced icosphere. Both models answer 512x512 camera rays; the triangle
    BLAS of the mesh gives the exact closest hits they are scored against."""
    import torch
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    spec = W.C1
    cfg = spec.model
    tris = W.scene_icosphere(level=8)
    batch, seed, lr, n_leaves = 1 << 16, SEED + 50, 1e-2, spec.n_leaves
    info = B.build_leaves(tris, 1)["info"]

    def fresh():
        desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
        lay = B.level_layout(desc)
        tab = torch.as_tensor(W.init_table(lay["total"], cfg.n_features, SEED + 51, 1e-4)).cuda()
        mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 52))).cuda()
        return desc, B.Optimizer(desc, tab, mlp, loss_scale=32768.0)

    # error-driven: grows from the root; its rounds and final round use the budget
    desc_e, opt_e = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lv_e, scene_e, hist, step_e = B.optimize_cut(tris, desc_e, opt_e, n_leaves, base_max_leaf=16, iters=10,
                                                 splits=16, factor=1.4, final_iters=1, batch=batch, seed=seed,
                                                 lr=lr, mode=B.TRAIN_PAPER)
    used = step_e - 1
    rest = max(0, args.cut_steps - used)
    ws_e = B.new_workspace(B.train_workspace_size(desc_e, batch, n_leaves))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    stats = {"hits": torch.zeros(n_leaves, dtype=torch.int32, device="cuda"),
             "trained": torch.zeros(n_leaves, dtype=torch.int32, device="cuda"),
             "loss": torch.zeros(n_leaves, dtype=torch.float32, device="cuda")}
    pdev = None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(rest):
        B.train_step_weighted(desc_e, opt_e, scene_e, B.TRAIN_PAPER, batch, seed, step_e, lr, ws_e, leaf_prob=pdev,
                              stats=stats, loss_out=loss)
        step_e += 1
        if i == 50:  # from here on, error-weighted selection from the measured statistics
            h, t, l = (stats[k].cpu().numpy() for k in ("hits", "trained", "loss"))
            pdev = torch.as_tensor(B.node_rank(h, t, l, batch * 51)[3].astype(np.float32)).cuda()
    e1.record()
    e1.synchronize()
    weighted_ms = e0.elapsed_time(e1) / max(1, rest)
    cut_s = time.perf_counter() - t0
    # median split: the same number of steps
    desc_m, opt_m = fresh()
    lv_m = B.build_leaves(tris, n_leaves, spec.inflate_rel)
    scene_m = B.DeviceScene(tris, lv_m)
    ws_m = B.new_workspace(B.train_workspace_size(desc_m, batch, n_leaves))
    for s in range(1, step_e):
        B.train_step(desc_m, opt_m, scene_m, B.TRAIN_PAPER, batch, seed, s, lr, ws_m, loss_out=loss)
    torch.cuda.synchronize()
    # score both on camera rays against the exact closest triangle hits
    rays_np = W.camera_rays(512, 512)
    rays = B.to_device_rays(rays_np)
    blas = B.build_tri_blas(tris, 4)
    gt = B.trace_triangles(B.DeviceTriBlas(tris, blas), rays)

    def score(desc, opt, lv):
        nodes = torch.as_tensor(lv["nodes"]).cuda()
        h = B.query_rays(desc, opt.table, opt.mlp, nodes, lv["n_nodes"], rays, 48)
        g_hit = gt["hit"].bool()
        m_hit = h["hit"].bool()
        both = g_hit & m_hit
        dt = (h["t"] - gt["t"]).abs()[both]
        cosang = (h["nx"] * gt["nx"] + h["ny"] * gt["ny"] + h["nz"] * gt["nz"])[both].clamp(-1, 1)
        return {"hit_agreement": float((g_hit == m_hit).float().mean()),
                "depth_mean_abs": float(dt.mean()) if both.any() else None,
                "depth_p95_abs": float(dt.quantile(0.95)) if both.any() else None,
                "normal_mean_deg": float(torch.rad2deg(torch.arccos(cosang)).mean()) if both.any() else None}

    out = {"workload": "icosphere-l8 2048 leaves, 2^16-ray steps, paper ray distribution, fp16",
           "steps": step_e - 1, "rays_per_step": batch,
           "error_driven": {"rounds": len(hist), "leaves": len(lv_e["leaf_ref"]), "construction_steps": used,
                            "wall_s": cut_s, "weighted_step_ms": weighted_ms,
                            "weighted_train_rays_s": batch / (weighted_ms * 1e-3) if rest else None,
                            **score(desc_e, opt_e, lv_e)},
           "median_split": score(desc_m, opt_m, lv_m),
           "scored_on": "512x512 camera rays vs the closest triangle hit (triangle BLAS of the mesh)"}
    if B.device_status() != 0:
        raise RuntimeError("device status after the cut comparison")
    return out


# ---------------------------------------------------------------------------- levels of detail (NEXT-3)
def time_lod(args, world):
    """Levels of detail (Sec. 5.3, Sec. 6.1): an error-driven construction on
    the icosphere registers LoDs every 100 training steps and trains a random
    one per step. Primary rays (1920x1080) are answered on the finest LoD;
    their bounce rays once on the finest and once on a coarse LoD (about 1/8
    of its leaves), each also with the reversed query of the leaf the ray
    starts in (NBVH_FLAG_REVERSE_INSIDE). Every bounce query is timed
    (graph-captured, L2 flushed) and scored against the closest triangle hits
    of the same bounce rays."""
    import torch
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    spec = W.C1
    cfg = spec.model
    tris = W.scene_icosphere(level=8)
    info = B.build_leaves(tris, 1)["info"]
    desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
    lay = B.level_layout(desc)
    opt = B.Optimizer(desc, torch.as_tensor(W.init_table(lay["total"], cfg.n_features, SEED + 61, 1e-4)).cuda(),
                      torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 62))).cuda(), loss_scale=32768.0)
    lods = []
    _, _, hist, step = B.optimize_cut(tris, desc, opt, spec.n_leaves, base_max_leaf=16, iters=10, splits=16,
                                      factor=1.4, final_iters=max(1, args.lod_steps - 1000), batch=1 << 16,
                                      seed=SEED + 63, lr=1e-2, mode=B.TRAIN_PAPER, lod_every=100, lods_out=lods)
    fine = lods[-1][0]
    target = max(1, len(fine["leaf_ref"]) // 8)
    coarse = min((x[0] for x in lods), key=lambda lv: abs(len(lv["leaf_ref"]) - target))
    rays = B.to_device_rays(W.camera_rays(1920, 1080))
    n = rays["ox"].numel()
    fine_nodes = torch.as_tensor(fine["nodes"]).cuda()
    h1 = B.query_rays(desc, opt.table, opt.mlp, fine_nodes, fine["n_nodes"], rays, 48)
    rays2 = B.bounce_rays(rays, h1, SEED + 64)
    blas = B.DeviceTriBlas(tris, B.build_tri_blas(tris, 4))
    gt = B.trace_triangles(blas, rays2)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = {"workload": "icosphere-l8, LoDs every 100 steps, 2^16-ray steps, fp16; 1920x1080 primary rays + bounce",
           "training_steps": step - 1, "lods": [len(x[0]["leaf_ref"]) for x in lods], "bounce_rays": int(h1["hit"].sum())}
    desc_rev = B.with_flags(desc, B.FLAG_REVERSE_INSIDE)
    for name, lv, dq in (("finest", fine, desc), ("coarse", coarse, desc), ("finest_reversed_inside", fine, desc_rev),
                         ("coarse_reversed_inside", coarse, desc_rev)):
        nodes = torch.as_tensor(lv["nodes"]).cuda()
        h2 = B.new_hits(n)
        ws = B.new_workspace(B.query_workspace_size(dq, n, 48))
        g = B.Graph.record(lambda: B.query_rays(dq, opt.table, opt.mlp, nodes, lv["n_nodes"], rays2, 48, out=h2,
                                                workspace=ws))
        for _ in range(3):
            g.launch()
        total = 0.0
        for _ in range(5):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.launch()
            e1.record()
            e1.synchronize()
            total += e0.elapsed_time(e1)
        g.destroy()
        segs, _ = B.query_stats(ws, n, 48)
        gh, mh = gt["hit"].bool(), h2["hit"].bool()
        live = rays2["tmax"] >= 0  # bounce rays spawned from a hit
        both = gh & mh
        dt = (h2["t"] - gt["t"]).abs()[both]
        out[name] = {"leaves": len(lv["leaf_ref"]), "ms": total / 5, "segments": int(segs),
                     "hit_agreement": float((gh == mh)[live].float().mean()),
                     "depth_mean_abs": float(dt.mean()) if both.any() else None}
    out["speedup_coarse_vs_finest"] = out["finest"]["ms"] / out["coarse"]["ms"]
    if B.device_status() != 0:
        raise RuntimeError("device status after the LoD measurement")
    return out


# ---------------------------------------------------------------------------- hybrid scene (S9)
HYBRID_BOUNCES = 4
HYBRID_MAX_SEGS = 16


class HybridWorkload:
    """16 neural assets (BF16 tables, BF16 tensor-core MLPs) on a 500,000-
    triangle classical ground, one frame = the primary pass plus 4 bounce
    passes of nbvh_hybrid_trace + nbvh_bounce_rays, recorded as one graph."""

    def __init__(self, width, height):
        import torch
        from paper_2405_16237_b300 import nbvh as B
        from paper_2405_16237_b300 import workloads as W
        self.B = B
        self.ground, self.assets = W.scene_hybrid()
        self.blas = B.build_tri_blas(self.ground, 4)
        self.dev_blas = B.DeviceTriBlas(self.ground, self.blas)
        self.instances = [B.tri_instance(self.dev_blas)]
        self.keep, self.models = [], []
        for k, a in enumerate(self.assets):
            lv = B.build_leaves(a.tris, a.n_leaves, 1e-4)
            info = lv["info"]
            desc = B.model_desc(a.model, B.BF16, B.BF16, info["centre"], info["extent"])
            lay = B.level_layout(desc)
            tab = torch.as_tensor(W.init_table(lay["total"], a.model.n_features, SEED + 100 + k, 1e-4)).cuda()
            table = tab.to(torch.bfloat16)
            layers = W.init_mlp(a.model.mlp_dims(), SEED + 200 + k)
            mlp = torch.as_tensor(B.pack_mlp(layers)).cuda()
            nodes = torch.as_tensor(lv["nodes"]).cuda()
            self.keep += [table, mlp, nodes]
            self.models.append((a, layers, table))
            self.instances.append(B.neural_instance(desc, table, mlp, nodes, lv["n_nodes"], HYBRID_MAX_SEGS))
        self.rays_np = W.hybrid_camera_rays(width, height)
        self.n = len(self.rays_np["ox"])
        self.rays = [B.to_device_rays(self.rays_np)] + [B.new_rays(self.n) for _ in range(HYBRID_BOUNCES)]
        self.hits = [B.new_hits(self.n) for _ in range(HYBRID_BOUNCES + 1)]
        self.inst = [torch.empty(self.n, dtype=torch.int32, device="cuda") for _ in range(HYBRID_BOUNCES + 1)]
        self.ws = B.new_workspace(B.hybrid_workspace_size(self.instances, self.n))
        self.flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        self.graph = None
        self.launches = 0

    def frame(self):
        B = self.B
        for b in range(HYBRID_BOUNCES + 1):
            B.hybrid_trace(self.instances, self.rays[b], out=self.hits[b], inst_out=self.inst[b], workspace=self.ws)
            if b < HYBRID_BOUNCES:
                B.bounce_rays(self.rays[b], self.hits[b], SEED + 30 + b, out=self.rays[b + 1])

    def graph_frame(self):
        if self.graph is None:
            n0 = self.B.launch_count()
            self.graph = self.B.Graph.record(self.frame)
            self.launches = self.B.launch_count() - n0
        self.graph.launch()

    def rays_per_frame(self):
        """Rays traced with a non-empty interval: every primary ray, and each
        bounce ray spawned from a hit."""
        return self.n + sum(int(self.hits[b]["hit"].sum().item()) for b in range(HYBRID_BOUNCES))


def time_hybrid(args, world):
    import torch
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import workloads as W
    w, h = (int(x) for x in args.hybrid_size.split("x"))
    t0 = time.perf_counter()
    hw = HybridWorkload(w, h)
    setup_s = time.perf_counter() - t0
    B = hw.B
    hw.frame()
    torch.cuda.synchronize()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the first hybrid frame")
    rays = hw.rays_per_frame()
    kinds = {"triangle": int((hw.inst[0] == 0).sum().item()), "neural": int((hw.inst[0] > 0).sum().item())}
    for _ in range(3):
        hw.graph_frame()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(args.hybrid_frames):
        hw.flush_buf.fill_(1)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        hw.graph_frame()
        e.record()
        e.synchronize()
        total += s.elapsed_time(e)
    if B.device_status() != 0:
        raise RuntimeError("device status after hybrid frames")
    ms = dist_max(total, world) / args.hybrid_frames
    out = {"workload": f"hybrid-16-neural-assets+500000-tri-ground_{w}x{h}_primary+{HYBRID_BOUNCES}-bounces",
           "value": world * rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_frame": ms,
           "rays_per_frame": rays, "primary_hits": kinds, "frames": args.hybrid_frames,
           "gpu_launches_per_frame": hw.launches, "dtype": "bf16 tables + bf16 tensor-core MLPs, fp32 triangles",
           "setup_s": setup_s, "l2": "flushed (256 MB write) between timed frames"}
    if args.hybrid_cpu_rays > 0 and not args.no_cpu_baseline:
        rng = np.random.default_rng(SEED + 6)
        idx = np.sort(rng.choice(hw.n, size=args.hybrid_cpu_rays, replace=False))
        sub = W.subset(hw.rays_np, idx)
        oinst = [{"kind": "triangles", "tris": hw.ground}]
        for a, layers, table in hw.models:
            oinst.append({"kind": "neural", "leaves": O.build_leaves(a.tris, a.n_leaves, 1e-4),
                          "table": table.float().cpu().numpy().astype(np.float64), "layers": layers,
                          "layout": O.level_layout(a.model.n_levels, a.model.base_res, a.model.growth,
                                                   a.model.log2_table), "n_samples": a.model.n_samples})
        t1 = time.perf_counter()
        ref = O.hybrid_trace(sub, oinst)
        dt = time.perf_counter() - t1
        g_inst = hw.inst[0].cpu().numpy()[idx]
        g = {k: v.cpu().numpy()[idx] for k, v in hw.hits[0].items()}
        same = (g_inst == ref["inst"]) & (g["leaf"] == ref["leaf"]) & ref["hit"].astype(bool)
        acc = {"rays": int(len(idx)), "instance_agreement": float(np.mean(g_inst == ref["inst"]))}
        if same.any():
            acc["depth_max_abs"] = float(np.max(np.abs(g["t"][same] - ref["t"][same])))
            gn = np.stack([g["nx"], g["ny"], g["nz"]], 1)[same]
            c = np.clip(np.sum(gn * ref["normal"][same], 1), -1, 1)
            acc["normal_mean_deg"] = float(np.degrees(np.arccos(c)).mean())
        out["accuracy_vs_oracle"] = acc
        out["cpu_baseline"] = {"value": len(idx) / dt / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                               "sample": f"{len(idx)} seeded primary rays of the {w}x{h} image, primary pass only, "
                                         f"{dt:.1f} s"}
    return out


# ---------------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_init(args.gpus)
    spec, tris, rays_np = make_scene(args.primary)

    if args.impl == "reference":
        if rank != 0:
            return
        rates, secs = [], []
        n = min(args.cpu_rays, 4096)
        for s in range(args.warmup + args.steps):
            v, dt, nr, _, _ = oracle_sample(spec, tris, rays_np, n)
            if s >= args.warmup:
                rates.append(v)
                secs.append(dt)
        val = float(np.mean(rates))
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mrays/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs) * 1e3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": spec.name, "sample_primary_rays": n},
                "cpu_baseline": {"value": val, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{n} seeded primary rays of the 1920x1080 image + their bounce rays"},
                "e2e": {"value": val, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_2405_16237_b300 import nbvh as B
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()  # a created stream: CUDA graphs cannot record the legacy default stream
    with torch.cuda.stream(stream):
        run_gpu(args, world, rank, spec, tris, rays_np)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_gpu(args, world, rank, spec, tris, rays_np):
    import torch
    from paper_2405_16237_b300 import nbvh as B
    wl = GpuWorkload(spec, tris, rays_np, args.max_segs)
    d16 = B.with_mlp_prec(wl.desc, B.FP16)
    d32 = B.with_mlp_prec(wl.desc, B.FP32)
    dbf = B.with_mlp_prec(wl.desc, B.BF16)

    # autotuner (untimed): pick the query schedule on this workload's primary rays
    if args.no_autotune:
        tune_best, tune_all = dict(B.options_dict(B.query_options()), ms=None), []
    else:
        tune_best, tune_all = B.autotune_query(d16, wl.table, wl.mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays,
                                               args.max_segs, out=wl.h1, workspace=wl.ws1, reps=3)
    wl.options = B.options_from_dict(tune_best)

    # untimed reference step: statistics of the work one step does
    wl.step(d16)
    torch.cuda.synchronize()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the first step")
    rays_step = wl.rays_per_step()
    seg1, waves1 = B.query_stats(wl.ws1, wl.n, args.max_segs)
    seg2, waves2 = B.query_stats(wl.ws2, wl.n, args.max_segs)

    # per-stage kernel times (CUDA events the library records on this stream
    # around traversal and evaluation waves) from eager steps
    B.set_timing(True)
    B.get_timing()
    time_steps(wl, d16, args.steps, args.warmup, graph=False)
    tr_ms, ev_ms, calls = B.get_timing()
    B.set_timing(False)
    eval_ms_step = ev_ms / (args.steps + args.warmup)
    tr_ms_step = tr_ms / (args.steps + args.warmup)

    # main measurement: FP16 tensor-core form, each step one CUDA-graph launch
    barrier(world)
    clocks = ClockSampler()
    clocks.start()
    total_ms = time_steps(wl, d16, args.steps, args.warmup)
    total_ms = dist_max(total_ms, world)
    ms_step = total_ms / args.steps
    value = world * rays_step / (ms_step * 1e-3) / 1e6
    launches_per_step = wl.launches_per_step[(d16.mlp_prec, d16.table_prec)]

    if args.quick:
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "Mrays/s", "ms_per_step": ms_step,
                              "quick": True, "segments_per_step": seg1 + seg2, "eval_ms_per_step": eval_ms_step,
                              "traverse_ms_per_step": tr_ms_step, "clocks": clk}), flush=True)
        return

    # other forms on the same workload
    ms32 = dist_max(time_steps(wl, d32, max(3, args.steps // 2), 2), world) / max(3, args.steps // 2)
    msbf = dist_max(time_steps(wl, dbf, max(3, args.steps // 2), 2), world) / max(3, args.steps // 2)
    wl.step(d16)
    torch.cuda.synchronize()

    # training throughput (train rays/s)
    train = time_training(spec, tris, wl, args.train_steps, 3) if args.train_steps > 0 else None
    if train is not None:
        train["value"] = dist_max_rate(train["value"], world)

    # uneven segment counts (64 sphere clusters, 8,192 leaves, 4M rays)
    uneven = time_uneven(args, world) if args.uneven_steps > 0 else None

    # error-driven cut vs median split (same leaves, same training budget)
    cutcmp = time_cut(args, world) if args.cut_steps > 0 else None

    # levels of detail: bounce rays on a coarse LoD vs the finest
    lod = time_lod(args, world) if args.lod_steps > 0 else None

    # the hybrid two-level scene (16 neural assets + 500,000 classical triangles)
    hybrid = time_hybrid(args, world) if args.hybrid_frames > 0 else None

    # the same step and training with the albedo head (8 outputs)
    albedo = time_albedo(args, world, spec, tris, wl) if not args.no_albedo else None

    # end to end through the public API with host buffers (graph step between the copies)
    # a stream of steps: the first copy-in and the last read-back are not
    # overlapped, so at least 30 steps keep that fill and drain below ~10 %
    e2e_steps = max(args.steps, 30)
    wl.e2e_pipelined(d16, args.warmup)
    e2e_ms = dist_max(wl.e2e_pipelined(d16, e2e_steps), world) / e2e_steps
    clk = clocks.stop()  # clocks sampled over every timed form above
    h2d = sum(v.numel() * v.element_size() for v in wl.rays_host.values())
    d2h = 2 * sum(v.numel() * v.element_size() for v in wl.h1_host.values())

    # roofline of the dominant kernel (the fused encode + MLP waves)
    cfg = spec.model
    bytes_seg = cfg.n_samples * cfg.n_levels * 8 * cfg.n_features * 2 + 48
    seg_step = seg1 + seg2
    achieved = seg_step * bytes_seg / (eval_ms_step * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    traffic = profiled_traffic()
    l2_ceiling = B.probe_l2_gather()  # 1e9 random 32-byte sectors per second
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind,
            "kernel": "eval_tc_kernel (query mode): gather + trilinear + tcgen05 MLP + resolve",
            "bytes_per_segment": bytes_seg, "segments_per_step": seg_step,
            "kernel_ms_per_step": eval_ms_step, "traverse_ms_per_step": tr_ms_step,
            "traffic": (traffic["dram_bytes_per_segment"] * seg_step / max(1, waves1 + waves2)
                        if traffic else None),
            "l2_gather": {
                "ceiling_gsectors_s": l2_ceiling,
                "how": "nbvh_probe_l2_gather: random 4-byte loads from a 64 MB L2-resident table, one 1024-thread "
                       "CTA per SM, 16 loads in flight per thread",
                "kernel_gsectors_s": (traffic["l2_sectors_per_segment"] * seg_step / (eval_ms_step * 1e-3) / 1e9
                                      if traffic and "l2_sectors_per_segment" in traffic else None),
                "frac": (traffic["l2_sectors_per_segment"] * seg_step / (eval_ms_step * 1e-3) / 1e9 / l2_ceiling
                         if traffic and "l2_sectors_per_segment" in traffic else None)}}

    line = {"metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": spec.name, "rays_per_step": rays_step, "primary_rays": wl.n,
                       "bounce_rays": rays_step - wl.n, "segments_per_step": seg_step,
                       "eval_launches": [waves1, waves2],
                       "schedule": {"options": B.options_dict(wl.options),
                                    "plan": B.eval_plan(d16, wl.options),
                                    "autotuner": {"best": tune_best, "candidates": tune_all}},
                       "l2": "flushed (256 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "train": train,
            "uneven": uneven,
            "cut_optimization": cutcmp,
            "levels_of_detail": lod,
            "hybrid": hybrid,
            "albedo_head": albedo,
            "fp32_plain": {"value": world * rays_step / (ms32 * 1e-3) / 1e6, "ms_per_step": ms32},
            "bf16_tc": {"value": world * rays_step / (msbf * 1e-3) / 1e6, "ms_per_step": msbf},
            "roofline": roof,
            "e2e": {"value": world * rays_step / (e2e_ms * 1e-3) / 1e6, "unit": "Mrays/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "steps": e2e_steps,
                    "how": "per step: H2D of the rays from pinned memory, graph step, D2H of both hit records; "
                           "two buffer sets, copies on their own streams overlap the neighbouring steps; the "
                           "first copy-in and last read-back are not overlapped; no L2 flush (per-step working "
                           "set ~250 MB > L2)"},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clk}

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        v, dt, nr, idx, res = oracle_sample(spec, tris, rays_np, args.cpu_rays)
        line["cpu_baseline"] = {"value": v, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_rays} seeded primary rays of the 1920x1080 image + their "
                                          f"{nr - args.cpu_rays} bounce rays, {dt:.1f} s"}
        acc = {}
        for nm, dsc in (("fp16_tc", d16), ("bf16_tc", dbf), ("fp32_plain", d32)):
            wl.step(dsc)
            torch.cuda.synchronize()
            acc[nm] = accuracy(wl, idx, res)
        line["accuracy_vs_oracle"] = acc
        tv, tdt = oracle_train_sample(spec, tris)
        line["cpu_baseline_train"] = {"value": tv, "unit": "rays/s", "cores": 1, "kind": "oracle",
                                      "sample": f"one FP64 oracle training step on 256 rays, {tdt:.1f} s"}
    elif rank == 0 and world == 1:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
