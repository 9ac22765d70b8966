#!/usr/bin/env python
"""Neural ray query benchmark on one or more B300s (one process per GPU).

Headline workload (printed as ``value``): the mixed scene. 16 neural assets
(displaced icospheres; per asset a 16-level hash grid with F in {2, 4, 8} and
2^16..2^22 entries per hashed level, BF16 tables, 16 samples per segment, a
3x64 BF16 tensor-core MLP, each trained by the library before the timed
region) stand on a 500,000-triangle classical ground. One step is one frame:
3840x2160 primary rays plus 4 bounces, each pass nbvh_hybrid_trace (top-level
cull, triangle BLAS, every neural BLAS) + nbvh_bounce_rays, replayed from one
CUDA graph. The metric counts the rays each frame traces (primary rays and
the bounce rays spawned from hits) per second.

Also measured, under their own keys: the displaced icosphere (1,310,720
triangles, 2,048 leaves, L16 F2 T2^20 FP16 table, a 3x64 MLP), trained with
the library's training step (the training throughput) and then queried with
1920x1080 primary rays plus one bounce in the FP16 and BF16 tensor-core forms
and the FP32 CUDA-core form at the same accuracy; the 4,096-ray latency case;
uneven segment counts; the error-driven cut; levels of detail; the albedo
head.

The CPU baselines are the FP64 oracle on the host cores: single-threaded and
in one process per core (a spawned pool over rays). ``--impl reference`` times
that oracle on bounded samples of the headline workload.

Printed as one JSON line by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import pickle
import shutil
import subprocess
import sys
import tempfile
import time

# The oracle runs single-threaded per process: pin numpy's BLAS before numpy
# loads (the spawned pool's workers import this module too). The GPU path
# does not use numpy arithmetic.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neural ray queries Mrays/s (fp16 TC vs fp32 plain, same GPU, same err); train rays/s"
SEED = 240516237
HYBRID_BOUNCES = 4
HYBRID_MAX_SEGS = 16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10, help="timed frames of the headline workload")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--hybrid-size", default="3840x2160")
    p.add_argument("--hybrid-train-steps", type=int, default=300, help="training steps per neural asset")
    p.add_argument("--hybrid-train-batch", type=int, default=1 << 16)
    p.add_argument("--accuracy-rays", type=int, default=4096, help="oracle sample of the accuracy comparisons")
    p.add_argument("--single-rays", type=int, default=48,
                   help="single-threaded oracle sample of the headline workload (primary rays)")
    p.add_argument("--ref-rays", type=int, default=0,
                   help="rays per step of the reference arm (0: 8 per host core, at least 64)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--max-segs", type=int, default=48)
    p.add_argument("--train-steps", type=int, default=2000,
                   help="training steps (2^18 rays) of the icosphere model; the query forms use the result")
    p.add_argument("--uneven-steps", type=int, default=5,
                   help="timed queries of the uneven-segment workload (0: skip it)")
    p.add_argument("--cut-steps", type=int, default=1700,
                   help="training-step budget of the error-driven-cut comparison (0: skip it)")
    p.add_argument("--lod-steps", type=int, default=1200,
                   help="training steps of the level-of-detail measurement (0: skip it)")
    p.add_argument("--no-albedo", action="store_true", help="skip the albedo-head measurement")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the library's default query options (no autotuning before the timed region)")
    p.add_argument("--primary", default="1920x1080",
                   help="primary image of the icosphere workload (smaller only for profiling captures)")
    p.add_argument("--only", default="all", choices=["all", "hybrid", "icosphere", "train", "latency", "uneven"],
                   help="run one workload only, without CPU baselines (profiling captures)")
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


# ---------------------------------------------------------------------------- measurement helpers
class ClockSampler:
    """nvidia-smi samples of this GPU's clocks and throttle reasons while the
    timed regions run (started before the first, stopped after the last)."""

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


# the sources of the query's evaluation kernel (eval_tc_kernel, its argument
# struct and device helpers): the committed DRAM traffic is valid for them
KERNEL_SOURCES = ("eval_tc.cuh", "eval_plain.cuh", "nbvh_internal.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2405_16237_b300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(key: str):
    """DRAM bytes per unit of work of a kernel from the committed ncu summary
    (profiles/traffic.json), if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        t = json.load(open(p))
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    return t.get(key)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def timed(fn, steps, flush=None):
    """Device milliseconds of `steps` calls of fn (CUDA events on the current
    stream around each call, synchronised), L2 flushed before each call."""
    import torch
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        total += s.elapsed_time(e)
    return total


def kernel_times(B, fn, steps, flush):
    """Per kernel class, milliseconds, timed groups and launches per step from
    the library's event pairs (eager calls, L2 flushed before each step)."""
    import torch
    torch.cuda.synchronize()
    B.get_kernel_times()
    B.set_timing(True)
    try:
        for _ in range(steps):
            flush()
            fn()
        torch.cuda.synchronize()
        t = B.get_kernel_times()
    finally:
        B.set_timing(False)
    return {k: {"ms": v["ms"] / steps, "groups": v["groups"] / steps, "launches": v["launches"] / steps}
            for k, v in t.items() if v["groups"] > 0}


def roof(ms, bound, amount, peak, unit, how, peak_source="measured"):
    """One roofline entry: `amount` algorithmic bytes (GB/s) or operations per
    step over `ms` device milliseconds against `peak`."""
    achieved = amount / (ms * 1e-3) / 1e9  # GB/s, or 1e9 operations per second
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "ms_per_step": ms, "per_step": amount, "how": how, "peak_source": peak_source}


class Flusher:
    """A buffer larger than L2 (126 MB), rewritten between timed steps."""

    def __init__(self):
        import torch
        self.buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.buf.fill_(1)


def pipelined_e2e(sets, copy_in, launch, copy_out, steps):
    """End to end with host buffers: every step copies its inputs in from
    pinned host memory (copy_in), runs (launch) and reads its results back
    (copy_out). Two device buffer sets and separate copy streams let step
    s+1's copy-in and step s-1's read-back run under step s's compute.
    Returns the device milliseconds of `steps` steps (events on the compute
    stream, which waits for the last read-back)."""
    import torch
    comp = torch.cuda.current_stream()
    s_in = torch.cuda.Stream()
    s_out = torch.cuda.Stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(comp)
    s_in.wait_event(start)
    s_out.wait_event(start)
    done_out = [None, None]
    done_comp = [None, None]
    for i in range(steps):
        st = sets[i % 2]
        with torch.cuda.stream(s_in):
            if done_comp[i % 2] is not None:
                s_in.wait_event(done_comp[i % 2])  # inputs of this set no longer read
            copy_in(st)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
        comp.wait_event(ev_in)
        if done_out[i % 2] is not None:
            comp.wait_event(done_out[i % 2])  # results of this set already read back
        launch(st)
        ev_c = torch.cuda.Event()
        ev_c.record(comp)
        done_comp[i % 2] = ev_c
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_c)
            copy_out(st)
            ev_o = torch.cuda.Event()
            ev_o.record(s_out)
        done_out[i % 2] = ev_o
    for ev in done_out:
        if ev is not None:
            comp.wait_event(ev)
    end.record(comp)
    end.synchronize()
    return start.elapsed_time(end)


def tensor_bytes(d):
    return sum(v.numel() * v.element_size() for v in d.values())


# ---------------------------------------------------------------------------- oracle pool
# The FP64 oracle over rays in one spawned process per host core. A job (the
# instances of a scene, tables as .npy files mapped read-only) is written
# once to a temporary folder; each task answers one chunk of rays.
_JOBS = {}


def _job(path):
    if path not in _JOBS:
        with open(path, "rb") as f:
            job = pickle.load(f)
        for x in job["instances"]:
            if x.get("table_path"):
                x["table"] = np.load(x.pop("table_path"), mmap_mode="r")
        _JOBS[path] = job
    return _JOBS[path]


def _oracle_task(arg):
    """Worker: the oracle's answer for one chunk of rays (the hybrid trace over
    the job's instances, or the query of its single neural instance)."""
    from oracle import nbvh_oracle as O
    path, rays = arg
    job = _job(path)
    t0 = time.perf_counter()
    if job["kind"] == "hybrid":
        r = O.hybrid_trace(rays, job["instances"])
        out = {k: r[k] for k in ("hit", "t", "normal", "leaf", "inst")}
    else:
        x = job["instances"][0]
        r = O.query(rays, x["leaves"], x["table"], x["layers"], x["layout"], x["n_samples"])
        out = {k: r[k] for k in ("hit", "t", "normal", "leaf")}
    out["seconds"] = time.perf_counter() - t0
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A spawned pool (no fork of the CUDA process) of single-threaded oracle
    workers, one per host core (at most `cap`)."""

    def __init__(self, cap=192):
        import multiprocessing as mp
        self.n = max(1, min(host_cores(), cap))
        self.dir = tempfile.mkdtemp(prefix="nbvh_oracle_", dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
        self.pool = mp.get_context("spawn").Pool(self.n)
        self.jobs = 0

    def add_job(self, kind, instances):
        """Writes a job: instances as the oracle takes them; large tables go
        to .npy files that the workers map."""
        inst = []
        for i, x in enumerate(instances):
            x = dict(x)
            if x.get("kind") == "neural":
                tp = os.path.join(self.dir, f"job{self.jobs}_table{i}.npy")
                np.save(tp, np.ascontiguousarray(x.pop("table")))
                x["table_path"] = tp
            inst.append(x)
        path = os.path.join(self.dir, f"job{self.jobs}.pkl")
        with open(path, "wb") as f:
            pickle.dump({"kind": kind, "instances": inst}, f, protocol=pickle.HIGHEST_PROTOCOL)
        self.jobs += 1
        return path

    def run(self, path, rays, warm=True):
        """The oracle's answers for `rays` (dict of arrays), concatenated in
        ray order, and the wall seconds of the pool pass (a first untimed pass
        over a small part lets every worker load the job)."""
        from paper_2405_16237_b300 import workloads as W
        n = len(rays["ox"])
        if warm:
            k = min(n, 2 * self.n)
            idx = np.arange(k)
            self.pool.map(_oracle_task, [(path, W.subset(rays, idx[i:i + 1])) for i in range(k)], chunksize=1)
        n_chunks = min(n, 4 * self.n)
        bounds = np.linspace(0, n, n_chunks + 1).astype(int)
        tasks = [(path, W.subset(rays, np.arange(bounds[i], bounds[i + 1]))) for i in range(n_chunks)]
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        out = {k: np.concatenate([p[k] for p in parts]) for k in parts[0] if k != "seconds"}
        return out, wall

    def close(self):
        self.pool.terminate()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def oracle_single(kind, instances, rays):
    """The oracle in this process (one thread) on `rays`: (answers, seconds)."""
    import contextlib
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # BLAS threads are pinned through the environment above
        def threadpool_limits(limits):
            return contextlib.nullcontext()
    from oracle import nbvh_oracle as O
    with threadpool_limits(limits=1):
        t0 = time.perf_counter()
        if kind == "hybrid":
            r = O.hybrid_trace(rays, instances)
        else:
            x = instances[0]
            r = O.query(rays, x["leaves"], x["table"], x["layers"], x["layout"], x["n_samples"])
        return r, time.perf_counter() - t0


def compare_hits(g, ref, g_inst=None):
    """Hit agreement, depth and normal error of GPU records g (numpy arrays)
    against the oracle's on the same rays; with g_inst, the winning instance
    too. Depth and normal over the rays where both sides hit the same leaf
    (and instance)."""
    g_hit = g["hit"].astype(bool)
    o_hit = ref["hit"].astype(bool)
    out = {"rays": int(len(g_hit)), "hit_agreement": float(np.mean(g_hit == o_hit))}
    same = g_hit & o_hit & (g["leaf"] == ref["leaf"])
    if g_inst is not None:
        out["instance_agreement"] = float(np.mean(g_inst == ref["inst"]))
        same &= g_inst == ref["inst"]
    out["compared_hits"] = int(same.sum())
    if same.any():
        dt = np.abs(g["t"][same] - ref["t"][same])
        out["depth_max_abs"] = float(dt.max())
        out["depth_mean_abs"] = float(dt.mean())
        gn = np.stack([g["nx"], g["ny"], g["nz"]], 1)[same]
        c = np.clip(np.sum(gn * ref["normal"][same], 1), -1, 1)
        out["normal_mean_deg"] = float(np.degrees(np.arccos(c)).mean())
    return out


# ---------------------------------------------------------------------------- headline: hybrid scene (S9)
def hybrid_name(w, h):
    return f"hybrid-16-neural-assets-L16-bf16+500000-tri-ground_{w}x{h}_primary+{HYBRID_BOUNCES}-bounces"


def build_hybrid_host(seed_tables=True):
    """The mixed scene on the host: (ground, assets, oracle instances without
    tables). Used by both arms."""
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import workloads as W
    ground, assets = W.scene_hybrid()
    oinst = [{"kind": "triangles", "tris": ground}]
    for a in assets:
        oinst.append({"kind": "neural", "leaves": O.build_leaves(a.tris, a.n_leaves, 1e-4),
                      "layout": O.level_layout(a.model.n_levels, a.model.base_res, a.model.growth,
                                               a.model.log2_table), "n_samples": a.model.n_samples})
    return ground, assets, oinst


class HybridWorkload:
    """The mixed scene on the device: each neural asset's BF16 table and MLP
    trained by the library (BF16 tensor-core training steps on its own
    triangles), then one frame = the primary pass plus 4 bounce passes of
    nbvh_hybrid_trace + nbvh_bounce_rays, recorded as one graph."""

    def __init__(self, width, height, train_steps, train_batch):
        import torch
        from paper_2405_16237_b300 import nbvh as B
        from paper_2405_16237_b300 import workloads as W
        self.B = B
        t0 = time.perf_counter()
        self.ground, self.assets = W.scene_hybrid()
        self.blas = B.build_tri_blas(self.ground, 4)
        self.dev_blas = B.DeviceTriBlas(self.ground, self.blas)
        self.instances = [B.tri_instance(self.dev_blas)]
        self.keep, self.models, self.asset_info = [], [], []
        self.scene_s = time.perf_counter() - t0
        t1 = time.perf_counter()
        for k, a in enumerate(self.assets):
            lv = B.build_leaves(a.tris, a.n_leaves, 1e-4)
            info = lv["info"]
            desc = B.model_desc(a.model, B.BF16, B.BF16, info["centre"], info["extent"])
            lay = B.level_layout(desc)
            gen = torch.Generator(device="cuda")
            gen.manual_seed(SEED + 100 + k)
            master = torch.empty((lay["total"], a.model.n_features), dtype=torch.float32, device="cuda")
            master.uniform_(-1e-4, 1e-4, generator=gen)
            layers = W.init_mlp(a.model.mlp_dims(), SEED + 200 + k)
            mlp = torch.as_tensor(B.pack_mlp(layers)).cuda()
            nodes = torch.as_tensor(lv["nodes"]).cuda()
            loss_first = loss_last = None
            if train_steps > 0:
                scene = B.DeviceScene(a.tris, lv)
                opt = B.Optimizer(desc, master, mlp, loss_scale=32768.0)
                ws = B.new_workspace(B.train_workspace_size(desc, train_batch, scene.n_leaves))
                loss = torch.zeros(1, dtype=torch.float32, device="cuda")
                for step in range(1, train_steps + 1):
                    B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, train_batch, SEED + 300 + k, step, 1e-2, ws,
                                 loss_out=loss)
                    if step == 1:
                        loss_first = float(loss.item())
                torch.cuda.synchronize()
                loss_last = float(loss.item())
                table = opt.table.clone()
                mlp = opt.mlp.clone()
                del opt, ws, scene
            else:
                table = master.to(torch.bfloat16)
            del master
            torch.cuda.empty_cache()
            self.keep += [table, mlp, nodes]
            self.models.append((a, table, mlp))
            self.instances.append(B.neural_instance(desc, table, mlp, nodes, lv["n_nodes"], HYBRID_MAX_SEGS))
            K = a.model.n_samples * a.model.n_levels * a.model.n_features
            self.asset_info.append({"triangles": int(len(a.tris)), "leaves": a.n_leaves, "F": a.model.n_features, "log2_T": a.model.log2_table,
                                    "levels": a.model.n_levels, "inputs": K, "table_entries": int(lay["total"]),
                                    "train_loss_first": loss_first, "train_loss_last": loss_last})
        if B.device_status() != 0:
            raise RuntimeError("device status after training the hybrid assets")
        self.train_s = time.perf_counter() - t1
        self.rays_np = W.hybrid_camera_rays(width, height)
        self.n = len(self.rays_np["ox"])
        self.rays_host = {k: torch.as_tensor(np.ascontiguousarray(self.rays_np[k])).pin_memory() for k in B.RAY_KEYS}
        self.bufs = self.new_buffers()
        self.bufs["rays"][0] = {k: v.cuda() for k, v in self.rays_host.items()}
        self.graph = None
        self.launches = 0

    def new_buffers(self):
        import torch
        B = self.B
        return {"rays": [B.new_rays(self.n) for _ in range(HYBRID_BOUNCES + 1)],
                "hits": [B.new_hits(self.n) for _ in range(HYBRID_BOUNCES + 1)],
                "inst": [torch.empty(self.n, dtype=torch.int32, device="cuda") for _ in range(HYBRID_BOUNCES + 1)],
                "ws": B.new_workspace(B.hybrid_workspace_size(self.instances, self.n))}

    def frame(self, bufs=None, options=None):
        B = self.B
        b_ = bufs or self.bufs
        for b in range(HYBRID_BOUNCES + 1):
            B.hybrid_trace(self.instances, b_["rays"][b], out=b_["hits"][b], inst_out=b_["inst"][b],
                           workspace=b_["ws"], options=options)
            if b < HYBRID_BOUNCES:
                B.bounce_rays(b_["rays"][b], b_["hits"][b], SEED + 30 + b, out=b_["rays"][b + 1])

    def graph_frame(self):
        if self.graph is None:
            n0 = self.B.launch_count()
            self.graph = self.B.Graph.record(self.frame)
            self.launches = self.B.launch_count() - n0
        self.graph.launch()

    def rays_per_frame(self):
        """Rays traced with a non-empty interval: every primary ray, and each
        bounce ray spawned from a hit."""
        h = self.bufs["hits"]
        return self.n + sum(int(h[b]["hit"].sum().item()) for b in range(HYBRID_BOUNCES))

    def oracle_instances(self, oinst):
        """The oracle's instances with the trained tables (float32 copies of the
        BF16 values, exact) and MLP weights."""
        from paper_2405_16237_b300 import nbvh as B
        out = [oinst[0]]
        for (a, table, mlp), x in zip(self.models, oinst[1:]):
            layers = B.unpack_mlp(mlp.cpu().numpy(), a.model.mlp_dims())
            out.append(dict(x, table=table.float().cpu().numpy(), layers=layers))
        return out


def time_hybrid(args, world, rank, clocks_cb):
    """The headline: trained mixed scene, graph-replayed frames."""
    import torch
    w, h = (int(x) for x in args.hybrid_size.split("x"))
    hw = HybridWorkload(w, h, args.hybrid_train_steps, args.hybrid_train_batch)
    B = hw.B
    flush = Flusher()
    hw.frame()
    torch.cuda.synchronize()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the first hybrid frame")
    rays = hw.rays_per_frame()
    kinds = {"triangle": int((hw.bufs["inst"][0] == 0).sum().item()),
             "neural": int((hw.bufs["inst"][0] > 0).sum().item())}
    for _ in range(args.warmup):
        hw.graph_frame()
    torch.cuda.synchronize()
    barrier(world)
    clocks_cb("start")
    total = timed(hw.graph_frame, args.steps, flush)
    clocks_cb("stop")
    if B.device_status() != 0:
        raise RuntimeError("device status after the timed hybrid frames")
    ms = dist_max(total, world) / args.steps
    res = {"rays_per_frame": rays, "ms_per_frame": ms, "value": world * rays / (ms * 1e-3) / 1e6,
           "primary_hits": kinds, "launches_per_frame": hw.launches, "hw": hw, "flush": flush}
    return res


def hybrid_details(args, world, hw, flush, pool, oinst, frame_ms):
    """Everything around the headline's timed frames: kernel times, evaluated
    segments per asset, the roofline, end to end with host buffers, and the
    accuracy and CPU baselines on the oracle."""
    import torch
    B = hw.B
    out = {}
    # evaluated segments of every neural instance over a frame (statistics pass)
    seg = torch.zeros(len(hw.instances), dtype=torch.int64, device="cuda")
    hw.frame(options=B.query_options(segments_out=seg))
    torch.cuda.synchronize()
    seg = seg.cpu().numpy()
    kt = kernel_times(B, hw.frame, 3, flush)
    peaks, peak_kind = measured_peaks()
    bytes_eval = 0
    per_asset = []
    for (a, _, _), s_i in zip(hw.models, seg[1:]):
        b_seg = a.model.n_samples * a.model.n_levels * 8 * a.model.n_features * 2 + 48
        bytes_eval += int(s_i) * b_seg
        per_asset.append({"segments": int(s_i), "bytes_per_segment": b_seg})
    n = hw.n
    live = hw.rays_per_frame()
    kernels = {}
    if "eval" in kt:
        kernels["eval"] = dict(kt["eval"], **roof(kt["eval"]["ms"], "hbm", bytes_eval, peaks["hbm_gbs"], "GB/s",
                                                   "per neural segment N*L*8 corners*F*2 B (BF16) + 48 B of ray "
                                                   "and segment; summed over the assets' evaluated segments",
                                                   peak_kind))
    hits_b = sum(int(hw.bufs["hits"][b]["hit"].sum().item()) for b in range(HYBRID_BOUNCES))
    for k, amount, how in (
            ("tri_trace", (32 + 4 + 24 + 4) * n * (HYBRID_BOUNCES + 1),
             "per ray 32 B ray + 4 B record t in, 24 B record + 4 B instance out, every ray of every pass (BVH "
             "nodes and triangles stay in L2: the traversal is bound by dependent fetches, not bytes)"),
            ("bounce", 57 * n * HYBRID_BOUNCES + 16 * hits_b,
             "per ray 24 B origin and direction + 1 B hit flag in, 32 B ray out; per hit 16 B t and normal in"),
            ("tlas_cull", (32 + 4) * n * (HYBRID_BOUNCES + 1),
             "per ray 32 B ray + 4 B record t in (list entries written only for rays meeting a root box)")):
        if k in kt:
            kernels[k] = dict(kt[k], **roof(kt[k]["ms"], "hbm", amount, peaks["hbm_gbs"], "GB/s", how, peak_kind))
    for k in ("traverse", "other"):
        if k in kt:
            kernels[k] = kt[k]
    dom = max(kernels, key=lambda k: kernels[k]["ms"] if "ms" in kernels[k] else 0.0)
    traffic = profiled_traffic("hybrid_eval")
    r = kernels.get("eval", {})
    out["roofline"] = {"bound": "hbm", "achieved": r.get("achieved"), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": r.get("frac"), "peak_source": peak_kind,
                       "note": "the neural instances of a pass run on two streams: the event time of the "
                               "evaluation groups sums overlapping launches (it exceeds the frame), so achieved is "
                               "a lower bound; over_frame divides the same bytes by the whole frame's time",
                       "over_frame": {"achieved": bytes_eval / (frame_ms * 1e-3) / 1e9,
                                      "frac": bytes_eval / (frame_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                       "kernel": "eval_tc_kernel (query mode, every neural BLAS of every pass): gather + trilinear "
                                 "+ tcgen05 MLP + resolve",
                       "dominant_kernel_class": dom,
                       "launches_per_frame": r.get("groups"), "ms_per_frame": r.get("ms"),
                       "bytes_per_frame": bytes_eval,
                       "traffic": traffic["dram_bytes_per_launch"] if traffic else None}
    out["kernels"] = kernels
    out["segments_per_frame"] = {"total": int(seg[1:].sum()), "per_asset": per_asset}

    # end to end through the public API with host buffers: per frame the
    # primary rays in from pinned memory, every pass's hit record and instance
    # out to pinned memory; two buffer sets overlap neighbouring frames
    second = hw.new_buffers()
    sets = [hw.bufs, second]
    for st in sets:
        st["host_out"] = [{k: torch.empty_like(v, device="cpu").pin_memory() for k, v in dict(
            st["hits"][b], inst=st["inst"][b]).items()} for b in range(HYBRID_BOUNCES + 1)]
        st["graph"] = B.Graph.record(lambda st=st: hw.frame(st))

    def copy_in(st):
        for k in B.RAY_KEYS:
            st["rays"][0][k].copy_(hw.rays_host[k], non_blocking=True)

    def copy_out(st):
        for b in range(HYBRID_BOUNCES + 1):
            src = dict(st["hits"][b], inst=st["inst"][b])
            for k, v in src.items():
                st["host_out"][b][k].copy_(v, non_blocking=True)

    e2e_steps = max(args.steps, 10)
    pipelined_e2e(sets, copy_in, lambda st: st["graph"].launch(), copy_out, args.warmup)
    e2e_ms = dist_max(pipelined_e2e(sets, copy_in, lambda st: st["graph"].launch(), copy_out, e2e_steps),
                      world) / e2e_steps
    for st in sets:
        st["graph"].destroy()
    h2d = tensor_bytes(hw.rays_host)
    d2h = sum(tensor_bytes(x) for x in sets[0]["host_out"])
    out["e2e"] = {"value": world * live / (e2e_ms * 1e-3) / 1e6, "unit": "Mrays/s", "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
                  "how": "per frame: H2D of the primary rays from pinned memory, graph-replayed frame, D2H of every "
                         "pass's hit record and instance id; two buffer sets, copies on their own streams overlap "
                         "the neighbouring frames; no L2 flush (per-frame working set > L2)"}
    del second, sets
    torch.cuda.empty_cache()

    # accuracy against the oracle on a seeded sample of the primary rays
    if pool is not None:
        from paper_2405_16237_b300 import workloads as W
        rng = np.random.default_rng(SEED + 6)
        idx = np.sort(rng.choice(hw.n, size=min(args.accuracy_rays, hw.n), replace=False))
        sub = W.subset(hw.rays_np, idx)
        inst = hw.oracle_instances(oinst)
        job = pool.add_job("hybrid", inst)
        ref, wall = pool.run(job, sub)
        g = {k: v.cpu().numpy()[idx] for k, v in hw.bufs["hits"][0].items()}
        out["accuracy_vs_oracle"] = compare_hits(g, ref, hw.bufs["inst"][0].cpu().numpy()[idx])
        out["cpu_baseline"] = {"value": len(idx) / wall / 1e6, "unit": "Mrays/s", "cores": pool.n, "kind": "oracle",
                               "cpu_count": os.cpu_count(),
                               "sample": f"{len(idx)} seeded primary rays of the {hw.n}-ray image, primary pass (the "
                                         f"triangle ground and all 16 neural assets, every segment evaluated), "
                                         f"{pool.n} single-threaded processes, {wall:.1f} s wall"}
        k = min(args.single_rays, len(idx))
        _, dt = oracle_single("hybrid", inst, W.subset(sub, np.arange(k)))
        out["cpu_baseline_single"] = {"value": k / dt / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                                      "sample": f"the first {k} rays of the same sample, one thread, {dt:.1f} s"}
    return out


# ---------------------------------------------------------------------------- icosphere (C1, C2)
def make_scene(primary="1920x1080"):
    from paper_2405_16237_b300 import workloads as W
    tris = W.scene_icosphere(level=8)
    w, h = (int(x) for x in primary.split("x"))
    return W.C1, tris, W.camera_rays(w, h)


class GpuWorkload:
    """The displaced icosphere: model, rays and buffers of its query step
    (primary query -> bounce rays -> secondary query)."""

    def __init__(self, spec, tris, rays_np, max_segs):
        import torch
        from paper_2405_16237_b300 import nbvh as B
        from paper_2405_16237_b300 import workloads as W
        self.B = B
        self.spec = spec
        self.tris = tris
        self.max_segs = max_segs
        self.leaves = B.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
        info = self.leaves["info"]
        cfg = spec.model
        self.desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
        lay = B.level_layout(self.desc)
        self.table_master = torch.as_tensor(W.init_table(lay["total"], cfg.n_features, SEED + 21, 1e-4)).cuda()
        self.table = self.table_master.half()
        self.mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 22))).cuda()
        self.nodes = torch.as_tensor(self.leaves["nodes"]).cuda()
        self.n = len(rays_np["ox"])
        self.rays_np = rays_np
        self.rays_host = {k: torch.as_tensor(np.ascontiguousarray(rays_np[k])).pin_memory() for k in B.RAY_KEYS}
        self.rays = {k: v.cuda() for k, v in self.rays_host.items()}
        self.rays2 = B.new_rays(self.n)
        self.h1 = B.new_hits(self.n)
        self.h2 = B.new_hits(self.n)
        ws = B.query_workspace_size(self.desc, self.n, max_segs)
        self.ws1 = B.new_workspace(ws)
        self.ws2 = B.new_workspace(ws)
        self.graphs = {}
        self.launches_per_step = {}
        self.options = None  # query options (None: the library's defaults), set from the autotuner

    def step(self, desc, bufs=None):
        B = self.B
        b = bufs or {"rays": self.rays, "rays2": self.rays2, "h1": self.h1, "h2": self.h2, "ws1": self.ws1,
                     "ws2": self.ws2}
        B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], b["rays"], self.max_segs,
                     out=b["h1"], workspace=b["ws1"], options=self.options)
        B.bounce_rays(b["rays"], b["h1"], SEED + 3, out=b["rays2"])
        B.query_rays(desc, self.table, self.mlp, self.nodes, self.leaves["n_nodes"], b["rays2"], self.max_segs,
                     out=b["h2"], workspace=b["ws2"], options=self.options)

    def graph_step(self, desc):
        """The step replayed from a CUDA graph recorded on first use."""
        key = (desc.mlp_prec, desc.table_prec)
        if key not in self.graphs:
            n0 = self.B.launch_count()
            self.graphs[key] = self.B.Graph.record(lambda: self.step(desc))
            self.launches_per_step[key] = self.B.launch_count() - n0
        self.graphs[key].launch()

    def drop_graphs(self):
        for g in self.graphs.values():
            g.destroy()
        self.graphs = {}

    def rays_per_step(self):
        return self.n + int(self.h1["hit"].sum().item())


def train_icosphere(args, world, wl, flush):
    """Training of the icosphere model (the training throughput): steps of 2^18
    rays (BVH-probed rays through random leaves and rays on the bounding
    sphere, brute-force labels), FP16 tensor-core compute on FP32 masters,
    Adam lr 1e-2, dynamic loss scale. The trained table and MLP replace the
    workload's for the query measurements."""
    import torch
    B = wl.B
    batch = 1 << 18
    scene = B.DeviceScene(wl.tris, wl.leaves)
    desc = B.with_mlp_prec(wl.desc, B.FP16)
    opt = B.Optimizer(desc, wl.table_master.clone(), wl.mlp.clone(), loss_scale=32768.0)
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    step = 0

    def one():
        nonlocal step
        step += 1
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, SEED + 9, step, 1e-2, ws, loss_out=loss)

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    first = float(loss.item())
    kt = kernel_times(B, one, 5, flush)
    n_timed = max(1, args.train_steps - 8)
    curve = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n_timed):
        one()
        if (i + 1) % max(1, n_timed // 8) == 0:
            curve.append((step, loss.clone()))
    e1.record()
    e1.synchronize()
    ms = dist_max(e0.elapsed_time(e1), world) / n_timed
    if B.device_status() != 0:
        raise RuntimeError("device status after the training steps")
    wl.table = opt.table.clone()
    wl.mlp = opt.mlp.clone()
    wl.table_master = opt.table_master.clone()
    res = {"value": world * batch / (ms * 1e-3), "unit": "rays/s", "batch": batch, "ms_per_step": ms,
           "steps": step, "timed_steps": n_timed,
           "dtype": "f16 compute, f32 masters", "loss_after_warmup": first, "loss_last": float(loss.item()),
           "loss_curve": [(s, float(l.item())) for s, l in curve], "loss_scale": float(opt.loss_scale.item()),
           "timing": "all timed steps between two CUDA events (no flush: a step's working set, ~1 GB, exceeds L2)"}
    res["kernels"] = train_rooflines(kt, wl, batch, scene.n_leaves, scene)
    del opt, ws
    torch.cuda.empty_cache()
    return res


def scatter_adds(wl, scene, n=8192):
    """Table-gradient atomic adds the tensor-core backward issues per training
    ray, counted on a sample of training rays from the library: walking each
    ray's samples level by level, a move to another cell flushes the corner
    sums the two cells do not share (8 - prod(2 - |d|) of them) and the last
    cell flushes all 8; without the level-major walk every (sample, level)
    adds its 8 corners. Returns (adds per training ray, algorithmic adds =
    N * L * 8 per valid ray, valid fraction)."""
    B = wl.B
    cfg = wl.spec.model
    rays, leaf, t0, t1, _ = B.train_rays(B.TRAIN_PROBED_MIX, SEED + 9, 0, scene, n)
    v = leaf.cpu().numpy() >= 0
    o = np.stack([rays[k].cpu().numpy() for k in ("ox", "oy", "oz")], 1)[v].astype(np.float64)
    d = np.stack([rays[k].cpu().numpy() for k in ("dx", "dy", "dz")], 1)[v].astype(np.float64)
    a, b = t0.cpu().numpy()[v].astype(np.float64), t1.cpu().numpy()[v].astype(np.float64)
    info = wl.leaves["info"]
    u = (np.arange(cfg.n_samples) + 0.5) / cfg.n_samples
    t = a[:, None] + u[None, :] * (b - a)[:, None]
    x = np.clip((o[:, None, :] + t[..., None] * d[:, None, :] - np.asarray(info["centre"])) / float(info["extent"])
                + 0.5, 0.0, 1.0)
    level_major = cfg.n_features <= 2 and 128 % (cfg.n_samples * cfg.n_features) == 0
    per_ray = np.zeros(len(a))
    for res in B.level_layout(wl.desc)["res"]:
        if not level_major:
            per_ray += 8 * cfg.n_samples
            continue
        c = np.minimum(np.floor(x * res), res - 1)
        dc = np.abs(np.diff(c, axis=1))  # [rays, samples - 1, 3]
        moved = np.any(dc > 0, axis=2)
        kept = np.where(np.all(dc <= 1, axis=2), np.prod(2 - dc, axis=2), 0)
        per_ray += 8 + np.sum(np.where(moved, 8 - kept, 0), axis=1)
    frac = v.mean()
    return float(per_ray.mean() * frac), float(cfg.n_samples * cfg.n_levels * 8 * frac), float(frac)


def train_rooflines(kt, wl, batch, n_leaves, scene):
    """Roofline entries of the training kernels per step (2^18 rays)."""
    from paper_2405_16237_b300 import nbvh as B
    peaks, peak_kind = measured_peaks()
    cfg = wl.spec.model
    K = cfg.n_samples * cfg.n_levels * cfg.n_features
    W_, nh = cfg.width, cfg.n_hidden
    n_params_tab = int(wl.table_master.numel())
    n_params_mlp = int(wl.mlp.numel())
    red = B.probe_l2_reduce()
    tris_per_leaf = len(wl.tris) / max(1, n_leaves)
    issued, algo, valid = scatter_adds(wl, scene)
    out = {"l2_reduce_ceiling_gadds_s": red,
           "scatter": {"issued_adds_per_ray": issued, "algorithmic_adds_per_ray": algo, "valid_fraction": valid}}
    spec = {
        "train_rays": ("hbm", batch * (32 + 12 + 12), "GB/s", "per ray 32 B ray + leaf, t0, t1 + 12 B grouping"),
        "train_forward": ("hbm", batch * (K // cfg.n_features * 8 * cfg.n_features * 2 + K * 2 + nh * W_ * 2
                                          + (nh - 1) * W_ * 2 + 44),
                          "GB/s", "per ray the gather (N*L*8 corners*F*2 B) + stored features (K*2 B) + hidden "
                                  "activations (n_hidden*W*2 B) and the neuron-major copies of those feeding a "
                                  "hidden layer ((n_hidden-1)*W*2 B) + outputs, dL/draw, loss term (44 B)"),
        "train_backward": ("l2_atomic", batch * issued, "Gadds/s",
                           "float2 table-gradient adds the kernel issues per training ray (the method's N*L*8 "
                           "corner updates per valid ray, merged along the ray: scatter) against "
                           "nbvh_probe_l2_reduce"),
        "weight_grad": ("hbm", batch * (K * 2 + 2 * nh * W_ * 2 + cfg.n_out * 4), "GB/s",
                        "per ray the operands read: features (K*2 B), each layer's dZ and input activations "
                        "(2*n_hidden*W*2 B), dL/draw (n_out*4 B)"),
        "adam": ("hbm", (n_params_tab + n_params_mlp) * 30, "GB/s",
                 "per parameter 30 B (master, gradient, two moments read; master, moments, 16-bit copy written; "
                 "gradient cleared)"),
        "labels": ("alu", batch * tris_per_leaf, "Gtests/s",
                   "per ray one Moller-Trumbore test per triangle of its leaf; peak: FP32 lanes x clock / 30 "
                   "FP32 operations per test"),
    }
    lanes_peak = 148 * 128 * 2.032e9 / 30 / 1e9  # ray-triangle tests per second (1e9), FP32 issue-bound
    for k, (bound, amount, unit, how) in spec.items():
        if k not in kt:
            continue
        if bound == "hbm":
            out[k] = dict(kt[k], **roof(kt[k]["ms"], bound, amount, peaks["hbm_gbs"], unit, how, peak_kind))
        elif bound == "l2_atomic":
            out[k] = dict(kt[k], **roof(kt[k]["ms"], bound, amount, red, unit, how, "probe"))
        else:
            out[k] = dict(kt[k], **roof(kt[k]["ms"], bound, amount, lanes_peak, unit, how, "derived"))
    for k in ("other",):
        if k in kt:
            out[k] = kt[k]
    return out


def time_icosphere(args, world, rank, wl, flush, pool, clocks_cb):
    """The icosphere query step with the trained network: FP16 (autotuned
    options), BF16 and FP32 forms, kernel times and rooflines, end to end, and
    the accuracy of each form against the oracle on 4,096 primary rays."""
    import torch
    B = wl.B
    d16 = B.with_mlp_prec(wl.desc, B.FP16)
    d32 = B.with_mlp_prec(wl.desc, B.FP32)
    dbf = B.with_mlp_prec(wl.desc, B.BF16)
    if args.no_autotune:
        tune_best, tune_all = dict(B.options_dict(B.query_options()), ms=None), []
    else:
        tune_best, tune_all = B.autotune_query(d16, wl.table, wl.mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays,
                                               args.max_segs, out=wl.h1, workspace=wl.ws1, reps=3)
    wl.options = B.options_from_dict(tune_best)
    wl.step(d16)
    torch.cuda.synchronize()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the first icosphere step")
    rays_step = wl.rays_per_step()
    seg1, _ = B.query_stats(wl.ws1, wl.n, args.max_segs)
    seg2, _ = B.query_stats(wl.ws2, wl.n, args.max_segs)
    # listed segments (traversal output), untimed
    listed = 0
    for r in (wl.rays, wl.rays2):
        tr = B.traverse(wl.nodes, wl.leaves["n_nodes"], r, args.max_segs)
        listed += int(tr["count"].sum().item())
        del tr
    kt = kernel_times(B, lambda: wl.step(d16), 5, flush)
    steps = max(args.steps, 5)
    for _ in range(args.warmup):
        wl.graph_step(d16)
    torch.cuda.synchronize()
    clocks_cb("start")
    ms16 = dist_max(timed(lambda: wl.graph_step(d16), steps, flush), world) / steps
    for _ in range(2):
        wl.graph_step(dbf)
        wl.graph_step(d32)
    msbf = dist_max(timed(lambda: wl.graph_step(dbf), steps, flush), world) / steps
    ms32 = dist_max(timed(lambda: wl.graph_step(d32), steps, flush), world) / steps
    clocks_cb("stop")
    launches16 = wl.launches_per_step[(d16.mlp_prec, d16.table_prec)]
    peaks, peak_kind = measured_peaks()
    cfg = wl.spec.model
    b_seg = cfg.n_samples * cfg.n_levels * 8 * cfg.n_features * 2 + 48
    seg_step = seg1 + seg2
    kernels = {}
    if "eval" in kt:
        kernels["eval"] = dict(kt["eval"], **roof(kt["eval"]["ms"], "hbm", seg_step * b_seg, peaks["hbm_gbs"], "GB/s",
                                                   "per evaluated segment N*L*8 corners*F*2 B (FP16) + 48 B",
                                                   peak_kind))
    if "traverse" in kt:
        kernels["traverse"] = dict(kt["traverse"], **roof(kt["traverse"]["ms"], "hbm",
                                                          2 * wl.n * 36 + listed * 12, peaks["hbm_gbs"], "GB/s",
                                                          "per ray 32 B ray in + 4 B count out, per listed segment "
                                                          "12 B (leaf, t0, t1) out; node reads are L1/L2-resident",
                                                          peak_kind))
    if "bounce" in kt:
        kernels["bounce"] = dict(kt["bounce"], **roof(kt["bounce"]["ms"], "hbm", wl.n * 57 + (rays_step - wl.n) * 16,
                                                      peaks["hbm_gbs"], "GB/s",
                                                      "per ray 24 B origin and direction + 1 B hit flag in, 32 B "
                                                      "ray out; per hit 16 B t and normal in (the hit record is "
                                                      "L2-hot from the query)", peak_kind))
    traffic = profiled_traffic("icosphere_eval")
    l2_ceiling = B.probe_l2_gather()
    ev = kernels.get("eval", {})
    roofline = {"bound": "hbm", "achieved": ev.get("achieved"), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ev.get("frac"), "peak_source": peak_kind,
                "kernel": "eval_tc_kernel (query mode): gather + trilinear + tcgen05 MLP + resolve",
                "bytes_per_segment": b_seg, "segments_per_step": seg_step,
                "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                "traffic_how": traffic["note"] if traffic else None,
                "l2_gather": {
                    "ceiling_gsectors_s": l2_ceiling,
                    "how": "nbvh_probe_l2_gather: random 4-byte loads from a 64 MB L2-resident table, one "
                           "1024-thread CTA per SM, 16 loads in flight per thread",
                    "kernel_gsectors_s": (traffic["l2_sectors_per_segment"] * seg_step / (ev["ms"] * 1e-3) / 1e9
                                          if traffic and ev else None),
                    "sectors_per_segment_from": "the committed 960x540 capture (profiles/traffic.json)"}}
    if roofline["l2_gather"]["kernel_gsectors_s"]:
        roofline["l2_gather"]["frac"] = roofline["l2_gather"]["kernel_gsectors_s"] / l2_ceiling

    # end to end with host buffers (the FP16 graph step between the copies)
    second = {"rays": {k: torch.empty_like(v) for k, v in wl.rays.items()}, "rays2": B.new_rays(wl.n),
              "h1": B.new_hits(wl.n), "h2": B.new_hits(wl.n), "ws1": B.new_workspace(wl.ws1.numel()),
              "ws2": B.new_workspace(wl.ws2.numel())}
    first = {"rays": wl.rays, "rays2": wl.rays2, "h1": wl.h1, "h2": wl.h2, "ws1": wl.ws1, "ws2": wl.ws2}
    sets = [first, second]
    for st_ in sets:
        st_["host"] = {("h1", k): torch.empty_like(v, device="cpu").pin_memory() for k, v in st_["h1"].items()}
        st_["host"].update({("h2", k): torch.empty_like(v, device="cpu").pin_memory() for k, v in st_["h2"].items()})
        st_["graph"] = B.Graph.record(lambda st_=st_: wl.step(d16, st_))

    def copy_in(st_):
        for k in B.RAY_KEYS:
            st_["rays"][k].copy_(wl.rays_host[k], non_blocking=True)

    def copy_out(st_):
        for (which, k), v in st_["host"].items():
            v.copy_(st_[which][k], non_blocking=True)

    e2e_steps = max(args.steps, 30)
    pipelined_e2e(sets, copy_in, lambda st_: st_["graph"].launch(), copy_out, args.warmup)
    e2e_ms = dist_max(pipelined_e2e(sets, copy_in, lambda st_: st_["graph"].launch(), copy_out, e2e_steps),
                      world) / e2e_steps
    for st_ in sets:
        st_["graph"].destroy()
    h2d = tensor_bytes(wl.rays_host)
    d2h = tensor_bytes(sets[0]["host"])
    del second, sets
    out = {"workload": wl.spec.name, "value": world * rays_step / (ms16 * 1e-3) / 1e6, "unit": "Mrays/s",
           "ms_per_step": ms16, "steps": steps, "rays_per_step": rays_step, "primary_rays": wl.n,
           "bounce_rays": rays_step - wl.n, "segments_per_step": seg_step, "segments_primary": seg1,
           "segments_bounce": seg2, "listed_segments_per_step": listed,
           "gpu_launches_per_step": launches16, "dtype": "f16 table, f16 tensor-core MLP",
           "fp32_plain": {"value": world * rays_step / (ms32 * 1e-3) / 1e6, "ms_per_step": ms32},
           "bf16_tc": {"value": world * rays_step / (msbf * 1e-3) / 1e6, "ms_per_step": msbf},
           "network": ("trained by the training measurement above" if "train" in args.__dict__.get("_ran", ())
                       else "untrained (initial weights)"),
           "schedule": {"options": B.options_dict(wl.options), "plan": B.eval_plan(d16, wl.options),
                        "autotuner": {"best": tune_best, "candidates": tune_all}},
           "kernels": kernels, "roofline": roofline,
           "e2e": {"value": world * rays_step / (e2e_ms * 1e-3) / 1e6, "unit": "Mrays/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                   "steps": e2e_steps,
                   "how": "per step: H2D of the rays from pinned memory, graph step, D2H of both hit records; two "
                          "buffer sets, copies on their own streams overlap the neighbouring steps; no L2 flush"},
           "l2": "flushed (256 MB write) between timed steps"}

    if pool is not None:
        from oracle import nbvh_oracle as O
        from paper_2405_16237_b300 import workloads as W
        rng = np.random.default_rng(SEED + 5)
        idx = np.sort(rng.choice(wl.n, size=min(args.accuracy_rays, wl.n), replace=False))
        sub = W.subset(wl.rays_np, idx)
        inst = [{"kind": "neural", "leaves": O.build_leaves(wl.tris, wl.spec.n_leaves, wl.spec.inflate_rel),
                 "table": wl.table.float().cpu().numpy(),
                 "layers": B.unpack_mlp(wl.mlp.cpu().numpy(), cfg.mlp_dims()),
                 "layout": O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table),
                 "n_samples": cfg.n_samples}]
        job = pool.add_job("query", inst)
        ref, wall = pool.run(job, sub)
        acc = {}
        for nm, dsc in (("fp16_tc", d16), ("bf16_tc", dbf), ("fp32_plain", d32)):
            wl.step(dsc)
            torch.cuda.synchronize()
            g = {k: v.cpu().numpy()[idx] for k, v in wl.h1.items()}
            acc[nm] = compare_hits(g, ref)
        out["accuracy_vs_oracle"] = acc
        out["cpu_baseline"] = {"value": len(idx) / wall / 1e6, "unit": "Mrays/s", "cores": pool.n, "kind": "oracle",
                               "cpu_count": os.cpu_count(),
                               "sample": f"{len(idx)} seeded primary rays of the {wl.n}-ray image (every segment "
                                         f"evaluated), {pool.n} single-threaded processes, {wall:.1f} s wall"}
        k = min(1024, len(idx))
        _, dt = oracle_single("query", inst, W.subset(sub, np.arange(k)))
        out["cpu_baseline_single"] = {"value": k / dt / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                                      "sample": f"the first {k} rays of the same sample, one thread, {dt:.1f} s"}
        tv, tdt = oracle_train_sample(wl)
        out["cpu_baseline_train"] = {"value": tv, "unit": "rays/s", "cores": 1, "kind": "oracle",
                                     "sample": f"one FP64 oracle training step on 256 rays, {tdt:.1f} s"}
    return out


def oracle_train_sample(wl, n=256):
    """One FP64 oracle training step (rays, labels, loss, gradient, Adam) on n
    rays of the icosphere scene and model. Returns rays/s and seconds."""
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import nbvh as B
    cfg = wl.spec.model
    leaves = O.build_leaves(wl.tris, wl.spec.n_leaves, wl.spec.inflate_rel)
    lay = O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table)
    tab = wl.table_master.cpu().numpy().astype(np.float64)
    layers = B.unpack_mlp(wl.mlp.cpu().numpy(), cfg.mlp_dims())
    fr = leaves["frame"]
    t0 = time.perf_counter()
    R = O.train_rays(O.TRAIN_MODE_PROBED_MIX, SEED + 9, 0, n, leaves)
    valid = R["leaf"] >= 0
    lab = O.labels(R["o"], R["d"], R["leaf"], R["t0"], R["t1"], wl.tris, leaves["tri_perm"], leaves["leaf_range"])
    L, g_tab, g_layers, _ = O.forward_backward(R["o"], R["d"], R["t0"], R["t1"], valid, lab["hit"], lab["depth"],
                                               lab["normal"], tab, layers, lay, fr["model_centre"],
                                               fr["model_extent"], cfg.n_samples)
    O.adam(tab, g_tab, np.zeros_like(tab), np.zeros_like(tab), 1)
    for (w_, b_), (gw, gb) in zip(layers, g_layers):
        O.adam(w_, gw, np.zeros_like(gw), np.zeros_like(gw), 1)
        O.adam(b_, gb, np.zeros_like(gb), np.zeros_like(gb), 1)
    dt = time.perf_counter() - t0
    return n / dt, dt


# ---------------------------------------------------------------------------- latency floor (C0)
def time_latency(args, world, flush):
    """The 4,096-ray case (4,096 random triangles, 64 leaves, L4 F2 T2^12 FP32
    table, 8 samples, 2x32 MLP, 64x64 camera rays): device time of one query
    (graph replay) and host latency of one eager call to completion, for the
    FP32 CUDA-core and FP16 tensor-core forms; and the oracle on all 4,096
    rays."""
    import torch
    from oracle import nbvh_oracle as O
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    spec = W.C0
    cfg = spec.model
    tris = W.scene_random_tris(4096, seed=W.SEED_BASE)
    rays_np = W.camera_rays(64, 64)
    lv = B.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
    info = lv["info"]
    d32 = B.model_desc(cfg, B.FP32, B.FP32, info["centre"], info["extent"])
    lay = B.level_layout(d32)
    tab_np = W.init_table(lay["total"], cfg.n_features, SEED + 71, 1e-4)
    layers = W.init_mlp(cfg.mlp_dims(), SEED + 72)
    table = torch.as_tensor(tab_np).cuda()
    mlp = torch.as_tensor(B.pack_mlp(layers)).cuda()
    nodes = torch.as_tensor(lv["nodes"]).cuda()
    rays = B.to_device_rays(rays_np)
    n = rays["ox"].numel()
    out = {"workload": spec.name, "rays": n}
    for nm, desc in (("fp32_plain", d32), ("fp16_tc", B.with_mlp_prec(d32, B.FP16))):
        ws = B.new_workspace(B.query_workspace_size(desc, n, 32))
        h = B.new_hits(n)

        def q():
            B.query_rays(desc, table, mlp, nodes, lv["n_nodes"], rays, 32, out=h, workspace=ws)

        q()
        torch.cuda.synchronize()
        n0 = B.launch_count()
        g = B.Graph.record(q)
        launches = B.launch_count() - n0
        for _ in range(20):
            g.launch()
        torch.cuda.synchronize()
        reps = 200
        dev_ms = timed(lambda: [g.launch() for _ in range(reps)], 1) / reps
        g.destroy()
        lat = []
        for _ in range(100):
            t0 = time.perf_counter()
            q()
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0)
        out[nm] = {"graph_device_us_per_query": dev_ms * 1e3, "eager_host_us_median": float(np.median(lat)) * 1e6,
                   "eager_host_us_p99": float(np.percentile(lat, 99)) * 1e6, "launches_per_query": launches,
                   "mrays_s_graph": n / (dev_ms * 1e-3) / 1e6}
        if nm == "fp32_plain":
            g32 = {k: v.cpu().numpy() for k, v in h.items()}
    if B.device_status() != 0:
        raise RuntimeError("device status after the latency case")
    if not args.no_cpu_baseline:
        ol = O.build_leaves(tris, spec.n_leaves, spec.inflate_rel)
        inst = [{"kind": "neural", "leaves": ol, "table": tab_np, "layers": layers,
                 "layout": O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table),
                 "n_samples": cfg.n_samples}]
        ref, dt = oracle_single("query", inst, rays_np)
        out["fp32_plain"]["accuracy_vs_oracle"] = compare_hits(g32, ref)
        out["cpu_baseline"] = {"value": n / dt / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                               "sample": f"all {n} rays, one thread, {dt:.1f} s"}
    return out


# ---------------------------------------------------------------------------- uneven segments (S6)
def time_uneven(args, world, flush, pool=None):
    """64 displaced sphere clusters (1k-200k triangles each) in one 8,192-leaf
    N-BVH; 4,194,304 rays (60% from a camera, 40% sphere chords) with 1-40
    segments each; the icosphere model in FP16. The autotuner picks the
    options on this workload; each timed step is one graph-captured query."""
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
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    total = timed(g.launch, args.uneven_steps, flush)
    g.destroy()
    st = B.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the uneven-segment queries")
    segs, _ = B.query_stats(ws, n, ms_max)
    ms = dist_max(total, world) / args.uneven_steps
    hit = cnt > 0
    cpu = None
    if pool is not None:
        from oracle import nbvh_oracle as O
        rng = np.random.default_rng(SEED + 7)
        idx = np.sort(rng.choice(n, size=min(args.accuracy_rays, n), replace=False))
        inst = [{"kind": "neural", "leaves": O.build_leaves(tris, spec.n_leaves, spec.inflate_rel),
                 "table": table.float().cpu().numpy(),
                 "layers": B.unpack_mlp(mlp.cpu().numpy(), cfg.mlp_dims()),
                 "layout": O.level_layout(cfg.n_levels, cfg.base_res, cfg.growth, cfg.log2_table),
                 "n_samples": cfg.n_samples}]
        _, wall = pool.run(pool.add_job("query", inst), W.subset(rays_np, idx))
        cpu = {"value": len(idx) / wall / 1e6, "unit": "Mrays/s", "cores": pool.n, "kind": "oracle",
               "sample": f"{len(idx)} seeded rays of the 4,194,304 (every segment evaluated), {pool.n} "
                         f"single-threaded processes, {wall:.1f} s wall"}
    return {"workload": spec.name, "value": world * n / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_query": ms,
            "cpu_baseline": cpu,
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
def time_lod(args, world, flush):
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
    out = {"workload": "icosphere-l8, LoDs every 100 steps, 2^16-ray steps, fp16; 1920x1080 primary rays + bounce",
           "training_steps": step - 1, "lods": [len(x[0]["leaf_ref"]) for x in lods],
           "bounce_rays": int(h1["hit"].sum())}
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
        total = timed(g.launch, 5, flush)
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


# ---------------------------------------------------------------------------- albedo head (NEXT-4)
def time_albedo(args, world, wl, flush):
    """The icosphere step with the albedo head (8 outputs, FP16 tensor cores):
    both queries write albedo into their hit records; and training steps with
    per-triangle albedo labels (smooth fBm colours) and the relative L2 term."""
    import torch
    from dataclasses import replace
    from paper_2405_16237_b300 import nbvh as B
    from paper_2405_16237_b300 import workloads as W
    cfg = replace(wl.spec.model, n_out=8)
    info = wl.leaves["info"]
    desc = B.model_desc(cfg, B.FP16, B.FP16, info["centre"], info["extent"])
    mlp = torch.as_tensor(B.pack_mlp(W.init_mlp(cfg.mlp_dims(), SEED + 22))).cuda()
    scene = B.DeviceScene(wl.tris, wl.leaves, albedo=W.tri_albedo(wl.tris))
    batch = 1 << 18
    opt = B.Optimizer(desc, wl.table_master.clone(), mlp, loss_scale=32768.0)
    ws = B.new_workspace(B.train_workspace_size(desc, batch, scene.n_leaves))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(1, 4):
        B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, SEED + 9, step, 1e-2, ws, loss_out=loss)
    torch.cuda.synchronize()
    n_t = 20
    ms_t = timed(lambda: B.train_step(desc, opt, scene, B.TRAIN_PROBED_MIX, batch, SEED + 9, 4, 1e-2, ws,
                                      loss_out=loss), n_t, flush) / n_t
    h1 = B.new_hits(wl.n, albedo=True)
    h2 = B.new_hits(wl.n, albedo=True)

    def step():
        B.query_rays(desc, opt.table, opt.mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays, wl.max_segs, out=h1,
                     workspace=wl.ws1)
        B.bounce_rays(wl.rays, h1, SEED + 3, out=wl.rays2)
        B.query_rays(desc, opt.table, opt.mlp, wl.nodes, wl.leaves["n_nodes"], wl.rays2, wl.max_segs, out=h2,
                     workspace=wl.ws2)

    step()
    torch.cuda.synchronize()
    g = B.Graph.record(step)
    for _ in range(args.warmup):
        g.launch()
    torch.cuda.synchronize()
    steps = max(args.steps, 5)
    total = timed(g.launch, steps, flush)
    g.destroy()
    if B.device_status() != 0:
        raise RuntimeError("device status after the albedo query")
    ms = dist_max(total, world) / steps
    rays = wl.n + int(h1["hit"].sum().item())
    a = torch.stack([h1["ar"], h1["ag"], h1["ab"]], 1)[h1["hit"] > 0]
    return {"query": {"value": world * rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms,
                      "rays_per_step": rays, "albedo_mean_on_hits": a.float().mean(0).tolist(),
                      "network": "table from the trained icosphere model, 8-output MLP after 24 albedo steps"},
            "train": {"value": dist_max_rate(batch / (ms_t * 1e-3), world), "unit": "rays/s", "batch": batch,
                      "ms_per_step": ms_t, "loss_last": float(loss.item())}}


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 oracle on the host cores, on bounded samples of the headline
    workload: per step a seeded sample of the primary rays, the hybrid trace
    over the triangle ground and the 16 neural assets (the oracle evaluates
    every segment, so its cost does not depend on the weights: the tables and
    MLPs have the trained models' shapes with seeded initial values)."""
    from paper_2405_16237_b300 import workloads as W
    w, h = (int(x) for x in args.hybrid_size.split("x"))
    t0 = time.perf_counter()
    ground, assets, oinst = build_hybrid_host()
    inst = [oinst[0]]
    for k, (a, x) in enumerate(zip(assets, oinst[1:])):
        tab = W.init_table(x["layout"]["total"], a.model.n_features, SEED + 100 + k, 1e-4)
        inst.append(dict(x, table=tab, layers=W.init_mlp(a.model.mlp_dims(), SEED + 200 + k)))
    rays_np = W.hybrid_camera_rays(w, h)
    n_all = len(rays_np["ox"])
    pool = OraclePool()
    if args.ref_rays <= 0:
        args.ref_rays = max(64, 8 * pool.n)
    try:
        job = pool.add_job("hybrid", inst)
        setup_s = time.perf_counter() - t0
        rates, secs = [], []
        for s in range(args.warmup + args.steps):
            rng = np.random.default_rng(SEED + 1000 + s)
            idx = np.sort(rng.choice(n_all, size=args.ref_rays, replace=False))
            _, wall = pool.run(job, W.subset(rays_np, idx), warm=(s == 0))
            if s >= args.warmup:
                rates.append(args.ref_rays / wall / 1e6)
                secs.append(wall)
    finally:
        pool.close()
    val = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs) * 1e3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": hybrid_name(w, h), "sample_primary_rays": args.ref_rays,
                                            "setup_s": setup_s},
            "cpu_baseline": {"value": val, "unit": "Mrays/s", "cores": pool.n, "kind": "oracle",
                             "cpu_count": os.cpu_count(),
                             "sample": f"per step {args.ref_rays} seeded primary rays of the {w}x{h} image, primary "
                                       f"pass over the ground and 16 neural assets, {pool.n} single-threaded "
                                       f"processes"},
            "e2e": {"value": val, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_init(args.gpus)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()  # a created stream: CUDA graphs cannot record the legacy default stream
    with torch.cuda.stream(stream):
        run_gpu(args, world, rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_gpu(args, world, rank):
    import torch
    from paper_2405_16237_b300 import nbvh as B
    only = args.only
    with_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline and only == "all"
    pool = OraclePool() if with_cpu else None
    clocks = ClockSampler()
    clock_state = {"started": False}

    def clocks_cb(what):
        # one sampler over every timed region (started at the first)
        if what == "start" and not clock_state["started"]:
            clocks.start()
            clock_state["started"] = True

    try:
        line = {}
        if only in ("all", "hybrid"):
            w, h = (int(x) for x in args.hybrid_size.split("x"))
            oinst = build_hybrid_host()[2] if pool is not None else None
            hy = time_hybrid(args, world, rank, clocks_cb)
            hw = hy.pop("hw")
            flush = hy.pop("flush")
            det = hybrid_details(args, world, hw, flush, pool, oinst, hy["ms_per_frame"]) if only == "all" else {}
            line = {"metric": METRIC, "value": hy["value"], "unit": "Mrays/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": hy["ms_per_frame"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                    "data": "synthetic (seeded scenes and rays; networks trained on them by the library)",
                    "config": {"workload": hybrid_name(w, h), "frame": f"{w}x{h} primary rays + "
                                                                       f"{HYBRID_BOUNCES} bounce passes",
                               "rays_per_frame": hy["rays_per_frame"], "primary_rays": hw.n,
                               "primary_hits": hy["primary_hits"], "ground_triangles": int(len(hw.ground)),
                               "assets": hw.asset_info,
                               "asset_training": {"steps": args.hybrid_train_steps, "batch": args.hybrid_train_batch,
                                                  "mode": "probed mix, BF16 tensor-core compute, FP32 masters, "
                                                          "Adam lr 1e-2", "seconds": hw.train_s},
                               "l2": "flushed (256 MB write) between timed frames",
                               "parallelism": f"replicas x{world}"},
                    "gpu_launches": int(hy["launches_per_frame"] * args.steps)}
            line.update({k: det[k] for k in ("roofline", "e2e", "cpu_baseline", "cpu_baseline_single",
                                             "accuracy_vs_oracle", "kernels", "segments_per_frame") if k in det})
            del hw
            torch.cuda.empty_cache()
        if only in ("all", "icosphere", "train"):
            spec, tris, rays_np = make_scene(args.primary)
            wl = GpuWorkload(spec, tris, rays_np, args.max_segs)
            flush = Flusher()
            args._ran = ()
            if args.train_steps > 0 and only in ("all", "train"):
                line["train"] = train_icosphere(args, world, wl, flush)
                args._ran = ("train",)
            if only in ("all", "icosphere"):
                line["icosphere"] = time_icosphere(args, world, rank, wl, flush, pool, clocks_cb)
                if not line.get("value"):
                    line.update({"metric": METRIC, "value": line["icosphere"]["value"], "unit": "Mrays/s",
                                 "ms_per_step": line["icosphere"]["ms_per_step"], "config": {
                                     "workload": spec.name}})
            if only == "all":
                line["uneven"] = time_uneven(args, world, flush, pool) if args.uneven_steps > 0 else None
                line["cut_optimization"] = time_cut(args, world) if args.cut_steps > 0 else None
                line["levels_of_detail"] = time_lod(args, world, flush) if args.lod_steps > 0 else None
                line["albedo_head"] = time_albedo(args, world, wl, flush) if not args.no_albedo else None
            wl.drop_graphs()
            del wl
            torch.cuda.empty_cache()
        if only in ("all", "latency"):
            line["latency_4096_rays"] = time_latency(args, world, Flusher())
        if only == "uneven":
            line["uneven"] = time_uneven(args, world, Flusher())
        if B.device_status() != 0:
            raise RuntimeError("device status at the end of the run")
    finally:
        clk = clocks.stop()
        if pool is not None:
            pool.close()
    line["clocks"] = clk
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
