"""Python binding of libnbvh.so (include/nbvh.h): argument marshalling only.

Every step of the neural ray query runs in the library's kernels. PyTorch
provides device memory and the current CUDA stream. Loading fails loudly when
the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_float, c_int32, c_int64, c_size_t, c_uint8, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbvh.so")

FP32, FP16, BF16 = 0, 1, 2
MAX_LEVELS = 32

STATUS = {
    0: "NBVH_OK", 1: "NBVH_ERR_INVALID_ARG", 2: "NBVH_ERR_CUDA", 3: "NBVH_ERR_OOM",
    4: "NBVH_ERR_WORKSPACE_TOO_SMALL", 5: "NBVH_ERR_SEGMENT_OVERFLOW", 6: "NBVH_ERR_TIMEOUT",
    7: "NBVH_ERR_UNSUPPORTED",
}


class NBVHError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class ModelDesc(ctypes.Structure):
    _fields_ = [("n_levels", c_int32), ("n_features", c_int32), ("log2_table", c_int32),
                ("base_res", c_int32), ("growth", c_float), ("n_samples", c_int32),
                ("n_hidden", c_int32), ("width", c_int32), ("n_out", c_int32),
                ("table_prec", c_int32), ("mlp_prec", c_int32), ("frame_centre", c_float * 3),
                ("frame_extent", c_float), ("flags", c_int32)]


FLAG_REVERSE_INSIDE = 1


class Rays(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")] + [("n", c_int64)]


HIT_KEYS = ("hit", "t", "nx", "ny", "nz", "leaf")
ALBEDO_KEYS = ("ar", "ag", "ab")


class Hits(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in HIT_KEYS + ALBEDO_KEYS]


class RaysOut(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")] + [("n", c_int64)]


class Node(ctypes.Structure):
    _fields_ = [("lo0", c_float * 3), ("hi0", c_float * 3), ("lo1", c_float * 3), ("hi1", c_float * 3),
                ("child0", c_int32), ("child1", c_int32), ("pad", c_int32 * 2)]


class SceneInfo(ctypes.Structure):
    _fields_ = [("lo", c_float * 3), ("hi", c_float * 3), ("centre", c_float * 3), ("extent", c_float),
                ("sphere_radius", c_float)]


class TrainScene(ctypes.Structure):
    _fields_ = [("nodes", c_void_p), ("n_nodes", c_int32), ("leaf_box", c_void_p), ("n_leaves", c_int32),
                ("tris", c_void_p), ("tri_perm", c_void_p), ("leaf_range", c_void_p), ("leaf_tris", c_void_p),
                ("info", SceneInfo), ("tri_albedo", c_void_p)]


LABEL_KEYS = ("hit", "depth", "nx", "ny", "nz")


class Labels(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in LABEL_KEYS + ALBEDO_KEYS]


class Optim(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ("table_master", "table_work", "table_m", "table_v", "grad_table", "mlp",
                                        "mlp_m", "mlp_v", "grad_mlp", "loss_scale", "counters")]


TRAIN_PROBED_MIX, TRAIN_PAPER = 0, 1


class LeafStats(ctypes.Structure):
    _fields_ = [("hits", c_void_p), ("trained", c_void_p), ("loss", c_void_p)]


class QueryOptions(ctypes.Structure):
    _fields_ = [("schedule", c_int32), ("patience_cycles", c_int64), ("traverse_block", c_int32),
                ("eval_threads", c_int32), ("w1_mode", c_int32), ("eval_pipeline", c_int32),
                ("wait_spins", c_int64), ("test_phantom_items", c_int32), ("segments_out", c_void_p),
                ("instance_streams", c_int32), ("partial_items", c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("opt", QueryOptions), ("ms", c_float)]


class TriBlas(ctypes.Structure):
    _fields_ = [("nodes", c_void_p), ("n_nodes", c_int32), ("tris", c_void_p), ("leaf_range", c_void_p),
                ("tri_id", c_void_p), ("albedo", c_void_p)]


class Instance(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("tri", TriBlas), ("desc", ModelDesc), ("table", c_void_p), ("mlp", c_void_p),
                ("nodes", c_void_p), ("n_nodes", c_int32), ("max_segs", c_int32)]


BLAS_TRIANGLES, BLAS_NEURAL = 0, 1

_lib = None

_SIGS = {
    "nbvh_status_string": (ctypes.c_char_p, [c_int32]),
    "nbvh_version": (c_int32, []),
    "nbvh_built_arch": (c_int32, []),
    "nbvh_level_layout": (c_int32, [POINTER(ModelDesc), POINTER(c_int32), POINTER(c_int32), POINTER(c_int64),
                                    POINTER(c_int64), POINTER(c_int64)]),
    "nbvh_mlp_param_count": (c_int32, [POINTER(ModelDesc), POINTER(c_int64)]),
    "nbvh_build_leaves": (c_int32, [c_void_p, c_int64, c_int32, c_double, c_void_p, c_int32, POINTER(c_int32),
                                    c_void_p, c_void_p, c_void_p, POINTER(SceneInfo)]),
    "nbvh_traverse": (c_int32, [c_void_p, c_int32, Rays, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p]),
    "nbvh_encode": (c_int32, [POINTER(ModelDesc), c_void_p, Rays, c_void_p, c_void_p, c_void_p, c_int64,
                              c_void_p, c_void_p]),
    "nbvh_query_options_default": (c_int32, [POINTER(QueryOptions)]),
    "nbvh_eval_workspace_size": (c_int32, [POINTER(ModelDesc), POINTER(c_size_t)]),
    "nbvh_eval_plan": (c_int32, [POINTER(ModelDesc), POINTER(QueryOptions), POINTER(c_int32), POINTER(c_int32),
                                 POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "nbvh_eval_segments": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, Rays, c_void_p, c_void_p, c_void_p,
                                     c_int64, c_void_p, POINTER(QueryOptions), c_void_p, c_size_t, c_void_p]),
    "nbvh_query_workspace_size": (c_int32, [POINTER(ModelDesc), c_int64, c_int32, POINTER(c_size_t)]),
    "nbvh_query_rays": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, c_void_p, c_int32, Rays, c_int32,
                                  Hits, c_void_p, c_size_t, c_void_p]),
    "nbvh_query_rays_opt": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, c_void_p, c_int32, Rays, c_int32,
                                      Hits, c_void_p, c_size_t, POINTER(QueryOptions), c_void_p]),
    "nbvh_bounce_rays": (c_int32, [Rays, Hits, ctypes.c_uint64, RaysOut, c_void_p]),
    "nbvh_autotune_query": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, c_void_p, c_int32, Rays, c_int32, Hits,
                                      c_void_p, c_size_t, c_int32, POINTER(TuneResult), POINTER(TuneResult), c_int32,
                                      POINTER(c_int32), c_void_p]),
    "nbvh_query_stats": (c_int32, [c_void_p, c_int64, c_int32, POINTER(c_int64), POINTER(c_int32), c_void_p]),
    "nbvh_set_timing": (c_int32, [c_int32]),
    "nbvh_get_kernel_times": (c_int32, [POINTER(c_double), POINTER(c_int64), POINTER(c_int64), c_int32]),
    "nbvh_launch_count": (c_int64, []),
    "nbvh_query_rays_static": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, c_void_p, c_int32, Rays, c_int32,
                                         Hits, c_void_p]),
    "nbvh_train_rays": (c_int32, [c_int32, ctypes.c_uint64, c_int64, POINTER(TrainScene), RaysOut, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p]),
    "nbvh_train_labels": (c_int32, [Rays, c_void_p, c_void_p, c_void_p, POINTER(TrainScene), Labels, c_void_p]),
    "nbvh_train_workspace_size": (c_int32, [POINTER(ModelDesc), c_int64, c_int32, POINTER(c_size_t)]),
    "nbvh_train_workspace_budget": (c_int32, [POINTER(ModelDesc), c_int64, c_int32, c_size_t, POINTER(c_size_t),
                                              POINTER(c_int64)]),
    "nbvh_loss_fp64": (c_int32, [POINTER(ModelDesc), c_int64, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "nbvh_forward_train": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, Rays, c_void_p, c_void_p, c_void_p,
                                     Labels, c_void_p, c_float, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                     c_void_p]),
    "nbvh_backward": (c_int32, [POINTER(ModelDesc), c_void_p, c_void_p, Rays, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nbvh_adam": (c_int32, [POINTER(ModelDesc), POINTER(Optim), c_int64, c_float, c_float, c_float, c_float, c_int32,
                            c_void_p]),
    "nbvh_train_step": (c_int32, [POINTER(ModelDesc), POINTER(Optim), POINTER(TrainScene), c_int32, c_int64,
                                  ctypes.c_uint64, c_int64, c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nbvh_train_step_weighted": (c_int32, [POINTER(ModelDesc), POINTER(Optim), POINTER(TrainScene), c_int32,
                                           c_int64, ctypes.c_uint64, c_int64, c_float, c_void_p, c_void_p, c_void_p,
                                           c_void_p, c_size_t, c_void_p]),
    "nbvh_build_cut": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_double, c_float,
                                 c_void_p, c_int32, POINTER(c_int32), c_void_p, c_void_p, c_void_p]),
    "nbvh_rank_leaves": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "nbvh_refine_cut": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p,
                                  c_void_p, c_int32, POINTER(c_int32)]),
    "nbvh_graph_begin": (c_int32, [c_void_p]),
    "nbvh_graph_end": (c_int32, [c_void_p, POINTER(c_void_p)]),
    "nbvh_graph_launch": (c_int32, [c_void_p, c_void_p]),
    "nbvh_graph_destroy": (c_int32, [c_void_p]),
    "nbvh_build_tri_blas": (c_int32, [c_void_p, c_int64, c_int32, c_void_p, c_int32, POINTER(c_int32), c_void_p,
                                      c_void_p, c_int32, POINTER(c_int32)]),
    "nbvh_trace_triangles": (c_int32, [POINTER(TriBlas), Rays, Hits, c_void_p]),
    "nbvh_hybrid_workspace_size": (c_int32, [POINTER(Instance), c_int32, c_int64, POINTER(c_size_t)]),
    "nbvh_hybrid_trace": (c_int32, [POINTER(Instance), c_int32, Rays, Hits, c_void_p, c_void_p, c_size_t,
                                    POINTER(QueryOptions), c_void_p]),
    "nbvh_probe_l2_gather": (c_int32, [c_void_p, c_int64, c_void_p, POINTER(c_double), c_void_p]),
    "nbvh_probe_l2_reduce": (c_int32, [c_void_p, c_int64, POINTER(c_double), c_void_p]),
    "nbvh_get_device_status": (c_int32, [c_void_p]),
}

STATIC_SCRATCH_BYTES = 33554432

EXPORTED = tuple(_SIGS)


def lib():
    """The loaded library; raises if it is missing (build it with build_lib.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libnbvh.so not built ({LIB_PATH}); run paper_2405_16237_b300.build_lib.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise NBVHError(code, what)


# ---------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _stream():
    torch = _torch()
    return c_void_p(torch.cuda.current_stream().cuda_stream)


TORCH_DTYPE = {FP32: "float32", FP16: "float16", BF16: "bfloat16"}


def table_dtype(prec: int):
    return getattr(_torch(), TORCH_DTYPE[prec])


# ---------------------------------------------------------------- model description
def model_desc(cfg, table_prec: int, mlp_prec: int, centre, extent) -> ModelDesc:
    d = ModelDesc()
    d.n_levels = cfg.n_levels
    d.n_features = cfg.n_features
    d.log2_table = cfg.log2_table
    d.base_res = cfg.base_res
    d.growth = cfg.growth
    d.n_samples = cfg.n_samples
    d.n_hidden = cfg.n_hidden
    d.width = cfg.width
    d.n_out = cfg.n_out
    d.table_prec = table_prec
    d.mlp_prec = mlp_prec
    for i in range(3):
        d.frame_centre[i] = float(centre[i])
    d.frame_extent = float(extent)
    return d


def with_mlp_prec(desc: ModelDesc, mlp_prec: int) -> ModelDesc:
    d = ModelDesc()
    ctypes.pointer(d)[0] = desc
    d.mlp_prec = mlp_prec
    return d


def with_flags(desc: ModelDesc, flags: int) -> ModelDesc:
    d = ModelDesc()
    ctypes.pointer(d)[0] = desc
    d.flags = flags
    return d


def level_layout(desc: ModelDesc) -> dict:
    res = (c_int32 * MAX_LEVELS)()
    dense = (c_int32 * MAX_LEVELS)()
    size = (c_int64 * MAX_LEVELS)()
    off = (c_int64 * MAX_LEVELS)()
    total = c_int64()
    _check(lib().nbvh_level_layout(ctypes.byref(desc), res, dense, size, off, ctypes.byref(total)), "level_layout")
    L = desc.n_levels
    return {"res": np.array(res[:L], np.int64), "dense": np.array(dense[:L], bool),
            "size": np.array(size[:L], np.int64), "offset": np.array(off[:L], np.int64), "total": total.value}


def mlp_param_count(desc: ModelDesc) -> int:
    n = c_int64()
    _check(lib().nbvh_mlp_param_count(ctypes.byref(desc), ctypes.byref(n)), "mlp_param_count")
    return n.value


def pack_mlp(layers) -> np.ndarray:
    """Flatten [(W [out,in], b [out])] into the library's float parameter order."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32)])
                           for w, b in layers]).astype(np.float32)


def unpack_mlp(flat, dims):
    """The library's flat parameter order back to [(W [out, in], b [out])]
    float32 arrays (the inverse of pack_mlp)."""
    flat = np.asarray(flat, np.float32)
    layers, off = [], 0
    for i in range(len(dims) - 1):
        w = flat[off:off + dims[i + 1] * dims[i]].reshape(dims[i + 1], dims[i])
        off += dims[i + 1] * dims[i]
        b = flat[off:off + dims[i + 1]]
        off += dims[i + 1]
        layers.append((w.copy(), b.copy()))
    if off != len(flat):
        raise ValueError("parameter count does not match the layer sizes")
    return layers


# ---------------------------------------------------------------- leaf build (host)
def build_leaves(tris: np.ndarray, n_leaves: int, inflate_rel: float = 1e-4) -> dict:
    tris = np.ascontiguousarray(tris, np.float32)
    n = len(tris)
    cap = max(1, n_leaves - 1)
    nodes = (Node * cap)()
    n_nodes = c_int32()
    perm = np.zeros(n, np.int32)
    rng = np.zeros(2 * n_leaves, np.int32)
    box = np.zeros((n_leaves, 6), np.float32)
    info = SceneInfo()
    _check(lib().nbvh_build_leaves(tris.ctypes.data_as(c_void_p), n, n_leaves, float(inflate_rel), nodes, cap,
                                   ctypes.byref(n_nodes), perm.ctypes.data_as(c_void_p),
                                   rng.ctypes.data_as(c_void_p), box.ctypes.data_as(c_void_p),
                                   ctypes.byref(info)), "build_leaves")
    node_bytes = np.frombuffer(bytes(nodes), np.uint8).copy()
    return {
        "nodes": node_bytes, "n_nodes": n_nodes.value, "tri_perm": perm, "leaf_range": rng.reshape(-1, 2),
        "leaf_lo": box[:, :3].copy(), "leaf_hi": box[:, 3:].copy(),
        "info": {"lo": np.array(info.lo[:]), "hi": np.array(info.hi[:]), "centre": np.array(info.centre[:]),
                 "extent": info.extent, "sphere_radius": info.sphere_radius},
    }


def node_array(leaves: dict) -> np.ndarray:
    """Nodes as a structured view (lo0, hi0, lo1, hi1, child0, child1)."""
    dt = np.dtype([("lo0", "<f4", 3), ("hi0", "<f4", 3), ("lo1", "<f4", 3), ("hi1", "<f4", 3),
                   ("child0", "<i4"), ("child1", "<i4"), ("pad", "<i4", 2)])
    return leaves["nodes"].view(dt)


# ---------------------------------------------------------------- device calls
RAY_KEYS = ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")


def to_device_rays(rays: dict, device="cuda"):
    torch = _torch()
    return {k: torch.as_tensor(np.ascontiguousarray(rays[k], np.float32), device=device) for k in RAY_KEYS}


def rays_struct(rays: dict) -> Rays:
    r = Rays()
    for k in RAY_KEYS:
        setattr(r, k, rays[k].data_ptr())
    r.n = rays["ox"].numel()
    return r


def new_hits(n: int, device="cuda", albedo: bool = False) -> dict:
    """Device hit record of n rays; albedo=True adds the ar/ag/ab arrays."""
    torch = _torch()
    h = {"hit": torch.empty(n, dtype=torch.uint8, device=device),
         "t": torch.empty(n, dtype=torch.float32, device=device),
         "nx": torch.empty(n, dtype=torch.float32, device=device),
         "ny": torch.empty(n, dtype=torch.float32, device=device),
         "nz": torch.empty(n, dtype=torch.float32, device=device),
         "leaf": torch.empty(n, dtype=torch.int32, device=device)}
    if albedo:
        for k in ALBEDO_KEYS:
            h[k] = torch.empty(n, dtype=torch.float32, device=device)
    return h


def hits_struct(h: dict) -> Hits:
    s = Hits()
    for k in HIT_KEYS:
        setattr(s, k, h[k].data_ptr())
    if "ar" in h:
        for k in ALBEDO_KEYS:
            setattr(s, k, h[k].data_ptr())
    return s


def traverse(nodes, n_nodes: int, rays: dict, max_segs: int, out=None):
    torch = _torch()
    n = rays["ox"].numel()
    dev = rays["ox"].device
    if out is None:
        out = {"count": torch.empty(n, dtype=torch.int32, device=dev),
               "leaf": torch.empty(max_segs * n, dtype=torch.int32, device=dev),
               "t0": torch.empty(max_segs * n, dtype=torch.float32, device=dev),
               "t1": torch.empty(max_segs * n, dtype=torch.float32, device=dev)}
    _check(lib().nbvh_traverse(_ptr(nodes), n_nodes, rays_struct(rays), max_segs, _ptr(out["count"]),
                               _ptr(out["leaf"]), _ptr(out["t0"]), _ptr(out["t1"]), _stream()), "traverse")
    return out


def encode(desc: ModelDesc, table, rays: dict, seg_ray, t0, t1, out=None):
    torch = _torch()
    n = seg_ray.numel()
    K = desc.n_samples * desc.n_levels * desc.n_features
    if out is None:
        out = torch.empty((n, K), dtype=torch.float32, device=seg_ray.device)
    _check(lib().nbvh_encode(ctypes.byref(desc), _ptr(table), rays_struct(rays), _ptr(seg_ray), _ptr(t0), _ptr(t1),
                             n, _ptr(out), _stream()), "encode")
    return out


def eval_plan(desc: ModelDesc, options=None):
    """nbvh_eval_plan: the evaluation's launch plan as a dict, or None when
    the kernels cannot run this model under these options."""
    th, st, sm, tm, pl = c_int32(), c_int32(), c_int32(), c_int32(), c_int32()
    code = lib().nbvh_eval_plan(ctypes.byref(desc), _opt_ref(options), ctypes.byref(th), ctypes.byref(st),
                                ctypes.byref(sm), ctypes.byref(tm), ctypes.byref(pl))
    if code == 7:
        return None
    _check(code, "eval_plan")
    return {"threads": th.value, "w1_streamed": bool(st.value), "smem_bytes": sm.value, "tmem_cols": tm.value,
            "pipeline": PIPELINES[pl.value]}


def eval_workspace_size(desc: ModelDesc) -> int:
    b = c_size_t()
    _check(lib().nbvh_eval_workspace_size(ctypes.byref(desc), ctypes.byref(b)), "eval_workspace_size")
    return b.value


def eval_segments(desc: ModelDesc, table, mlp, rays: dict, seg_ray, t0, t1, out=None, options=None, workspace=None):
    torch = _torch()
    n = seg_ray.numel()
    if out is None:
        out = torch.empty((n, desc.n_out), dtype=torch.float32, device=seg_ray.device)
    need = eval_workspace_size(desc)
    if workspace is None and need > 0:
        workspace = new_workspace(need, seg_ray.device)
    base = aligned_ptr(workspace) if workspace is not None else None
    avail = workspace.numel() - (base - workspace.data_ptr()) if workspace is not None else 0
    _check(lib().nbvh_eval_segments(ctypes.byref(desc), _ptr(table), _ptr(mlp), rays_struct(rays), _ptr(seg_ray),
                                    _ptr(t0), _ptr(t1), n, _ptr(out), _opt_ref(options),
                                    c_void_p(base) if base else None, avail, _stream()), "eval_segments")
    return out


def query_workspace_size(desc: ModelDesc, n_rays: int, max_segs: int) -> int:
    b = c_size_t()
    _check(lib().nbvh_query_workspace_size(ctypes.byref(desc), n_rays, max_segs, ctypes.byref(b)),
           "query_workspace_size")
    return b.value


def new_workspace(nbytes: int, device="cuda"):
    torch = _torch()
    return torch.empty(max(256, nbytes + 256), dtype=torch.uint8, device=device)


def aligned_ptr(ws) -> int:
    p = ws.data_ptr()
    return (p + 255) & ~255


SCHEDULE_WAVES, SCHEDULE_PERSISTENT = 0, 1
W1_AUTO, W1_RESIDENT, W1_STREAMED = 0, 1, 2
PIPELINE_AUTO, PIPELINE_PHASES, PIPELINE_WARP_SPECIALISED = 0, 1, 2
PIPELINES = ("auto", "phases", "warp_specialised")


def query_options(**kw) -> QueryOptions:
    """nbvh_query_options_default with the given fields replaced (schedule,
    patience_cycles, traverse_block, eval_threads, w1_mode, eval_pipeline,
    wait_spins, test_phantom_items; segments_out: a device int64 tensor)."""
    o = QueryOptions()
    _check(lib().nbvh_query_options_default(ctypes.byref(o)), "query_options_default")
    for k, v in kw.items():
        if k == "segments_out" and v is not None and not isinstance(v, int):
            assert v.dtype == _torch().int64 and v.is_cuda and v.is_contiguous()
            v = v.data_ptr()
        setattr(o, k, v)
    return o


def options_dict(o: QueryOptions) -> dict:
    return {"schedule": ["waves", "persistent"][o.schedule], "patience_cycles": o.patience_cycles,
            "traverse_block": o.traverse_block, "eval_threads": o.eval_threads,
            "w1_mode": ["auto", "resident", "streamed"][o.w1_mode], "eval_pipeline": PIPELINES[o.eval_pipeline],
            "instance_streams": o.instance_streams, "partial_items": o.partial_items}


def options_from_dict(d: dict) -> QueryOptions:
    return query_options(schedule=["waves", "persistent"].index(d["schedule"]), patience_cycles=d["patience_cycles"],
                         traverse_block=d["traverse_block"], eval_threads=d["eval_threads"],
                         w1_mode=["auto", "resident", "streamed"].index(d["w1_mode"]),
                         eval_pipeline=PIPELINES.index(d.get("eval_pipeline", "auto")),
                         instance_streams=d.get("instance_streams", 0), partial_items=d.get("partial_items", 0))


def _opt_ref(options):
    if options is None:
        return None
    if isinstance(options, dict):
        options = options_from_dict(options)
    return ctypes.byref(options)


def query_rays(desc: ModelDesc, table, mlp, nodes, n_nodes: int, rays: dict, max_segs: int, out=None,
               workspace=None, options=None):
    n = rays["ox"].numel()
    if out is None:
        out = new_hits(n, rays["ox"].device, albedo=desc.n_out >= 8)
    need = query_workspace_size(desc, n, max_segs)
    if workspace is None:
        workspace = new_workspace(need, rays["ox"].device)
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    _check(lib().nbvh_query_rays_opt(ctypes.byref(desc), _ptr(table), _ptr(mlp), _ptr(nodes), n_nodes,
                                     rays_struct(rays), max_segs, hits_struct(out), c_void_p(base), avail,
                                     _opt_ref(options), _stream()), "query_rays")
    return out


def device_status() -> int:
    """Reads and clears the device status word (synchronises the current stream)."""
    return int(lib().nbvh_get_device_status(_stream()))


def new_rays(n: int, device="cuda") -> dict:
    torch = _torch()
    return {k: torch.empty(n, dtype=torch.float32, device=device) for k in RAY_KEYS}


def bounce_rays(rays: dict, hits: dict, seed: int, out=None):
    n = rays["ox"].numel()
    if out is None:
        out = new_rays(n, rays["ox"].device)
    o = RaysOut()
    for k in RAY_KEYS:
        setattr(o, k, out[k].data_ptr())
    o.n = n
    _check(lib().nbvh_bounce_rays(rays_struct(rays), hits_struct(hits), ctypes.c_uint64(seed), o, _stream()),
           "bounce_rays")
    return out


def _tune_dict(r: TuneResult) -> dict:
    d = options_dict(r.opt)
    d["ms"] = r.ms
    return d


def autotune_query(desc: ModelDesc, table, mlp, nodes, n_nodes: int, rays: dict, max_segs: int, out=None,
                   workspace=None, reps: int = 3):
    """nbvh_autotune_query: times the query under each candidate option set
    and returns (best, [all candidates]) as dicts (options_from_dict turns
    one back into options); the library keeps no state."""
    n = rays["ox"].numel()
    if out is None:
        out = new_hits(n, rays["ox"].device, albedo=desc.n_out >= 8)
    if workspace is None:
        workspace = new_workspace(query_workspace_size(desc, n, max_segs), rays["ox"].device)
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    best = TuneResult()
    cap = 32
    arr = (TuneResult * cap)()
    n_all = c_int32()
    _check(lib().nbvh_autotune_query(ctypes.byref(desc), _ptr(table), _ptr(mlp), _ptr(nodes), n_nodes,
                                     rays_struct(rays), max_segs, hits_struct(out), c_void_p(base), avail, reps,
                                     ctypes.byref(best), arr, cap, ctypes.byref(n_all), _stream()), "autotune_query")
    return _tune_dict(best), [_tune_dict(arr[i]) for i in range(min(cap, n_all.value))]


def query_stats(workspace, n_rays: int, max_segs: int):
    segs = c_int64()
    waves = c_int32()
    _check(lib().nbvh_query_stats(c_void_p(aligned_ptr(workspace)), n_rays, max_segs, ctypes.byref(segs),
                                  ctypes.byref(waves), _stream()), "query_stats")
    return segs.value, waves.value


def set_timing(enable: bool):
    _check(lib().nbvh_set_timing(1 if enable else 0), "set_timing")


# kernel classes of the library's timing (NBVH_KERNEL_* in the header)
KERNEL_KINDS = ("traverse", "eval", "tri_trace", "tlas_cull", "bounce", "train_rays", "labels", "train_forward",
                "train_backward", "weight_grad", "adam", "other")


def get_kernel_times() -> dict:
    """Per kernel class, since the previous call: summed milliseconds of the
    timed groups, the number of groups and the kernels they launched."""
    n = len(KERNEL_KINDS)
    ms = (c_double * n)()
    sec = (c_int64 * n)()
    lau = (c_int64 * n)()
    _check(lib().nbvh_get_kernel_times(ms, sec, lau, n), "get_kernel_times")
    return {k: {"ms": ms[i], "groups": int(sec[i]), "launches": int(lau[i])} for i, k in enumerate(KERNEL_KINDS)}


def launch_count() -> int:
    return int(lib().nbvh_launch_count())


def query_rays_static(desc: ModelDesc, table, mlp, nodes, n_nodes: int, rays: dict, max_segs: int, out=None):
    """nbvh_query_rays_static: the query with the library's built-in scratch,
    for callers that cannot allocate device memory (see include/nbvh.h)."""
    n = rays["ox"].numel()
    if out is None:
        out = new_hits(n, rays["ox"].device, albedo=desc.n_out >= 8)
    _check(lib().nbvh_query_rays_static(ctypes.byref(desc), _ptr(table), _ptr(mlp), _ptr(nodes), n_nodes,
                                        rays_struct(rays), max_segs, hits_struct(out), _stream()),
           "query_rays_static")
    return out


# ---------------------------------------------------------------- training
class DeviceScene:
    """Device copies of the geometry the training step reads."""

    def __init__(self, tris: np.ndarray, leaves: dict, device="cuda", albedo: np.ndarray = None):
        """albedo: optional [n_tris][3] RGB in [0, 1]; the labels then carry
        the hit triangle's albedo (trained by a model with n_out = 8)."""
        torch = _torch()
        self.tris = torch.as_tensor(np.ascontiguousarray(tris, np.float32).reshape(-1, 9), device=device)
        self.albedo = None if albedo is None else torch.as_tensor(
            np.ascontiguousarray(albedo, np.float32).reshape(-1, 3), device=device)
        self.nodes = torch.as_tensor(leaves["nodes"], device=device)
        box = np.concatenate([leaves["leaf_lo"], leaves["leaf_hi"]], 1).astype(np.float32)
        self.leaf_box = torch.as_tensor(np.ascontiguousarray(box), device=device)
        self.tri_perm = torch.as_tensor(leaves["tri_perm"], device=device)
        self.leaf_range = torch.as_tensor(np.ascontiguousarray(leaves["leaf_range"], np.int32), device=device)
        self.leaf_tris = self.tris[self.tri_perm.long()].contiguous()
        self.n_nodes = leaves["n_nodes"]
        self.n_leaves = len(leaves["leaf_lo"])
        sc = TrainScene()
        sc.nodes = self.nodes.data_ptr()
        sc.n_nodes = self.n_nodes
        sc.leaf_box = self.leaf_box.data_ptr()
        sc.n_leaves = self.n_leaves
        sc.tris = self.tris.data_ptr()
        sc.tri_perm = self.tri_perm.data_ptr()
        sc.leaf_range = self.leaf_range.data_ptr()
        sc.leaf_tris = self.leaf_tris.data_ptr()
        sc.tri_albedo = self.albedo.data_ptr() if self.albedo is not None else None
        inf = leaves["info"]
        for i in range(3):
            sc.info.lo[i] = float(inf["lo"][i])
            sc.info.hi[i] = float(inf["hi"][i])
            sc.info.centre[i] = float(inf["centre"][i])
        sc.info.extent = float(inf["extent"])
        sc.info.sphere_radius = float(inf["sphere_radius"])
        self.struct = sc


def train_rays(mode: int, seed: int, step: int, scene: DeviceScene, n: int):
    torch = _torch()
    dev = scene.nodes.device
    rays = new_rays(n, dev)
    leaf = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = torch.empty(n, dtype=torch.float32, device=dev)
    t1 = torch.empty(n, dtype=torch.float32, device=dev)
    n_valid = torch.zeros(1, dtype=torch.int32, device=dev)
    o = RaysOut()
    for k in RAY_KEYS:
        setattr(o, k, rays[k].data_ptr())
    o.n = n
    _check(lib().nbvh_train_rays(mode, ctypes.c_uint64(seed), step, ctypes.byref(scene.struct), o, _ptr(leaf),
                                 _ptr(t0), _ptr(t1), _ptr(n_valid), _stream()), "train_rays")
    return rays, leaf, t0, t1, n_valid


def new_labels(n: int, device="cuda", albedo: bool = False) -> dict:
    torch = _torch()
    keys = ("depth", "nx", "ny", "nz") + (ALBEDO_KEYS if albedo else ())
    return {"hit": torch.empty(n, dtype=torch.uint8, device=device),
            **{k: torch.empty(n, dtype=torch.float32, device=device) for k in keys}}


def labels_struct(lab) -> Labels:
    s = Labels()
    if lab is not None:
        for k in LABEL_KEYS + (ALBEDO_KEYS if "ar" in lab else ()):
            setattr(s, k, lab[k].data_ptr())
    return s


def train_labels(rays: dict, leaf, t0, t1, scene: DeviceScene, out=None):
    n = rays["ox"].numel()
    if out is None:
        out = new_labels(n, rays["ox"].device, albedo=scene.albedo is not None)
    _check(lib().nbvh_train_labels(rays_struct(rays), _ptr(leaf), _ptr(t0), _ptr(t1), ctypes.byref(scene.struct),
                                   labels_struct(out), _stream()), "train_labels")
    return out


def train_workspace_size(desc: ModelDesc, n: int, n_leaves: int = 0) -> int:
    b = c_size_t()
    _check(lib().nbvh_train_workspace_size(ctypes.byref(desc), n, n_leaves, ctypes.byref(b)),
           "train_workspace_size")
    return b.value


def train_workspace_budget(desc: ModelDesc, n: int, n_leaves: int, max_bytes: int):
    """(bytes, rays per activation chunk) of a training workspace within
    max_bytes: the stored mode (chunk = n) when it fits, else recompute mode."""
    b, c = c_size_t(), c_int64()
    _check(lib().nbvh_train_workspace_budget(ctypes.byref(desc), n, n_leaves, max_bytes, ctypes.byref(b),
                                             ctypes.byref(c)), "train_workspace_budget")
    return b.value, c.value


def workspace_bytes(workspace) -> int:
    """Usable bytes of a workspace tensor from its 256-byte aligned start."""
    base = aligned_ptr(workspace)
    return workspace.numel() - (base - workspace.data_ptr())


def loss_fp64(desc: ModelDesc, n: int, n_valid, workspace, out):
    """nbvh_loss_fp64: the last forward's loss with FP64 accumulation (the
    finite-difference check's reduction); out: device float64 scalar."""
    _check(lib().nbvh_loss_fp64(ctypes.byref(desc), n, _ptr(n_valid), c_void_p(aligned_ptr(workspace)),
                                workspace_bytes(workspace), _ptr(out), _stream()), "loss_fp64")


def forward_train(desc: ModelDesc, table, mlp, rays: dict, leaf, t0, t1, workspace, labels=None, n_valid=None,
                  loss_scale: float = 1.0, loss_scale_dev=None, raw_out=None, loss_out=None):
    torch = _torch()
    n = rays["ox"].numel()
    if raw_out is None:
        raw_out = torch.empty((n, desc.n_out), dtype=torch.float32, device=rays["ox"].device)
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    _check(lib().nbvh_forward_train(ctypes.byref(desc), _ptr(table), _ptr(mlp), rays_struct(rays), _ptr(leaf),
                                    _ptr(t0), _ptr(t1), labels_struct(labels), _ptr(n_valid), float(loss_scale),
                                    _ptr(loss_scale_dev), _ptr(raw_out), _ptr(loss_out), c_void_p(base), avail,
                                    _stream()), "forward_train")
    return raw_out


def backward(desc: ModelDesc, table, mlp, rays: dict, leaf, t0, t1, workspace, grad_table, grad_mlp,
             grad_out=None):
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    _check(lib().nbvh_backward(ctypes.byref(desc), _ptr(table), _ptr(mlp), rays_struct(rays), _ptr(leaf), _ptr(t0),
                               _ptr(t1), _ptr(grad_out), _ptr(grad_table), _ptr(grad_mlp), c_void_p(base), avail,
                               _stream()), "backward")


class Optimizer:
    """FP32 master parameters, Adam moments, gradients and the loss scale, all
    device tensors owned here and handed to the library as plain pointers."""

    def __init__(self, desc: ModelDesc, table_master, mlp, loss_scale: float = 1.0):
        torch = _torch()
        self.desc = desc
        self.table_master = table_master.contiguous()
        dev = self.table_master.device
        self.table_work = None
        if desc.table_prec != FP32:
            self.table_work = self.table_master.to(table_dtype(desc.table_prec))
        self.table_m = torch.zeros_like(self.table_master)
        self.table_v = torch.zeros_like(self.table_master)
        self.grad_table = torch.zeros_like(self.table_master)
        self.mlp = mlp.contiguous()
        self.mlp_m = torch.zeros_like(self.mlp)
        self.mlp_v = torch.zeros_like(self.mlp)
        self.grad_mlp = torch.zeros_like(self.mlp)
        self.loss_scale = torch.tensor([loss_scale], dtype=torch.float32, device=dev)
        self.counters = torch.zeros(4, dtype=torch.int32, device=dev)
        o = Optim()
        for k in ("table_master", "table_m", "table_v", "grad_table", "mlp", "mlp_m", "mlp_v", "grad_mlp",
                  "loss_scale", "counters"):
            setattr(o, k, getattr(self, k).data_ptr())
        o.table_work = self.table_work.data_ptr() if self.table_work is not None else None
        self.struct = o

    @property
    def table(self):
        return self.table_work if self.table_work is not None else self.table_master

    def adam(self, step: int, lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             dynamic_scale: bool = False):
        _check(lib().nbvh_adam(ctypes.byref(self.desc), ctypes.byref(self.struct), step, lr, beta1, beta2, eps,
                               1 if dynamic_scale else 0, _stream()), "adam")


def train_step(desc: ModelDesc, opt: Optimizer, scene: DeviceScene, mode: int, batch: int, seed: int, step: int,
               lr: float, workspace, loss_out=None):
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    _check(lib().nbvh_train_step(ctypes.byref(desc), ctypes.byref(opt.struct), ctypes.byref(scene.struct), mode,
                                 batch, ctypes.c_uint64(seed), step, lr, _ptr(loss_out), c_void_p(base), avail,
                                 _stream()), "train_step")


class Graph:
    """A recorded sequence of library calls replayed with one launch
    (nbvh_graph_*). Record on a created torch stream:

        with torch.cuda.stream(s):
            g = Graph.record(lambda: query_rays(...))
            g.launch()
    """

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def record(cls, fn):
        _check(lib().nbvh_graph_begin(_stream()), "graph_begin")
        try:
            fn()
        finally:
            h = c_void_p()
            st = lib().nbvh_graph_end(_stream(), ctypes.byref(h))
        _check(st, "graph_end")
        return cls(h)

    def launch(self):
        _check(lib().nbvh_graph_launch(self.handle, _stream()), "graph_launch")

    def destroy(self):
        if self.handle:
            lib().nbvh_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------- hybrid hierarchy (S9)
def build_tri_blas(tris: np.ndarray, max_leaf: int = 4) -> dict:
    """Host binned-SAH BVH over triangles (nbvh_build_tri_blas)."""
    tris = np.ascontiguousarray(tris, np.float32)
    n = len(tris)
    cap = max(1, n - 1)
    nodes = np.zeros(cap * 64, np.uint8)
    n_nodes = c_int32()
    n_leaves = c_int32()
    perm = np.zeros(n, np.int32)
    rng = np.zeros(2 * n, np.int32)
    _check(lib().nbvh_build_tri_blas(tris.ctypes.data_as(c_void_p), n, max_leaf, nodes.ctypes.data_as(c_void_p),
                                     cap, ctypes.byref(n_nodes), perm.ctypes.data_as(c_void_p),
                                     rng.ctypes.data_as(c_void_p), n, ctypes.byref(n_leaves)), "build_tri_blas")
    return {"nodes": nodes[:n_nodes.value * 64].copy(), "n_nodes": n_nodes.value, "tri_perm": perm,
            "leaf_range": rng[:2 * n_leaves.value].reshape(-1, 2).copy(), "n_leaves": n_leaves.value}


class DeviceTriBlas:
    """Device copy of a triangle BLAS: nodes, leaf-order triangles, leaf
    ranges and the caller index of every leaf-order triangle."""

    def __init__(self, tris: np.ndarray, blas: dict, device="cuda", albedo: np.ndarray = None):
        torch = _torch()
        t = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
        self.albedo = None if albedo is None else torch.as_tensor(
            np.ascontiguousarray(albedo, np.float32).reshape(-1, 3), device=device)
        self.nodes = torch.as_tensor(blas["nodes"], device=device)
        self.tris = torch.as_tensor(np.ascontiguousarray(t[blas["tri_perm"]]), device=device)
        self.leaf_range = torch.as_tensor(np.ascontiguousarray(blas["leaf_range"], np.int32), device=device)
        self.tri_id = torch.as_tensor(blas["tri_perm"], device=device)
        s = TriBlas()
        s.nodes = self.nodes.data_ptr()
        s.n_nodes = blas["n_nodes"]
        s.tris = self.tris.data_ptr()
        s.leaf_range = self.leaf_range.data_ptr()
        s.tri_id = self.tri_id.data_ptr()
        s.albedo = self.albedo.data_ptr() if self.albedo is not None else None
        self.struct = s


def trace_triangles(blas: DeviceTriBlas, rays: dict, out=None):
    n = rays["ox"].numel()
    if out is None:
        out = new_hits(n, rays["ox"].device, albedo=blas.albedo is not None)
    _check(lib().nbvh_trace_triangles(ctypes.byref(blas.struct), rays_struct(rays), hits_struct(out), _stream()),
           "trace_triangles")
    return out


def tri_instance(blas: DeviceTriBlas) -> Instance:
    x = Instance()
    x.kind = BLAS_TRIANGLES
    x.tri = blas.struct
    return x


def neural_instance(desc: ModelDesc, table, mlp, nodes, n_nodes: int, max_segs: int) -> Instance:
    x = Instance()
    x.kind = BLAS_NEURAL
    x.desc = desc
    x.table = table.data_ptr()
    x.mlp = mlp.data_ptr()
    x.nodes = nodes.data_ptr()
    x.n_nodes = n_nodes
    x.max_segs = max_segs
    return x


def instance_array(instances) -> ctypes.Array:
    arr = (Instance * len(instances))()
    for i, x in enumerate(instances):
        arr[i] = x
    return arr


def hybrid_workspace_size(instances, n_rays: int) -> int:
    arr = instance_array(instances)
    b = c_size_t()
    _check(lib().nbvh_hybrid_workspace_size(arr, len(arr), n_rays, ctypes.byref(b)), "hybrid_workspace_size")
    return b.value


def hybrid_trace(instances, rays: dict, out=None, inst_out=None, workspace=None, options=None):
    """Closest hit over the instances of the two-level hierarchy
    (nbvh_hybrid_trace). Returns (hits, instance index per ray)."""
    torch = _torch()
    n = rays["ox"].numel()
    dev = rays["ox"].device
    if out is None:
        alb = any((x.kind == BLAS_NEURAL and x.desc.n_out >= 8) or (x.kind == BLAS_TRIANGLES and x.tri.albedo)
                  for x in instances)
        out = new_hits(n, dev, albedo=alb)
    if inst_out is None:
        inst_out = torch.empty(n, dtype=torch.int32, device=dev)
    arr = instance_array(instances)
    if workspace is None:
        workspace = new_workspace(hybrid_workspace_size(instances, n), dev)
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    _check(lib().nbvh_hybrid_trace(arr, len(arr), rays_struct(rays), hits_struct(out), _ptr(inst_out),
                                   c_void_p(base), avail, _opt_ref(options), _stream()), "hybrid_trace")
    return out, inst_out


def probe_l2_gather(n_entries: int = 1 << 24) -> float:
    """nbvh_probe_l2_gather: the L2 random-gather ceiling in 1e9 sector loads/s
    (a measurement utility for the gather's roofline)."""
    torch = _torch()
    tab = torch.ones(n_entries, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = c_double()
    _check(lib().nbvh_probe_l2_gather(_ptr(tab), n_entries, _ptr(sink), ctypes.byref(g), _stream()),
           "probe_l2_gather")
    return g.value


def probe_l2_reduce(n_entries: int = 1 << 23) -> float:
    """nbvh_probe_l2_reduce: the L2 float2 atomic-add ceiling in 1e9 adds/s
    (a measurement utility for the table-gradient scatter's roofline)."""
    torch = _torch()
    grad = torch.zeros(2 * n_entries, dtype=torch.float32, device="cuda")
    g = c_double()
    _check(lib().nbvh_probe_l2_reduce(_ptr(grad), n_entries, ctypes.byref(g), _stream()), "probe_l2_reduce")
    return g.value


# ---------------------------------------------------------------- error-driven cut (Sec. 5.1)
def build_cut(base: dict, cut, inflate_rel: float, info: dict) -> dict:
    """nbvh_build_cut: the N-BVH whose leaves are the base-BVH references in
    ``cut`` (the base BVH from build_tri_blas). Returns a leaves dict in the
    format of build_leaves (triangle order: the base BVH's) plus leaf_ref."""
    cut = np.ascontiguousarray(cut, np.int32)
    n_cut = len(cut)
    cap = max(1, n_cut - 1)
    nodes = np.zeros(cap * 64, np.uint8)
    n_nodes = c_int32()
    rng = np.zeros(2 * n_cut, np.int32)
    box = np.zeros((n_cut, 6), np.float32)
    ref = np.zeros(n_cut, np.int32)
    base_nodes = np.ascontiguousarray(base["nodes"])
    base_rng = np.ascontiguousarray(base["leaf_range"], np.int32)
    _check(lib().nbvh_build_cut(base_nodes.ctypes.data_as(c_void_p), base["n_nodes"], base_rng.ctypes.data_as(c_void_p),
                                base["n_leaves"], cut.ctypes.data_as(c_void_p), n_cut, float(inflate_rel),
                                float(info["extent"]), nodes.ctypes.data_as(c_void_p), cap, ctypes.byref(n_nodes),
                                rng.ctypes.data_as(c_void_p), box.ctypes.data_as(c_void_p),
                                ref.ctypes.data_as(c_void_p)), "build_cut")
    return {"nodes": nodes[:n_nodes.value * 64].copy(), "n_nodes": n_nodes.value, "tri_perm": base["tri_perm"],
            "leaf_range": rng.reshape(-1, 2), "leaf_lo": box[:, :3].copy(), "leaf_hi": box[:, 3:].copy(),
            "leaf_ref": ref, "info": info}


def base_children(base: dict, ref: int):
    """Child references of an internal base reference (ref >= 0)."""
    nd = node_array({"nodes": base["nodes"]})[ref]
    out = [int(nd["child0"])]
    if int(nd["child1"]) != 0x7fffffff:
        out.append(int(nd["child1"]))
    return out


def train_step_weighted(desc: ModelDesc, opt, scene, mode: int, batch: int, seed: int, step: int, lr: float,
                        workspace, leaf_prob=None, stats=None, loss_out=None):
    """nbvh_train_step_weighted. stats: dict of device tensors hits (int32),
    trained (int32), loss (float32), n_leaves entries each, accumulated."""
    base = aligned_ptr(workspace)
    avail = workspace.numel() - (base - workspace.data_ptr())
    st = None
    if stats is not None:
        st = LeafStats()
        st.hits, st.trained, st.loss = (stats["hits"].data_ptr(), stats["trained"].data_ptr(),
                                        stats["loss"].data_ptr())
    _check(lib().nbvh_train_step_weighted(ctypes.byref(desc), ctypes.byref(opt.struct), ctypes.byref(scene.struct),
                                          mode, batch, ctypes.c_uint64(seed), step, lr, _ptr(leaf_prob),
                                          ctypes.byref(st) if st is not None else None, _ptr(loss_out),
                                          c_void_p(base), avail, _stream()), "train_step_weighted")


def node_rank(hits, trained, loss, n_rays):
    """nbvh_rank_leaves (Sec. 5.1 "Node error", Sec. 5.2 training
    probability): per leaf q, p, the ranking r and the training probability."""
    n = len(hits)
    h = np.ascontiguousarray(hits, np.uint32)
    t = np.ascontiguousarray(trained, np.uint32)
    l = np.ascontiguousarray(loss, np.float32)
    q, p, r = (np.zeros(n, np.float64) for _ in range(3))
    prob = np.zeros(n, np.float32)
    _check(lib().nbvh_rank_leaves(h.ctypes.data_as(c_void_p), t.ctypes.data_as(c_void_p), l.ctypes.data_as(c_void_p),
                                  n, int(n_rays), q.ctypes.data_as(c_void_p), p.ctypes.data_as(c_void_p),
                                  r.ctypes.data_as(c_void_p), prob.ctypes.data_as(c_void_p)), "rank_leaves")
    return q, p, r, prob


def refine_cut(base: dict, cut, r, prob, k_splits: int):
    """nbvh_refine_cut (Sec. 5.1): the cut with its k_splits best-ranked
    splittable leaves replaced by their base children, and every new leaf's
    training probability. Returns (new cut, new probabilities)."""
    cut = np.ascontiguousarray(cut, np.int32)
    r = np.ascontiguousarray(r, np.float64)
    prob = np.ascontiguousarray(prob, np.float32)
    cap = 2 * len(cut)
    out = np.zeros(cap, np.int32)
    out_p = np.zeros(cap, np.float32)
    m = c_int32()
    nodes = np.ascontiguousarray(base["nodes"])
    _check(lib().nbvh_refine_cut(nodes.ctypes.data_as(c_void_p), base["n_nodes"], cut.ctypes.data_as(c_void_p),
                                 len(cut), r.ctypes.data_as(c_void_p), prob.ctypes.data_as(c_void_p), int(k_splits),
                                 out.ctypes.data_as(c_void_p), out_p.ctypes.data_as(c_void_p), cap, ctypes.byref(m)),
           "refine_cut")
    return out[:m.value].tolist(), out_p[:m.value].tolist()


def optimize_cut(tris, desc: ModelDesc, opt, n_target: int, *, base_max_leaf: int = 16, iters: int = 50,
                 splits: int = 4, factor: float = 1.5, final_iters: int = 200, batch: int = 1 << 16,
                 seed: int = 240516237, lr: float = 1e-2, mode: int = TRAIN_PROBED_MIX, inflate_rel: float = 1e-4,
                 step0: int = 1, max_rounds: int = 1000, lod_every: int = 0, lods_out=None):
    """Error-driven cut optimization (Sec. 5.1): start with the root of the
    base BVH (binned SAH over the triangles); train ``iters`` steps on the
    current cut's N-BVH with error-weighted ray selection; split the
    ``splits`` leaves of largest ranking r into their base children; grow
    both counts by ``factor``; stop at ``n_target`` leaves and train
    ``final_iters`` more steps. Returns (leaves dict of the final cut, the
    DeviceScene, per-round history, next step number).

    Levels of detail (Sec. 5.3): with ``lod_every`` > 0 the current cut is
    registered as an LoD whenever another ``lod_every`` training steps have
    passed (at a round's end, before its splits), and from then on every step
    trains a cut drawn uniformly from the registered LoDs and the current cut
    (seeded host draws; error weighting applies to the current cut only).
    ``lods_out`` (a list) receives (leaves, DeviceScene) of every LoD, coarse
    to fine, the final cut last."""
    torch = _torch()
    base = build_tri_blas(tris, base_max_leaf)
    info = build_leaves(tris, 1, inflate_rel)["info"]
    cut = [0]
    prob = None
    step = step0
    history = []
    ws = None
    ws_leaves = -1
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    lods = []  # registered (leaves, scene), coarse to fine
    lod_rng = np.random.default_rng(seed ^ 0x10D)
    trained_steps = 0
    next_lod = lod_every

    def run(cut, prob, n_iters):
        nonlocal step, ws, ws_leaves, trained_steps
        lv = build_cut(base, cut, inflate_rel, info)
        scene = DeviceScene(tris, lv)
        if ws is None or ws_leaves < len(cut):
            ws = new_workspace(train_workspace_size(desc, batch, max(len(cut), n_target)))
            ws_leaves = max(len(cut), n_target)
        n = len(cut)
        stats = {"hits": torch.zeros(n, dtype=torch.int32, device="cuda"),
                 "trained": torch.zeros(n, dtype=torch.int32, device="cuda"),
                 "loss": torch.zeros(n, dtype=torch.float32, device="cuda")}
        pdev = torch.as_tensor(np.asarray(prob, np.float32)).cuda() if prob is not None else None
        for _ in range(n_iters):
            k = int(lod_rng.integers(0, len(lods) + 1)) if lods else len(lods)
            if k == len(lods):
                train_step_weighted(desc, opt, scene, mode, batch, seed, step, lr, ws, leaf_prob=pdev,
                                    stats=stats, loss_out=loss)
            else:
                train_step_weighted(desc, opt, lods[k][1], mode, batch, seed, step, lr, ws, loss_out=loss)
            step += 1
        trained_steps += n_iters
        h = stats["hits"].cpu().numpy()
        t = stats["trained"].cpu().numpy()
        l = stats["loss"].cpu().numpy()
        return lv, scene, h, t, l

    rounds = 0
    while len(cut) < n_target and rounds < max_rounds:
        rounds += 1
        lv, scene, h, t, l = run(cut, prob, iters)
        if lod_every > 0 and trained_steps >= next_lod:
            lods.append((lv, scene))
            while next_lod <= trained_steps:
                next_lod += lod_every
        q, p, r, pr = node_rank(h, t, l, batch * iters)
        history.append({"leaves": len(cut), "iters": iters, "loss": float(loss.item()),
                        "mean_q": float(np.sum(l) / max(1, np.sum(t)))})
        k = min(int(splits), n_target - len(cut))
        if k <= 0:
            break
        new_cut, new_prob = refine_cut(base, lv["leaf_ref"], r, pr, k)
        if len(new_cut) == len(cut):
            break  # nothing left to split
        cut, prob = new_cut, new_prob
        iters = int(math.ceil(iters * factor))
        splits = int(math.ceil(splits * factor))
    lv, scene, h, t, l = run(cut, prob, final_iters)
    history.append({"leaves": len(cut), "iters": final_iters, "loss": float(loss.item()),
                    "mean_q": float(np.sum(l) / max(1, np.sum(t))), "final": True,
                    "lods": [len(x[0]["leaf_ref"]) for x in lods]})
    if lods_out is not None:
        lods_out.extend(lods)
        lods_out.append((lv, scene))
    return lv, scene, history, step
