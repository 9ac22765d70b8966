"""Builds libnbvh.so (sm_103a) in-tree with nvcc.

The kernel families live in separate translation units so they compile in
parallel: tu_eval_tc.cu once per (table type, mode), tu_eval_plain.cu and
tu_train.cu once per table type, tu_train_tc.cu, nbvh_lib.cu (entry points and
small kernels) and host.cpp. Objects go to _build/ next to this file; a unit is
recompiled when its source or a header it includes (nvcc dependency file) is
newer than its object.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libnbvh.so")
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-Xcompiler", "-fPIC", "-O3", "-std=c++17", "-lineinfo", *ARCH, "-I", os.path.join(ROOT, "include")]


def units():
    """(object name, source, extra defines) of every translation unit."""
    u = [("nbvh_lib", "nbvh_lib.cu", []), ("host", "host.cpp", []), ("train_tc", "tu_train_tc.cu", [])]
    for t in range(3):
        for m in range(3):
            u.append((f"eval_tc_t{t}_m{m}", "tu_eval_tc.cu", [f"-DNBVH_TU_TABLE={t}", f"-DNBVH_TU_MODE={m}"]))
        u.append((f"eval_plain_t{t}", "tu_eval_plain.cu", [f"-DNBVH_TU_TABLE={t}"]))
        u.append((f"train_t{t}", "tu_train.cu", [f"-DNBVH_TU_TABLE={t}"]))
    return u


def _deps(dep_file):
    """Files listed in an nvcc/gcc make-style dependency file."""
    try:
        text = open(dep_file).read().replace("\\\n", " ")
    except OSError:
        return None
    if ":" not in text:
        return None
    return [f for f in text.split(":", 1)[1].split() if f]


def _stale(obj, src, dep_file):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = _deps(dep_file)
    if deps is None:
        return True
    return any(not os.path.exists(f) or os.path.getmtime(f) > t for f in deps + [src])


def _compile(nvcc, name, src, defs, extra, verbose):
    obj = os.path.join(OBJ, name + ".o")
    dep = os.path.join(OBJ, name + ".d")
    path = os.path.join(CSRC, src)
    if not _stale(obj, path, dep):
        return obj
    cmd = [nvcc, "-c", *FLAGS, *defs, *extra, "-MD", "-MF", dep, "-o", obj + ".tmp", path]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), jobs: int = 0) -> str:
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    if force:
        for f in os.listdir(OBJ):
            if f.endswith(".o") or f.endswith(".d"):
                os.remove(os.path.join(OBJ, f))
    jobs = jobs or max(1, os.cpu_count() or 1)
    us = units()
    # the largest units first so the pool stays busy
    order = sorted(us, key=lambda u: 0 if u[0].startswith("eval_tc") else 1)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(nvcc, u[0], u[1], u[2], list(extra), verbose), order))
    if os.path.exists(LIB) and all(os.path.getmtime(o) <= os.path.getmtime(LIB) for o in objs):
        return LIB
    cmd = [nvcc, "-shared", *ARCH, "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=("-Xptxas", "-v") if "--ptxas-v" in sys.argv else ())
