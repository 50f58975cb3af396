"""Build the in-tree CUDA library libgvqe.so for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process in parallel, then
linked into one shared object next to this file.  No torch, no cmake.
build(debug=True) makes libgvqe_debug.so instead: the same sources with
GVQE_DEBUG defined (guarded device workspaces, gvqe_debug_check).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from typing import List, Optional

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgvqe.so")
LIB_DEBUG = os.path.join(HERE, "libgvqe_debug.so")
SOURCES = ["gvqe_api.cu", "gvqe_kernels.cu", "gvqe_static.cu", "gvqe_batch.cu", "gvqe_grad_l0.cu", "gvqe_readout.cu",
           "gvqe_graph.cu", "gvqe_tune.cu", "gvqe_mps.cu"]
# gvqe_inst.cu is compiled once per (amplitude type, tile bits) pair
INSTANCES = [("float", tb) for tb in (10, 11, 12, 13)] + [("double", tb) for tb in (10, 11, 12)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _deps() -> List[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return files + [os.path.join(INCLUDE, "gvqe.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(job, extra: List[str], out_dir: str = BUILD) -> str:
    src, defs, tag = job
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + tag + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra: Optional[List[str]] = None, debug: bool = False) -> str:
    """Compile libgvqe.so (debug: libgvqe_debug.so) if any source changed; returns the library path."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    out_dir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(out_dir, exist_ok=True)
    extra = list(extra or []) + (["-DGVQE_DEBUG"] if debug else [])
    jobs = [(s, [], "") for s in SOURCES]
    jobs += [("gvqe_inst.cu", [f"-DGVQE_INST_T={t}", f"-DGVQE_INST_TB={tb}"], f"_{t}_{tb}") for t, tb in INSTANCES]
    # the heaviest units first
    jobs.sort(key=lambda j: (j[0] != "gvqe_inst.cu", -int(j[1][1].split("=")[1]) if j[1] else 0))
    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda j: _compile(j, extra, out_dir), jobs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
