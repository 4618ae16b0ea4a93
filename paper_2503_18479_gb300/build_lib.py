"""Build libmts.so (the sm_103a CUDA library behind include/mts.h) in-tree.

Each translation unit is compiled by nvcc in parallel (one -gencode for sm_103a), then
linked into paper_2503_18479_gb300/lib/libmts.so. Rebuilds only what is stale.
Run: python -m paper_2503_18479_gb300.build_lib [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libmts.so")
SOURCES = ["abi.cu", "basis.cu", "solve.cu", "solve_mixed.cu", "solve_large.cu", "superpose.cu", "superpose_tc.cu",
           "backward.cu",
           "static_solve.cu", "optim.cu", "sroute.cu", "field_adjoint_tc.cu"]
HEADERS = ["common.cuh", "kernels.h", "solve_common.cuh", "tc_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmts.so")


def _newest_header() -> float:
    hs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mts.h")]
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, force: bool) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    path = os.path.join(CSRC, src)
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _newest_header()):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force), SOURCES))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    _build_peak_probe(force)
    if verbose:
        print(f"built {LIB}")
    return LIB


PEAK_PROBE = os.path.join(LIBDIR, "fp32_peak")


def _build_peak_probe(force: bool) -> str:
    """The FP32 throughput probe (csrc/fp32_peak.cu) that bench.py runs for the measured
    denominator of its ALU rooflines; a standalone program, not part of libmts.so."""
    src = os.path.join(CSRC, "fp32_peak.cu")
    if not force and os.path.exists(PEAK_PROBE) and os.path.getmtime(PEAK_PROBE) >= os.path.getmtime(src):
        return PEAK_PROBE
    tmp = PEAK_PROBE + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-O3", "-o", tmp, src], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for fp32_peak.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PEAK_PROBE)
    return PEAK_PROBE


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
