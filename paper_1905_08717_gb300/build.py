"""Build the CUDA library libmrlt.so in-tree for sm_103a (GB300) with nvcc.

The translation units are compiled in parallel and linked with the
static CUDA runtime.  Run as `python -m paper_1905_08717_gb300.build`.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(CSRC, "libmrlt.so")
# (source, extra flags, object tag): the stage kernels are compiled once per
# equation so that the heaviest translation units build in parallel
UNITS = [("mrlt_api.cu", [], "api"), ("mrlt_tree.cu", [], "tree"), ("mrlt_stage.cu", [], "stage"),
         ("mrlt_noalloc.cu", [], "noalloc")] + [
            ("mrlt_stage_eq.cu", [f"-DMRLT_STAGE_EQ={e}"], f"stage_eq{e}") for e in range(4)] + [
            ("mrlt_macro_eq.cu", [f"-DMRLT_STAGE_EQ={e}"], f"macro_eq{e}") for e in range(4)]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["mrlt_impl.cuh", "mrlt_tree.cuh", "mrlt_tree_dev.cuh", "mrlt_stage.cuh", "mrlt_macro.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "mrlt.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    objs, procs = [], []
    for src, extra, tag in UNITS:
        obj = os.path.join(CSRC, f"{tag}.{os.getpid()}.o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    bad = [cmd for p, cmd in procs if p.wait() != 0]
    try:
        if bad:
            raise RuntimeError("nvcc failed: " + " ".join(bad[0]))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
