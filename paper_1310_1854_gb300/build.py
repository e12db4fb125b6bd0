"""Compile libvgrid (CUDA for sm_103a plus the host grid builder) in-tree.

Each translation unit is compiled separately and in parallel with nvcc, then
linked into ``_build/libvgrid.so``. Host code is built without floating-point
contraction so the host-side arithmetic does not depend on the CPU's FMA.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libvgrid.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "aux.cu", "trace_lpr1.cu", "trace_lpr2.cu", "trace_lpr4.cu", "trace_lpr8.cu", "build.cpp",
           "noalloc.cu", "build_gpu.cu", "probe.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INC, "-I", SRC,
                   "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "--expt-relaxed-constexpr"]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INC, "vgrid.h"))
    cmds = []
    objs = []
    for src in SOURCES:
        path = os.path.join(SRC, src)
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
            cmds.append([cc] + _flags() + lang + ["-c", path, "-o", obj])
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        if verbose and (p.stderr or p.stdout):
            print(p.stdout + p.stderr)

    with cf.ThreadPoolExecutor(jobs) as ex:
        list(ex.map(run, cmds))
    if force or cmds or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
