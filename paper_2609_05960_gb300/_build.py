"""Build the engine's shared library (libgtpower.so) in-tree with nvcc for
sm_103a.  Translation units are compiled in parallel and linked with the
static CUDA runtime."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from typing import List, Optional

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgtpower.so")
ROOT = os.path.dirname(PKG)

SOURCES = ["gtp_engine.cu", "gtp_kernels.cu", "gtp_walk.cu", "gtp_walk_glitch.cu", "gtp_walk_comp.cu", "gtp_scheme.cu",
           "gtp_sipl.cu", "gtp_noalloc.cu", "gtp_tiled.cu", "gtp_pattern.cu", "gtp_walk_whole.cu",
           "gtp_walk_glitch_whole.cu", "gtp_walk_adjoint_whole.cu", "gtp_walk_adjoint_staged.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _deps() -> List[str]:
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdr + [os.path.join(ROOT, "include", "gtpower.h")]


def _stale(out: str, inputs: List[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(i) > t for i in inputs if os.path.exists(i))


def build(force: bool = False, verbose: bool = False, extra: Optional[List[str]] = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not os.path.exists(LIB):
        force = True  # objects left from another machine must not be reused
    deps = _deps()
    cc = nvcc()
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + deps):
            cmd = [cc, "-c", s, "-o", o] + ARCH + NVCC_FLAGS + (extra or [])
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
