"""Build the in-tree CUDA library libqtm.so for sm_103a.

Host planner sources (.cpp) compile with g++, kernels and the C ABI (.cu) with
nvcc for compute_103a/sm_103a, in parallel; the objects link into one shared
library next to this file.  Nothing is installed into site-packages.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqtm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["capi.cu", "fused.cu", "naive.cu", "noalloc.cu", "multi.cu", "pauli.cu"]
CPP_SOURCES = ["plan.cpp", "emulate.cpp", "jit.cpp"]
# device headers embedded as the prelude of run-time generated kernels (NVRTC)
PRELUDE_HEADERS = ["pod.h", "finalize_math.h", "tile.cuh", "f32x2.cuh", "tile_cpx.cuh"]


def _write_prelude() -> str:
    parts = []
    for h in PRELUDE_HEADERS:
        for line in open(os.path.join(CSRC, h)):
            t = line.strip()
            if t == "#pragma once" or (t.startswith("#include \"") and t.endswith("\"")):
                continue
            parts.append(line)
    text = "".join(parts)
    assert ")QTMJIT\"" not in text
    out = os.path.join(BUILD, "jit_prelude.cpp")
    src = ("namespace qtm {\nextern const char *const kJitPrelude;\nconst char *const kJitPrelude = R\"QTMJIT(" +
           text + ")QTMJIT\";\n}\n")
    if not os.path.exists(out) or open(out).read() != src:
        with open(out, "w") as f:
            f.write(src)
    return out


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
           [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return deps


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _sources() + [__file__])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
    ptxas_v = ["-Xptxas", "-v"] if os.environ.get("QTM_PTXAS_VERBOSE") == "1" else []
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-Wall", *ptxas_v, "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    prelude = _write_prelude()
    for f in CPP_SOURCES + [prelude]:
        src = f if os.path.isabs(f) else os.path.join(CSRC, f)
        obj = os.path.join(BUILD, os.path.basename(f) + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC, "-I", cuda_inc, "-c",
               src, "-o", obj]
        jobs.append((cmd, obj))

    def run(job):
        cmd, obj = job
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if r.stderr and (verbose or r.returncode != 0 or ptxas_v):
            print(r.stderr, file=sys.stderr)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp] + [o for _, o in jobs] + ["-ldl"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        print(r.stderr, file=sys.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
