"""Build the CUDA library libseg.so in-tree for sm_103a (GB300).

Compiles the translation units of csrc/ in parallel with nvcc and links them
into paper_1408_2355_gb300/_build/<machine>/libseg.so (CUDA runtime linked statically).
Re-uses object files that are newer than every source and header.

    python paper_1408_2355_gb300/build.py [--force]
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(BUILD, "libseg.so")

SOURCES = ["api.cu", "kernels_f32.cu", "kernels_f64.cu", "mesh.cpp", "assemble.cpp", "noalloc.cu", "server.cpp"]
HEADERS = ["seg_internal.h", "kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libseg")
    return exe


def _flags():
    return ARCH + [
        "-O3",
        "-lineinfo",
        "-std=c++17",
        "-I" + INCLUDE,
        "-I" + CSRC,
        "-Xcompiler",
        "-fPIC,-ffp-contract=off,-O2",
    ]


def _newest_dep():
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "seg.h"), __file__]
    return max(os.path.getmtime(d) for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    dep_time = _newest_dep()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.rsplit(".", 1)[0] + ".o")
        objs.append(o)
        stale = force or not os.path.exists(o) or os.path.getmtime(o) < max(dep_time, os.path.getmtime(s))
        if stale:
            jobs.append([nvcc] + _flags() + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
