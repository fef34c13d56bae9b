"""Build libshearlet.so in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit is compiled in its own process, in parallel; the
shared object is relinked only when a source or header is newer than it.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libshearlet.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["fast.cu", "fused.cu", "general.cu", "noalloc.cu", "nn.cu", "nn_tc.cu", "bank_gpu.cu", "ray.cu"]
CPP_SOURCES = ["api.cpp", "bank_build.cpp"]


def _deps():
    out = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))] + [__file__]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libshearlet.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest(_deps()):
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError("nvcc not found at %s" % NVCC)
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs = []
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append((o, [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, s),
                         "-o", o] + (["-Xptxas", "-v"] if verbose else [])))
    gxx = shutil.which("g++") or "g++"
    for s in CPP_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append((o, [gxx, "-O2", "-fPIC", "-std=c++17", "-Wall", "-Wno-unused-function",
                         "-I" + os.path.join(CUDA_HOME, "include"), *inc, "-c",
                         os.path.join(CSRC, s), "-o", o]))
    logs = []
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for out in ex.map(lambda j: _run(j[1]), jobs):
            logs.append(out)
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-o", tmp] + [j[0] for j in jobs] + ["-lpthread"])
    os.replace(tmp, LIB)
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
