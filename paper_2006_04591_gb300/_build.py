"""Build libshearlet.so (and its bounds-checked variant
libshearlet_checked.so) in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit is compiled in its own process, in parallel; a shared
object is relinked only when a source or header is newer than it.
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

CU_SOURCES = ["fast.cu", "fused.cu", "general.cu", "noalloc.cu", "nn.cu", "nn_tc.cu", "bank_gpu.cu", "ray.cu",
              "tc_dft.cu"]
CPP_SOURCES = ["api.cpp", "bank_build.cpp"]
# The checked library: every source again with -DSHL_CHECKED (bounds guards
# with a device error word in the transform kernels), the same C ABI.
LIB_CHECKED = os.path.join(PKG, "libshearlet_checked.so")
CU_CHECKED = CU_SOURCES


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


def _jobs(cu, cpp, tag, defines, verbose):
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs = []
    for s in cu:
        o = os.path.join(BUILD, tag + s + ".o")
        jobs.append((o, [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "--expt-relaxed-constexpr", *defines, *inc, "-c", os.path.join(CSRC, s),
                         "-o", o] + (["-Xptxas", "-v"] if verbose else [])))
    gxx = shutil.which("g++") or "g++"
    for s in cpp:
        o = os.path.join(BUILD, tag + s + ".o")
        jobs.append((o, [gxx, "-O2", "-fPIC", "-std=c++17", "-Wall", "-Wno-unused-function",
                         *defines, "-I" + os.path.join(CUDA_HOME, "include"), *inc, "-c",
                         os.path.join(CSRC, s), "-o", o]))
    return jobs


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libshearlet.so and libshearlet_checked.so (all
    translation units of both in parallel); returns the main library's path."""
    newest = _newest(_deps())
    stale = [lib for lib in (LIB, LIB_CHECKED)
             if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest]
    if not stale:
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError("nvcc not found at %s" % NVCC)
    os.makedirs(BUILD, exist_ok=True)
    plan = {LIB: _jobs(CU_SOURCES, CPP_SOURCES, "", [], verbose),
            LIB_CHECKED: _jobs(CU_CHECKED, CPP_SOURCES, "checked_", ["-DSHL_CHECKED"], verbose)}
    jobs = [j for lib in stale for j in plan[lib]]
    logs = []
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for out in ex.map(lambda j: _run(j[1]), jobs):
            logs.append(out)
    for lib in stale:
        tmp = lib + ".tmp"
        _run([NVCC, *ARCH, "-shared", "-o", tmp] + [j[0] for j in plan[lib]] + ["-lpthread"])
        os.replace(tmp, lib)
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
