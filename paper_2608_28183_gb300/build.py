"""Build the in-tree CUDA library libnlos_gb300.so for sm_103a.

Each .cu file under csrc/ is compiled to an object in parallel, then the
objects are linked into a shared library next to this file. Objects are
rebuilt when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnlos_gb300.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
          "-I", CSRC, "-I", INCLUDE] + ARCH


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return r


def bounds_checked() -> bool:
    """NLOS_BOUNDS_CHECK=1 in the environment selects the bounds-checked debug
    build (every checked global access outside its buffer is recorded in the
    workspace's error word and skipped)."""
    return os.environ.get("NLOS_BOUNDS_CHECK", "0") not in ("", "0")


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile csrc/*.cu for sm_103a and link libnlos_gb300.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    extra_flags = list(extra_flags or []) + (["-DNLOS_BOUNDS_CHECK"] if bounds_checked() else [])
    # objects built with other flags are rebuilt
    stamp = os.path.join(BUILD, "flags.txt")
    sig = " ".join(CFLAGS + extra_flags)
    if not os.path.exists(stamp) or open(stamp).read() != sig:
        force = True
    srcs = _sources()
    keep = {os.path.basename(x)[:-3] + ".o" for x in srcs}
    for stale in glob.glob(os.path.join(BUILD, "*.o")):
        if os.path.basename(stale) not in keep:
            os.remove(stale)
    hdr_time = _newest(_headers())
    flags = CFLAGS + list(extra_flags or [])
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            jobs.append([NVCC] + flags + ["-c", s, "-o", o])
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda c: _run(c, verbose), jobs))
    if force or jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        _run([NVCC] + ARCH + ["-shared", "-o", LIB] + objs
             + ["-cudart", "shared", "-Xlinker", "-rpath," + os.path.join(CUDA_HOME, "lib64")], verbose)
    with open(stamp, "w") as f:
        f.write(sig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
