"""Build librogs.so (sm_103a) in-tree with nvcc: one object per translation
unit, compiled in parallel, then linked into a shared library next to this
file.  Usage: python -m paper_2405_14342_gb300.build [--force] [--verbose]."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build", "librogs")
LIB = os.path.join(HERE, "librogs.so")
LIB_CHECKED = os.path.join(HERE, "librogs_checked.so")
SOURCES = ["api.cu", "project.cu", "sort.cu", "bin.cu", "composite.cu", "backward.cu", "loss.cu", "init.cu",
           "noalloc.cu", "serve.cu", "smooth.cu", "adam.cu", "lidar.cu", "bev.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "rogs.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose, checked=False):
    out = os.path.join(OBJ + ("_checked" if checked else ""), os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", out, "-O3", "-std=c++17", *ARCH, "-lineinfo",
           "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I", os.path.join(ROOT, "include")]
    if checked:
        cmd += ["-DROGS_CHECKED"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return out, r.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build librogs.so, or with checked=True the bounds-checked variant
    librogs_checked.so (-DROGS_CHECKED, see rogs_bounds_checked in rogs.h)."""
    lib = LIB_CHECKED if checked else LIB
    deps = _deps()
    if not force and not _stale(lib, deps):
        return lib
    os.makedirs(OBJ + ("_checked" if checked else ""), exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, checked), SOURCES))
    if verbose:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
