"""Build libqtreeshap.so for sm_103a (GB300) with nvcc, in-tree.

Every translation unit under csrc/ is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked into one
shared library next to this file.  Objects go to ``_build/`` (git-ignored).
A source whose first lines say ``qts-build-parts: N`` is compiled N times, with
``-DQTS_PART=0`` .. ``N-1``, each part holding a share of its kernels, so the
heaviest files compile in parallel too.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqtreeshap.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _parts(src: str) -> int:
    """Number of build parts a source declares in its first 30 lines (1 if none)."""
    with open(src) as fh:
        for _, line in zip(range(30), fh):
            m = re.search(r"qts-build-parts:\s*(\d+)", line)
            if m:
                return max(1, int(m.group(1)))
    return 1


def _units():
    """(source, part) pairs; part None for a source compiled as one unit."""
    out = []
    for src in _sources():
        n = _parts(src)
        out += [(src, None)] if n == 1 else [(src, k) for k in range(n)]
    return out


def _compile(unit, extra: list[str]) -> str:
    src, part = unit
    suffix = "" if part is None else f".p{part}"
    obj = os.path.join(BUILD, os.path.basename(src) + suffix + ".o")
    newest = max(os.path.getmtime(p) for p in [src] + _headers() + [__file__])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    defs = [] if part is None else [f"-DQTS_PART={part}"]
    cmd = [nvcc()] + ARCH + COMMON + defs + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    wanted = {os.path.basename(u[0]) + ("" if u[1] is None else f".p{u[1]}") + ".o" for u in units}
    for o in glob.glob(os.path.join(BUILD, "*.o")):
        if force or os.path.basename(o) not in wanted:  # stale objects of an older layout
            os.remove(o)
    extra = list(extra or [])
    # kernel parts of the largest sources first (the slowest units), host parts last
    units.sort(key=lambda u: (u[1] is None or u[1] == 0, -os.path.getsize(u[0]), u[1] or 0))
    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda u: _compile(u, extra), units))
    if (not os.path.exists(LIB) or force or
            os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs)):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
