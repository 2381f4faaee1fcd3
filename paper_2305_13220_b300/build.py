"""Builds libsdg.so (every CUDA source of the package) for sm_103a with nvcc, in-tree.

Usage: python paper_2305_13220_b300/build.py [--force] [--verbose-ptxas]
(run by path: importing the package itself loads the library this script builds)
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int = 0, out: str = None,
          extra_flags=()) -> str:
    """Compiles every source and links libsdg.so (or `out`); extra_flags are added to each compile."""
    lib = out or LIB
    if out is None and not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build" if out is None else "_build_" + os.path.basename(out))
    os.makedirs(objdir, exist_ok=True)
    common = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        common += ["-Xptxas", "-v"]
    common += list(extra_flags)
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = common + ["-c", src, "-o", obj]
        procs.append((src, subprocess.Popen(cmd)))
    bad = [s for s, p in procs if p.wait() != 0]
    if bad:
        raise RuntimeError(f"nvcc failed for {bad}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, lib)
    return lib


CHECKED_LIB = os.path.join(HERE, "libsdg_checked.so")


def build_checked(force: bool = False) -> str:
    """The bounds-checked build (-DSDG_CHECKED) as libsdg_checked.so, selected at run time with
    SDG_LIBRARY=libsdg_checked.so.  Rebuilt when a source is newer than it."""
    if not force and os.path.exists(CHECKED_LIB):
        t = os.path.getmtime(CHECKED_LIB)
        deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
            glob.glob(os.path.join(INCLUDE, "*.h"))
        if not any(os.path.getmtime(p) > t for p in deps):
            return CHECKED_LIB
    return build(force=True, out=CHECKED_LIB, extra_flags=["-DSDG_CHECKED"])


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="--verbose-ptxas" in sys.argv)
    print(LIB)
    if "--checked" in sys.argv:
        print(build_checked(force="--force" in sys.argv))
