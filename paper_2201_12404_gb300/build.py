"""Build liblbm.so from csrc/ with nvcc for sm_103a (in-tree, no CMake).

Each translation unit compiles in its own nvcc process, in parallel; the link
step makes ``paper_2201_12404_gb300/liblbm.so``.  Rebuilds only when a source or
header is newer than the library.  ``build_bounds_checked()`` makes a second
library, ``_build_bc/liblbm_bounds_check.so``, with -DLBM_BOUNDS_CHECK: every
computed population address and auxiliary-field index is checked against its
buffer (LBM_ERR_BOUNDS instead of an out-of-range access); the binding loads it
when LBM_LIBRARY names it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
# extra nvcc flags (e.g. -DLBM_K2_MINBLOCKS_F32=3) for tuning builds
FLAGS += os.environ.get("LBM_NVCC_FLAGS", "").split()


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, defines=(), obj_dir: str = OBJ, lib: str = LIB) -> str:
    os.makedirs(obj_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                     + glob.glob(os.path.join(ROOT, "include", "*.h")))
    objs = []
    jobs = []
    for src in sources:
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, *defines, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if res.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + res.stdout + res.stderr)
            if verbose and (res.stdout or res.stderr):
                print(res.stdout + res.stderr)
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + res.stdout + res.stderr)
        os.replace(tmp, lib)
    return lib


OBJ_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(OBJ_BC, "liblbm_bounds_check.so")


def build_bounds_checked(force: bool = False) -> str:
    """The library with -DLBM_BOUNDS_CHECK (objects and library under _build_bc/)."""
    return build(force=force, defines=("-DLBM_BOUNDS_CHECK",), obj_dir=OBJ_BC, lib=LIB_BC)


if __name__ == "__main__":
    print(build(verbose=True))
