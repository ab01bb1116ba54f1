"""Build the CUDA library libasd.so in-tree for sm_103a (nvcc, no cmake).

Translation units compile in parallel; the shared object links the CUDA runtime
statically, so it only needs the NVIDIA driver at run time.  build(check_bounds=True)
makes the index-checked variant libasd_checked.so (ASD_CHECK_BOUNDS=1: every computed
shared-memory and table index of the kernels is tested before use; a failure is recorded
in the device error word and the access skipped), loaded by the binding when ASD_CHECKED=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
OBJ = os.path.join(OUT, "obj")
SO = os.path.join(OUT, "libasd.so")
OBJ_CHECKED = os.path.join(OUT, "obj_checked")
SO_CHECKED = os.path.join(OUT, "libasd_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(HERE, "..", "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose_ptxas=False, checked=False):
    obj = os.path.join(OBJ_CHECKED if checked else OBJ, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + _headers()):
        return obj, ""
    cmd = ([NVCC] + ARCH + FLAGS + (["-DASD_CHECK_BOUNDS=1"] if checked else []) +
           (["-Xptxas", "-v"] if verbose_ptxas else []) + ["-c", src, "-o", obj])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False, check_bounds: bool = False) -> str:
    obj_dir, so = (OBJ_CHECKED, SO_CHECKED) if check_bounds else (OBJ, SO)
    os.makedirs(obj_dir, exist_ok=True)
    srcs = _sources()
    if force:
        for o in glob.glob(os.path.join(obj_dir, "*.o")):
            os.remove(o)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 8))) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose_ptxas, check_bounds), srcs))
    objs = [o for o, _ in res]
    if verbose_ptxas:
        for _, log in res:
            if log:
                sys.stderr.write(log)
    if force or _stale(so, objs):
        tmp = so + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                check_bounds="--checked" in sys.argv))
