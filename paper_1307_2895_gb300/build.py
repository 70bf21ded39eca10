"""Build the CUDA library ``_lib/libhif.so`` in-tree with nvcc for sm_103a.

Every translation unit is compiled in parallel, then linked into one shared
library exporting the C ABI of ``include/hif.h``.  Rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libhif.so")
SOURCES = ["kernels_factor.cu", "kernels_apply.cu", "kernels_solve.cu", "hif_api.cu", "hif_factor.cu",
           "hif_apply.cu", "hif_solve.cu", "geometry.cpp",
           "noalloc.cu", "kernels_mlp.cu", "kernels_tiled.cu", "kernels_bigfront.cu", "kernels_tc.cu",
           "host_pool.cpp", "symbolic3x.cpp", "kernels_dense3x.cu",
           "kernels_root.cu", "kernels_bigapply.cu", "kernels_svdfront.cu", "kernels_twosided.cu"]
HEADERS = ["hif_internal.h", "kernels.h", "blockops.cuh", "geometry.h", "tile_mma.cuh", "front_common.cuh",
           "host_pool.h", "symbolic3x.h", "hif_host.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhif")
    return cand


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "hif.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library; returns its path."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC] + ARCH

    def compile_one(src: str) -> str:
        obj = os.path.join(LIBDIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
