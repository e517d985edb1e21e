"""Build libsalf.so (sm_103a) in-tree with nvcc.

Usage: python -m paper_2507_18713_gb300.build [--force] [--verbose-ptxas]
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsalf.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["render.cu", "backward.cu", "params.cu", "noalloc.cu", "raster.cu", "actors.cu",
                "refine.cu", "scene_build_gpu.cu", "secondary.cu", "measure.cu"]
CXX_SOURCES = ["capi.cpp", "scene_build.cpp", "serve.cpp", "checkpoint.cpp"]
HEADERS = ["salf_internal.h", "traverse.cuh", "scan.cuh", "sort.cuh"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsalf")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in CUDA_SOURCES + CXX_SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "salf.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, verbose_ptxas: bool, out_dir: str = OUT_DIR, defines=(),
             csrc: str = CSRC) -> str:
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", csrc, *[f"-D{d}" for d in defines], "-c",
           os.path.join(csrc, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["-x", "cu"]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd[1:1] = ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, out_dir: str = OUT_DIR,
          defines=(), csrc: str = CSRC) -> str:
    """Compile every translation unit (in parallel) and link libsalf.so into
    out_dir (default: the package's _build/), with optional -D defines and an
    alternative source directory."""
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libsalf.so")
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    with cf.ThreadPoolExecutor(max_workers=len(CUDA_SOURCES) + len(CXX_SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, out_dir, defines, csrc),
                           CUDA_SOURCES + CXX_SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--verbose-ptxas" in sys.argv))
