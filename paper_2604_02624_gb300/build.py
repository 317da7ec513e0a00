"""Builds libdos.so (the C-ABI CUDA library) in-tree for sm_103a.

Every ``csrc/*.cu`` translation unit is compiled by its own nvcc process (in
parallel) and the objects are linked into ``paper_2604_02624_gb300/libdos.so``
against the shared CUDA runtime.  No CMake, no setuptools.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdos.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libdos")
    return cand


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def compile_flags() -> list:
    return ["-std=c++17", "--expt-relaxed-constexpr", "-O3", ARCH, "-lineinfo",
            "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", os.path.join(ROOT, "include")]


def _compile(nvcc: str, src: str, verbose: bool) -> tuple:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc, *compile_flags(), "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    p = subprocess.run(cmd, capture_output=True, text=True)
    return obj, p.returncode, p.stdout + p.stderr, " ".join(cmd)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile all translation units and link libdos.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    objs, logs = [], []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, rc, out, cmd in ex.map(lambda s: _compile(nvcc, s, verbose), srcs):
            logs.append(f"$ {cmd}\n{out}")
            if rc != 0:
                raise RuntimeError(f"nvcc failed for {obj}:\n{out}")
            objs.append(obj)
    with open(os.path.join(BUILD, "build.log"), "w") as f:
        f.write("\n".join(logs))
    tmp = LIB + ".tmp"
    link = [nvcc, "-shared", ARCH, "-o", tmp, *objs, "-cudart", "shared",
            "-Xlinker", "-rpath," + _cuda_lib_dir(nvcc)]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    path = build(verbose="-v" in sys.argv)
    print(path)
