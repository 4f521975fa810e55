"""Build liblbmwet.so in-tree for sm_103a with nvcc (no CMake, no torch extension machinery).

Each translation unit is compiled in parallel, then linked into a shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblbmwet.so")
OBJ = os.path.join(ROOT, "_build")
SOURCES = ["step.cu", "step2p.cu", "step2d.cu", "step3d.cu", "step3p.cu", "reduce.cu", "adjoint.cu", "probe.cu", "api.cu",
           "eos_host.cpp", "plan.cpp", "wall_gf.cpp", "maskscan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
EXTRA_FLAGS = os.environ.get("LBMWET_NVCC_FLAGS", "").split()   # e.g. tile-shape macros for measurements


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, verbose_ptxas: bool) -> str:
    out = os.path.join(OBJ, os.path.basename(src) + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", out, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-lineinfo", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH + EXTRA_FLAGS
    if verbose_ptxas and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return out


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in os.listdir(CSRC)
                                                       if h.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(ROOT, "include", "lbmwet.h"))
    if not force and os.path.exists(LIB):
        lib_t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) < lib_t for s in srcs):
            return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force=True))
