"""Builds the in-tree shared library libhhg.so for sm_103a with nvcc.

Usage: python -m paper_2010_13513_gb300.build   (or build() from Python)

Each translation unit is compiled in parallel into _build/, then linked
into paper_2010_13513_gb300/libhhg.so (CUDA runtime linked statically, so the
library needs nothing beyond the driver at run time).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhhg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, extra flags): fast.cu and stream.cu are compiled once per precision
SOURCES = [("kernels.cu", "kernels", []), ("fast.cu", "fast64", ["-DHHG_FAST_ONLY=64"]),
           ("fast.cu", "fast32", ["-DHHG_FAST_ONLY=32"]),
           ("fast.cu", "fast64b", ["-DHHG_FAST_ONLY=64", "-DHHG_FAST_BATCHED"]),
           ("fast.cu", "fast32b", ["-DHHG_FAST_ONLY=32", "-DHHG_FAST_BATCHED"]), ("stream.cu", "stream64", ["-DHHG_STREAM_ONLY=64"]),
           ("stream.cu", "stream32", ["-DHHG_STREAM_ONLY=32"]),
           ("stream.cu", "stream32v2", ["-DHHG_STREAM_ONLY=32", "-DHHG_STREAM_V=2"]),
           ("stream.cu", "stream64b", ["-DHHG_STREAM_ONLY=64", "-DHHG_STREAM_BATCHED"]),
           ("stream.cu", "stream32b", ["-DHHG_STREAM_ONLY=32", "-DHHG_STREAM_BATCHED"]),
           ("stream.cu", "stream32v2b", ["-DHHG_STREAM_ONLY=32", "-DHHG_STREAM_V=2", "-DHHG_STREAM_BATCHED"]),
           ("small.cu", "small", []),
           ("nn.cu", "nn", []), ("noalloc.cu", "noalloc", []), ("stencils.cpp", "stencils", []),
           ("dfres.cu", "dfres", []), ("batch.cpp", "batch", []), ("problem.cpp", "problem", [])]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(unit, verbose):
    src, name, extra = unit
    nvcc = _nvcc()
    obj = os.path.join(OUT, name + ".o")
    cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-I", OUT] + extra
    if src.endswith(".cu"):
        cmd += ARCH + ["-lineinfo", "--expt-relaxed-constexpr"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd += ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _generate_structure():
    """Compiles and runs the stencil-structure generator (host C++), which
    writes the compile-time row term counts used by fast.cu."""
    exe = os.path.join(OUT, "gen_structure")
    cxx = shutil.which("g++") or shutil.which("c++")
    cmd = [cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), os.path.join(CSRC, "gen_structure.cpp"),
           os.path.join(CSRC, "stencils.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"generator build failed: {' '.join(cmd)}\n{r.stderr}")
    r = subprocess.run([exe], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"generator failed: {r.stderr}")
    path = os.path.join(OUT, "structure.inc")
    old = open(path).read() if os.path.exists(path) else None
    if old != r.stdout:
        with open(path, "w") as f:
            f.write(r.stdout)


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    _generate_structure()
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    cmd = [_nvcc(), "-shared", "-o", LIB + ".tmp"] + objs + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
