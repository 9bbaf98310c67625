"""Build the CUDA library in-tree with nvcc for sm_103a.

Produces ``paper_1102_5071_gb300/libcfet_gb300.so`` from ``csrc/``.  Each
translation unit is compiled in parallel, then linked with the static CUDA
runtime.  Run ``python -m paper_1102_5071_gb300.build`` or call ``build()``.
Extra nvcc flags (for example ``-DCFET_CTL_MAX_THREADS=544``) can be given in the
environment variable ``CFET_NVCC_FLAGS``; a change of them triggers a rebuild.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libcfet_gb300.so"
LIB_PATH = os.path.join(PKG, LIB_NAME)
BUILD_DIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS_STAMP = os.path.join(BUILD_DIR, "extra_flags.txt")


def _extra_flags() -> list:
    return os.environ.get("CFET_NVCC_FLAGS", "").split()
SOURCES = ["kernels.cu", "kernels_fx.cu", "kernels_c64.cu", "kernels_cheb.cu", "capi.cu", "schemes.cpp", "chebyshev.cpp",
           "noalloc.cu", "batch.cu", "adjoint.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the extension")


def _compile(nvcc: str, src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-I", INCLUDE,
           *_extra_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
    else:
        cmd += ["-x", "c++"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def _up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    try:
        with open(FLAGS_STAMP) as fh:
            if fh.read() != " ".join(_extra_flags()):
                return False
    except OSError:
        return False
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "cfet.h"), __file__]
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and _up_to_date():
        return LIB_PATH
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, verbose), SOURCES))
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB_PATH)
    with open(FLAGS_STAMP, "w") as fh:
        fh.write(" ".join(_extra_flags()))
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
