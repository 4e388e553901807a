"""Build the CUDA library (sm_103a) in-tree: paper_2012_07266_gb300/libpmlens.so.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library against the shared CUDA runtime.  No CMake, no torch extension
machinery: the library exposes a plain C ABI (include/pm.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpmlens.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "--expt-relaxed-constexpr"]

# (source, object, extra defines)
UNITS = [
    ("fft.cu", "fft_f32.o", ["-DPM_REAL=float"]),
    ("fft.cu", "fft_f64.o", ["-DPM_REAL=double"]),
    ("particles.cu", "particles.o", []),
    ("lens.cu", "lens.o", []),
    ("capi.cu", "capi.o", []),
    ("cosmo.cpp", "cosmo.o", []),
    ("prof.cpp", "prof.o", []),
    ("tma_map.cpp", "tma_map.o", []),
    ("static_forces.cu", "static_forces.o", []),
    ("adjoint.cu", "adjoint.o", []),
    ("sort.cu", "sort.o", []),
    ("jvp.cu", "jvp.o", []),
    ("shotnoise.cu", "shotnoise.o", []),
]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src, obj, extra):
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def sources_newer_than(path) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    for root, _, files in os.walk(CSRC):
        for f in files:
            if os.path.getmtime(os.path.join(root, f)) > t:
                return True
    hdr = os.path.join(os.path.dirname(HERE), "include", "pm.h")
    return os.path.getmtime(hdr) > t if os.path.exists(hdr) else False


def build(force: bool = False, verbose: bool = True) -> str:
    if not force and not sources_newer_than(OUT):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        list(ex.map(lambda u: _compile(*u), UNITS))
    objs = [os.path.join(BUILD, u[1]) for u in UNITS]
    tmp = OUT + ".tmp"
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-Xlinker", f"-rpath,{cudalib}", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print(f"built {OUT}", file=sys.stderr)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv)
