"""Build the in-tree shared library libsem.so (C ABI in include/sem.h).

Compiles the host preprocessing (g++) and the CUDA sources (nvcc, sm_103a
only) in parallel, then links them into paper_2104_08416_gb300/libsem.so.
Usage: python -m paper_2104_08416_gb300.build  (or build() from Python).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


# sem_kernels.cu is compiled once per element order (SEM_KERNEL_NP = p + 1,
# orders 1..8) for the kernels templated on the order, and once without it
# for the dispatchers and the order-independent kernels: nine translation
# units that compile in parallel.
KERNEL_NP = tuple(range(2, 10))


def _units():
    """(source, object name, extra flags) of every translation unit."""
    u = [(os.path.join(CSRC, "sem_host.cpp"), "sem_host.o", []),
         (os.path.join(CSRC, "sem_api.cu"), "sem_api.o", []),
         (os.path.join(CSRC, "sem_kernels.cu"), "sem_kernels.o", [])]
    for n in KERNEL_NP:
        u.append((os.path.join(CSRC, "sem_kernels.cu"), f"sem_kernels_np{n}.o", [f"-DSEM_KERNEL_NP={n}"]))
    return u


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "sem.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def _compile(unit, nvcc: str) -> str:
    src, name, extra = unit
    obj = os.path.join(OUT_DIR, name)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if src.endswith(".cpp"):
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall", *inc, "-c", src, "-o", obj]
    else:
        cmd = [nvcc, *ARCH, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
               *extra, *inc, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsem.so if any input is newer than it; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    units = _units()
    with ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda u: _compile(u, nvcc), units))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
