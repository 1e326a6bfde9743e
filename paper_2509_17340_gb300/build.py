"""Build ``libaero_mppi.so`` in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into one shared
library exporting the C ABI of ``include/aero_mppi.h``.  Host code is compiled
with ``-ffp-contract=off`` (the binary32 partition decisions depend on the exact
operation order).
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaero_mppi.so")
# the same sources with AERO_CHECKED: every index the kernels rely on is
# checked on the device and a failed check is reported by aero_sync_status
CHECKED_LIB = os.path.join(PKG, "libaero_mppi_checked.so")
SOURCES = ["aero_mppi.cu", "partition.cu", "rollout.cu", "accum.cu"]
HEADERS = ["internal.h", "device.cuh", "adjoint.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaero_mppi.so")


def _flags(verbose_ptxas: bool, checked: bool = False) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                "-I", os.path.join(ROOT, "include")]
    if checked:
        f += ["-DAERO_CHECKED"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "aero_mppi.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Compile and link; returns the library path.  Skips work when up to date.
    checked: the checked build (CHECKED_LIB) instead of the product library."""
    lib = CHECKED_LIB if checked else LIB
    if not force and not _stale(lib):
        return lib
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = _flags(verbose_ptxas, checked)

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose_ptxas:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                checked="--checked" in sys.argv))
