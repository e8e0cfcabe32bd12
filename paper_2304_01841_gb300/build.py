"""Build the CUDA library (sm_103a) in-tree: paper_2304_01841_gb300/_build/libwctsim.so.

Each translation unit is compiled by nvcc in parallel and linked into one shared library
against the shared CUDA runtime (so the library and PyTorch use one runtime instance).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwctsim.so")
SOURCES = ["wct_sim.cu", "k_depo.cu", "k_raster.cu", "k_fft.cu", "k_adc.cu", "wct_response.cu"]
HEADERS = ["wct_internal.cuh", "wct_device.cuh", "wct_tma.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _stale(outputs, inputs) -> bool:
    if not all(os.path.exists(o) for o in outputs):
        return True
    t_out = min(os.path.getmtime(o) for o in outputs)
    return any(os.path.getmtime(i) > t_out for i in inputs)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, bounds_check: bool = False) -> str:
    """Compile every translation unit (in parallel, only what changed) and link the library.
    bounds_check builds the debugging variant (-DWCT_BOUNDS_CHECK: the kernels check their
    computed indices) into _build_checked/ instead; returns the library's path."""
    nvcc = _nvcc()
    BUILD = os.path.join(HERE, "_build_checked" if bounds_check else "_build")
    LIB = os.path.join(BUILD, "libwctsim_checked.so" if bounds_check else "libwctsim.so")
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "wct_sim.h"),
                                                       os.path.abspath(__file__)]
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]
    if bounds_check:
        common += ["-DWCT_BOUNDS_CHECK"]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale([o], [s] + hdrs):
            jobs.append([nvcc, *common, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(run, jobs):
                if verbose or ptxas_verbose:
                    sys.stdout.write(out)
    if force or jobs or _stale([LIB], objs):
        tmp = LIB + f".tmp{os.getpid()}"
        libdir = _cuda_lib_dir(nvcc)
        run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
             "-Xlinker", "-rpath", "-Xlinker", libdir])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
