"""Build libhphi.so (the CUDA library behind include/hphi.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel and linked into one
shared library in paper_2307_13222_gb300/_build/.  Run `python -m
paper_2307_13222_gb300.build` or call build().
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhphi.so")
SOURCES = ["basis.cu", "ham.cu", "hv.cu", "hv_lean.cu", "hv_fly.cu", "hv_staged.cu", "hv_phased.cu", "hv_seg.cu", "hv_tile.cu", "vec.cu", "pattern.cu", "capi.cu", "drivers.cu",
           "spectrum.cu", "evolve.cu", "batch.cu", "serve.cu",
           "lobpcg.cu", "tune.cu", "methods.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "hphi.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


# sources every H*x kernel's code and tables depend on: the shared headers and
# the basis / Hamiltonian table builders
HV_COMMON = ["basis.cu", "ham.cu", "hvcommon.cuh", "rowvisit.cuh", "hphi_internal.cuh"]
# units that name kernels defined in other files (hv.cu launches the lean and
# the on-the-fly kernels)
TAG_DEPS = {"hv.cu": ["hv_lean.cu", "hv_fly.cu"]}


def source_tag(unit: str = "hv.cu") -> str:
    """Short hash of one translation unit and the sources its H*x kernels
    depend on: hphi_last_kernel appends it to the kernel name, so a profile
    taken on other sources of that kernel does not match (and one taken
    before a change to another kernel's file still does)."""
    import hashlib
    h = hashlib.sha1()
    for f in [unit] + TAG_DEPS.get(unit, []) + HV_COMMON:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:10]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT, exist_ok=True)
    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        inc = ["-I", os.path.join(ROOT, "include"), f"-DHPHI_SRC_TAG=\"{source_tag(src)}\""]
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + FLAGS + inc
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
