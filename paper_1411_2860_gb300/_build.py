"""Builds the CUDA library ``libprojgemm.so`` in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` is compiled to an object in parallel, then linked into one
shared library (static CUDA runtime) under ``paper_1411_2860_gb300/_lib/``.
A rebuild happens only when a source or header is newer than the library.

Two variants of the same sources exist:
  "pairs" -- ``libprojgemm.so``: the reduced GEMMs may run on clusters of two
             CTAs that share operand tiles through cluster-multicast TMA loads
             (one process on one GPU);
  "solo"  -- ``libprojgemm_solo.so``: compiled with ``-DPJ_CTA_PAIRS=0``, which
             leaves every multicast form out (``csrc/tc_pair.cuh`` is not
             included); the build that processes running one per GPU on
             several GPUs load.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(OUT_DIR, "obj")
LIB_PATH = os.path.join(OUT_DIR, "libprojgemm.so")
VARIANTS = {"pairs": [], "solo": ["-DPJ_CTA_PAIRS=0"]}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I" + INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libprojgemm")
    return path


def _sources():
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return srcs, deps


def lib_path(variant: str = "pairs") -> str:
    if variant not in VARIANTS:
        raise ValueError(f"unknown library variant {variant!r} (one of {sorted(VARIANTS)})")
    return LIB_PATH if variant == "pairs" else os.path.join(OUT_DIR, f"libprojgemm_{variant}.so")


def compile_flags(variant: str = "pairs"):
    """nvcc flags of one translation unit of `variant` (before -c / -o)."""
    if variant not in VARIANTS:
        raise ValueError(f"unknown library variant {variant!r}")
    return [*ARCH, *NVCC_FLAGS, *VARIANTS[variant]]


def sources():
    """The translation units every variant compiles."""
    return _sources()[0]


def up_to_date(variant: str = "pairs") -> bool:
    path = lib_path(variant)
    if not os.path.exists(path):
        return False
    _, deps = _sources()
    t = os.path.getmtime(path)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, variant: str = "pairs") -> str:
    """Compile and link one variant of libprojgemm; returns its path.  Processes
    that build at the same time (one per GPU) take turns on a lock file."""
    path = lib_path(variant)
    if not force and up_to_date(variant):
        return path
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, f".build_{variant}.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and up_to_date(variant):
                return path
            return _build_locked(path, verbose, variant)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(path: str, verbose: bool, variant: str) -> str:
    obj_dir = OBJ_DIR if variant == "pairs" else os.path.join(OUT_DIR, f"obj_{variant}")
    os.makedirs(obj_dir, exist_ok=True)
    srcs, _ = _sources()
    cc = nvcc()
    flags = compile_flags(variant)

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = path + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    import sys
    for v in (sys.argv[1:] or ["pairs"]):
        print(build(force=True, verbose=True, variant=v))
