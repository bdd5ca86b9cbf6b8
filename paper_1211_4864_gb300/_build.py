"""Builds the CUDA library in-tree for sm_103a with nvcc.

Two variants: libhacc_sr.so (the product) and libhacc_sr_debug.so, the same
sources compiled with -DHACC_DEBUG_BOUNDS=1, whose pair kernels check every
index a task leads to before using it and report violations in the device
status word (HACC_STATUS_BOUNDS) instead of touching memory out of range.
Each translation unit compiles in parallel, then one link step per variant
produces the shared library next to this file.  A rebuild happens only when a
source or the public header is newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhacc_sr.so")
LIB_DEBUG = os.path.join(PKG, "libhacc_sr_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
VARIANTS = {"release": (LIB, os.path.join(BUILD, "release"), []),
            "debug": (LIB_DEBUG, os.path.join(BUILD, "debug"), ["-DHACC_DEBUG_BOUNDS=1"])}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(variant: str = "release") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def compile_flags(verbose_ptxas: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC,
                "-Xcompiler", "-fPIC,-ffp-contract=off,-O2"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          variants=("release", "debug")) -> str:
    """Build the requested variants (all translation units of all of them in
    one parallel pool); returns the release library's path."""
    todo = [v for v in variants if force or not up_to_date(v)]
    if not todo:
        return LIB
    cc = nvcc()
    srcs = _sources()
    jobs_list = []
    for v in todo:
        lib, out_dir, extra = VARIANTS[v]
        os.makedirs(out_dir, exist_ok=True)
        for src in srcs:
            jobs_list.append((v, src, os.path.join(out_dir, os.path.basename(src)[:-3] + ".o"), extra))

    def one(job):
        v, src, obj, extra = job
        cmd = [cc, "-c", src, "-o", obj] + compile_flags(verbose_ptxas) + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} ({v}):\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(16, os.cpu_count() or 8, len(jobs_list))) as ex:
        logs = list(ex.map(one, jobs_list))
    for v in todo:
        lib, out_dir, _ = VARIANTS[v]
        objs = [j[2] for j in jobs_list if j[0] == v]
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([cc, "-shared"] + ARCH + ["-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed ({v}):\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose_ptxas:
        for (v, src, _, _), log in zip(jobs_list, logs):
            print(f"== {v} {os.path.basename(src)}\n{log}")
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
          variants=("release",) if "--release-only" in sys.argv else ("release", "debug"))
    print(LIB)
