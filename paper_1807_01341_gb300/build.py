"""Build libsph_gb300.so in-tree with nvcc for sm_103a, and beside it
libsph_gb300_checks.so, the same sources compiled with -DSPH_CHECKS (device
bounds checks that record SPH_ERR_BOUNDS instead of accessing out of range).

The translation units of both libraries compile in parallel; each shared
library links against the CUDA runtime only (no torch symbols cross the C ABI).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsph_gb300.so")
CHECKS_LIB = os.path.join(OUT_DIR, "libsph_gb300_checks.so")
SOURCES = ["sph_cells.cu", "sph_integrate.cu", "sph_pairs.cu", "sph_adjoint.cu", "sph_api.cu",
           "sph_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checks: bool = True) -> str:
    """Builds the library (and, with checks, the bounds-checked one); returns
    the path of the plain library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdrs = [os.path.join(CSRC, "sph_internal.cuh"), os.path.join(CSRC, "sph_pairloop.cuh"),
            os.path.join(CSRC, "sph_diag.cuh"),
            os.path.join(os.path.dirname(HERE), "include", "sph.h")]
    variants = [(LIB, OUT_DIR, [])]
    if checks:
        variants.append((CHECKS_LIB, os.path.join(OUT_DIR, "checks"), ["-DSPH_CHECKS"]))
    jobs, links = [], []
    for lib, odir, defs in variants:
        os.makedirs(odir, exist_ok=True)
        objs = []
        stale = False
        for src in SOURCES:
            path = os.path.join(CSRC, src)
            obj = os.path.join(odir, src.replace(".cu", ".o"))
            objs.append(obj)
            if force or _stale(obj, [path] + hdrs):
                cmd = [nvcc(), *ARCH, *FLAGS, *defs, *extra, "-c", path, "-o", obj]
                if verbose:
                    cmd.insert(1, "-Xptxas=-v")
                jobs.append(cmd)
                stale = True
        if force or stale or not os.path.exists(lib):
            links.append((lib, objs))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    for lib, objs in links:
        tmp = lib + ".tmp.%d" % os.getpid()
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
