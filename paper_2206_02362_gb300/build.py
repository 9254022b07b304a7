"""Builds libfwime.so (the sm_103a CUDA library behind include/fwime.h) in-tree.

Each .cu translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
``paper_2206_02362_gb300/_build/libfwime.so``.  No cmake, no torch extension
machinery: the library exports a plain C ABI and is loaded with ctypes.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfwime.so")
SOURCES = ["fwime_api.cu", "k_prop.cu", "k_ext.cu", "k_misc.cu", "k_spline.cu", "k_tlag.cu", "fwime_static.cu", "fwime_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfwime")
    return cand


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            f"-I{os.path.join(ROOT, 'include')}", "--expt-relaxed-constexpr", *extra]


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, defines=(), build_dir=None) -> str:
    """Compile every translation unit for sm_103a and link libfwime.so; returns its path.

    `defines` (e.g. ["FWIME_PROP_AUX_SLOTS=6"]) and `build_dir` build a variant of the library
    into another directory (tuning experiments); the default build is the one the package loads."""
    global BUILD, LIB
    if build_dir is not None:
        saved = BUILD, LIB
        BUILD, LIB = build_dir, os.path.join(build_dir, "libfwime.so")
        try:
            return build(force, verbose, ptxas_info, [f"-D{d}" for d in defines] if defines else ())
        finally:
            BUILD, LIB = saved
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, "fwime_kernels.cuh"), os.path.join(CSRC, "fwime_internal.h"),
               os.path.join(ROOT, "include", "fwime.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s, *headers, __file__]):
            extra = (["-Xptxas", "-v"] if ptxas_info else []) + list(defines)
            jobs.append([nvcc(), *_flags(extra), "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or ptxas_info:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
