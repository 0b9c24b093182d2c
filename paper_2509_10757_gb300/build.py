"""Build libfasttrack.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit compiles in parallel to an object file, then one
link step makes the shared library.  Host code is built without FP
contraction; device floating point uses explicitly rounded intrinsics.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfasttrack.so")
SOURCES = ["ft_kernels.cu", "ft_pyramid.cu", "ft_orb.cu", "ft_api.cu", "ft_noalloc.cu", "ft_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfasttrack.so")


def _flags(debug: bool = False) -> list:
    f = ARCH + ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"]
    if debug:
        f += ["-DFT_DEBUG=1"]
    return f


def _stale(target: str, deps: list) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          defines: tuple = (), out: str | None = None) -> str:
    """Compile (if stale) and return the library path.  `defines` adds -D
    flags and `out` names another output (a variant build: its objects go to
    a build folder of their own)."""
    global BUILD, LIB
    if defines or out:
        tag = "_".join(d.replace("=", "") for d in defines) or "variant"
        saved = (BUILD, LIB)
        BUILD = os.path.join(HERE, "_build", tag)
        LIB = out or os.path.join(BUILD, "libfasttrack.so")
        try:
            return _build(force, verbose, ptxas_info, ["-D" + d for d in defines])
        finally:
            BUILD, LIB = saved
    return _build(force, verbose, ptxas_info, [])


def _build(force: bool, verbose: bool, ptxas_info: bool, dflags: list) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
    headers.append(os.path.join(INCLUDE, "fasttrack.h"))
    exe = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [exe] + _flags() + dflags + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", path, "-o", obj]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or ptxas_info or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libfasttrack.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
