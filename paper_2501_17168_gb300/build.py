"""Builds the in-tree shared library ``_build/libtgp.so`` for sm_103a.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel (one -gencode for
sm_103a, -lineinfo), then linked into one shared library exporting the C ABI
of ``include/tgp.h``.  Also builds the host-side tree generator.  Usage:
``python -m paper_2501_17168_gb300.build [--force] [--verbose]``.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtgp.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtgp.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(INCLUDE, "tgp.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def generate(force: bool = False):
    """Regenerates the inline-PTX interpreter headers (and the forward
    instruction-set header) when their generator changed."""
    gen = os.path.join(CSRC, "gen_interp.py")
    gen_b = os.path.join(CSRC, "gen_interp_bwd.py")
    if force or any(_stale(os.path.join(CSRC, f), [gen]) for f in ("interp_fwd.cuh", "isa_fwd.cuh")):
        subprocess.check_call([sys.executable, gen], cwd=CSRC)
    if force or _stale(os.path.join(CSRC, "interp_bwd.cuh"), [gen, gen_b]):
        subprocess.check_call([sys.executable, gen_b], cwd=CSRC)


def build_library(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    generate()
    srcs = _sources()
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "tgp.h")]
    if not force and not _stale(LIB, _deps()):
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_all(force: bool = False, verbose: bool = False) -> str:
    from . import workloads
    workloads.build_treegen(force=force)
    return build_library(force=force, verbose=verbose)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build_all(force=a.force, verbose=a.verbose))


if __name__ == "__main__":
    main()
