"""Build libtucker.so (all CUDA sources under csrc/) for sm_103a, in-tree.

    python -m paper_2010_10638_gb300.build [--force] [--verbose] [--checked]

Each translation unit compiles in its own nvcc process (in parallel); the objects
are linked into paper_2010_10638_gb300/_build/libtucker.so.  A unit is rebuilt
when it or any header is newer than its object.  `--checked` (build_checked) also links
_build/checked/libtucker.so, the same library with the cluster QRP compiled with
TUCKER_QRP_CHECKED (every array index compared with its array's length), for the tests.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtucker.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                     "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdr_mtime = max((os.path.getmtime(h) for h in headers()), default=0.0)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + list(extra_flags or [])
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_mtime):
            jobs.append([nvcc] + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            rcs = list(ex.map(run, jobs))
        if any(rcs):
            raise RuntimeError("nvcc failed")
    if jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        if run(cmd) != 0:
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


CHECKED_DIR = os.path.join(BUILD, "checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "libtucker.so")
CHECKED_UNITS = ("qrp_cluster.cu",)


def build_checked(verbose: bool = False) -> str:
    """The library with the units in CHECKED_UNITS compiled with -DTUCKER_QRP_CHECKED and
    the other objects of the normal build."""
    build(verbose=verbose)
    os.makedirs(CHECKED_DIR, exist_ok=True)
    hdr_mtime = max((os.path.getmtime(h) for h in headers()), default=0.0)
    nvcc = _nvcc()
    objs = []
    for src in sources():
        name = os.path.basename(src)
        if name not in CHECKED_UNITS:
            objs.append(os.path.join(BUILD, name[:-3] + ".o"))
            continue
        obj = os.path.join(CHECKED_DIR, name[:-3] + ".o")
        objs.append(obj)
        if not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_mtime):
            cmd = [nvcc] + NVCC_FLAGS + ["-DTUCKER_QRP_CHECKED", "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed (checked build)")
    if not os.path.exists(CHECKED_LIB) or os.path.getmtime(CHECKED_LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = CHECKED_LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs,
                           capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed (checked build)")
        os.replace(tmp, CHECKED_LIB)
    return CHECKED_LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
    if "--checked" in sys.argv:
        print(build_checked(verbose="--verbose" in sys.argv))
