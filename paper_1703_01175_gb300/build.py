"""Compile the native libraries of the package in-tree.

libh2.so       CUDA C-ABI library (csrc/*.cu), sm_103a only.
libh2con.so    GPU kernels of the H^2 constructor (csrc_con/*.cu), sm_103a only.
libh2build.so  host constructor helpers (csrc_host/*.cpp).

Each translation unit is compiled by its own nvcc process in parallel and the
objects are linked into a shared library next to this file. Rebuilds only when
a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBH2 = os.path.join(HERE, "libh2.so")
CSRC_HOST = os.path.join(HERE, "csrc_host")
LIBH2BUILD = os.path.join(HERE, "libh2build.so")
CSRC_CON = os.path.join(HERE, "csrc_con")
LIBH2CON = os.path.join(HERE, "libh2con.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-fopenmp,-O3", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_libh2(verbose: bool = False, force: bool = False, srcdir: str = CSRC, target: str = LIBH2) -> str:
    srcs = sorted(glob.glob(os.path.join(srcdir, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(srcdir, "*.h")) + glob.glob(os.path.join(srcdir, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))
    if not force and not _stale(target, srcs + hdrs + [__file__]):
        return target
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(os.path.dirname(s)) + "_" + os.path.basename(s) + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(f"{s}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = target + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lgomp"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, target)
    return target


def build_libh2con(verbose: bool = False, force: bool = False) -> str:
    """GPU kernels of the H^2 constructor (setup)."""
    return build_libh2(verbose, force, CSRC_CON, LIBH2CON)


def build_libh2build(verbose: bool = False, force: bool = False) -> str:
    """Host-only constructor helpers (plain C++, portable: no -march flags)."""
    srcs = sorted(glob.glob(os.path.join(CSRC_HOST, "*.cpp")))
    hdrs = [os.path.join(INCLUDE, "h2build.h")]
    if not force and not _stale(LIBH2BUILD, srcs + hdrs + [__file__]):
        return LIBH2BUILD
    cxx = os.environ.get("CXX") or shutil.which("g++") or "c++"
    tmp = LIBH2BUILD + ".tmp"
    cmd = [cxx, "-O3", "-std=c++17", "-fcx-limited-range", "-fPIC", "-shared", "-I" + INCLUDE, *srcs, "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("g++ failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIBH2BUILD)
    return LIBH2BUILD


def build_all(verbose: bool = False, force: bool = False) -> None:
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(3) as ex:
        futs = [ex.submit(build_libh2, verbose, force), ex.submit(build_libh2build, verbose, force),
                ex.submit(build_libh2con, verbose, force)]
        for f in futs:
            f.result()


if __name__ == "__main__":
    build_all(verbose=True, force="--force" in sys.argv)
