"""Builds the casim CUDA library (libcasim.so) and its bounds-checked twin
(libcasim_checked.so, -DCASIM_CHECKED) in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel; the shared objects land next to
this file, where the Python binding loads them.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
BUILD_CHECKED = os.path.join(HERE, "_build", "checked")
LIB = os.path.join(HERE, "libcasim.so")
LIB_CHECKED = os.path.join(HERE, "libcasim_checked.so")

SOURCES = ["api.cu", "collision.cu", "solve.cu", "adjoint.cu", "noalloc.cu", "remesh.cu", "anderson.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _compile(src: str, extra, build_dir: str = None) -> str:
    obj = os.path.join(build_dir or BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + FLAGS + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def _link(objs, lib: str, verbose: bool) -> str:
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


def build(extra_flags=(), verbose: bool = False, checked: bool = True) -> str:
    """Compiles every source and links libcasim.so and, with checked=True,
    libcasim_checked.so (-DCASIM_CHECKED: bounds-checked gathers), all
    translation units in parallel; returns the path of libcasim.so."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = [(s, BUILD, tuple(extra_flags)) for s in SOURCES]
    if checked:
        os.makedirs(BUILD_CHECKED, exist_ok=True)
        jobs += [(s, BUILD_CHECKED, tuple(extra_flags) + ("-DCASIM_CHECKED",)) for s in SOURCES]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], j[2], j[1]), jobs))
    _link(objs[: len(SOURCES)], LIB, verbose)
    if checked:
        _link(objs[len(SOURCES):], LIB_CHECKED, verbose)
    return LIB


if __name__ == "__main__":
    build(extra_flags=sys.argv[1:], verbose=True)
