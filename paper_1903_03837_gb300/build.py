"""Builds the sm_103a shared library liblumipath.so in-tree with nvcc.

Each .cu of csrc/ compiles to an object in parallel, then nvcc links them
into paper_1903_03837_gb300/_build/liblumipath.so (CUDA runtime linked
statically). Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblumipath.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblumipath.so")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


DEBUG_DIR = os.path.join(BUILD, "debug")


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_dir: str = None) -> str:
    """Compile every .cu of csrc/ in parallel and link liblumipath.so. With
    `out_dir` the objects and the library go there instead of _build/ (e.g. the
    debug build: extra_flags=["-DLF_DEBUG_CHECKS"], out_dir=DEBUG_DIR)."""
    bdir = out_dir or BUILD
    lib = os.path.join(bdir, "liblumipath.so")
    if not force and not extra_flags and out_dir is None and up_to_date():
        return LIB
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    srcs = _sources()
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def comp(pair):
        s, o = pair
        cmd = [cc, *NVCC_FLAGS, *extra_flags, "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with ThreadPoolExecutor(len(srcs)) as ex:
        logs = list(ex.map(comp, zip(srcs, objs)))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    build(force=True, verbose=True, extra_flags=sys.argv[1:])
    print(LIB)
