"""Compile the sm_103a CUDA library (libflbm) in-tree with nvcc.

The shared object goes to paper_1909_01092_gb300/_build/libflbm_<machine>.so
and is rebuilt when any source under csrc/ or the public header is newer.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def lib_path() -> str:
    return os.path.join(BUILD, f"libflbm_{platform.machine()}.so")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the FLBM CUDA library cannot be built")
    return exe


def _compile(src: str, obj: str, verbose: bool) -> str:
    cmd = [nvcc(), *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17", "-c", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-o", obj, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every csrc/*.cu in parallel (one translation unit each) and
    link them into the shared library."""
    out = lib_path()
    srcs = _sources()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(s) for s in srcs):
        return out
    tag = f".tmp{os.getpid()}"
    objdir = os.path.join(BUILD, f"obj_{platform.machine()}{tag}")
    os.makedirs(objdir, exist_ok=True)
    units = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs = [os.path.join(objdir, os.path.basename(u)[:-3] + ".o") for u in units]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(units)) as pool:
        logs = list(pool.map(lambda uo: _compile(uo[0], uo[1], verbose), zip(units, objs)))
    if verbose:
        print("".join(logs))
    tmp = out + tag
    r = subprocess.run([nvcc(), *ARCH_FLAGS, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    shutil.rmtree(objdir, ignore_errors=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
