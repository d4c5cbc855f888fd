"""Build step of the package: compiles csrc/ into libdecbpm.so (in-tree) for
sm_103a with nvcc, and the same sources with -DDECBPM_BOUNDS_CHECK into
libdecbpm_checked.so (the march kernels test every gather index and report
DECBPM_ERR_DEVICE_CHECK instead of reading out of bounds).  Needs no GPU.
Usage: ``python -m paper_2608_03587_b300.build [--force] [--checked | --all]``."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libdecbpm.so")
CHECKED_LIB = os.path.join(HERE, "libdecbpm_checked.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("api.cu", "assembly.cpp")]
HEADERS = [os.path.join(HERE, "csrc", f) for f in ("internal.h", "kernels.cuh")] + [
    os.path.join(ROOT, "include", "decbpm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def lib_path(checked: bool = False) -> str:
    return CHECKED_LIB if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    LIB = lib_path(checked)
    if not force and up_to_date(checked):
        return LIB
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"),
           *(["-DDECBPM_BOUNDS_CHECK"] if checked else []),
           "-o", LIB + ".tmp", *SOURCES, *(extra or [])]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose and (res.stdout or res.stderr):
        print(res.stdout + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    variants = [False, True] if "--all" in sys.argv else [("--checked" in sys.argv)]
    for chk in variants:
        build(force="--force" in sys.argv, verbose=True, checked=chk,
              extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
