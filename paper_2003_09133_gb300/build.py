"""Compile the lfbp CUDA library (sm_103a) in-tree with nvcc.

The library is written to ``paper_2003_09133_gb300/_build/liblfbp.so``; the
Python binding loads it from there and refuses to run without it.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblfbp.so")
# self-checking variant (-DLFBP_CHECK): bounds/alignment checks on every access
LIB_CHECK = os.path.join(BUILD, "liblfbp_check.so")

SOURCES = ["lfbp.cu", "lfbp_project.cu"]
HEADERS = ["lfbp_device.cuh", "lfbp_stripes.cuh", "lfbp_pairs.cuh", "lfbp_project.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the lfbp CUDA library cannot be built")
    return cand


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "lfbp.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    """Build liblfbp.so (or the self-checking liblfbp_check.so) if it is missing
    or older than its sources; return its path."""
    lib = LIB_CHECK if check else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    objs, procs = [], []
    if check:
        extra = list(extra) + ["-DLFBP_CHECK"]
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".check.o" if check else ".o"))
        cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
        objs.append(obj)
    logs = []
    for p in procs:
        out, _ = p.communicate()
        logs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + "\n".join(logs))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    if verbose:
        print("\n".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
