"""Build libgmaf.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each .cu file is compiled in parallel, then linked into a shared object next to
this file.  Host code is compiled with -ffp-contract=off so that the lattice
set-up takes the same floating-point decisions on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgmaf.so")
SOURCES = ["gmaf_api.cu", "gmaf_assemble.cu", "gmaf_pcg.cu", "gmaf_tma.cu", "gmaf_drec.cu",
           "gmaf_server.cu", "gmaf_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return (ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC])


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "gmaf.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = _flags() + list(extra_flags or [])

    # per-process object names: ranks that build at the same time never link
    # each other's half-written objects (the library itself is replaced atomically)
    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", f".{os.getpid()}.o"))
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, "-shared"] + ARCH + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
