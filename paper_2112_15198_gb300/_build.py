"""Compile the CUDA sources into the in-tree shared library (sm_103a only).

The translation units are compiled in parallel with nvcc and linked into
``_build/libifgf_<arch>.so`` (static CUDA runtime, no torch dependency).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, f"libifgf_{platform.machine()}.so")
# the same sources with every bounds check compiled in (-DIFGF_CHECKS)
CHECKS_LIB = os.path.join(BUILD, f"libifgf_checks_{platform.machine()}.so")
SOURCES = ["util.cu", "plan.cu", "apply.cu", "api.cu", "noalloc.cu", "batch.cu", "batch_queue.cu", "shard.cu", "prop_tc.cu", "tune.cu", "solve.cu"]
# throughput probes for the roofline denominators (a library of their own)
PEAKS_LIB = os.path.join(BUILD, f"libifgf_peaks_{platform.machine()}.so")
PEAKS_SOURCES = ["peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the IFGF CUDA library cannot be built")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ifgf.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Build the libraries if a source is newer than them; return the IFGF library's path (the
    checked variant, compiled with -DIFGF_CHECKS, when checks is true)."""
    os.makedirs(BUILD, exist_ok=True)
    lib_path = CHECKS_LIB if checks else LIB
    if not force and all(os.path.exists(f) and os.path.getmtime(f) >= _deps_mtime() for f in (lib_path, PEAKS_LIB)):
        return lib_path
    nvcc = _nvcc()
    tag = "_checks" if checks else ""
    extra = ["-DIFGF_CHECKS"] if checks else []

    def compile_one(src: str) -> str:
        t = tag if src in SOURCES else ""
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + f"{t}_{platform.machine()}.o")
        cmd = [nvcc, *ARCH, *FLAGS, *(extra if src in SOURCES else []), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + len(PEAKS_SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES + PEAKS_SOURCES))
    for lib, lo in ((lib_path, objs[:len(SOURCES)]), (PEAKS_LIB, objs[len(SOURCES):])):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *lo], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib_path


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
