"""Compile libebit.so for sm_103a in-tree (paper_2309_00338_gb300/_build).

Each translation unit is compiled to an object in parallel, then linked."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libebit.so")
SOURCES = ["ebit.cu", "ebit_noalloc.cu", "ebit_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "ebit.h"))
    return files


CHECK_LIB_PATH = os.path.join(OUT_DIR, "libebit_check.so")


def build_library(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA library (idempotent; rebuilds when a source changed).
    checked=True builds the debug variant libebit_check.so, compiled with
    EBIT_CHECK: the step kernels check every global index against its array
    and record a miss instead of making the access (ebit_check_status)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib_path = CHECK_LIB_PATH if checked else LIB_PATH
    newest = max(os.path.getmtime(f) for f in _inputs())
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    pid = os.getpid()
    tag = "chk." if checked else ""

    def compile_one(src):
        obj = os.path.join(OUT_DIR, f"{os.path.splitext(src)[0]}.{tag}{pid}.o")
        cmd = [nvcc(), *ARCH, *FLAGS, *(["-DEBIT_CHECK"] if checked else []), "-I", INCLUDE, "-I", CSRC,
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".{pid}.tmp"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
    for o in objs:
        os.unlink(o)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose="-v" in sys.argv))
