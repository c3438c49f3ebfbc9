"""Compile the CUDA library (csrc/*.cu) into paper_2404_17344_gb300/_lib/libaddker.so for sm_103a.

Each translation unit is compiled to an object in parallel, then nvcc links the shared library.
Only the sm_103a target is built (one -gencode), so a build takes well under a minute.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libaddker.so")
SOURCES = ["addker.cu", "fft.cu", "spread_gather.cu", "noalloc.cu", "gradients.cu", "solver.cu", "gsi.cu"]
RATES_SOURCE = "rates.cu"                 # the device-rate microbenchmark: its own library, not the product's
RATES_LIB = os.path.join(OUT_DIR, "libaddker_rates.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", 
         "-Xptxas", "-v"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "addker.h"))
    files.append(os.path.join(HERE, "..", "include", "addker_rates.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.exists(RATES_LIB):
        newest = max(os.path.getmtime(f) for f in _deps())
        if min(os.path.getmtime(LIB), os.path.getmtime(RATES_LIB)) >= newest:
            return LIB
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(r.stderr)
        if verbose:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [RATES_SOURCE]))
    rates_obj = objs.pop()
    tmp_r = RATES_LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", rates_obj, "-o", tmp_r, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed (rates):\n{r.stdout}\n{r.stderr}")
    os.replace(tmp_r, RATES_LIB)
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
