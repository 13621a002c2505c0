"""Build the in-tree shared library ``_lib/libemrkc.so`` for sm_103a.

The CUDA translation units are compiled with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` only; the host runtime with g++
(OpenMP for the assembly).  Units are compiled in parallel and linked with
nvcc into one shared library exposing the C ABI of include/emrkc.h.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libemrkc.so")

GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_UNITS = ["kernels_fp64.cu", "kernels_mixed.cu", "batch.cu", "noalloc.cu", "rl_methods.cu", "mrkc.cu"]
HOST_UNITS = ["solver.cpp", "assemble.cpp", "batch_host.cpp"]
FAST_MATH_UNITS = {"kernels_mixed.cu", "batch.cu"}


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.isdir(c):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("CUDA toolkit not found (nvcc)")


def _sources_newer(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build(verbose: bool = False, force: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "emrkc.h"))
    cuda_units = [u for u in CUDA_UNITS if os.path.exists(os.path.join(CSRC, u))]
    host_units = [u for u in HOST_UNITS if os.path.exists(os.path.join(CSRC, u))]
    all_src = [os.path.join(CSRC, u) for u in cuda_units + host_units] + headers
    if not force and not _sources_newer(LIB, all_src):
        return LIB
    procs = []
    objs = []
    for u in cuda_units:
        obj = os.path.join(BUILD_DIR, u + ".o")
        objs.append(obj)
        # the mixed-precision unit uses approximate FP32 division/sqrt and
        # flush-to-zero (FP64 code in it is unaffected)
        fast = ["-use_fast_math"] if u in FAST_MATH_UNITS else []
        # a non-void function without a return is undefined behaviour that
        # the optimiser turns into a function that never returns: an error
        cmd = [nvcc, *GENCODE, "-O3", "-lineinfo", "-std=c++17", *fast, "--diag-error", "940",
               "-Xcompiler", "-fPIC,-Werror=return-type",
               "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, u), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for u in host_units:
        obj = os.path.join(BUILD_DIR, u + ".o")
        objs.append(obj)
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-Werror=return-type", "-I", INCLUDE, "-I", CSRC,
               "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, u), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("build failed:\n" + msg)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *GENCODE, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
