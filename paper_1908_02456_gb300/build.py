"""Builds the native library ``_lib/libabc.so`` in-tree.

CUDA sources are compiled by nvcc for sm_103a only; the FP64 host setup by g++
with OpenMP.  Translation units compile in parallel.  A stamp of the sources and
flags skips the rebuild when nothing changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libabc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-fopenmp", "-I", INC, "-I", CSRC]
CXX_FLAGS = ["-std=c++17", "-O3", "-fPIC", "-fopenmp", "-I", INC, "-I", CSRC]

CU_SOURCES = ["api.cu", "noalloc.cu", "one_d.cu"]
CXX_SOURCES = ["dense.cpp", "setup.cpp", "symmetry.cpp", "host_api.cpp", "one_d_setup.cpp"]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stamp() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/abc.h", "../../include/abc1d.h"]:
        path = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(path):
            h.update(name.encode())
            h.update(open(path, "rb").read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    stamp_path = os.path.join(OUT, "stamp")
    st = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_path) and open(stamp_path).read() == st:
        return LIB
    nvcc = _nvcc()
    procs, objs = [], []
    for src in CU_SOURCES:
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for src in CXX_SOURCES:
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen(["g++", *CXX_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    failed = []
    for p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(p.args))
    if failed:
        raise RuntimeError("native build failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    with open(stamp_path, "w") as f:
        f.write(st)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
