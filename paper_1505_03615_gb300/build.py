"""Build liblbmg.so in-tree: CUDA sources for sm_103a with nvcc, the host
hierarchy builder with g++ and OpenMP, compiled in parallel and linked into one
shared library under paper_1505_03615_gb300/_build/."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["assemble.cu", "relax.cu", "packed.cu", "persist.cu", "narrow.cu", "learned.cu", "noalloc.cu", "cmcf.cu", "lobpcg.cu", "tune.cu", "clip.cu", "basis.cu", "api.cu"]
CPP = ["hier.cpp", "batch.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, h) for h in ("hier.h", "lbmg_internal.h")] + [
        os.path.join(os.path.dirname(HERE), "include", "lbmg.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for f in CU:
        o = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
               "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    for f in CPP:
        o = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or (verbose and out):
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace") + "\n")
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("liblbmg build failed")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC,-fopenmp", "-o", tmp, *objs, "-lgomp"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
