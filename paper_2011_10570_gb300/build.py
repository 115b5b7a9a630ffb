"""Builds libltsoct.so in-tree for sm_103a (nvcc + g++, translation units in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libltsoct.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libltsoct")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp", ".h", ".cuh")))


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    hdr = os.path.join(os.path.dirname(HERE), "include", "ltsoct.h")
    return all(os.path.getmtime(s) <= t for s in sources() + [hdr, os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"]
    jobs = []
    objs = []
    for src in ("kernels.cu", "api.cu", "octree.cu"):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, *ARCH, *common, "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append(cmd)
        objs.append(obj)
    obj = os.path.join(BUILD, "host.cpp.o")
    jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-c", os.path.join(CSRC, "host.cpp"),
                 "-o", obj])
    objs.append(obj)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in jobs]
    for cmd, pr in zip(jobs, procs):
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            print(out)
        if pr.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
