"""Build libgblu.so in-tree with nvcc for sm_103a (GB300).

CUDA sources are compiled with ``-gencode arch=compute_103a,code=sm_103a``;
host C++ sources with the system g++.  Translation units compile in
parallel; the result is ``paper_2411_14082_gb300/_build/libgblu.so``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libgblu.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgblu")


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(INCLUDE, "gblu.h")]
    return cu, cpp, hdr


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    cu, cpp, hdr = _sources()
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in cu + cpp + hdr + [__file__])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp, _ = _sources()
    jobs, objs = [], []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = ["g++", *CXX_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    procs = [(subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), s) for c, s in jobs]
    errors = []
    for p, src in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            (errors if p.returncode else []).append(f"--- {src}\n{out.decode(errors='replace')}")
            if verbose and out:
                print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("libgblu build failed:\n" + "\n".join(errors))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
