"""Builds the in-tree shared library ``librdm.so`` (CUDA for sm_103a + C++ host code).

Usage: ``python -m paper_2204_08147_gb300.build`` (or ``build_library()``). The
translation units compile in parallel; the output and objects stay in-tree under
``paper_2204_08147_gb300/_build`` (git-ignored) and ``paper_2204_08147_gb300/librdm.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librdm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librdm.so")
    return cand


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def build_library(verbose: bool = False, extra_nvcc: list[str] | None = None) -> str:
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    cu_flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                "-Xptxas", "-warn-spills"] + ARCH + (extra_nvcc or [])
    cxx_flags = ["-O3", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
                 "-I", os.path.join(cuda, "include")]
    jobs = []
    for name in sorted(os.listdir(CSRC)):
        src = os.path.join(CSRC, name)
        obj = os.path.join(BUILD, name + ".o")
        if name.endswith(".cu"):
            cmd = [nvcc] + cu_flags + inc + ["-c", src, "-o", obj]
        elif name.endswith(".cpp"):
            cmd = [shutil.which("g++") or "g++"] + cxx_flags + inc + ["-c", src, "-o", obj]
        else:
            continue
        jobs.append((cmd, obj))
    procs = [(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True), cmd, obj)
             for cmd, obj in jobs]
    failed = []
    for p, cmd, obj in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + (out or ""))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    tmp = LIB + ".tmp"
    link = [nvcc, "-shared"] + ARCH + ["-o", tmp] + [o for _, o in jobs] + ["-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout)
    if r.returncode != 0:
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(verbose="-v" in sys.argv))
