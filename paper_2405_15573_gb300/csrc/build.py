"""Build libuh.so in-tree: CUDA sources with nvcc for sm_103a, host sources with g++.

Run as `python -m paper_2405_15573_gb300.csrc.build` (or through __graft_entry__.build()).
Objects go to paper_2405_15573_gb300/_build/, the library to paper_2405_15573_gb300/libuh.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libuh.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["uh_stream.cu", "uh_noalloc.cu", "uh_panel.cu", "uh_solve.cu", "uh_probe.cu", "uh_gbuild.cu"]
CPP_SOURCES = ["uh_capi.cpp", "uh_program.cpp", "uh_build.cpp", "uh_panel_pack.cpp", "uh_serve.cpp"]


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith(".h")]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    jobs = []
    objs = []
    for s in CU_SOURCES:
        src = os.path.join(HERE, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _newer([src] + headers, obj):
            jobs.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-I", INCLUDE, "-I", HERE, "-c", src, "-o", obj])
    for s in CPP_SOURCES:
        src = os.path.join(HERE, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _newer([src] + headers, obj):
            jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-pthread", "-Wall", "-Wno-unused-function",
                         "-I", INCLUDE, "-I", HERE, "-I", os.path.join(CUDA_HOME, "include"),
                         "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for out in ex.map(_run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-Xcompiler", "-pthread", "-lgomp"])
        shutil.move(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
