"""Compile liblskum.so (CUDA kernels for sm_103a + host orchestration) in-tree.

Run as ``python -m paper_2406_07441_gb300.build``; ``__graft_entry__.build()``
calls :func:`build`.  Translation units compile in parallel with nvcc; one
``-gencode`` (compute_103a/sm_103a); the CUDA runtime is linked statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblskum.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lskum_kernels.cu", "lskum_host.cpp", "lskum_noalloc.cu", "lskum_mlp.cu"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblskum")


def _deps():
    files = ([os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
             + [__file__])
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tmpdir = os.path.join(OUT_DIR, f"obj{os.getpid()}")
    os.makedirs(tmpdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, *extra_flags]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(tmpdir, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, *common]
        if src.endswith(".cu"):
            cmd += [*ARCH, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        shutil.rmtree(tmpdir, ignore_errors=True)
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lrt", "-ldl"])
    os.replace(tmp, LIB)
    shutil.rmtree(tmpdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
