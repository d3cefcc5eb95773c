"""Build libpic.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_2004_03754_gb300.build

Translation units compile in parallel; the shared library lands next to this
file, where the Python binding loads it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpic.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "fields.cu", "particles.cu", "particles_f32.cu", "particles_f64.cu",
           "particles_dfl.cu", "batch.cu", "adjoint.cu", "noalloc.cu", "spectral.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "pic.h"))
    procs, objs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if _stale(o, [s] + headers):
            cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        for src, out in failed:
            sys.stderr.write("nvcc failed on %s:\n%s\n" % (src, out))
        raise RuntimeError("libpic build failed")
    if procs or not os.path.exists(OUT):
        tmp = OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcufft"])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
