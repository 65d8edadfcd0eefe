"""Build liblpic.so (CUDA for sm_103a) in-tree with nvcc, and on request the
checked library liblpic_check.so (LPIC_CHECK=1: bounds tests on the
data-dependent shared-memory indices of the tile kernels, which raise
LPIC_ST_BOUNDS instead of accessing).

    python -m paper_2607_13507_b300.build [--checked]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib", "liblpic.so")
OUT_CHECK = os.path.join(PKG, "_lib", "liblpic_check.so")
SOURCES = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = list(SOURCES)
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h")):
            files.append(os.path.join(CSRC, f))
    files.append(os.path.join(ROOT, "include", "lpic.h"))
    return files


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          checked: bool = False) -> str:
    out = OUT_CHECK if checked else OUT
    if checked:
        extra = list(extra or []) + ["-DLPIC_CHECK=1"]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tag = f"tmp{os.getpid()}"
    objdir = os.path.join(os.path.dirname(OUT), "obj." + tag)
    os.makedirs(objdir, exist_ok=True)
    try:
        # one translation unit per process (the tile-kernel instances are the
        # long ones), then one link
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", src, "-o", obj, *(extra or [])]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            objs.append(obj)
            procs.append((src, subprocess.Popen(cmd)))
        failed = [src for src, p in procs if p.wait() != 0]
        if failed:
            raise subprocess.CalledProcessError(1, "nvcc " + " ".join(os.path.basename(f) for f in failed))
        tmp = out + "." + tag
        cmd = [nvcc(), *ARCH, "--shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return out


if __name__ == "__main__":
    v = "-v" in sys.argv
    x = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else None
    print(build(force=True, verbose=v, extra=x, checked="--checked" in sys.argv))
