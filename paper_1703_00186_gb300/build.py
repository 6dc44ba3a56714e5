"""Builds liblbm.so in-tree for sm_103a (nvcc + g++, no cmake).

    python -m paper_1703_00186_gb300.build          # incremental
    python -m paper_1703_00186_gb300.build --force  # full rebuild

Translation units compile in parallel into ``_build/``; the shared library
is written next to this file.  The double-double quadrature solver is
compiled by the host compiler with -ffp-contract=off (its error-free
transforms need separately rounded operations).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _headers_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.join(HERE, "..", "include", "lbm.h"))
    paths.append(os.path.join(HERE, "..", "include", "lbm_batch.h"))
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def _compile(cmd, obj, src, hdr_mtime, force):
    if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
            and os.path.getmtime(obj) >= hdr_mtime):
        return None
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
    return None


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = _sources()
    hdr = _headers_mtime()
    jobs = []
    objs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f[:-3] + ".o")
        cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "--extended-lambda",
               "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
        jobs.append((cmd, obj, src))
        objs.append(obj)
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f[:-4] + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off",
               "-I/usr/local/cuda/include", "-c", src, "-o", obj]
        jobs.append((cmd, obj, src))
        objs.append(obj)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        errs = [e for e in ex.map(lambda j: _compile(j[0], j[1], j[2], hdr, force), jobs) if e]
    if errs:
        raise RuntimeError("liblbm build failed:\n" + "\n".join(errs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [nvcc, "-shared", *ARCH, "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("liblbm link failed:\n" + r.stdout + r.stderr)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    args = ap.parse_args()
    try:
        build(force=args.force, verbose=True)
    except RuntimeError as e:
        print(e, file=sys.stderr)
        sys.exit(1)
