"""Build libwcns.so (the CUDA C-ABI library) in-tree for sm_103a.

Compiles every translation unit under csrc/ in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and links them into
paper_2102_05287_gb300/_build/libwcns.so.  Also builds the peak
microbenchmark binary used for the roofline denominators.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwcns.so")
PEAKS = os.path.join(BUILD, "peaks")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["wcns_fp64.cu", "wcns_mixed.cu", "wcns_api.cu", "wcns_batch.cu"]
DEPS = ["wcns_sweep.cuh", "wcns_internal.h", "wcns_mixed_body.cuh"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwcns")
    return exe


def _stale(target, inputs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.exists(i) and os.path.getmtime(i) > t for i in inputs)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    header = os.path.join(os.path.dirname(HERE), "include", "wcns.h")
    deps = [os.path.join(CSRC, d) for d in DEPS] + [header]
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + deps):
            jobs.append([cc] + flags + ["-c", s, "-o", o])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        _run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, LIB)
    psrc = os.path.join(CSRC, "peaks.cu")
    if force or _stale(PEAKS, [psrc]):
        _run([cc] + ARCH + ["-O3", "-o", PEAKS, psrc])
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    if logs:  # keep the last compile's register / spill report when nothing was rebuilt
        with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
            f.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
