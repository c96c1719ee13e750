"""Build the CUDA library (sm_103a) in-tree: csrc/*.cu + csrc/*.cpp -> _build/libmmsim.so.

Translation units compile in parallel; the shared library links the CUDA
runtime statically so it loads on any machine with a matching driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmmsim.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    srcs = sorted(os.listdir(CSRC))
    cu = [os.path.join(CSRC, f) for f in srcs if f.endswith(".cu")]
    cpp = [os.path.join(CSRC, f) for f in srcs if f.endswith(".cpp")]
    hdr = [os.path.join(CSRC, f) for f in srcs if f.endswith(".h")]
    hdr.append(os.path.join(os.path.dirname(HERE), "include", "mm.h"))
    return cu, cpp, hdr


def _run(cmd, verbose):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}")
    return r.stdout


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    cu, cpp, hdr = _sources()
    os.makedirs(OUT, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in cu + cpp + hdr + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    ch = cuda_home()
    nvcc = os.path.join(ch, "bin", "nvcc")
    inc = ["-I" + os.path.join(os.path.dirname(HERE), "include"), "-I" + CSRC]
    jobs = []
    objs = []
    for s in cu:
        o = os.path.join(OUT, os.path.basename(s) + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc, "-c", s, "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
        objs.append(o)
    for s in cpp:
        o = os.path.join(OUT, os.path.basename(s) + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + os.path.join(ch, "include"), *inc,
                     "-c", s, "-o", o])
        objs.append(o)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), jobs))
    if ptxas_info:
        for o in outs:
            sys.stderr.write(o)
    tmp = LIB + f".{os.getpid()}.tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
