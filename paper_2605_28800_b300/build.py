"""Build libtdgl.so (the C-ABI library of include/tdgl.h) for sm_103a with nvcc, in-tree."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libtdgl.so")
SOURCES = [os.path.join(HERE, "csrc", "tdgl.cu"), os.path.join(HERE, "csrc", "unet.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in ("fft.cuh", "fft_reg.cuh", "kernels.cuh", "kernels_fast.cuh", "kernels_rows.cuh", "tensor.cuh", "runtime.cuh", "tc.cuh", "unet_kernels.cuh", "philox.cuh")] + [
    os.path.join(ROOT, "include", "tdgl.h")]

NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(HERE, os.path.basename(s) + tag + ".o") for s in SOURCES]
    compile_flags = [f for f in NVCC_FLAGS if f != "-shared"]
    procs = []
    try:
        # one nvcc per translation unit, in parallel, then one link
        for s, o in zip(SOURCES, objs):
            cmd = [nvcc()] + compile_flags + ["-c", "-o", o, s]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append(subprocess.Popen(cmd))
        for p in procs:
            if p.wait() != 0:
                raise subprocess.CalledProcessError(p.returncode, p.args)
        tmp = LIB + tag
        cmd = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
