"""ORACLE (test infrastructure).  Compiles the oracle's C part (tensor.c) with gcc."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "liboracle_tensor.so")


def build() -> str:
    out = library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-Wall",
                           os.path.join(_HERE, "tensor.c"), "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build())
