"""Compile the FP64 oracle (plain C, OpenMP) into oracle/_build/liboracle.so.

Test infrastructure: built by the package build step so that the checker
exists on every machine, used only by tests, the smoke check and the bench's
CPU-baseline leg.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "pf_oracle.c"), os.path.join(_HERE, "or_elastic.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    deps = _SRCS + [os.path.join(_HERE, "pf_oracle.h")]
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= max(os.path.getmtime(d) for d in deps)):
        return _OUT
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, *_SRCS,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


if __name__ == "__main__":
    print(build(force=True))
