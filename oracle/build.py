"""Compile the FP64 CPU oracle into a shared library (``oracle/_build/liboracle.so``).

TEST INFRASTRUCTURE ONLY: the oracle is the correctness reference for the CUDA
library and is used by the tests, the smoke check and the CPU-baseline leg of
the benchmark.  Plain g++ (C++17, OpenMP when available), no -ffast-math so the
arithmetic stays IEEE double.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")


def sources():
    return sorted(os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith(".cpp"))


def headers():
    return sorted(os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith(".h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in sources() + headers() + [__file__])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    base = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas"]
    tmp = LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + sources() + ["-o", tmp]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
        err = r.stderr
    raise RuntimeError(f"oracle build failed:\n{err}")


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
