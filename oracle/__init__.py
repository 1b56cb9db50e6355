"""CPU oracle for RNS-CKKS and the PackVFL MatMult.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the
GPU library (`paper_2405_00482_gb300`), and the library never imports it.

Pieces:
  he_oracle.c   exact integer ring arithmetic, samplers and the scheme (C, built by `build()`)
  encoding.py   CKKS encode/decode (numpy FFT and the O(N^2) defining sums)
  layout.py     planner, diagonal layout, lazy rotate-and-sum, cleartext model
  ckks.py       the scheme and the MatMult composed from the C primitives
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhe_oracle.so")
SRC_PATH = os.path.join(_HERE, "he_oracle.c")


def build(force: bool = False) -> str:
    """Compile he_oracle.c into libhe_oracle.so with gcc (plain -O2, no fast-math), with OpenMP
    when the compiler has it (the parallel loops give the same results on any thread count)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC_PATH, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH
