"""Compile the oracle's C core into oracle/_build/libckks_oracle.so.

TEST INFRASTRUCTURE: built so the tests and the CPU baseline can run it; the
GPU library neither builds against nor loads it.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ckks_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libckks_oracle.so")


def _compile(flags) -> bool:
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", *flags, SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        return False
    os.replace(tmp, LIB)
    return True


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    if not _compile(["-fopenmp"]) and not _compile([]):
        raise RuntimeError("gcc failed to build the oracle")
    return LIB


if __name__ == "__main__":
    print(build(force=True))
