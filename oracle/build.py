"""Compile the C oracle into oracle/_build/libqmc_oracle.so with gcc.

Test infrastructure (see oracle/__init__.py).  Portable flags only (the library is built
on x86_64 and on aarch64 hosts): no -march, no intrinsics.  -ffp-contract=off keeps
every multiply and add individually rounded, as the source reads.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qmc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "libqmc_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    cc = os.environ.get("CC", "gcc")
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", SRC, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
