"""Builds the oracle's shared library (plain C, gcc) in-tree.

TEST INFRASTRUCTURE ONLY: the library is loaded by ``oracle/__init__.py``.
Flags keep IEEE double semantics identical on x86_64 and aarch64: no fast-math
and no FMA contraction.
"""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "liboracle.so")


def build_oracle(verbose: bool = False) -> str:
    out = library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    src = os.path.join(_HERE, "grover_oracle.c")
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(verbose=True))
