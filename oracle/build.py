"""Compile the CPU oracle (``oracle.cpp``) into ``liboracle.so`` beside it.

Plain g++ with portable flags, so the same source builds on x86_64 and on
aarch64 hosts. ``-ffp-contract=off`` keeps the HyperLogLog estimate evaluated
as written (no fused multiply-add contraction).
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def build_oracle(verbose: bool = False) -> str:
    src = os.path.join(HERE, "oracle.cpp")
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-pthread", "-shared", "-fPIC", src, "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(verbose=True))
