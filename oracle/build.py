"""Compile the FP64 CPU oracle (test infrastructure) into oracle/libbipp_oracle.so.

Usage: python oracle/build.py   (also called by the test suite and by the
package build step; it only rebuilds when the source is newer).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bipp_oracle.c")
HDR = os.path.join(HERE, "bipp_oracle.h")
LIB = os.path.join(HERE, "libbipp_oracle.so")


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-D_GNU_SOURCE",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
