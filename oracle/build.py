"""Builds the plain CPU reference as oracle/liboracle.so (g++, no CUDA).

Test infrastructure only: the product library never links or loads it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_bgv.cpp", "oracle_eval.cpp", "oracle_capi.cpp"]
TARGET = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.hpp")]
    if not force and os.path.exists(TARGET):
        t = os.path.getmtime(TARGET)
        if all(os.path.getmtime(d) <= t for d in deps):
            return TARGET
    tmp = TARGET + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
