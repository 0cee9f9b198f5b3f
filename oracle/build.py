"""Builds the oracle shared library (plain g++, FP64, no FP contraction).

Test infrastructure only: tests/, the smoke check and the benchmark's CPU
baseline leg are the only users of the oracle.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SOURCES = ["amr_oracle.cpp", "maps_oracle.cpp", "opcount.cpp"]


def build(force=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "mhd_core.hpp")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
