"""Compile the OpenMP CPU twin into cpu_twin/libtwin.so (a measured CPU
baseline; the GPU library never loads it)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lcc_twin.c")
LIB = os.path.join(HERE, "libtwin.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O3", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-Wextra", SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
