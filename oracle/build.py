"""Compile the FP64 CPU oracle (plain C + OpenMP) into oracle/libmsm_oracle.so.

Test infrastructure only: the oracle checks the CUDA library, it is never part
of it.  gcc only, portable flags (the same source builds on x86-64 and Arm).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "msm_oracle.c")
LIB = os.path.join(HERE, "libmsm_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_DEFAULT_SOURCE",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
