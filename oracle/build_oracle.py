"""Build the plain-C FP64 oracle (test infrastructure) into oracle/librhd_oracle.so.

Compiled with -ffp-contract=off so that the same source gives the same bits on x86-64 and
aarch64 hosts, and with OpenMP so the CPU-baseline leg can use every host core (OpenMP only
splits loops over independent cells; it changes no arithmetic).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rhd_oracle.c")
LIB = os.path.join(HERE, "librhd_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rhd_oracle.h"))
    ):
        return LIB
    cmd = [
        "gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
        "-Wall", "-shared", "-fPIC", "-o", LIB + ".tmp", SRC, "-lm",
    ]
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
