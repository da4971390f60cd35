"""Compile the FP64 CPU oracle (test infrastructure) into oracle/libkgs_oracle.so.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark load
the result.  Plain C11, -O2, no fast-math, so that the arithmetic follows the
source literally.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kgs_oracle.c")
LIB = os.path.join(HERE, "libkgs_oracle.so")


def build_oracle(force: bool = False) -> str:
    hdr = os.path.join(HERE, "kgs_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    # OpenMP only serves the optional concurrent velocity ranges; without it
    # the ranges run one after another
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
