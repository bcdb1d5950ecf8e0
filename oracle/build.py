"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain C, no GPU: contraction of a*b+c into fused multiply-adds is switched off
so that every expression in fpt_oracle.c is rounded as written on any host
(gcc contracts by default on Arm).
"""
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fpt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "fpt_oracle.h"))
    ):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}.{threading.get_ident()}"  # unique per process and thread
    cmd = [
        os.environ.get("CC", "cc"), "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
        "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
        "-o", tmp, SRC, "-lm",
    ]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
