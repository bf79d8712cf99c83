"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain gcc, no FMA contraction, so every operation rounds as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "es_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "es_oracle.h"))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


OPC_SRC = os.path.join(HERE, "opcount.cpp")
OPC_LIB = os.path.join(HERE, "libopcount.so")


def build_opcount(force: bool = False) -> str:
    """The operation-counting build of the same oracle source (opcount.cpp includes
    es_oracle.c with double replaced by a counting binary64 type), oracle/libopcount.so."""
    deps = [SRC, OPC_SRC, os.path.join(HERE, "es_oracle.h")]
    if not force and os.path.exists(OPC_LIB) and os.path.getmtime(OPC_LIB) >= max(os.path.getmtime(d) for d in deps):
        return OPC_LIB
    tmp = OPC_LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, OPC_SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, OPC_LIB)
    return OPC_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
