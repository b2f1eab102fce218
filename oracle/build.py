"""Compile the CPU oracle (plain C) into oracle/_liboracle.so.

Test infrastructure: the oracle is the independent reference the CUDA library
is checked against; nothing in the library links it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_liboracle.so")
SOURCES = ["bn.c", "paillier.c"]


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "bn.h")]
    if not force and os.path.exists(SO) and all(os.path.getmtime(SO) >= os.path.getmtime(d) for d in deps):
        return SO
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", SO + ".tmp"] + srcs
    subprocess.check_call(cmd)
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
