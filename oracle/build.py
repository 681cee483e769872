"""Compile the oracle's C++ source into oracle/_oracle.so (test infrastructure).

Plain g++ -O2, no FMA contraction (the quantisation step must round exactly
as written), portable to x86_64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
OUT = os.path.join(HERE, "_oracle.so")


def compile_source(src: str, out: str) -> str:
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    return compile_source(SRC, OUT)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
