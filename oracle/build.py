"""ORACLE — test infrastructure only.

Compiles the plain-C oracle (lhaf_oracle.c) into oracle/_build/liblhaf_oracle.so with gcc
and OpenMP. Portable flags only (no -march=native), so it builds the same way on x86-64
and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblhaf_oracle.so")
SOURCES = [os.path.join(HERE, "lhaf_oracle.c")]
DEPS = SOURCES + [os.path.join(HERE, "lhaf_subset_body.h")]


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_m for s in DEPS):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
           "-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
