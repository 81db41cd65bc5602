"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain g++ with OpenMP; floating-point contraction is disabled so the host
quadrature arithmetic is reproducible on x86_64 and aarch64 alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sclbm_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if it is missing or older than its sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [SRC, os.path.join(HERE, "sclbm_oracle.h")]
    if not force and os.path.exists(OUT):
        if os.path.getmtime(OUT) >= max(os.path.getmtime(s) for s in srcs):
            return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
