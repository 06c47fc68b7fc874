"""Compile the FP64 CPU oracle (plain C) into oracle/libram_oracle.so.

Test infrastructure: the oracle is the independent reference that the CUDA
library is checked against.  It is built with gcc only, shares no source with
the CUDA path, and is never a fallback for it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ram_oracle.c")
LIB = os.path.join(HERE, "libram_oracle.so")


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, SRC, "-lm"]
    try:
        subprocess.run(cmd, check=True)
    except subprocess.CalledProcessError:
        # a compiler without OpenMP still builds the (single-threaded) oracle
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
