"""Compile the oracle's C part (wilson.c) into oracle/_build/liboracle.so with gcc.

Test infrastructure only.  Plain gcc, -O2, OpenMP when the compiler has it (the loop
bodies are independent per site, so threading does not change any result bit).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "wilson.c")


def build(force=False, verbose=False):
    """Build liboracle.so if missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:2] + extra + base[2:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    sys.stderr.write(r.stderr)
    raise RuntimeError("failed to compile the oracle (oracle/wilson.c)")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
