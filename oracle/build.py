"""Build the FP64 oracle shared library (plain C, gcc, OpenMP).

Test infrastructure: the oracle is compiled next to this file as
``liboracle.so`` and loaded only by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rick_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile rick_oracle.c into liboracle.so unless it is up to date."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    # -ffp-contract=off: the binary32 placement decisions must be evaluated
    # exactly as written (explicit fmaf only), never fused by the compiler.
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas",
           SRC, "-o", LIB + ".tmp", "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
