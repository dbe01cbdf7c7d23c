"""Compile the C oracle (seeds_ref.c) into a shared library next to it.

Test infrastructure: see the package docstring.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "seeds_ref.c")
LIB = os.path.join(HERE, "_seeds_ref.so")


def build(force: bool = False) -> str:
    """Build `_seeds_ref.so` if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    # no fused multiply-add: the floating-point means distances (R17) must
    # round after every operation
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-Wall", "-Wextra", "-shared", "-fPIC", "-o", tmp, SRC,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
