"""Compile the C oracle into ``oracle/_build/liboracle.so`` (test infrastructure).

Plain gcc, strict IEEE double arithmetic: no fast-math and no floating-point
contraction, so every product and sum is rounded as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["mie.c", "table.c", "philox.c", "walk.c", "walk32.c", "adjoint.c"]
LIB = os.path.join(HERE, "_build", "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force=False):
    """Build the oracle library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-Wall",
           "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
