"""Build step for the FP64 CPU oracle (test infrastructure only).

Compiles the plain-C oracle in this folder into ``liboracle.so`` next to it.
The flags keep the arithmetic identical on x86-64 and aarch64: no fused
multiply-add contraction, no fast-math, no machine-specific tuning.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["lattice.c", "vacuum.c", "u1.c", "surrogate.c", "gw.c"]


def _sources():
    return [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(HERE, "oracle.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False):
    """Compile liboracle.so if it is missing or older than its sources."""
    if not force and not needs_build():
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + _sources() + ["-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
