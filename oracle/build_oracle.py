"""Build step for the FP64 CPU oracle (test infrastructure only).

Compiles the plain-C oracle in this folder into ``liboracle.so`` next to it.
The flags keep the arithmetic identical on x86-64 and aarch64: no fused
multiply-add contraction, no fast-math, no machine-specific tuning.

``build(omp=True)`` compiles the same sources with OpenMP into
``liboracle_omp.so``, which only the CPU-baseline timing loads (its sums run
in a different order; the tests use the serial library).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")
SOURCES = ["lattice.c", "vacuum.c", "u1.c", "surrogate.c", "gw.c"]


def _sources():
    return [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]


def needs_build(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = _sources() + [os.path.join(HERE, "oracle.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, omp=False):
    """Compile liboracle.so (or, with omp, liboracle_omp.so) if it is missing or older than
    its sources."""
    lib = LIB_OMP if omp else LIB
    if not force and not needs_build(lib):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall"] + (["-fopenmp"] if omp else []) + ["-o", tmp] + _sources() + ["-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, omp=True))
