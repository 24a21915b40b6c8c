"""Build the oracle's shared library (plain C, FP64, OpenMP).

Test infrastructure only: the CUDA library never links or loads this.
Compiled with -ffp-contract=off so that the cluster tree is reproducible bit
for bit by any other implementation that performs the same IEEE operations.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_geom.c", "orc_freq.c", "orc_tree.c", "orc_aca.c", "orc_mlp.c"]
LIB = os.path.join(HERE, "liborc.so")


def build(force=False, verbose=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "orc.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unused-function", "-o", LIB + ".tmp"] + srcs + ["-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
