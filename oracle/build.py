"""Build step for the CPU oracle (test infrastructure only).

Compiles ``gp_oracle.c`` with gcc into ``libgp_oracle.so`` beside it, and the
same source in long double into ``libgp_oracle_ext.so``.  Plain
-O2, OpenMP only across independent theta candidates; no -march flags, so the
same source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gp_oracle.c")
LIB = os.path.join(HERE, "libgp_oracle.so")
# the same source in long double, used only to bound the double build's own
# rounding error on small cases
LIB_EXT = os.path.join(HERE, "libgp_oracle_ext.so")


def build_oracle(force: bool = False, extended: bool = False) -> str:
    lib = LIB_EXT if extended else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
           *(["-DGPO_EXTENDED"] if extended else []), SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_oracle(force=True))
    print(build_oracle(force=True, extended=True))
