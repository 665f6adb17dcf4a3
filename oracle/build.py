"""Build step for the CPU oracle (test infrastructure only).

Compiles ``gp_oracle.c`` with gcc into ``libgp_oracle.so`` beside it.  Plain
-O2, OpenMP only across independent theta candidates; no -march flags, so the
same source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gp_oracle.c")
LIB = os.path.join(HERE, "libgp_oracle.so")


def build_oracle(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
