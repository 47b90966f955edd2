"""Compile the CPU oracle into oracle/liboracle.so (test infrastructure only).

Plain gcc, no CUDA headers, -ffp-contract=off so that the double-precision
threshold tables are evaluated without fused multiply-adds.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "snc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
SRC_PAR = os.path.join(HERE, "snc_oracle_par.c")
LIB_PAR = os.path.join(HERE, "liboracle_par.so")
FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-shared", "-fPIC",
         "-D_DEFAULT_SOURCE"]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc"] + FLAGS + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def build_oracle_par(force: bool = False) -> str:
    """The same oracle on host threads (OpenMP): snc_oracle_par.c includes
    snc_oracle.c and only reorders its work."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(SRC_PAR))
    if not force and os.path.exists(LIB_PAR) and os.path.getmtime(LIB_PAR) >= newest:
        return LIB_PAR
    tmp = LIB_PAR + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc"] + FLAGS + ["-fopenmp", "-o", tmp, SRC_PAR, "-lm"], check=True)
    os.replace(tmp, LIB_PAR)
    return LIB_PAR


if __name__ == "__main__":
    print(build_oracle(force=True))
    print(build_oracle_par(force=True))
