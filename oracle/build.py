"""Builds the CPU oracle into oracle/liboracle_pcz.so with the host C compiler.

Test infrastructure only (see pcz_oracle.c).  Floating-point contraction is
turned off so that every sum and difference is a single IEEE operation in the
field type, on x86-64 and on AArch64 alike.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcz_oracle.c")
LIB = os.path.join(HERE, "liboracle_pcz.so")

BASE_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
              "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    tmp = LIB + ".tmp"
    for omp in (["-fopenmp"], []):
        cmd = [cc, *BASE_FLAGS, *omp, SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
