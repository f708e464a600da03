"""Build the oracle shared library (plain C, gcc, no GPU).

Test infrastructure: the oracle is only loaded by tests, the smoke check and
the benchmark's CPU-baseline leg.  Output: oracle/_build/liboracle.so.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "scan_oracle.c")


def build(force: bool = False) -> str:
    """Compile scan_oracle.c into liboracle.so (portable flags: x86 and Arm)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(
                os.path.join(HERE, "scan_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # -O2 without -ffast-math: the FP64 accumulation order must stay the
    # sequential order of the definition.
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
