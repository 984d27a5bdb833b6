"""Build the FP64 CPU oracle (test infrastructure only) into a shared library.

The oracle is plain C compiled with the host gcc.  Floating-point contraction is
switched off so that x86_64 and aarch64 hosts produce the same roundings.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "chcpic_oracle.c")
LIB = os.path.join(HERE, "libchcpic_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile ``chcpic_oracle.c`` unless an up-to-date library exists; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
