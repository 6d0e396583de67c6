"""Compile the CPU oracle (plain C, FP64) into a shared library next to it.

The oracle is test infrastructure: the library built here is loaded only by the
tests, the smoke check and the CPU-baseline leg of the benchmark.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "srfmg_oracle.c")
LIBRARY = os.path.join(HERE, "_build", "libsrfmg_oracle.so")

# -ffp-contract=off keeps a*b+c unfused so x86 and Arm hosts round identically.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-Wall"]


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    os.makedirs(os.path.dirname(LIBRARY), exist_ok=True)
    if (not force and os.path.exists(LIBRARY)
            and os.path.getmtime(LIBRARY) >= os.path.getmtime(SOURCE)):
        return LIBRARY
    tmp = LIBRARY + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, SOURCE, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIBRARY)
    return LIBRARY


if __name__ == "__main__":
    print(build(force=True))
