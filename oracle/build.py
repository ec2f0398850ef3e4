"""Compile the FP64 CPU oracle into oracle/liboracle.so (gcc, OpenMP).

Test infrastructure: the library built here is loaded only by the test
suite, the smoke check and the benchmark's CPU-baseline leg.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dgsm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

# -ffp-contract=off and no -ffast-math: the f32 index/binning functions must
# round every operation on its own, exactly as the GPU side does.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math", "-Wall", "-Wno-misleading-indentation"]


# The same source under AddressSanitizer and UndefinedBehaviorSanitizer,
# aborting on the first report (the sanitized oracle test runs the oracle's
# pins against it in a child process that preloads the ASan runtime).
SAN_LIB = os.path.join(HERE, "liboracle_san.so")
SAN_FLAGS = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
             "-fno-sanitize-recover=all"]


def build(force: bool = False, sanitize: bool = False) -> str:
    lib = SAN_LIB if sanitize else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    flags = [f for f in CFLAGS if f != "-O2"] + SAN_FLAGS if sanitize else CFLAGS
    cmd = ["gcc", *flags, SRC, "-o", lib + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, sanitize="--sanitize" in sys.argv))
