"""Compile the C oracle (lbm_oracle.c) into oracle/_build/liboracle.so.

Test infrastructure only.  Plain gcc, FP64, no fused multiply-add
(-ffp-contract=off), OpenMP over rows.  Works unchanged on x86_64 and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
# the same source with long double arithmetic (the extended-precision
# reference; see the header of lbm_oracle.c)
LIB_EXT = os.path.join(OUT_DIR, "liboracle_ext.so")


def build(force=False, ext=False):
    """Build the oracle library if it is missing or older than its source
    (ext=True: the extended-precision build)."""
    lib = LIB_EXT if ext else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    if ext:
        cmd.insert(1, "-DORC_REAL=long double")
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
