"""Build liblbm.so (the CUDA library behind include/lbm.h) in-tree for sm_103a.

nvcc compiles each translation unit in parallel and links one shared
library with the CUDA runtime linked statically.  aux.cu and step_f64.cu are
compiled with -fmad=false: the plain FP64 path keeps the operation order of
a straightforward FP64 implementation.  Host code is compiled with
-ffp-contract=off for the same reason.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                 "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr"]
UNITS = {
    "lbm_api.cu": [],
    "batch.cu": [],
    "step_f32.cu": [],
    "step_f16.cu": [],
    "step_bf16.cu": [],
    "step_f64dev.cu": [],
    "step_f64.cu": ["-fmad=false"],
    "aux.cu": ["-fmad=false"],
    "io_dev.cu": [],
    "serve.cu": [],
    "drift_noalloc.cu": [],
    "slabs.cu": [],
    "vn.cu": [],
    "optcost.cu": [],
}
HEADERS = ["lbm_internal.h", "d2q9_pull.cuh", "collide.cuh", "step_impl.cuh", "bounds.cuh",
           "resident.cuh", "runtime.h", "node_xy.cuh", "slots.h"]
# the debug build: device-side index checks that record failures in a word
# (lbm_debug_bounds) instead of trapping
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "liblbm.so")


def _newest_input():
    paths = [os.path.join(SRC, f) for f in list(UNITS) + HEADERS]
    paths.append(os.path.join(HERE, "..", "include", "lbm.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False, debug=False):
    """Compile (if stale) and return the path of liblbm.so; debug=True builds
    the index-checking library in _build_debug instead."""
    out, lib = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    flags = COMMON + (["-DLBM_DEBUG_BOUNDS"] if debug else [])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(out, exist_ok=True)
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(out, unit.replace(".cu", ".o"))
        cmd = ["nvcc"] + flags + extra + ["-c", os.path.join(SRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                             stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = lib + ".tmp.%d" % os.getpid()
    subprocess.run(["nvcc"] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"],
                   check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
