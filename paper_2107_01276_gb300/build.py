"""Build the CUDA library libsph_gb300.so in-tree (sm_103a only).

Each .cu file compiles to an object in parallel with nvcc, then one link
step makes the shared library.  Output goes to ``_build/`` next to this
file (git-ignored).  Nothing here runs a GPU.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsph_gb300.so")
# the debug build: device-side bounds checks compiled in (-DSPH_DEBUG)
BUILD_DEBUG = os.path.join(BUILD, "debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libsph_gb300_debug.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--extended-lambda",
                     "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                     "-I", INCLUDE]
# Per-file flags.  The pair passes flush FP32 subnormals to zero: a
# subnormal term is below 1e-38 of the sums it enters, and the approximate
# reciprocal and reciprocal square root of the FP32 pair arithmetic then
# need no subnormal fix-up instructions (3-4 % of pass A and pass B).
# FP64 arithmetic is not affected.
FILE_FLAGS = {"pair_passes.cu": ["-ftz=true"]}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"),
                        "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          debug: bool = False) -> str:
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    if debug:
        extra += ["-DSPH_DEBUG"]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + FILE_FLAGS.get(os.path.basename(src), []) + extra + \
            ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose or ptxas_v:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_v="-v" in sys.argv))
