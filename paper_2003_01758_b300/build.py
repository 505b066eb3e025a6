"""Builds libpcba.so in-tree with nvcc for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpcba.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("pcba.cu", "pcba_noalloc.cu", "pcba_mlp.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in ("pcba_device.cuh", "pcba_kernels.cuh",
                                                          "pcba_subdivide.cuh", "pcba_eval.cuh",
                                                          "pcba_polish.cuh")] \
    + [os.path.join(ROOT, "include", f) for f in ("pcba.h", "pcba_warmstart.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include")]


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in DEPS)


def build(force=False, verbose=False):
    if not force and not needs_build():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp] + SOURCES
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
