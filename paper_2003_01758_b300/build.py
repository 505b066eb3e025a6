"""Builds libpcba.so in-tree with nvcc for sm_103a (B300).

The library is compiled as several translation units in parallel (the
subdivision kernels once per arithmetic, the polish kernel, the engine, the
network and the allocation-free conversion), then linked into one shared
object next to this file; object files go to _build/ at the repository root.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpcba.so")
CSRC = os.path.join(HERE, "csrc")
OBJDIR = os.path.join(ROOT, "_build")
# (source, object name, extra flags)
UNITS = [
    ("pcba.cu", "pcba", []),
    ("pcba_k2.cu", "pcba_k2_f32", ["-DPCBA_K2_F64=0"]),
    ("pcba_k2.cu", "pcba_k2_f64", ["-DPCBA_K2_F64=1"]),
    ("pcba_polish.cu", "pcba_polish", []),
    ("pcba_noalloc.cu", "pcba_noalloc", []),
    ("pcba_mlp.cu", "pcba_mlp", []),
]
DEPS = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
        if f.endswith((".cu", ".cuh", ".h"))] \
    + [os.path.join(ROOT, "include", f) for f in ("pcba.h", "pcba_warmstart.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I" + os.path.join(ROOT, "include")]


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in DEPS)


def build(force=False, verbose=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    procs = []
    for src, name, extra in UNITS:
        obj = os.path.join(OBJDIR, name + ".o")
        cmd = [NVCC] + FLAGS + extra + (["-Xptxas", "-v"] if verbose else []) + \
            ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((obj, subprocess.Popen(cmd)))
    failed = [obj for obj, p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, "nvcc", "failed: " + ", ".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-o", tmp] + [obj for obj, _ in procs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
