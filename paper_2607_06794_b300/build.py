"""Build the CUDA library liblbm.so in-tree for sm_103a with nvcc."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblbm.so")
ROOT = os.path.dirname(HERE)

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def sources():
    out = [os.path.join(ROOT, "include", "lbm.h")]
    for f in sorted(os.listdir(SRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(SRC, f))
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    units = [os.path.join(SRC, f) for f in sorted(os.listdir(SRC)) if f.endswith(".cu")]
    cmd = ["nvcc"] + NVCC_FLAGS + ["-o", LIB] + units
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
