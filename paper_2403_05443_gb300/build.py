"""Build liblbsph.so (sm_103a) in-tree with nvcc: one object per translation
unit, compiled in parallel, then linked into a shared library."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbsph.so")
UNITS = ["bulk_kernel.cu", "boundary_kernel.cu", "lattice_kernel.cu", "particle_kernel.cu", "step_kernel.cu", "lbsph_api.cu",
         "q27.cu",
         "mlp_kernel.cu", "warm_kernel.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without contraction of a*b+c (aarch64 gcc contracts by default): the
# quaternion normalised on input must round the same on every host
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I",
         os.path.join(ROOT, "include")]


def _deps():
    inc = os.path.join(ROOT, "include")
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(unit):
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
