"""Build of the CUDA library libsrm.so (sm_103a) in the package tree.

Each translation unit is compiled by its own nvcc process, in parallel; the
input generator (srm_inputs/gen.c, used by srm_init for starting
configurations) is compiled with gcc and linked in.  Rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
GEN_C = os.path.join(ROOT, "srm_inputs", "gen.c")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libsrm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC] + ARCH
# translation units whose binary64 arithmetic must round every multiply and
# add separately (they reproduce the reference bit for bit without explicit
# rounding intrinsics)
NO_FMAD = {"platelet.cu"}
# tuning knobs: blocks per SM the register allocation of the sweep kernels
# (staged, general) must allow
for _k in ("SRM_SWEEP_MIN_BLOCKS", "SRM_SWEEP_MIN_BLOCKS_GENERAL"):
    if os.environ.get(_k):
        NVCC_FLAGS += [f"-D{_k}={int(os.environ[_k])}"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, hdr


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    cu, hdr = sources()
    t = os.path.getmtime(LIB)
    stamp = os.path.join(OUT_DIR, "flags.txt")
    flags = " ".join(NVCC_FLAGS)
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        return True
    return any(os.path.getmtime(f) > t for f in cu + hdr + [GEN_C, __file__])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    cu, _ = sources()
    jobs = []
    for src in cu:
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        extra = ["--fmad=false"] if os.path.basename(src) in NO_FMAD else []
        jobs.append([nvcc] + NVCC_FLAGS + extra + ["-c", src, "-o", obj])
    gen_obj = os.path.join(OUT_DIR, "gen.o")
    jobs.append(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-c", GEN_C, "-o", gen_obj])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or p.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
        if p.returncode:
            raise RuntimeError(f"compile failed: {cmd[-3]}")
        return cmd[-1]

    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + f".{os.getpid()}.tmp"
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lm"])
    os.replace(tmp, LIB)
    with open(os.path.join(OUT_DIR, "flags.txt"), "w") as f:
        f.write(" ".join(NVCC_FLAGS))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
