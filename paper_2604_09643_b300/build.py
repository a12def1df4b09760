"""Build ``lib/libpasfm.so`` (sm_103a) from ``csrc/`` with nvcc.

The hot kernels are instantiated once per pulse profile and sample-slot count
from ``kernels_s.cu`` (sphere: S = 2..16, Gaussian: S = 2..32); those
translation units compile in parallel.  The library is
built in-tree so that it travels with the source tree.

    python -m paper_2604_09643_b300.build [--force]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "lib", "libpasfm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (pulse profile, slot count) pairs: the sphere (0) for S = 2..16, the Gaussian (1) for S = 2..32
KS_VALUES = [(0, s) for s in range(2, 17)] + [(1, s) for s in range(2, 33)]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpasfm")


def _flags():
    return ["-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            f"-I{os.path.join(ROOT, 'include')}"]


def _sources():
    return glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "pasfm.h"), os.path.abspath(__file__)]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _sources())


def _compile(job):
    src, obj, extra = job
    cmd = [nvcc(), *_flags(), *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libpasfm.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    # The hot kernels flush FP32 subnormals to zero: none of their quantities comes near
    # 1e-38, and without it rsqrtf, __fdividef and exp2f each carry extra instructions to
    # handle subnormal operands (measured: 10-17% of the forward and backward time).
    work = [(os.path.join(CSRC, "kernels_s.cu"), os.path.join(OBJ, f"kernels_k{k}_s{s}.o"),
             [f"-DPASFM_K={k}", f"-DPASFM_S={s}", "-ftz=true"]) for k, s in KS_VALUES]
    work += [(os.path.join(CSRC, "aux.cu"), os.path.join(OBJ, "aux.o"), []),
             (os.path.join(CSRC, "launchers.cu"), os.path.join(OBJ, "launchers.o"), []),
             (os.path.join(CSRC, "tgv.cu"), os.path.join(OBJ, "tgv.o"), ["-ftz=true"]),
             (os.path.join(CSRC, "pasfm.cu"), os.path.join(OBJ, "pasfm.o"), []),
             (os.path.join(CSRC, "noalloc.cu"), os.path.join(OBJ, "noalloc.o"), [])]
    jobs = jobs or max(1, min(len(work), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, work))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    build(force=a.force, verbose=True)
    sys.exit(0)
