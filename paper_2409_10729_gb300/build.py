"""Build libmfc5.so (the CUDA library behind include/mfc.h) for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into ``lib/libmfc5.so`` inside the package (in-tree; git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libmfc5.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++20", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# per-unit extra flags: the mixed form uses fast FP32 division/square root; the
# reference-order FP64 units must not contract a*b+c into FMAs
FAST32 = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
EXTRA = {"sweep_mixed.cu": FAST32, "sweep_gated.cu": FAST32,
         "sweep_fp64x.cu": ["-fmad=false"], "aux.cu": ["-fmad=false"], "mlp.cu": ["-fmad=false"]}
# extra nvcc flags for every unit (e.g. -DMFC_MIN_BLOCKS_MIXED=3); changing them
# needs build(force=True)
USER_FLAGS = os.environ.get("MFC5_NVCC_FLAGS", "").split()
UNITS = ["capi.cu", "aux.cu", "sweep_fp64.cu", "sweep_fp64x.cu", "sweep_mixed.cu", "sweep_gated.cu", "mlp.cu",
         "noalloc.cu", "grid.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmfc5")


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mfc.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_unit(unit):
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *EXTRA.get(unit, []), *USER_FLAGS, "-c", os.path.join(CSRC, unit), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
