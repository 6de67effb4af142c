"""Build libmfc5.so (the CUDA library behind include/mfc.h) for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into ``lib/libmfc5.so`` inside the package (in-tree; git-ignored).

A build is keyed on a SHA-256 of every source and header, this file, the
nvcc command lines and the nvcc version; the key is stored beside the
library (``lib/libmfc5.so.key``).  A library whose key does not match -- a
stale one, or one copied from another machine -- is rebuilt, whatever its
modification time.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
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
KEY = LIB + ".key"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++20", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# per-unit extra flags: the mixed form uses fast FP32 division/square root; the
# reference-order FP64 units must not contract a*b+c into FMAs
FAST32 = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
EXTRA = {"sweep_mixed.cu": FAST32, "sweep_gated.cu": FAST32,
         "sweep_fp64x.cu": ["-fmad=false"], "aux.cu": ["-fmad=false"], "mlp.cu": ["-fmad=false"]}
# extra nvcc flags for every unit (e.g. -DMFC_MIN_BLOCKS_MIXED=3); they are part
# of the build key
USER_FLAGS = os.environ.get("MFC5_NVCC_FLAGS", "").split()
UNITS = ["capi.cu", "aux.cu", "sweep_fp64.cu", "sweep_fp64x.cu", "sweep_mixed.cu", "sweep_gated.cu", "mlp.cu",
         "noalloc.cu", "grid.cu", "blocks.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmfc5")


def _unit_cmd(cc: str, unit: str, obj: str) -> list:
    return [cc, *ARCH, *COMMON, *EXTRA.get(unit, []), *USER_FLAGS, "-c", os.path.join(CSRC, unit), "-o", obj]


def build_key(cc: str) -> str:
    """SHA-256 of the sources, headers, this file, the compile commands and
    the compiler version."""
    h = hashlib.sha256()
    files = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")))
    for path in files + [os.path.join(INCLUDE, "mfc.h"), os.path.abspath(__file__)]:
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as fh:
            h.update(fh.read())
    for unit in UNITS:
        h.update(" ".join(_unit_cmd("nvcc", unit, "x.o")).encode())
    try:
        ver = subprocess.run([cc, "--version"], capture_output=True, text=True).stdout
    except OSError:
        ver = ""
    h.update(ver.encode())
    return h.hexdigest()


_REPORTED = set()


def _stored_key() -> str:
    try:
        with open(KEY) as fh:
            return fh.read().strip()
    except OSError:
        return ""


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    cc = nvcc()
    key = build_key(cc)
    if not force and os.path.exists(LIB) and _stored_key() == key:
        if key not in _REPORTED:
            _REPORTED.add(key)
            print(f"libmfc5: reusing {LIB} (key {key[:16]})", file=sys.stderr)
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_unit(unit):
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = _unit_cmd(cc, unit, obj)
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
    with open(KEY + f".tmp{os.getpid()}", "w") as fh:
        fh.write(key + "\n")
    os.replace(KEY + f".tmp{os.getpid()}", KEY)
    _REPORTED.add(key)
    print(f"libmfc5: compiled {LIB} (key {key[:16]})", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
