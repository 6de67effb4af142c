"""Host-side checks of the C ABI library (no GPU calls).

The library builds for sm_103a, loads, exports every entry point declared in
include/mfc.h, its parameter struct matches the binding's layout, and
parameter validation rejects bad input before touching the device.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2409_10729_gb300 import build as B
from paper_2409_10729_gb300 import mfc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mfc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mfc.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mfc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mfc_create", "mfc_destroy", "mfc_set_state", "mfc_get_state", "mfc_rhs",
                     "mfc_step_rk3", "mfc_max_wavespeed"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", mfc.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b[TW] (mfc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"not exported: {missing}"
    for n in declared_functions():
        assert hasattr(lib, n)


def test_params_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mfc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(mfc_params),'
                   ' offsetof(mfc_params, bc), offsetof(mfc_params, gamma),'
                   ' offsetof(mfc_params, weno_eps), offsetof(mfc_params, precision), offsetof(mfc_params, weno_order));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    P = mfc.MfcParams
    assert got == [ctypes.sizeof(P), P.bc.offset, P.gamma.offset, P.weno_eps.offset, P.precision.offset,
                   P.weno_order.offset]


def _params(**over):
    from paper_2409_10729_gb300 import inputs as I
    p = I.make_params(3, [8, 8, 8], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE)
    p.update(over)
    return p


@pytest.mark.parametrize("bad", [
    dict(ndim=0), dict(ndim=4), dict(n=[0, 8, 8]), dict(hi=[0.0, 1.0, 1.0]),
    dict(bc=[[0, 1], [0, 0], [0, 0]]), dict(bc=[[2, 2], [0, 0], [0, 0]]),
    dict(gamma=[1.0, 1.4]), dict(pi_inf=[-1.0, 0.0]), dict(weno_eps=0.0),
    dict(weno_order=4), dict(weno_order=7), dict(weno_order=3, precision="gated"),
    dict(gamma=[4.4, 1.4, 2.35], pi_inf=[6e8, 0.0, 1e9], precision="gated"),
    dict(gamma=[4.4, 1.4, 2.35], pi_inf=[6e8, 0.0, -1.0]),
])
def test_create_rejects_bad_params_before_touching_the_device(lib, bad):
    handle = ctypes.c_void_p()
    bad = dict(bad)
    prec = bad.pop("precision", "fp64")
    st = lib.mfc_create(ctypes.byref(mfc.make_params(_params(**bad), prec)), None, ctypes.byref(handle))
    assert st == mfc.MFC_EINVAL
    assert not handle.value


def test_null_arguments_are_rejected(lib):
    assert lib.mfc_create(None, None, None) == mfc.MFC_EINVAL
    assert lib.mfc_destroy(None) == mfc.MFC_OK
    assert lib.mfc_set_state(None, None, 0) == mfc.MFC_EINVAL
    assert lib.mfc_rhs(None, None, 0) == mfc.MFC_EINVAL
    assert lib.mfc_step_rk3(None, 0.4, 1, None) == mfc.MFC_EINVAL
    assert mfc.strerror(mfc.MFC_ENONPHYSICAL).startswith("non-physical")


@pytest.mark.parametrize("n", [[2 ** 21, 2 ** 21, 2 ** 22],        # 2^64 cells: wraps to 0 in 64 bits
                               [2 ** 31 - 1] * 3, [4096, 4096, 4097]])
def test_create_rejects_cell_counts_no_device_can_hold(lib, n):
    """More than 2^36 cells is refused with MFC_ENOMEM before any device call,
    including counts whose 64-bit product would wrap."""
    handle = ctypes.c_void_p()
    st = lib.mfc_create(ctypes.byref(mfc.make_params(_params(n=n), "fp64")), None, ctypes.byref(handle))
    assert st == mfc.MFC_ENOMEM
    assert not handle.value


@pytest.mark.parametrize("n", [[2 ** 21, 2 ** 21, 2 ** 22], [2 ** 31 - 1] * 3, [96, 96, 96], [66, 66, 69]])
def test_noalloc_rejects_problems_beyond_its_scratch_before_touching_the_device(lib, n):
    """mfc_rhs_noalloc's size check (neq * ncells + 32 doubles against the
    fixed scratch) runs before any device call and cannot be fooled by a
    wrapping cell count."""
    p = mfc.make_params(_params(n=n), "fp64")
    dummy = ctypes.c_void_p(16)   # never dereferenced: the call returns first
    assert lib.mfc_rhs_noalloc(ctypes.byref(p), dummy, dummy, None) == mfc.MFC_ETOOBIG


@pytest.mark.parametrize("offset_doubles", [0, 1, -1, 8 * 8 * 8 * 7 - 1, -(8 * 8 * 8 * 7 - 1)])
def test_noalloc_refuses_overlapping_buffers_before_touching_the_device(lib, offset_doubles):
    """mfc_rhs_noalloc refuses an output range that overlaps the input range
    (in place, or shifted by fewer cells than the state holds) with
    MFC_EINVAL before any device call; the addresses are never dereferenced."""
    p = mfc.make_params(_params(), "fp64")
    base = 1 << 40
    q = ctypes.c_void_p(base)
    rhs = ctypes.c_void_p(base + 8 * offset_doubles)
    assert lib.mfc_rhs_noalloc(ctypes.byref(p), q, rhs, None) == mfc.MFC_EINVAL


def test_tma_staging_build_option_compiles(tmp_path):
    """The measured-and-rejected TMA staging of the FP32 y/z sweeps stays a
    working build option: the FP32 sweep unit compiles with it for sm_103a."""
    out = tmp_path / "sweep_mixed_tma.o"
    cmd = [B.nvcc(), *B.ARCH, *B.COMMON, *B.FAST32, "-DMFC_TMA_YZ=1", "-c",
           os.path.join(B.CSRC, "sweep_mixed.cu"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    assert out.stat().st_size > 0
