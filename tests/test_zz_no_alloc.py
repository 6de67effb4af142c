"""mfc_rhs_noalloc: the FP64 right-hand side for callers that cannot allocate.

Callers that live inside a framework whose pool allocator owns the GPU, or
services that must keep a fixed device footprint after start-up, cannot call
cudaMalloc when they need a right-hand side; mfc_rhs_noalloc serves them with
caller-owned input/output buffers and a fixed scratch array compiled into the
library.  These tests call it through the C ABI and check it against the
context entry point mfc_rhs on the same device buffers, within the FP64 RHS
parity bar used by the other GPU tests (1e-12 of the flux scale
max(|L|, |q| S) per field), on calls made back to back.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_10729_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10729_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _noalloc(p, q, out, precision="fp64"):
    import torch
    from paper_2409_10729_gb300 import mfc
    return mfc.lib().mfc_rhs_noalloc(ctypes.byref(mfc.make_params(p, precision)), ctypes.c_void_p(q.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _reference(p, w):
    """State on the device and L(q) from the context entry point mfc_rhs."""
    import torch
    from paper_2409_10729_gb300 import mfc
    s = mfc.Solver(p, "fp64")
    s.set_state_prim(w)
    q = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.get_state(q)
    ref = torch.empty_like(q)
    s.rhs(ref, allow_nonphysical=True)
    S = s.max_wavespeed() if s.last_status == mfc.MFC_OK else 0.0
    status = s.last_status
    s.close()
    return q, ref, S, status


def _err(out, ref, q, S):
    o = out.cpu().numpy().reshape(out.shape[0], -1)
    r = ref.cpu().numpy().reshape(ref.shape[0], -1)
    qq = q.cpu().numpy().reshape(q.shape[0], -1)
    scale = np.maximum(np.abs(r).max(1), np.abs(qq).max(1) * S)
    return (np.abs(o - r).max(1) / np.maximum(scale, 1e-300)).max()


def test_noalloc_rhs_matches_context_rhs_on_consecutive_calls():
    import torch
    from paper_2409_10729_gb300 import mfc
    cases = [I.random_periodic(3, [24, 20, 18], seed=41), I.shock_droplets(48), I.random_periodic(2, [70, 37], 3)]
    for p, w in cases:
        q, ref, S, _ = _reference(p, w)
        for _ in range(2):   # two calls in a row on the same buffers
            out = torch.full_like(q, float("nan"))
            assert _noalloc(p, q, out) == mfc.MFC_OK
            torch.cuda.synchronize()
            assert _err(out, ref, q, S) <= TOL


def test_noalloc_status_is_cleared_between_calls():
    """A non-physical state is reported, and the next (physical) call is not
    polluted by the previous call's status word."""
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(2, [16, 12], seed=0)
    bad = w.copy()
    bad[0, 0, 5, 7] = -1.0
    bad[1, 0, 5, 7] = 0.0
    qb, refb, _, stb = _reference(p, bad)
    assert stb == mfc.MFC_ENONPHYSICAL
    out = torch.empty_like(qb)
    assert _noalloc(p, qb, out) == mfc.MFC_ENONPHYSICAL
    qg, refg, S, _ = _reference(p, w)
    out = torch.empty_like(qg)
    assert _noalloc(p, qg, out) == mfc.MFC_OK
    assert _err(out, refg, qg, S) <= TOL


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    from paper_2409_10729_gb300 import mfc
    big = I.make_params(3, [96, 96, 96], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE)   # 7 * 96^3 > 2 Mi doubles
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    assert _noalloc(big, dummy, dummy) == mfc.MFC_ETOOBIG
    small = I.make_params(1, [8], [0.0], [1.0], I.TRANSMISSIVE)
    assert _noalloc(small, dummy, dummy, precision="mixed") == mfc.MFC_EINVAL
    assert mfc.strerror(mfc.MFC_ETOOBIG).startswith("problem too large")
