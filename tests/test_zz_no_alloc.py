"""mfc_rhs_noalloc: the FP64 right-hand side for callers that cannot allocate.

Callers that live inside a framework whose pool allocator owns the GPU, or
services that must keep a fixed device footprint after start-up, cannot call
cudaMalloc when they need a right-hand side; mfc_rhs_noalloc serves them with
caller-owned input/output buffers and a fixed scratch array compiled into the
library.  These tests call it through the C ABI on two calls in a row and
check each result bit for bit against the serial oracle's L(q) (the FP64
form evaluates every formula in the oracle's operation order, as the other
GPU parity tests require) and against the context entry point mfc_rhs on the
same device buffers.  The state comes from the oracle's own primitive ->
conservative conversion.  Cases: 1-D (the last sweep is the only sweep), 2-D
and 3-D, both boundary conditions, WENO3, three fluids.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def _context_rhs(p, qd):
    """L(q) from the context entry point mfc_rhs on the same device state."""
    import torch
    from paper_2409_10729_gb300 import mfc
    s = mfc.Solver(p, "fp64")
    s.set_state(qd)
    ref = torch.empty_like(qd)
    s.rhs(ref, allow_nonphysical=True)
    status = s.last_status
    s.close()
    return ref, status


CASE_IDS = ["1-D tube, transmissive", "3-D periodic", "3-D droplets, transmissive", "2-D periodic", "2-D WENO3",
            "3-D three fluids"]


def _cases():
    p1, w1 = I.air_water_shock_tube(300)
    p3, w3 = I.random_periodic(3, [24, 20, 18], seed=41)
    pw, ww = I.random_periodic(2, [70, 37], 3)
    pn, wn = I.random_periodic_n(3, [20, 14, 11], nfluids=3, seed=12)
    return [("1-D tube, transmissive", p1, w1),
            ("3-D periodic", p3, w3),
            ("3-D droplets, transmissive", *I.shock_droplets(48)),
            ("2-D periodic", pw, ww),
            ("2-D WENO3", dict(pw, weno_order=3), ww),
            ("3-D three fluids", pn, wn)]


@pytest.mark.parametrize("case", range(len(CASE_IDS)), ids=CASE_IDS)
def test_noalloc_rhs_is_the_oracle_rhs_on_consecutive_calls(case):
    import torch
    from paper_2409_10729_gb300 import mfc
    name, p, w = _cases()[case]
    assert name == CASE_IDS[case]
    q = O.prim_to_cons(p, w)
    Lo = O.rhs(p, q)
    qd = torch.from_numpy(q).cuda()
    ref, st = _context_rhs(p, qd)
    assert st == mfc.MFC_OK
    for _ in range(2):   # two calls in a row on the same buffers
        out = torch.full_like(qd, float("nan"))
        assert _noalloc(p, qd, out) == mfc.MFC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, Lo), "not bit-identical to the oracle"
        assert torch.equal(out, ref), "differs from mfc_rhs"
    assert np.array_equal(qd.cpu().numpy(), q)   # the input is left as it was


def test_noalloc_status_is_cleared_between_calls():
    """A non-physical state is reported, and the next (physical) call is not
    polluted by the previous call's status word."""
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(2, [16, 12], seed=0)
    bad = w.copy()
    bad[0, 0, 5, 7] = -1.0
    bad[1, 0, 5, 7] = 0.0
    qb = torch.from_numpy(O.prim_to_cons(p, bad)).cuda()
    out = torch.empty_like(qb)
    assert _noalloc(p, qb, out) == mfc.MFC_ENONPHYSICAL
    q = O.prim_to_cons(p, w)
    qg = torch.from_numpy(q).cuda()
    out = torch.empty_like(qg)
    assert _noalloc(p, qg, out) == mfc.MFC_OK
    assert np.array_equal(out.cpu().numpy(), O.rhs(p, q))


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    from paper_2409_10729_gb300 import mfc
    big = I.make_params(3, [96, 96, 96], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE)   # 7 * 96^3 > 2 Mi doubles
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    assert _noalloc(big, dummy, dummy) == mfc.MFC_ETOOBIG
    small = I.make_params(1, [8], [0.0], [1.0], I.TRANSMISSIVE)
    assert _noalloc(small, dummy, dummy, precision="mixed") == mfc.MFC_EINVAL
    assert mfc.strerror(mfc.MFC_ETOOBIG).startswith("problem too large")


def test_noalloc_refuses_overlapping_input_and_output():
    """In place, or with ranges that overlap by a cell, the call is refused
    before anything is launched; the input is left untouched."""
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(2, [16, 12], seed=2)
    q = O.prim_to_cons(p, w)
    buf = torch.zeros(2 * q.size, dtype=torch.float64, device="cuda")
    qd = buf[:q.size]
    qd.copy_(torch.from_numpy(q.reshape(-1)))
    assert _noalloc(p, qd, qd) == mfc.MFC_EINVAL
    assert _noalloc(p, qd, buf[q.size - 1:2 * q.size - 1]) == mfc.MFC_EINVAL
    assert _noalloc(p, buf[1:q.size + 1], qd) == mfc.MFC_EINVAL
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy(), q.reshape(-1))
    out = buf[q.size:]
    assert _noalloc(p, qd, out) == mfc.MFC_OK      # adjacent but disjoint
    assert np.array_equal(out.cpu().numpy().reshape(q.shape), O.rhs(p, q))
