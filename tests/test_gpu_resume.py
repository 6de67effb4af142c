"""Checkpoint/resume: a run split at step N -- the state read out with
mfc_get_state, a fresh context, mfc_set_state, the remaining M steps -- equals
the unbroken run of N + M steps bit for bit, state and per-step dt alike.

That holds because a step depends only on q^n: dt_n = CFL / S(q^n), and S of
a state set through mfc_set_state is computed by the same reference-order
reduction the stepping kernels reach at the end of a step.  Checked in the
reference-order FP64 form, through host buffers and through device buffers.
The reorganised FP64 form reduces S at the end of a step with its own
(contracted) formula, so the dt of the first resumed step can differ from the
unbroken run's by rounding: it agrees to the FP64 parity bar.  The FP32 forms
keep an FP32 working copy of q^n whose pressure is formed by a different
kernel build at set-up than at the end of a step (contracted FMAs), so their
resumed run agrees to FP32 rounding; both are checked.
"""
import numpy as np
import pytest

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


def _steps(s, k):
    """k single steps; the dt of each."""
    return [s.step_rk3(0.4, 1) for _ in range(k)]


@pytest.mark.parametrize("via", ["host", "device"])
def test_resume_is_bitwise(via, form="fp64"):
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_droplets(32)
    N, M = 25, 35
    a = mfc.Solver(p, form)
    a.set_state_prim(w)
    dts_a = _steps(a, N + M)
    qa = a.get_state()
    a.close()

    b = mfc.Solver(p, form)
    b.set_state_prim(w)
    dts_b = _steps(b, N)
    if via == "host":
        ck = b.get_state()
    else:
        ck = torch.empty(b.shape, dtype=torch.float64, device="cuda")
        b.get_state(ck)
    b.close()
    c = mfc.Solver(p, form)
    c.set_state(ck)
    dts_b += _steps(c, M)
    qc = c.get_state()
    c.close()
    assert dts_a == dts_b
    assert np.array_equal(qa, qc)

    # one call of N + M steps replays the same graph: same state, and its
    # time advanced is the same sum of the same dt in the same order
    d = mfc.Solver(p, form)
    d.set_state_prim(w)
    t = d.step_rk3(0.4, N + M)
    assert np.array_equal(d.get_state(), qa)
    acc = 0.0
    for dt in dts_a:
        acc += dt
    assert t == acc
    d.close()


@pytest.mark.parametrize("form,tol", [("fp64_fast", 1e-12), ("mixed", 1e-5)])
def test_resume_agrees_to_rounding(form, tol):
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_droplets(32)
    N, M = 25, 35
    a = mfc.Solver(p, form)
    a.set_state_prim(w)
    ta = a.step_rk3(0.4, N + M)
    qa = a.get_state()
    b = mfc.Solver(p, form)
    b.set_state_prim(w)
    tb = b.step_rk3(0.4, N)
    c = mfc.Solver(p, form)
    c.set_state(b.get_state())
    tb += c.step_rk3(0.4, M)
    qc = c.get_state()
    scale = np.abs(qa).reshape(7, -1).max(1)
    scale[2:5] = scale[2:5].max()
    err = (np.abs(qc - qa).reshape(7, -1).max(1) / scale).max()
    assert err <= tol
    assert abs(tb - ta) <= tol * ta
