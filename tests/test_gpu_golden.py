"""Full-size FP64 parity at the stated step counts, against stored oracle
results written by tests/golden/make_golden.py (which calls only the oracle).

The 2-D shock / water-column case at 1024x512 for 500 steps and the 3-D
shock / droplet case at 128^3 and 256^3 for 100 steps (CFL 0.4) are run on
the GPU in the benchmark's launch configuration.  The FP64 form (reference
operation order) must reproduce the time advanced, the per-field sums over
all cells and the state at ~1000 sampled cells bit for bit, and, where the
stored result carries it, the SHA-256 of the whole final state.  The reorganised FP64 form
is checked against a bound set by the flows themselves: re-running the
oracle with FMA contraction (a change of rounding only) moves the 2-D
momentum by 6.6e-12 relative after 500 steps, so it is held to 5e-11
(momentum rows relative to the largest momentum component) and 1e-12 in t.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2409_10729_gb300 import inputs as I

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-12
CASES = {
    "column_1024x512": lambda: I.shock_water_column(1024, 512),
    "droplets_128": lambda: I.shock_droplets(128),
    "droplets_256": lambda: I.shock_droplets(256),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10729_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("form", ["fp64", "fp64_fast"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_full_size_run_matches_stored_oracle(name, form):
    from paper_2409_10729_gb300 import mfc
    path = os.path.join(HERE, "golden", f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle result {name}.json not generated (tests/golden/make_golden.py)")
    with open(path) as f:
        g = json.load(f)
    p, w = CASES[name]()
    assert hashlib.sha256(np.ascontiguousarray(w).tobytes()).hexdigest() == g["ic_sha256"], \
        "initial state differs from the one the stored oracle result was made from"
    s = mfc.Solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(g["cfl"], g["steps"])
    q = s.get_state()
    ne = q.shape[0]
    ndim = ne - 4
    qf = q.reshape(ne, -1)
    t_ref = float(g["t_final"])
    ref = np.array([[float(v) for v in row] for row in g["values"]]).T
    l1 = np.array([float(v) for v in g["field_l1"]])
    sums = np.array([float(v) for v in g["field_sum"]])
    if form == "fp64":
        assert t == t_ref
        assert np.array_equal(qf[:, g["cells"]], ref)
        if "state_sha256" in g:
            assert hashlib.sha256(np.ascontiguousarray(q, dtype=np.float64).tobytes()).hexdigest() == \
                g["state_sha256"], "whole final state differs from the oracle's"
        assert np.array_equal(np.abs(qf).max(1), np.array([float(v) for v in g["field_max_abs"]]))
        # numpy's summation order may differ between machines: sums to round-off
        assert np.all(np.abs(np.abs(qf).sum(1) - l1) <= 1e-14 * l1)
        assert np.all(np.abs(qf.sum(1) - sums) <= 1e-14 * l1)
    else:
        assert abs(t - t_ref) <= TOL * t_ref
        scale = np.array([float(v) for v in g["field_max_abs"]])
        scale[2:2 + ndim] = scale[2:2 + ndim].max()
        err = np.abs(qf[:, g["cells"]] - ref).max(1) / scale
        assert err.max() <= 5e-11, f"sampled-cell error per field {err}"
        assert np.all(np.abs(np.abs(qf).sum(1) - l1) <= 5e-11 * l1)
    s.close()
