"""GPU parity: the FP64 CUDA paths against the serial FP64 oracle.

Every comparison is element by element on the same seeded inputs, per field.
The FP64 form ("fp64", reference operation order, no FMA contraction) must
equal the oracle bit for bit.  The reorganised FP64 form ("fp64_fast") is held
to the FP64 parity bar: states (after the stated step counts) as relative
L-infinity, max|gpu - oracle| / max|oracle| <= 1e-12.

A single RHS is a difference of face fluxes divided by dx, so its round-off
scales with the flux magnitude, not with the (possibly much smaller) result:
RHS errors are taken relative to max(max|L_f|, max|q_f| * S), where
S = max sum_d (|u_d| + c)/dx_d makes |q| S the natural size of dq/dt; the bar
is again 1e-12.  A wrong term, sign or index shows up at 1e-6 or far above.

Sizes span several warps/segments and ragged tails; full-size workloads are
checked on sampled cells the oracle evaluates one by one, plus the wave speed
over every cell.
"""
import numpy as np
import pytest

import oracle as O
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


FORMS = ["fp64", "fp64_fast"]
_ORACLE_RUNS = {}


def oracle_run(key, p, w, steps):
    """The oracle's CFL run of a case, computed once per test session."""
    if key not in _ORACLE_RUNS:
        _ORACLE_RUNS[key] = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, steps)
    return _ORACLE_RUNS[key]


def check_state(form, got, ref):
    if form == "fp64":
        assert np.array_equal(got, ref), f"not bit-identical, rel err {rel_err(got, ref)}"
    else:
        assert rel_err(got, ref).max() <= TOL


def check_rhs(form, p, L, Lo, q, S):
    if form == "fp64":
        assert np.array_equal(L, Lo), f"not bit-identical, err {rhs_err(p, L, Lo, q, S)}"
    else:
        assert rhs_err(p, L, Lo, q, S).max() <= TOL


def solver(p, precision="fp64"):
    from paper_2409_10729_gb300 import mfc
    return mfc.Solver(p, precision)


def rel_err(a, b, nf=2):
    """Per-field relative L-infinity error of a against reference b.  The
    momentum components are rows of one vector field and share its scale,
    max over cells of |rho u| (otherwise a component that is ~0 in a given
    orientation, e.g. rho v in a flow along x, would be judged against its own
    round-off-sized values).  nf: number of fluids (momenta at rows nf ..)."""
    ndim = a.shape[0] - 2 * nf
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    scale = np.abs(b).max(1)
    mom = np.sqrt((b[nf:nf + ndim] ** 2).sum(0)).max()
    scale[nf:nf + ndim] = mom
    return np.abs(a - b).max(1) / np.maximum(scale, 1e-300)


def rhs_scale(p, q, Lo, S):
    """Per-field size of the fluxes a RHS is formed from, per unit length:
    max(max|L_f|, max|q_f| S), plus max(p) max(1/dx_d) on the momentum rows
    (their normal flux carries the pressure)."""
    nq = q.shape[0]
    qf = q.reshape(nq, -1)
    scale = np.maximum(np.abs(Lo.reshape(Lo.shape[0], -1)).max(1), np.abs(qf).max(1) * S)
    ndim = p["ndim"]
    nfl = len(p["gamma"])
    pmax = np.abs(O.cons_to_prim(p, q)[nfl + ndim]).max()
    inv_dx = max(p["n"][d] / (p["hi"][d] - p["lo"][d]) for d in range(ndim))
    scale[nfl:nfl + ndim] = np.maximum(scale[nfl:nfl + ndim], pmax * inv_dx)
    return scale


def rhs_err(p, L, Lo, q, S):
    """Per-field RHS error relative to rhs_scale."""
    d = np.abs(L.reshape(L.shape[0], -1) - Lo.reshape(Lo.shape[0], -1)).max(1)
    return d / np.maximum(rhs_scale(p, q, Lo, S), 1e-300)


SMALL = [
    (1, [33], 0), (1, [33], 1), (1, [200], 1),
    (2, [16, 8], 0), (2, [13, 9], 1), (2, [70, 37], 0),
    (3, [8, 8, 8], 0), (3, [13, 9, 7], 1), (3, [7, 5, 4], 0), (3, [40, 11, 35], 1),
]


def _case(ndim, n, bc, seed=0):
    p, w = I.random_periodic(ndim, n, seed=seed)
    p["bc"] = [[bc, bc]] * ndim + [[0, 0]] * (3 - ndim)
    return p, w


@pytest.mark.parametrize("ndim,n,bc", SMALL)
def test_prim_to_cons(ndim, n, bc):
    """The conversion of the seeded primitive state is bit-identical (every
    form starts from the same conservative state)."""
    p, w = _case(ndim, n, bc)
    s = solver(p)
    s.set_state_prim(w)
    assert np.array_equal(s.get_state(), O.prim_to_cons(p, w))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc", SMALL)
def test_rhs_parity_small(ndim, n, bc, form):
    p, w = _case(ndim, n, bc, seed=ndim)
    s = solver(p, form)
    s.set_state_prim(w)
    L = s.rhs()
    q = O.prim_to_cons(p, w)
    Lo = O.rhs(p, q)
    check_rhs(form, p, L, Lo, q, O.max_wavespeed(p, q))


@pytest.mark.parametrize("ndim,n,bc", SMALL)
def test_wavespeed_parity(ndim, n, bc):
    p, w = _case(ndim, n, bc, seed=ndim + 3)
    s = solver(p)
    s.set_state_prim(w)
    So = O.max_wavespeed(p, O.prim_to_cons(p, w))
    assert s.max_wavespeed() == So


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc", SMALL)
def test_cfl_steps_parity_small(ndim, n, bc, form):
    p, w = _case(ndim, n, bc, seed=ndim + 5)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 5)
    qo, to = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 5)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-13 * to


@pytest.mark.parametrize("form", FORMS)
def test_fixed_dt_parity(form):
    p, w = _case(3, [13, 9, 7], 1, seed=11)
    q = O.prim_to_cons(p, w)
    dt = 0.3 / O.max_wavespeed(p, q)
    s = solver(p, form)
    s.set_state(q)
    s.step_rk3_dt(dt, 3)
    qo = q
    for _ in range(3):
        qo = O.step_dt(p, qo, dt)
    check_state(form, s.get_state(), qo)


@pytest.mark.parametrize("form", FORMS)
def test_air_water_tube_full_run(form):
    """1000 cells, 200 CFL-0.4 steps, FP64: every field within 1e-12."""
    p, w = I.air_water_shock_tube(1000)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 200)
    qo, to = oracle_run("test_air_water_tube_full_run", p, w, 200)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-12 * to


@pytest.mark.parametrize("form", FORMS)
def test_shock_water_column_reduced_full_run(form):
    """The 2-D shock / water-column case on a 128x64 grid for its full 500 steps."""
    p, w = I.shock_water_column(128, 64)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 500)
    qo, to = oracle_run("test_shock_water_column_reduced_full_run", p, w, 500)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-12 * to


@pytest.mark.parametrize("form", FORMS)
def test_shock_droplets_reduced_full_run(form):
    """The 3-D shock / droplet case on a 32^3 grid for its full 100 steps."""
    p, w = I.shock_droplets(32)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 100)
    qo, to = oracle_run("test_shock_droplets_reduced_full_run", p, w, 100)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-12 * to


def _sample_cells(p, k, seed):
    rng = np.random.default_rng(seed)
    n = p["n"]
    nc = n[0] * n[1] * n[2]
    cells = list(rng.integers(0, nc, size=k))
    # faces and corners of the box (ghost handling)
    for z in (0, n[2] - 1):
        for y in (0, n[1] - 1):
            for x in (0, 1, 2, n[0] - 3, n[0] - 2, n[0] - 1):
                cells.append(x + n[0] * (y + n[1] * z))
    return np.unique(np.array(cells, dtype=np.int64))


def _check_sampled(p, s, q, seed):
    """RHS at sampled cells and the wave speed over all cells, against the
    oracle, bit for bit (FP64 form)."""
    cells = _sample_cells(p, 4096, seed)
    Lfull = s.rhs().reshape(q.shape[0], -1)
    Lo = O.rhs_points(p, q, cells).T
    So = O.max_wavespeed(p, q)
    assert np.array_equal(Lfull[:, cells], Lo)
    assert s.max_wavespeed() == So


@pytest.mark.parametrize("case", ["column_1024x512", "droplets_256"])
def test_full_size_sampled(case):
    """Full-size workloads in the benchmark's launch configuration: the RHS of
    the initial state and of the state after the full FP64 run, at 4096+
    sampled cells, and the wave speed, against the oracle."""
    if case == "column_1024x512":
        p, w = I.shock_water_column(1024, 512)
        steps = 500
    else:
        p, w = I.shock_droplets(256)
        steps = 100
    s = solver(p)
    s.set_state_prim(w)
    q0 = O.prim_to_cons(p, w)
    assert np.array_equal(s.get_state(), q0)
    _check_sampled(p, s, q0, 1)
    s.step_rk3(0.4, steps)
    qf = s.get_state()
    assert np.all(np.isfinite(qf))
    _check_sampled(p, s, qf, 2)


def test_largest_size_sampled():
    """The largest configuration (3-D droplets at 512^3, 134M cells, the mixed
    form's benchmark size): FP64 RHS at 4096+ sampled cells and the wave speed
    bit for bit, before and after two steps; the mixed form's RHS at the same
    cells within FP32 accuracy of the flux scale."""
    p, w = I.shock_droplets(512)
    q0 = O.prim_to_cons(p, w)
    s = solver(p)
    s.set_state(q0)
    _check_sampled(p, s, q0, 3)
    m = solver(p, "mixed")
    m.set_state(q0)
    cells = _sample_cells(p, 4096, 3)
    Lm = m.rhs().reshape(q0.shape[0], -1)[:, cells]
    m.close()
    Lo = O.rhs_points(p, q0, cells).T
    S = O.max_wavespeed(p, q0)
    # flux scale as in rhs_scale, from the whole state
    scale = np.maximum(np.abs(Lo).max(1), np.abs(q0.reshape(q0.shape[0], -1)).max(1) * S)
    pmax = np.abs(O.cons_to_prim(p, q0)[5]).max()
    scale[2:5] = np.maximum(scale[2:5], pmax * 512.0)
    assert (np.abs(Lm - Lo).max(1) / scale).max() <= 1e-5
    s.step_rk3(0.4, 2)
    _check_sampled(p, s, s.get_state(), 4)


@pytest.mark.parametrize("where", ["interior", "edge"])
def test_nonphysical_state_is_reported(where):
    """A cell with negative density: both sides report it (MFC_ENONPHYSICAL /
    the oracle's status), on the RHS and on a step."""
    from paper_2409_10729_gb300 import mfc
    p, w = _case(2, [16, 12], 0)
    y, x = (5, 7) if where == "interior" else (0, 15)
    w[0, 0, y, x] = -1.0
    w[1, 0, y, x] = 0.0
    s = solver(p)
    s.set_state_prim(w)
    s.rhs(allow_nonphysical=True)
    assert s.last_status == mfc.MFC_ENONPHYSICAL
    with pytest.raises(RuntimeError):
        O.rhs(p, O.prim_to_cons(p, w))
    s.step_rk3(0.4, 1, allow_nonphysical=True)
    assert s.last_status == mfc.MFC_ENONPHYSICAL


def test_device_arrays_and_timing_mode():
    """Torch device tensors in and out give the same result as host arrays,
    and stepping with per-kernel timing (direct launches) equals the graph."""
    import torch
    p, w = _case(3, [24, 20, 18], 1, seed=4)
    s1, s2 = solver(p), solver(p)
    s1.set_state_prim(torch.from_numpy(w).cuda())
    s2.set_state_prim(w)
    Ld = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    s1.rhs(Ld)
    np.testing.assert_array_equal(Ld.cpu().numpy(), s2.rhs())
    s1.set_timing(True)
    t1 = s1.step_rk3(0.4, 4)
    t2 = s2.step_rk3(0.4, 4)
    assert t1 == t2
    qd = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    s1.get_state(qd)
    np.testing.assert_array_equal(qd.cpu().numpy(), s2.get_state())
    kt = s1.kernel_times()
    assert kt["sweep_z"][1] == 12 and kt["step_begin"][1] == 4
    assert s1.launches_per_step() == 10


def test_integer_conversions_match_hardware():
    """The mixed form's integer-pipe float<->double conversions return the
    hardware conversions' bits on 16M pseudo-random patterns."""
    import ctypes
    from paper_2409_10729_gb300 import mfc
    bad = ctypes.c_longlong(-1)
    assert mfc.lib().mfc_selfcheck_conversions(1 << 24, 2409, ctypes.byref(bad)) == 0
    assert bad.value == 0


def test_integer_weno_operations_match_hardware():
    """The FP64 form's integer-pipe products K v (K = 3, 5, 7, 11) and
    quotients x/6 return the FP64 instructions' bits, and its integer-word
    compares (x > 0, 0 <= x, x < y) the FP64 compares' answers, on 64M
    patterns, zeros, subnormals, infinities, NaNs and the ends of the exponent
    range among them."""
    import ctypes
    from paper_2409_10729_gb300 import mfc
    bad = ctypes.c_longlong(-1)
    assert mfc.lib().mfc_selfcheck_exact_ops(1 << 26, 1729, ctypes.byref(bad)) == 0
    assert bad.value == 0


# ---------------------------------------------------------------- WENO3 ----
# The third-order reconstruction option (Sec. II-B; weno_order = 3) to the
# same bar: bit-identical in the FP64 form, 1e-12 in the reorganised one.

W3_SMALL = [(1, [33], 1), (2, [13, 9], 1), (2, [70, 37], 0), (3, [13, 9, 7], 1), (3, [40, 11, 35], 0)]


def _w3(p):
    return dict(p, weno_order=3)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc", W3_SMALL)
def test_weno3_rhs_parity_small(ndim, n, bc, form):
    p, w = _case(ndim, n, bc, seed=ndim + 20)
    p = _w3(p)
    s = solver(p, form)
    s.set_state_prim(w)
    L = s.rhs()
    q = O.prim_to_cons(p, w)
    Lo = O.rhs(p, q)
    assert not np.array_equal(Lo, O.rhs(dict(p, weno_order=5), q))
    check_rhs(form, p, L, Lo, q, O.max_wavespeed(p, q))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc", W3_SMALL)
def test_weno3_cfl_steps_parity_small(ndim, n, bc, form):
    p, w = _case(ndim, n, bc, seed=ndim + 25)
    p = _w3(p)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 5)
    qo, to = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 5)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-13 * to


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["tube_1000x200", "column_128x64x500", "droplets_32x100"])
def test_weno3_full_runs(case, form):
    """The three workloads at reduced size for their full step counts, WENO3."""
    gen = {"tube_1000x200": (lambda: I.air_water_shock_tube(1000), 200),
           "column_128x64x500": (lambda: I.shock_water_column(128, 64), 500),
           "droplets_32x100": (lambda: I.shock_droplets(32), 100)}
    mk, steps = gen[case]
    p, w = mk()
    p = _w3(p)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, steps)
    qo, to = oracle_run("weno3_" + case, p, w, steps)
    check_state(form, s.get_state(), qo)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-12 * to


def test_weno3_mixed_form_error_against_oracle():
    """Mixed precision with WENO3 on the 2-D column (128x64, 100 steps):
    per-field error against the oracle at the FP32 level."""
    p, w = I.shock_water_column(128, 64)
    p = _w3(p)
    s = solver(p, "mixed")
    s.set_state_prim(w)
    s.step_rk3(0.4, 100)
    qo, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 100)
    q = s.get_state()
    err = rel_err(q, qo)
    assert err.max() <= 2e-4, err
    l1 = np.abs(q - qo).reshape(6, -1).sum(1) / np.abs(qo).reshape(6, -1).sum(1)
    assert l1[[0, 1, 4, 5]].max() <= 1e-6, l1


# ---------------------------------------------------------------- non-uniform grids
# Directions refined with a hyperbolic tangent (Sec. III-A), set through
# mfc_set_grid from the same edges the oracle takes.  The library computes its
# WENO5 tables independently of the oracle (Lagrange derivatives of the
# primitive function versus cell-average solves), so the FP64 forms are held
# to 1e-12 rather than bit-identity; the wave speed (same widths, IEEE
# quotients) must still match exactly.

def _stretch(p, dirs, centre=0.45, strength=10.0, refine=0.6):
    edges = [None, None, None]
    for d in dirs:
        edges[d] = I.tanh_edges(p["n"][d], p["lo"][d], p["hi"][d], p["lo"][d] + centre * (p["hi"][d] - p["lo"][d]),
                                strength=strength, refine=refine)
    return dict(p, edges=edges)


NU_SMALL = [(1, [40], 1, (0,)), (1, [37], 0, (0,)), (2, [21, 13], 1, (0, 1)), (2, [33, 19], 0, (1,)),
            (3, [13, 9, 11], 1, (0, 1, 2)), (3, [40, 11, 35], 0, (0, 2))]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc,dirs", NU_SMALL)
def test_stretched_rhs_and_wavespeed_parity(ndim, n, bc, dirs, form):
    p, w = _case(ndim, n, bc, seed=ndim + 40)
    p = _stretch(p, dirs)
    s = solver(p, form)
    s.set_state_prim(w)
    L = s.rhs()
    q = O.prim_to_cons(p, w)
    Lo = O.rhs(p, q)
    So = O.max_wavespeed(p, q)
    assert not np.allclose(Lo, O.rhs(dict(p, edges=None), q), rtol=1e-6, atol=0)
    assert rhs_err(p, L, Lo, q, So).max() <= TOL
    if form == "fp64":
        assert s.max_wavespeed() == So
    else:
        assert s.max_wavespeed() == pytest.approx(So, rel=1e-14)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,bc,dirs", NU_SMALL)
def test_stretched_cfl_steps_parity(ndim, n, bc, dirs, form):
    p, w = _case(ndim, n, bc, seed=ndim + 45)
    p = _stretch(p, dirs)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 5)
    qo, to = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 5)
    assert rel_err(s.get_state(), qo).max() <= TOL
    assert abs(t - to) <= 1e-13 * to


@pytest.mark.parametrize("form", FORMS)
def test_stretched_shock_water_column(form):
    """2-D shock / water column at 128x64, both directions refined around the
    column, 100 steps: within 1e-11 (independent tables; rounding differences
    of 1e-16 grow through the shock-interface interaction as on uniform grids)."""
    p, w = I.shock_water_column(128, 64)
    p = _stretch(p, (0, 1), centre=0.3, strength=8.0, refine=0.5)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 100)
    qo, to = oracle_run("stretched_column_128x64x100", p, w, 100)
    assert rel_err(s.get_state(), qo).max() <= 1e-11
    assert abs(t - to) <= 1e-12 * to


def test_stretched_mixed_form_error_against_oracle():
    p, w = I.shock_water_column(128, 64)
    p = _stretch(p, (0, 1), centre=0.3, strength=8.0, refine=0.5)
    s = solver(p, "mixed")
    s.set_state_prim(w)
    s.step_rk3(0.4, 100)
    qo, _ = oracle_run("stretched_column_128x64x100", p, w, 100)
    q = s.get_state()
    # FP32 stencils at the shock: ~2e-4 of the momentum scale (as on uniform grids)
    assert rel_err(q, qo).max() <= 5e-4
    l1 = np.abs(q - qo).reshape(6, -1).sum(1) / np.abs(qo).reshape(6, -1).sum(1)
    assert l1[[0, 1, 4, 5]].max() <= 1e-6, l1


def test_set_grid_rejections():
    from paper_2409_10729_gb300 import mfc
    p, w = _case(2, [16, 8], 0)
    e = I.tanh_edges(16, 0.0, 1.0, 0.5)
    bad = e.copy()
    bad[5] = bad[4]
    s = solver(p, "fp64")
    for d, edges in ((2, e), (0, bad)):
        with pytest.raises(mfc.MfcError):
            s.set_grid(d, edges)
    for kw, prec in ((dict(weno_order=3), "fp64"), ({}, "gated")):
        g = solver(dict(p, **kw), prec)
        with pytest.raises(mfc.MfcError):
            g.set_grid(0, e)


# ---------------------------------------------------------------- N fluids
# The N-fluid model (N = 3, 4; the oracle's N-fluid pins fix the model) to
# the same bar: bit-identical in the FP64 form, 1e-12 in the reorganised one.

NF_SMALL = [(1, [33], 3), (2, [13, 9], 3), (3, [9, 7, 6], 3), (2, [14, 11], 4), (3, [8, 7, 5], 4)]


def check_state_n(form, got, ref, nf):
    if form == "fp64":
        assert np.array_equal(got, ref), f"not bit-identical, rel err {rel_err(got, ref, nf)}"
    else:
        assert rel_err(got, ref, nf).max() <= TOL


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,nf", NF_SMALL)
def test_nfluid_rhs_parity(ndim, n, nf, form):
    p, w = I.random_periodic_n(ndim, n, nf, seed=70 + ndim + nf)
    s = solver(p, form)
    s.set_state_prim(w)
    L = s.rhs()
    q = O.prim_to_cons(p, w)
    assert np.array_equal(s.get_state(), q)
    Lo = O.rhs(p, q)
    check_rhs(form, p, L, Lo, q, O.max_wavespeed(p, q))
    if form == "fp64":
        assert s.max_wavespeed() == O.max_wavespeed(p, q)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ndim,n,nf", NF_SMALL)
def test_nfluid_cfl_steps_parity(ndim, n, nf, form):
    p, w = I.random_periodic_n(ndim, n, nf, seed=80 + ndim + nf)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 5)
    qo, to = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 5)
    check_state_n(form, s.get_state(), qo, nf)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-13 * to


@pytest.mark.parametrize("form", FORMS)
def test_three_fluid_droplets_full_run(form):
    """Water and oil droplets in air (32^3), Mach-2 shock, 60 steps."""
    p, w = I.shock_droplets_3fluid(32)
    s = solver(p, form)
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 60)
    qo, to = oracle_run("droplets3_32x60", p, w, 60)
    check_state_n(form, s.get_state(), qo, 3)
    assert t == to if form == "fp64" else abs(t - to) <= 1e-12 * to


def test_three_fluid_mixed_form_error_against_oracle():
    p, w = I.shock_droplets_3fluid(32)
    s = solver(p, "mixed")
    s.set_state_prim(w)
    s.step_rk3(0.4, 60)
    qo, _ = oracle_run("droplets3_32x60", p, w, 60)
    q = s.get_state()
    assert rel_err(q, qo, 3).max() <= 1e-3
    l1 = np.abs(q - qo).reshape(9, -1).sum(1) / np.abs(qo).reshape(9, -1).sum(1)
    assert l1[[0, 1, 2, 6, 7, 8]].max() <= 1e-5, l1


def test_nfluid_rejections():
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic_n(2, [16, 8], 3, seed=1)
    with pytest.raises(mfc.MfcError):
        solver(p, "gated")
    s = solver(p, "fp64")
    with pytest.raises(mfc.MfcError):
        s.set_grid(0, I.tanh_edges(16, 0.0, 1.0, 0.5))


# ---------------------------------------------------------------- degenerate grids
# Directions with fewer cells than the five-cell stencil (1 or 2 cells: every
# ghost is a copy or a wrap of them), single cells, and segments of one cell.

DEGENERATE = [(1, [1], 0), (1, [1], 1), (1, [2], 0), (1, [3], 1), (2, [1, 9], 0), (2, [9, 1], 1),
              (2, [2, 2], 1), (3, [1, 1, 1], 0), (3, [5, 1, 3], 1), (3, [1, 33, 2], 0)]


@pytest.mark.parametrize("form", FORMS + ["mixed"])
@pytest.mark.parametrize("ndim,n,bc", DEGENERATE)
def test_degenerate_grids(ndim, n, bc, form):
    p, w = _case(ndim, n, bc, seed=90 + ndim)
    s = solver(p, form)
    s.set_state_prim(w)
    L = s.rhs()
    q = O.prim_to_cons(p, w)
    Lo = O.rhs(p, q)
    S = O.max_wavespeed(p, q)
    t = s.step_rk3(0.4, 3)
    qo, to = O.run_cfl(p, q, 0.4, 3)
    if form == "mixed":
        assert rhs_err(p, L, Lo, q, S).max() <= 1e-5
        assert rel_err(s.get_state(), qo).max() <= 1e-5
    else:
        check_rhs(form, p, L, Lo, q, S)
        check_state(form, s.get_state(), qo)
        assert t == to if form == "fp64" else abs(t - to) <= 1e-13 * to
