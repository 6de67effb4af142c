"""Pins for the oracle's N-fluid model (N = 3, 4).

The five-equation model of Sec. II-A carries, per fluid i, a partial density
alpha_i rho_i and (for i < N) a volume fraction alpha_i; the mixture rules sum
over the fluids.  Checks against things other than the N-fluid code itself:
the two-fluid model when one fluid is split into two identical copies (the
split is a passive scalar), the two-fluid model when the extra fluids are
absent, discrete conservation, and pressure/velocity equilibrium across
interfaces of three different materials.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

WATER, AIR = I.WATER, I.AIR
OIL = (2.35, 1.0e9)   # a third stiffened gas


def _split(p2, w2, s, eps=1e-150):
    """3-fluid copy of a 2-fluid state: fluid 2 (air) split into fluids 2 and
    3 of the same material in the fixed ratio s : 1 - s."""
    d = p2["ndim"]
    p3 = dict(p2, gamma=[p2["gamma"][0], p2["gamma"][1], p2["gamma"][1]],
              pi_inf=[p2["pi_inf"][0], p2["pi_inf"][1], p2["pi_inf"][1]], weno_eps=eps)
    a1 = w2[3 + d]
    w3 = np.empty((2 * 3 + d,) + w2.shape[1:])
    w3[0] = w2[0]
    w3[1] = s * w2[1]
    w3[2] = (1 - s) * w2[1]
    w3[3:3 + d] = w2[2:2 + d]
    w3[3 + d] = w2[2 + d]
    w3[4 + d] = a1
    w3[5 + d] = s * (1 - a1)
    return dict(p2, weno_eps=eps), p3, w3


@pytest.mark.parametrize("ndim,n", [(1, [40]), (2, [14, 11]), (3, [9, 7, 6])])
def test_split_fluid_is_the_two_fluid_model(ndim, n):
    """Splitting air into two identical fluids (ratio s) changes nothing: the
    summed partial densities, momenta, energy and alpha_1 have the two-fluid
    RHS, and alpha_2 = s (1 - alpha_1) evolves as -s times alpha_1 (WENO with a
    vanishing epsilon is scale- and shift-invariant, HLLC linear in the
    partial densities)."""
    p2, w2 = I.random_periodic(ndim, n, seed=60 + ndim)
    s = 0.3
    p2e, p3, w3 = _split(p2, w2, s)
    q2, q3 = O.prim_to_cons(p2e, w2), O.prim_to_cons(p3, w3)
    L2, L3 = O.rhs(p2e, q2), O.rhs(p3, q3)
    d = ndim
    scale = np.abs(q2).reshape(q2.shape[0], -1).max(1) * O.max_wavespeed(p2e, q2)

    def close(a, b, sc):
        assert np.max(np.abs(a - b)) <= 1e-12 * sc

    close(L3[0], L2[0], scale[0])
    close(L3[1] + L3[2], L2[1], scale[1])
    for k in range(d):
        close(L3[3 + k], L2[2 + k], scale[2 + k] + scale[2:2 + d].max())
    close(L3[3 + d], L2[2 + d], scale[2 + d])
    close(L3[4 + d], L2[3 + d], scale[3 + d])
    close(L3[5 + d], -s * L2[3 + d], scale[3 + d])
    assert O.max_wavespeed(p3, q3) == pytest.approx(O.max_wavespeed(p2e, q2), rel=1e-14)


def test_absent_fluids_leave_the_two_fluid_model():
    """Fluids 2 and 3 of a 4-fluid system absent everywhere (alpha 0): the air
    -water shock tube runs as in the two-fluid model."""
    p2, w2 = I.air_water_shock_tube(200)
    p4 = dict(p2, gamma=[WATER[0], OIL[0], OIL[0], AIR[0]], pi_inf=[WATER[1], OIL[1], OIL[1], AIR[1]])
    a1 = w2[4]
    w4 = I.assemble_n(p4, [a1, 0.0, 0.0], [1000.0, 900.0, 900.0, 50.0], [w2[2]], w2[3])
    w4[0], w4[3] = w2[0], w2[1]
    q2, _ = O.run_cfl(p2, O.prim_to_cons(p2, w2), 0.4, 50)
    q4, _ = O.run_cfl(p4, O.prim_to_cons(p4, w4), 0.4, 50)
    for a, b in ((q4[0], q2[0]), (q4[3], q2[1]), (q4[4], q2[2]), (q4[5], q2[3]), (q4[6], q2[4])):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    assert np.all(q4[1] == 0.0) and np.all(q4[2] == 0.0) and np.all(q4[7] == 0.0) and np.all(q4[8] == 0.0)


@pytest.mark.parametrize("nf", [3, 4])
def test_conservation_n_fluids(nf):
    """All partial masses, momenta and energy conserved to round-off on a
    periodic 2-D domain with N fluids."""
    fl = [WATER, AIR, OIL, (1.8, 2.0e8)][:nf]
    p = I.make_params(2, [12, 10], [0.0, 0.0], [1.0, 1.0], I.PERIODIC, gamma=[f[0] for f in fl],
                      pi_inf=[f[1] for f in fl])
    x, y, _ = I.cell_centres(p)
    X, Y = np.meshgrid(x, y)
    rng = np.random.default_rng(nf)
    raw = [0.5 + 0.4 * np.sin(2 * np.pi * (X * rng.integers(1, 3) + Y * rng.integers(1, 3)) + k) for k in range(nf)]
    tot = sum(raw)
    alphas = [(r / tot)[None] for r in raw[:-1]]
    w = I.assemble_n(p, alphas, [1000.0, 1.2, 900.0, 3.0][:nf],
                     [50.0 * np.cos(2 * np.pi * Y)[None], 30.0 * np.sin(2 * np.pi * X)[None]],
                     1e7 * (1 + 0.1 * np.cos(2 * np.pi * X))[None])
    q = O.prim_to_cons(p, w)
    S = O.max_wavespeed(p, q)
    for _ in range(3):
        q1 = O.step_dt(p, q, 0.4 / S)
        for f in range(nf + 3):
            scale = np.sum(np.abs(q[f]))
            assert abs(np.sum(q1[f]) - np.sum(q[f])) <= 1e-13 * scale, f
        q = q1


def test_three_material_equilibrium():
    """Water and oil slabs translating through air at 100 m/s, p = 1e5: p and
    u stay uniform to the round-off bound of the two-fluid pin."""
    n, steps = 64, 150
    p = I.make_params(1, [n], [0.0], [1.0], I.PERIODIC, gamma=[WATER[0], OIL[0], AIR[0]],
                      pi_inf=[WATER[1], OIL[1], AIR[1]])
    x, _, _ = I.cell_centres(p)
    e = I.ALPHA_EPS
    a_w = np.where((x >= 0.2) & (x < 0.45), 1 - 2 * e, e)
    a_o = np.where((x >= 0.55) & (x < 0.8), 1 - 2 * e, e)
    w = I.assemble_n(p, [a_w[None, None], a_o[None, None]], [1000.0, 900.0, 1.2], [100.0], 1e5)
    q, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, steps)
    wf = O.cons_to_prim(p, q)
    Pi_max = max(WATER[0] * WATER[1] / (WATER[0] - 1), OIL[0] * OIL[1] / (OIL[0] - 1))
    G_min = min(1 / (WATER[0] - 1), 1 / (OIL[0] - 1))
    tol = steps * 30 * np.finfo(float).eps * Pi_max / (G_min * 1e5)
    assert np.max(np.abs(wf[4] - 1e5)) / 1e5 <= tol
    assert np.max(np.abs(wf[3] - 100.0)) / 100.0 <= tol
    assert np.ptp(wf[5]) > 0.9 and np.ptp(wf[6]) > 0.9


def test_bad_fluid_counts_are_rejected():
    p, w = I.smooth_density_wave(8)
    q = O.prim_to_cons(p, w)
    for g in ([1.4], [1.4] * 5):
        with pytest.raises(Exception):
            O.rhs(dict(p, gamma=g, pi_inf=[0.0] * len(g)), q)
