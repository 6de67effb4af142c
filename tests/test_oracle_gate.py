"""Pins for the oracle's gated right-hand side (the gated form's rule; the
paper has no gate).  Each pin fixes a part of the rule by something other
than the oracle itself:

* limits: a gate that never fires is plain WENO5-JS bit for bit; one that
  always fires is WENO5 with epsilon -> infinity (linear weights);
* the linear reconstruction is exact for cell averages of quartics;
* the flat test: closed-form decisions for a single-cell bump just below and
  just above the round-off floor, and a uniform state (every stencil flat:
  linear everywhere, L = 0, whatever the network says);
* both sensors: a pressure step in uniform density is troubled by its
  pressure stencil alone;
* the network's input: hand-built networks whose logit is a known function
  of the normalised stencil (its orientation, its centring) give
  closed-form decisions on ramps;
* the fallback: across the sharp air-water interface linear faces leave
  [0, 1] in alpha1; exactly the cells with a non-admissible linear face fall
  back, and away from the gate's switches the RHS equals the plain or the
  linear-weight RHS cell by cell.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

DELTA = 1e-4


def _bias(b3):
    th = np.zeros(1281)
    th[1280] = b3
    return th


def _hand_net(kind):
    """z = (x4 - x0) - 1/2 ("orientation") or z = x0 + x4 + 1/2
    ("centring"), built from ReLU pairs and an identity second layer."""
    th = np.zeros(1281)
    W1 = th[0:160].reshape(32, 5)
    W1[0, 4], W1[0, 0] = 1.0, -1.0      # relu(x4 - x0)
    W1[1, 4], W1[1, 0] = -1.0, 1.0      # relu(x0 - x4)
    W1[2, 0], W1[2, 4] = 1.0, 1.0       # relu(x0 + x4)
    W1[3, 0], W1[3, 4] = -1.0, -1.0     # relu(-x0 - x4)
    W2 = th[192:1216].reshape(32, 32)
    for i in range(4):
        W2[i, i] = 1.0
    w3 = th[1248:1280]
    if kind == "orientation":
        w3[0], w3[1], th[1280] = 1.0, -1.0, -0.5
    else:
        w3[2], w3[3], th[1280] = 1.0, -1.0, 0.5
    return th


def _scale(p, L, q):
    S = O.max_wavespeed(p, q)
    return np.maximum(np.abs(L).reshape(L.shape[0], -1).max(1), np.abs(q).reshape(q.shape[0], -1).max(1) * S)


def _tube_like(n, rho_fn, p_fn):
    """1-D periodic air state with given density (second partial density)
    and pressure profiles, at rest; alpha1 = 1e-6."""
    p = I.make_params(1, [n], [0.0], [1.0], [[1, 1]])
    x = (np.arange(n) + 0.5) / n
    w = np.zeros((5, 1, 1, n))
    w[0, 0, 0] = 1e-6 * 1000.0
    w[1, 0, 0] = rho_fn(np.arange(n))
    w[2, 0, 0] = 0.0
    w[3, 0, 0] = p_fn(np.arange(n))
    w[4, 0, 0] = 1e-6
    return p, w, x


@pytest.mark.parametrize("ndim,n", [(2, [20, 14]), (3, [10, 9, 8])])
def test_gate_that_never_fires_is_plain_weno(ndim, n):
    p, w = I.random_periodic(ndim, n, seed=3)
    q = O.prim_to_cons(p, w)
    L, dec, info = O.rhs_gated(p, q, _bias(10.0), DELTA)
    assert np.array_equal(L, O.rhs(p, q))
    assert np.all(dec == 0)
    assert np.all(info[..., 0] == 10.0) and np.all(info[..., 1] == 10.0)   # every stencil non-flat: z = b3


def test_gate_that_always_fires_is_weno_with_infinite_epsilon():
    p, w = I.random_periodic(3, [10, 9, 8], seed=4)
    q = O.prim_to_cons(p, w)
    L, dec, _ = O.rhs_gated(p, q, _bias(-10.0), DELTA)
    assert np.all(dec == 1)
    Llin = O.rhs(dict(p, weno_eps=1e30), q)
    assert (np.abs(L - Llin).reshape(7, -1).max(1) / _scale(p, Llin, q)).max() <= 1e-13
    # and it is not the nonlinear scheme
    Lw = O.rhs(p, q)
    assert (np.abs(L - Lw).reshape(7, -1).max(1) / _scale(p, Lw, q)).max() > 1e-6


@pytest.mark.parametrize("seed", range(5))
def test_linear_reconstruction_is_exact_for_quartics(seed):
    """Cell averages of a quartic over cells [k - 1/2, k + 1/2] (k = -2..2):
    the face values at +-1/2 are the polynomial's values there, exactly."""
    c = np.random.default_rng(seed).normal(size=5)
    P = np.polynomial.Polynomial(c)
    I_ = P.integ()
    v = np.array([I_(k + 0.5) - I_(k - 0.5) for k in range(-2, 3)])
    vm, vp = O.linear5_cell(v)
    assert abs(vm - P(0.5)) <= 1e-13 * max(1.0, np.abs(c).sum())
    assert abs(vp - P(-0.5)) <= 1e-13 * max(1.0, np.abs(c).sum())


def test_uniform_state_is_flat_everywhere():
    p, w = I.random_periodic(2, [12, 10], seed=1)
    for f in range(w.shape[0]):
        w[f] = w[f].reshape(-1)[0]
    q = O.prim_to_cons(p, w)
    L, dec, info = O.rhs_gated(p, q, _bias(10.0), DELTA)
    assert np.all(dec == 1) and np.all(L == 0.0)
    assert np.all(np.isnan(info[..., 0])) and np.all(np.isnan(info[..., 1]))


@pytest.mark.parametrize("amp,flat", [(0.5, True), (2.0, False)])
def test_round_off_floor_closed_form(amp, flat):
    """One cell (i0) of the second partial density raised by amp * delta *
    rho: the five cells whose stencils contain it have max |s_k - s_2| =
    amp * delta * rho (flat exactly when amp <= 1); every other stencil is
    exactly flat.  With a network that calls every non-flat stencil
    troubled, the decisions follow in closed form."""
    n, i0, rho = 24, 11, 1.2
    p, w, _ = _tube_like(n, lambda i: rho + amp * DELTA * rho * (i == i0) - 1e-3, lambda i: 1e5 + 0 * i)
    q = O.prim_to_cons(p, w)
    L, dec, info = O.rhs_gated(p, q, _bias(10.0), DELTA)
    near = np.abs(np.arange(n) - i0) <= 2
    expect = np.where(near & (not flat), 0, 1)
    assert np.array_equal(dec[0, 0, 0], expect)
    s = w[0, 0, 0] + w[1, 0, 0]
    ratio = info[0, 0, 0, :, 2]
    m = amp * DELTA * rho
    assert np.allclose(ratio[near], m / (DELTA * s[near]), rtol=1e-9)
    assert np.all(ratio[~near] == 0.0)


def test_pressure_step_in_uniform_density_is_troubled_by_its_pressure():
    n, i0 = 24, 12
    p, w, _ = _tube_like(n, lambda i: 1.2 + 0 * i, lambda i: np.where(i < i0, 2e5, 1e5))
    q = O.prim_to_cons(p, w)
    L, dec, info = O.rhs_gated(p, q, _bias(10.0), DELTA)
    i = np.arange(n)
    # stencils i-2..i+2 that straddle the step (cells i0-1 | i0), and the wrap at 0 | n-1
    near = ((i >= i0 - 2) & (i <= i0 + 1)) | (i <= 1) | (i >= n - 2)
    assert np.array_equal(dec[0, 0, 0], np.where(near, 0, 1))
    assert np.all(np.isnan(info[0, 0, 0, :, 0]))            # the density sensor is flat everywhere


@pytest.mark.parametrize("kind,slope,expect", [("orientation", +1, 0), ("orientation", -1, 1),
                                               ("centring", +1, 0), ("centring", -1, 0)])
def test_hand_built_network_on_ramps(kind, slope, expect):
    """On a linear density ramp the normalised stencil is x = (k - 2)/2 times
    the slope's sign: orientation z = (x4 - x0) - 1/2 = 2 sign - 1/2;
    centring z = x0 + x4 + 1/2 = 1/2 for either sign."""
    n = 40
    p = I.make_params(1, [n], [0.0], [1.0], [[0, 0]])
    w = np.zeros((5, 1, 1, n))
    w[0, 0, 0] = 1e-6 * 1000.0
    w[1, 0, 0] = 1.2 + slope * 0.01 * np.arange(n)
    w[3, 0, 0] = 1e5
    w[4, 0, 0] = 1e-6
    q = O.prim_to_cons(p, w)
    _, dec, info = O.rhs_gated(p, q, _hand_net(kind), DELTA)
    inner = slice(2, n - 2)                  # stencils that do not reach the clamped boundary ghosts
    sg = 1.0 if slope > 0 else -1.0
    z = info[0, 0, 0, inner, 0]
    zexp = 2 * sg - 0.5 if kind == "orientation" else 0.5
    assert np.allclose(z, zexp, atol=1e-12)
    assert np.all(dec[0, 0, 0, inner] == expect)


def test_fallback_exactly_where_linear_faces_are_not_admissible():
    p, w = I.air_water_shock_tube(200)
    q = O.prim_to_cons(p, w)
    L, dec, info = O.rhs_gated(p, q, _bias(-10.0), DELTA)
    d, m = dec[0, 0, 0], info[0, 0, 0, :, 4:8]
    admissible = (m[:, 0] > 0) & (m[:, 1] >= 0) & (m[:, 2] >= 0) & (m[:, 3] > 0)
    assert np.any(d == 2) and np.any(d == 1) and not np.any(d == 0)
    assert np.array_equal(d == 1, admissible)
    assert np.any(m[d == 2, 1] < 0) or np.any(m[d == 2, 2] < 0)    # alpha1 leaves [0, 1]
    # cell by cell: where the cell and both neighbours use WENO, the plain
    # RHS; where all three are linear, the linear-weight RHS
    Lw = O.rhs(p, q)
    Ll = O.rhs(dict(p, weno_eps=1e30), q, allow_nonphysical=True)   # linear faces leave [0, 1] at the interface
    sc = _scale(p, Lw, q)
    for i in range(1, 199):
        tri = d[i - 1:i + 2]
        if np.all(tri != 1):
            assert np.array_equal(L[:, 0, 0, i], Lw[:, 0, 0, i])
        elif np.all(tri == 1):
            assert np.all(np.abs(L[:, 0, 0, i] - Ll[:, 0, 0, i]) <= 1e-13 * sc)
