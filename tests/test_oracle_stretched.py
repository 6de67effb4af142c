"""Pins for the oracle on non-uniform (tanh-stretched) grids.

Sec. III-A refines the mesh locally with a hyperbolic tangent; on such a grid
the WENO5 reconstruction (Shu's general form) has cell-dependent candidate
coefficients, smoothness indicators and linear weights, and the flux
divergence and CFL bound use the local cell width.  Each check compares the
oracle with something other than itself: the Jiang-Shu coefficients of the
uniform grid, polynomial exactness, a definition-based derivation through the
primitive function with numpy, the consistency of the linear weights with the
quartic reconstruction, the uniform solver, fifth-order convergence, discrete
conservation and pressure/velocity equilibrium.
"""
import math

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I


def _edges_from_widths(w):
    return np.concatenate([[0.0], np.cumsum(w)])


def _avgs(coef, edges):
    """Exact cell averages of the polynomial coef over consecutive cells."""
    integ = P.polyint(coef)
    return (P.polyval(edges[1:], integ) - P.polyval(edges[:-1], integ)) / np.diff(edges)


def test_table_of_uniform_cells_is_jiang_shu():
    t = O.weno5_table(np.full(5, 0.37))
    np.testing.assert_allclose(t["cp"] * 6, [[2, -7, 11], [-1, 5, 2], [2, 5, -1]], atol=1e-13)
    np.testing.assert_allclose(t["cm"] * 6, [[-1, 5, 2], [2, 5, -1], [11, -7, 2]], atol=1e-13)
    np.testing.assert_allclose(t["dp"], [0.1, 0.6, 0.3], atol=1e-14)
    np.testing.assert_allclose(t["dm"], [0.3, 0.6, 0.1], atol=1e-14)
    # beta_k = B.v^2 + 13/3 C.v^2 = 1/4 (..)^2 + 13/12 (..)^2 of Jiang-Shu
    np.testing.assert_allclose(t["B"] * 2, [[1, -4, 3], [-1, 0, 1], [-3, 4, -1]], atol=1e-13)
    np.testing.assert_allclose(t["C"] * 2, [[1, -2, 1]] * 3, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_candidates_exact_for_quadratics_and_weights_for_quartics(seed):
    """Random widths (ratios up to 3): each stencil's candidate reproduces the
    face values of any quadratic from its cell averages, and the linear-weight
    combination those of any quartic (both faces)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, 5)
    e = _edges_from_widths(w)
    xf_p, xf_m = e[3], e[2]
    t = O.weno5_table(w)
    for _ in range(5):
        c2 = rng.normal(size=3)
        v = _avgs(c2, e)
        for k in range(3):
            assert t["cp"][k] @ v[k:k + 3] == pytest.approx(P.polyval(xf_p, c2), rel=1e-12, abs=1e-12)
            assert t["cm"][k] @ v[k:k + 3] == pytest.approx(P.polyval(xf_m, c2), rel=1e-12, abs=1e-12)
        c4 = rng.normal(size=5)
        v = _avgs(c4, e)
        vm, vp = O.weno5_nu_cell(t, v, eps=1e100)
        assert vm == pytest.approx(P.polyval(xf_p, c4), rel=1e-11, abs=1e-11)
        assert vp == pytest.approx(P.polyval(xf_m, c4), rel=1e-11, abs=1e-11)


def _definition(w, v, eps):
    """Non-uniform WENO5-JS from its definitions with numpy: candidates from
    the derivative of the primitive function interpolated at each stencil's
    edges, beta_k = sum_l h^(2l-1) int_cell (p_k^(l))^2 (exact polynomial
    integrals), linear weights by least squares on all five coefficients of
    the quartic reconstruction (whose residual must vanish)."""
    e = _edges_from_widths(w)
    h = w[2]

    def recon(first, m):
        xe = e[first:first + m + 1]
        V = np.concatenate([[0.0], np.cumsum(v[first:first + m] * w[first:first + m])])
        return np.polyder(np.polyfit(xe, V, m))

    polys = [recon(k, 3) for k in range(3)]
    betas = []
    for pk in polys:
        b = 0.0
        for l in (1, 2):
            dl = np.polyder(pk, l)
            sq = np.polyint(np.polymul(dl, dl))
            b += h ** (2 * l - 1) * (np.polyval(sq, e[3]) - np.polyval(sq, e[2]))
        betas.append(b)

    def coeffs(first, m, xf):
        out = np.zeros(5)
        for j in range(m):
            vv = np.zeros(5)
            vv[first + j] = 1.0
            xe = e[first:first + m + 1]
            V = np.concatenate([[0.0], np.cumsum(vv[first:first + m] * w[first:first + m])])
            out[first + j] = np.polyval(np.polyder(np.polyfit(xe, V, m)), xf)
        return out

    res = []
    for xf in (e[3], e[2]):
        Q = coeffs(0, 5, xf)
        A = np.stack([coeffs(k, 3, xf) for k in range(3)], axis=1)
        d, *_ = np.linalg.lstsq(A, Q, rcond=None)
        assert np.max(np.abs(A @ d - Q)) < 1e-10
        a = d / (eps + np.array(betas)) ** 2
        om = a / a.sum()
        res.append(sum(om[k] * np.polyval(polys[k], xf) for k in range(3)))
    return res, d


def test_matches_definition_bruteforce():
    rng = np.random.default_rng(7)
    for trial in range(120):
        w = rng.uniform(0.6, 1.6, 5) * 10 ** rng.uniform(-3, 0)
        kind = trial % 3
        if kind == 0:
            v = rng.normal(size=5)
        elif kind == 1:
            v = 1.0 + 1e-3 * np.cumsum(rng.normal(size=5))
        else:
            v = np.where(np.arange(5) < rng.integers(1, 5), 1.0, 50.0) * (1 + 0.01 * rng.normal(size=5))
        (vm_ref, vp_ref), _ = _definition(w, v, 1e-6)
        vm, vp = O.weno5_nu_cell(O.weno5_table(w), v, eps=1e-6)
        s = np.max(np.abs(v))
        assert abs(vm - vm_ref) <= 1e-8 * s
        assert abs(vp - vp_ref) <= 1e-8 * s


def _wave(n, edges, amp=0.2):
    """The periodic density wave of inputs.smooth_density_wave, with exact cell
    averages on the given edges."""
    p = I.make_params(1, [n], [0.0], [1.0], I.PERIODIC, gamma=(1.4, 1.4), pi_inf=(0.0, 0.0))
    p["edges"] = [edges, None, None]
    xl, xr = edges[:-1], edges[1:]
    rho = 1.0 + amp * (np.cos(2 * math.pi * xl) - np.cos(2 * math.pi * xr)) / (2 * math.pi * (xr - xl))
    return p, I.assemble(p, 0.5, rho[None, None, :], rho[None, None, :], [1.0], 1.0)


def test_uniform_edges_reproduce_the_uniform_solver():
    """Edges given explicitly but uniform: the RHS equals the uniform scheme's
    to round-off of the flux scale (different but equivalent arithmetic)."""
    n = 40
    p0, w = I.smooth_density_wave(n)
    p1 = dict(p0, edges=[np.linspace(0.0, 1.0, n + 1), None, None])
    q = O.prim_to_cons(p0, w)
    L0, L1 = O.rhs(p0, q), O.rhs(p1, q)
    scale = np.abs(q).reshape(5, -1).max(1) * O.max_wavespeed(p0, q)
    assert np.all(np.abs(L1 - L0).reshape(5, -1).max(1) <= 1e-13 * scale)
    assert O.max_wavespeed(p1, q) == pytest.approx(O.max_wavespeed(p0, q), rel=1e-14)


def test_fifth_order_on_a_stretched_grid():
    """The smooth wave advected once around a periodic tanh-refined grid
    (cells near the centre half as wide), dt ~ dx^(5/3): L1 order >= 4.5."""
    errs = []
    for n in (32, 64, 128):
        e = I.tanh_edges(n, 0.0, 1.0, 0.5, strength=8.0, refine=0.5)
        p, w = _wave(n, e)
        q0 = O.prim_to_cons(p, w)
        c = math.sqrt(1.4 / 0.8) + 1.0
        dt0 = 0.4 * np.diff(e).min() / c * (32.0 / n) ** (2.0 / 3.0)
        nst = int(math.ceil(1.0 / dt0))
        q = q0
        for _ in range(nst):
            q = O.step_dt(p, q, 1.0 / nst)
        dxc = np.diff(e)
        errs.append(np.sum(np.abs((q[0] + q[1]) - (q0[0] + q0[1])).ravel() * dxc))
    orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert orders[-1] >= 4.5, orders


def test_conservation_on_a_stretched_periodic_grid():
    """sum_i dx_i q_i of the conserved fields is kept to round-off."""
    n = 48
    e = I.tanh_edges(n, 0.0, 1.0, 0.4, strength=12.0, refine=0.6)
    p, w = I.random_periodic(1, [n], seed=31)
    p["edges"] = [e, None, None]
    q = O.prim_to_cons(p, w)
    dx = np.diff(e)
    S = O.max_wavespeed(p, q)
    for _ in range(3):
        q1 = O.step_dt(p, q, 0.4 / S)
        for f in range(4):
            scale = np.sum(np.abs(q[f]).ravel() * dx)
            assert abs(np.sum(q1[f].ravel() * dx) - np.sum(q[f].ravel() * dx)) <= 1e-13 * scale, f
        q = q1


def test_equilibrium_on_a_stretched_grid():
    """The water slab translating through air (pressure/velocity equilibrium)
    on a refined grid: p and u stay uniform to the round-off bound of the
    uniform-grid pin."""
    n, steps = 64, 150
    p, _ = I.air_water_slab(1, n, 100.0, 0)
    e = I.tanh_edges(n, 0.0, 1.0, 0.45, strength=10.0, refine=0.6)
    p["edges"] = [e, None, None]
    xc = 0.5 * (e[1:] + e[:-1])
    inside = (xc >= 0.3) & (xc < 0.6)
    a1 = np.where(inside, 1.0 - I.ALPHA_EPS, I.ALPHA_EPS).reshape(1, 1, n)
    w = I.assemble(p, a1, 1000.0, 1.2, [100.0], 1.0e5)
    q, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, steps)
    wf = O.cons_to_prim(p, q)
    Pi_w, G_w = 4.4 * 6e8 / 3.4, 1.0 / 3.4
    tol = steps * 30 * np.finfo(float).eps * Pi_w / (G_w * 1e5)
    assert np.max(np.abs(wf[3] - 1e5)) / 1e5 <= tol
    assert np.max(np.abs(wf[2] - 100.0)) / 100.0 <= tol
    assert np.ptp(wf[4]) > 0.9


def test_stretched_grid_rejects_bad_edges_and_weno3():
    n = 8
    p, w = I.smooth_density_wave(n)
    q = O.prim_to_cons(p, w)
    bad = np.linspace(0.0, 1.0, n + 1)
    bad[4] = bad[3]
    for pp in (dict(p, edges=[bad, None, None]),
               dict(p, edges=[np.linspace(0, 1, n + 1), None, None], weno_order=3)):
        with pytest.raises(Exception):
            O.rhs(pp, q)


def test_wave_speed_uses_the_local_width():
    """S = max_i (|u_i| + c_i)/dx_i with the stiffened-gas mixture sound speed
    (c^2 = gamma (p + pi)/rho for a pure phase): the smallest cells bound dt."""
    n = 32
    e = I.tanh_edges(n, 0.0, 1.0, 0.3, strength=10.0, refine=0.7)
    p, w = I.smooth_density_wave(n)
    p["edges"] = [e, None, None]
    q = O.prim_to_cons(p, w)
    rho = (w[0] + w[1]).ravel()
    c = np.sqrt(1.4 * w[3].ravel() / rho)
    S_ref = np.max((np.abs(w[2].ravel()) + c) / np.diff(e))
    assert O.max_wavespeed(p, q) == pytest.approx(S_ref, rel=1e-14)
