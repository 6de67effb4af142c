"""Pins for the oracle's building blocks (EOS, WENO5-JS, HLLC, RHS assembly).

Every check compares the oracle against something other than itself: a closed
form, the defining integral of a quantity, an independent re-derivation, a
symmetry, or a special case with a known answer (Sec. II of arXiv 2409.10729
for the model; Jiang-Shu for WENO5; Toro for HLLC).
"""
import math

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

EPS = np.finfo(float).eps


def _p1(**kw):
    return I.make_params(1, [8], [0.0], [1.0], I.TRANSMISSIVE, **kw)


def _p3(**kw):
    return I.make_params(3, [4, 4, 4], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE, **kw)


# ---------------------------------------------------------------- EOS ------

def test_eos_single_fluid_limit():
    """alpha1 = 1: the mixture is the stiffened gas of Sec. II-A,
    rho E = p/(gamma-1) + gamma pi/(gamma-1) + rho u^2/2, c^2 = gamma (p+pi)/rho."""
    p = _p1()
    g, pi = I.WATER
    rho, u, pres = 998.0, 3.5, 2.0e7
    w = np.array([rho, 0.0, u, pres, 1.0]).reshape(5, 1, 1, 1)
    pp = dict(p, n=[1, 1, 1])
    q = O.prim_to_cons(pp, w).ravel()
    E_ref = pres / (g - 1.0) + g * pi / (g - 1.0) + 0.5 * rho * u * u
    assert q[3] == pytest.approx(E_ref, rel=4 * EPS)
    assert q[2] == pytest.approx(rho * u, rel=EPS)
    c2 = O.sound_speed2(pp, w.ravel())
    assert c2 == pytest.approx(g * (pres + pi) / rho, rel=8 * EPS)


@pytest.mark.parametrize("pi2", [0.0, 3.0e7])
def test_eos_mixture_is_linear_in_alpha(pi2):
    """Gamma and Pi are the alpha-weighted sums of 1/(gamma_i-1) and
    gamma_i pi_i/(gamma_i-1): the internal energy at alpha1 = a is the
    a-weighted combination of the two pure-phase internal energies at the same p."""
    pp = dict(_p1(gamma=(4.4, 2.1), pi_inf=(6e8, pi2)), n=[1, 1, 1])
    pres = 3.0e6
    e = {}
    for a in (0.0, 1.0, 0.3):
        w = np.array([a * 1000.0, (1 - a) * 1.2, 0.0, pres, a]).reshape(5, 1, 1, 1)
        e[a] = O.prim_to_cons(pp, w).ravel()[3]
    assert e[0.3] == pytest.approx(0.3 * e[1.0] + 0.7 * e[0.0], rel=1e-14)
    # the pure-phase end points are each fluid's own stiffened-gas relation
    for a, (g, pi) in ((1.0, (4.4, 6e8)), (0.0, (2.1, pi2))):
        assert e[a] == pytest.approx(pres / (g - 1) + g * pi / (g - 1), rel=1e-14)


def test_eos_roundtrip_random():
    """prim -> cons -> prim recovers the state; the pressure error is bounded
    by the cancellation in p = (rho E - rho u^2/2 - Pi)/Gamma."""
    rng = np.random.default_rng(1)
    p = I.make_params(3, [17, 5, 3], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE)
    shp = I.shape_of(p)
    a1 = rng.uniform(0, 1, shp[1:])
    w = I.assemble(p, a1, rng.uniform(900, 1100, shp[1:]), rng.uniform(0.5, 5, shp[1:]),
                   [rng.uniform(-300, 300, shp[1:]) for _ in range(3)],
                   rng.uniform(1e4, 1e9, shp[1:]))
    q = O.prim_to_cons(p, w)
    w2 = O.cons_to_prim(p, q)
    for f in (0, 1, 6):
        np.testing.assert_array_equal(w2[f], w[f])
    rho = w[0] + w[1]
    for k in range(3):
        np.testing.assert_allclose(w2[2 + k], w[2 + k], rtol=4 * EPS, atol=4 * EPS * 300)
    G = a1 / (4.4 - 1) + (1 - a1) / (1.4 - 1)
    Pi = a1 * 4.4 * 6e8 / 3.4
    bound = 16 * EPS * (np.abs(q[5]) + Pi + 0.5 * rho * (w[2] ** 2 + w[3] ** 2 + w[4] ** 2)) / G
    assert np.all(np.abs(w2[5] - w[5]) <= bound)


# ---------------------------------------------------------------- WENO -----

def _cell_avgs(coef, h, centers):
    """Exact cell averages of the polynomial with coefficients coef."""
    integ = P.polyint(coef)
    return (P.polyval(centers + h / 2, integ) - P.polyval(centers - h / 2, integ)) / h


def test_weno_linear_weights_exact_for_quartics():
    """With a huge epsilon the weights are the linear ones and the
    reconstruction is the fifth-order upwind one: exact for cell averages of
    any polynomial of degree <= 4 (both faces)."""
    rng = np.random.default_rng(2)
    h = 0.1
    xc = np.arange(-2, 3) * h
    for _ in range(20):
        coef = rng.normal(size=5)
        v = _cell_avgs(coef, h, xc)
        vm, vp = O.weno5_cell(v, eps=1e100)
        assert vm == pytest.approx(P.polyval(h / 2, coef), rel=1e-12, abs=1e-12)
        assert vp == pytest.approx(P.polyval(-h / 2, coef), rel=1e-12, abs=1e-12)


def _weno_independent(v, eps):
    """WENO5-JS from its definitions: candidate values from the interpolating
    polynomial of the primitive function on each 3-cell stencil, smoothness
    indicators from the integral sum_{l=1,2} h^(2l-1) int_cell (p_k^(l))^2,
    weights a_k = d_k/(eps+beta_k)^2 normalised (Jiang & Shu 1996)."""
    h = 1.0
    edges = np.arange(-2.5, 3.0, 1.0)   # cell i spans [-1/2, 1/2]

    def stencil_poly(cells):
        # primitive function V(x) = int_{x_left}^x v; interpolate at the 4 edges
        xe = edges[cells[0]:cells[0] + 4]
        V = np.concatenate([[0.0], np.cumsum(v[cells[0]:cells[0] + 3]) * h])
        cV = np.polyfit(xe, V, 3)
        return np.polyder(cV)            # reconstruction polynomial (numpy order)

    polys = [stencil_poly([k, k + 1, k + 2]) for k in range(3)]
    betas = []
    for pk in polys:
        b = 0.0
        for l in (1, 2):
            dl = np.polyder(pk, l)
            sq = np.polyint(np.polymul(dl, dl))
            b += h ** (2 * l - 1) * (np.polyval(sq, 0.5) - np.polyval(sq, -0.5))
        betas.append(b)
    out = []
    for d, xf in (((0.1, 0.6, 0.3), 0.5), ((0.3, 0.6, 0.1), -0.5)):
        a = np.array([d[k] / (eps + betas[k]) ** 2 for k in range(3)])
        wts = a / a.sum()
        out.append(sum(wts[k] * np.polyval(polys[k], xf) for k in range(3)))
    return out, betas


def test_weno_matches_definition_bruteforce():
    """Random 5-tuples (smooth, rough, with jumps): the oracle equals the
    definition-based WENO5-JS built from polynomial fits and integrals."""
    rng = np.random.default_rng(3)
    for trial in range(300):
        kind = trial % 3
        if kind == 0:
            v = rng.normal(size=5)
        elif kind == 1:
            v = 1.0 + 1e-3 * np.cumsum(rng.normal(size=5))
        else:
            v = np.where(np.arange(5) < rng.integers(1, 5), 1.0, 1e3) * (1 + 0.01 * rng.normal(size=5))
        (vm_ref, vp_ref), _ = _weno_independent(v, 1e-6)
        vm, vp = O.weno5_cell(v, eps=1e-6)
        scale = np.max(np.abs(v))
        assert abs(vm - vm_ref) <= 1e-10 * scale
        assert abs(vp - vp_ref) <= 1e-10 * scale


def test_weno_mirror_symmetry():
    """Reversing the stencil swaps the roles of the two faces."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        v = rng.normal(size=5) * 10 ** rng.uniform(-3, 3)
        vm, vp = O.weno5_cell(v)
        vm_r, vp_r = O.weno5_cell(v[::-1].copy())
        s = np.max(np.abs(v))
        assert vp_r == pytest.approx(vm, abs=8 * EPS * s)
        assert vm_r == pytest.approx(vp, abs=8 * EPS * s)


def test_weno_eno_property_at_jump():
    """A jump just downstream of the cell: the face value comes from the smooth
    stencil only (non-oscillatory), up to the epsilon-sized leakage."""
    v = np.array([1.0, 1.0, 1.0, 5.0, 5.0])
    vm, vp = O.weno5_cell(v)
    assert vm == pytest.approx(1.0, abs=1e-10)
    assert vp == pytest.approx(1.0, abs=1e-10)


def test_weno_fifth_order_on_smooth_data():
    """With epsilon 1e-6 on smooth data, halving h divides the face error by ~32."""
    errs = []
    for h in (0.05, 0.025, 0.0125):
        xc = np.arange(-2, 3) * h + 0.3
        v = (np.cos(xc + h / 2) - np.cos(xc - h / 2)) / h * -1.0   # averages of sin
        vm, _ = O.weno5_cell(v)
        errs.append(abs(vm - math.sin(0.3 + h / 2)))
    order = math.log2(errs[1] / errs[2])
    assert order > 4.5


# ---------------------------------------------------------------- WENO3 ----

def test_weno3_linear_weights_exact_for_quadratics():
    """With a huge epsilon the WENO3 weights are the linear ones (1/3, 2/3) and
    the reconstruction is the third-order upwind one: exact for cell averages
    of any polynomial of degree <= 2 (both faces); a cubic is not reproduced."""
    rng = np.random.default_rng(12)
    h = 0.1
    xc = np.arange(-2, 3) * h
    for _ in range(20):
        coef = rng.normal(size=3)
        v = _cell_avgs(coef, h, xc)
        vm, vp = O.weno3_cell(v, eps=1e100)
        assert vm == pytest.approx(P.polyval(h / 2, coef), rel=1e-12, abs=1e-12)
        assert vp == pytest.approx(P.polyval(-h / 2, coef), rel=1e-12, abs=1e-12)
    v = _cell_avgs([0.0, 0.0, 0.0, 1.0], 1.0, np.arange(-2, 3) * 1.0)
    vm, _ = O.weno3_cell(v, eps=1e100)
    assert abs(vm - 0.125) > 1e-3


def _weno3_independent(v, eps):
    """WENO3-JS from its definitions (Jiang & Shu 1996, r = 2): candidate
    values from the interpolating polynomial of the primitive function on
    each two-cell stencil, smoothness indicator h int_cell (p_k')^2, weights
    a_k = d_k/(eps+beta_k)^2 normalised, d = (1/3, 2/3) at i+1/2 and mirrored."""
    h = 1.0
    edges = np.arange(-2.5, 3.0, 1.0)

    def stencil_poly(first):
        xe = edges[first:first + 3]
        V = np.concatenate([[0.0], np.cumsum(v[first:first + 2]) * h])
        return np.polyder(np.polyfit(xe, V, 2))

    polys = [stencil_poly(1), stencil_poly(2)]      # {i-1, i}, {i, i+1}
    betas = []
    for pk in polys:
        d1 = np.polyder(pk, 1)
        sq = np.polyint(np.polymul(d1, d1))
        betas.append(h * (np.polyval(sq, 0.5) - np.polyval(sq, -0.5)))
    out = []
    for d, xf in (((1 / 3, 2 / 3), 0.5), ((2 / 3, 1 / 3), -0.5)):
        a = np.array([d[k] / (eps + betas[k]) ** 2 for k in range(2)])
        wts = a / a.sum()
        out.append(sum(wts[k] * np.polyval(polys[k], xf) for k in range(2)))
    return out


def test_weno3_matches_definition_bruteforce():
    """Random stencils (smooth, rough, with jumps): the oracle's WENO3 equals
    the definition-based one; cells i-2 and i+2 do not enter."""
    rng = np.random.default_rng(13)
    for trial in range(300):
        kind = trial % 3
        if kind == 0:
            v = rng.normal(size=5)
        elif kind == 1:
            v = 1.0 + 1e-3 * np.cumsum(rng.normal(size=5))
        else:
            v = np.where(np.arange(5) < rng.integers(1, 5), 1.0, 1e3) * (1 + 0.01 * rng.normal(size=5))
        vm_ref, vp_ref = _weno3_independent(v, 1e-6)
        vm, vp = O.weno3_cell(v, eps=1e-6)
        scale = np.max(np.abs(v))
        assert abs(vm - vm_ref) <= 1e-10 * scale
        assert abs(vp - vp_ref) <= 1e-10 * scale
        w = v.copy()
        w[0], w[4] = rng.normal(size=2) * 1e6
        assert O.weno3_cell(w, eps=1e-6) == (vm, vp)


def test_weno3_mirror_symmetry():
    """Reversing the stencil swaps the roles of the two faces."""
    rng = np.random.default_rng(14)
    for _ in range(100):
        v = rng.normal(size=5) * 10 ** rng.uniform(-3, 3)
        vm, vp = O.weno3_cell(v)
        vm_r, vp_r = O.weno3_cell(v[::-1].copy())
        s = np.max(np.abs(v))
        assert vp_r == pytest.approx(vm, abs=8 * EPS * s)
        assert vm_r == pytest.approx(vp, abs=8 * EPS * s)


def test_weno3_eno_property_at_jump():
    """A jump between cells i and i+1: both face values of cell i come from the
    smooth stencil {i-1, i}; a jump between i-1 and i: from {i, i+1}.  The
    leakage of the rough stencil is (beta_smooth/beta_rough)^2 relative."""
    vm, vp = O.weno3_cell(np.array([7.0, 1.0, 1.0, 5.0, -3.0]))
    assert vm == pytest.approx(1.0, abs=1e-10)
    assert vp == pytest.approx(1.0, abs=1e-10)
    vm, vp = O.weno3_cell(np.array([7.0, 1000.0, 1.0, 2.0, -3.0]))
    assert vm == pytest.approx(1.5, abs=5e-9)        # (v_i + v_{i+1})/2
    assert vp == pytest.approx(0.5, abs=5e-9)        # (3 v_i - v_{i+1})/2


def test_weno3_third_order_on_smooth_data():
    """Away from critical points, halving h divides the face error by ~8."""
    errs = []
    for h in (0.02, 0.01, 0.005):
        xc = np.arange(-2, 3) * h + 0.3
        v = (np.cos(xc + h / 2) - np.cos(xc - h / 2)) / h * -1.0   # averages of sin
        vm, _ = O.weno3_cell(v)
        errs.append(abs(vm - math.sin(0.3 + h / 2)))
    order = math.log2(errs[1] / errs[2])
    assert 2.5 < order < 3.5


# ---------------------------------------------------------------- HLLC -----

def _flux_ref(w, d, ndim, g, pi):
    """Physical flux of the five-equation model (Sec. II-A) from primitives."""
    a1 = w[3 + ndim]
    rho = w[0] + w[1]
    u = np.array(w[2:2 + ndim])
    pres = w[2 + ndim]
    G = a1 / (g[0] - 1) + (1 - a1) / (g[1] - 1)
    Pi = a1 * g[0] * pi[0] / (g[0] - 1) + (1 - a1) * g[1] * pi[1] / (g[1] - 1)
    E = G * pres + Pi + 0.5 * rho * np.dot(u, u)
    un = u[d]
    F = np.zeros(ndim + 4)
    F[0] = w[0] * un
    F[1] = w[1] * un
    F[2:2 + ndim] = rho * u * un
    F[2 + d] += pres
    F[2 + ndim] = (E + pres) * un
    F[3 + ndim] = a1 * un
    return F


def _rand_prim(rng, ndim):
    a1 = rng.uniform(0, 1)
    return np.array([a1 * rng.uniform(900, 1100), (1 - a1) * rng.uniform(0.5, 5)]
                    + list(rng.uniform(-200, 200, ndim)) + [rng.uniform(1e5, 1e8), a1])


def test_hllc_consistency():
    """F(w, w) is the physical flux, in every direction."""
    rng = np.random.default_rng(5)
    p = _p3()
    for _ in range(50):
        w = _rand_prim(rng, 3)
        for d in range(3):
            F, uf, st = O.hllc_face(p, d, w, w)
            assert st == 0
            Fr = _flux_ref(w, d, 3, p["gamma"], p["pi_inf"])
            np.testing.assert_allclose(F, Fr, rtol=1e-12, atol=1e-12 * np.max(np.abs(Fr)))
            assert uf == pytest.approx(w[2 + d], rel=1e-12, abs=1e-9)


def test_hllc_mirror_symmetry():
    """Reflecting x -> -x (swap sides, flip the normal velocity) flips the sign
    of every flux except the normal-momentum one, and flips u_face."""
    rng = np.random.default_rng(6)
    p = _p3()
    for _ in range(50):
        wL, wR = _rand_prim(rng, 3), _rand_prim(rng, 3)
        for d in range(3):
            F, uf, _ = O.hllc_face(p, d, wL, wR)
            mL, mR = wR.copy(), wL.copy()
            mL[2 + d] *= -1
            mR[2 + d] *= -1
            Fm, ufm, _ = O.hllc_face(p, d, mL, mR)
            sign = -np.ones(7)
            sign[2 + d] = 1.0
            np.testing.assert_allclose(Fm, sign * F, rtol=1e-10, atol=1e-10 * np.max(np.abs(F)))
            assert ufm == pytest.approx(-uf, rel=1e-10, abs=1e-8)


def test_hllc_upwind_side_identities():
    """In every region of the HLLC fan the selected side K (K = L exactly when
    the face velocity u_f >= 0) satisfies: alpha1 flux = alpha1_K u_f, and
    tangential momentum flux = v_K times the total mass flux (the tangential
    velocity jumps only across the contact)."""
    rng = np.random.default_rng(8)
    p = _p3(gamma=(4.4, 2.1), pi_inf=(6e8, 3e7))
    for _ in range(200):
        wL, wR = _rand_prim(rng, 3), _rand_prim(rng, 3)
        wL[2] += rng.uniform(-2000, 2000)
        wR[2] += rng.uniform(-2000, 2000)
        for d in range(3):
            F, uf, st = O.hllc_face(p, d, wL, wR)
            assert st == 0
            K = wL if uf >= 0 else wR
            assert F[6] == pytest.approx(K[6] * uf, rel=1e-14, abs=1e-300)
            mass = F[0] + F[1]
            for t in range(3):
                if t != d:
                    assert F[2 + t] == pytest.approx(K[2 + t] * mass, rel=1e-9,
                                                     abs=1e-9 * abs(K[2 + t] * mass) + 1e-9)


def test_hllc_isolated_contact():
    """Equal pressure and normal velocity across a material interface: S* = u,
    and the flux is the upwind side's advective flux plus p."""
    p = _p3()
    for u in (37.0, -12.5, 0.0):
        wL = np.array([999.0, 0.0012, u, 4.0, -2.0, 2.5e5, 1 - 1e-6])
        wR = np.array([1e-3, 1.19, u, 7.0, 1.0, 2.5e5, 1e-6])
        F, uf, st = O.hllc_face(p, 0, wL, wR)
        assert st == 0
        assert uf == pytest.approx(u, abs=1e-9)
        up = wL if u >= 0 else wR
        Fr = _flux_ref(up, 0, 3, p["gamma"], p["pi_inf"])
        np.testing.assert_allclose(F, Fr, rtol=1e-9, atol=1e-6)


def test_hllc_supersonic_upwind():
    """All waves moving right: the flux is F(w_L) exactly; all left: F(w_R)."""
    p = I.make_params(1, [4], [0.0], [1.0], I.TRANSMISSIVE, gamma=(1.4, 1.4), pi_inf=(0.0, 0.0))
    wL = np.array([1.0, 0.0, 5.0, 1.0, 1.0])
    wR = np.array([0.5, 0.0, 6.0, 0.8, 1.0])
    F, uf, _ = O.hllc_face(p, 0, wL, wR)
    np.testing.assert_allclose(F, _flux_ref(wL, 0, 1, p["gamma"], p["pi_inf"]), rtol=1e-14)
    assert uf == 5.0
    wL = np.array([1.0, 0.0, -5.0, 1.0, 1.0])
    wR = np.array([0.5, 0.0, -6.0, 0.8, 1.0])
    F, uf, _ = O.hllc_face(p, 0, wL, wR)
    np.testing.assert_allclose(F, _flux_ref(wR, 0, 1, p["gamma"], p["pi_inf"]), rtol=1e-14)
    assert uf == -6.0


def test_hllc_flags_nonphysical():
    p = _p3()
    w = _rand_prim(np.random.default_rng(7), 3)
    bad = w.copy()
    bad[0] = -1.0
    bad[1] = 0.0
    _, _, st = O.hllc_face(p, 0, w, bad)
    assert st == O.ENONPHYSICAL


# ---------------------------------------------------------------- RHS ------

def test_rhs_uniform_state_is_zero():
    p, w = I.random_periodic(3, 6, seed=0)
    w[:] = w[:, :1, :1, :1]
    q = O.prim_to_cons(p, w)
    assert np.all(O.rhs(p, q) == 0.0)


def test_rhs_points_equal_full_rhs():
    """The per-cell evaluation reproduces the full RHS bit for bit."""
    for ndim, n, bc in ((1, 19, 0), (2, 11, 1), (3, 7, 0), (3, 6, 1)):
        p, w = I.random_periodic(ndim, n, seed=ndim)
        p["bc"] = [[bc, bc]] * ndim + [[0, 0]] * (3 - ndim)
        q = O.prim_to_cons(p, w)
        L = O.rhs(p, q).reshape(ndim + 4, -1)
        cells = np.arange(L.shape[1])
        Lp = O.rhs_points(p, q, cells)
        np.testing.assert_array_equal(Lp.T, L)


@pytest.mark.parametrize("axis", [1, 2])
def test_rhs_direction_permutation(axis):
    """A 1-D problem laid along x, y or z gives the same RHS bit for bit."""
    p1, w1 = I.air_water_shock_tube(40)
    px, wx = I.embed_1d(p1, w1, 0)
    pa, wa = I.embed_1d(p1, w1, axis)
    Lx = O.rhs(px, O.prim_to_cons(px, wx))
    La = O.rhs(pa, O.prim_to_cons(pa, wa))
    ex = Lx[[0, 1, 2, 5, 6]][:, 0, 0, :]
    line = [slice(0, 1)] * 3
    line[2 - axis] = slice(None)
    ea = La[[0, 1, 2 + axis, 5, 6]][(slice(None),) + tuple(line)].reshape(5, -1)
    np.testing.assert_array_equal(ea, ex)
    others = [k for k in (2, 3, 4) if k != 2 + axis]
    assert np.all(La[others] == 0.0)


def test_max_wavespeed_closed_form():
    """Uniform state: S = sum_d (|u_d| + c)/dx_d."""
    p, w = I.random_periodic(3, 5, seed=9)
    p["n"] = [5, 4, 3]
    w = np.broadcast_to(w[:, :1, :1, :1], I.shape_of(p)).copy()
    q = O.prim_to_cons(p, w)
    S = O.max_wavespeed(p, q)
    g, pi = p["gamma"], p["pi_inf"]
    v = w[:, 0, 0, 0]
    a1 = v[6]
    G = a1 / (g[0] - 1) + (1 - a1) / (g[1] - 1)
    Pi = a1 * g[0] * pi[0] / (g[0] - 1) + (1 - a1) * g[1] * pi[1] / (g[1] - 1)
    c = math.sqrt(((G + 1) * v[5] + Pi) / (G * (v[0] + v[1])))
    ref = sum((abs(v[2 + d]) + c) * p["n"][d] for d in range(3))
    assert S == pytest.approx(ref, rel=1e-13)


def test_params_rejected():
    p = _p3()
    bad = dict(p, bc=[[0, 1], [0, 0], [0, 0]])
    with pytest.raises(RuntimeError):
        O.neq(bad)
    with pytest.raises(RuntimeError):
        O.neq(dict(p, gamma=[1.0, 1.4]))
