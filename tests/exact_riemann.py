"""Exact solution of the 1-D Riemann problem for two stiffened gases.

Independent of the oracle: used to pin it.  Each side K is a stiffened gas
(gamma_K, pi_K); with pbar = p + pi_K the gas behaves as an ideal gas in pbar,
so the classical exact solver (pressure function, star state, shock and
rarefaction sampling; Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4) applies per side with p replaced by p + pi_K.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


class Side:
    def __init__(self, rho, u, p, gamma, pi):
        self.rho, self.u, self.p, self.g, self.pi = float(rho), float(u), float(p), float(gamma), float(pi)
        self.c = math.sqrt(self.g * (self.p + self.pi) / self.rho)

    def f(self, ps):
        """Velocity change across the wave connecting this side to pressure ps."""
        g, pi = self.g, self.pi
        if ps > self.p:   # shock
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * (self.p + pi)
            return (ps - self.p) * math.sqrt(A / (ps + pi + B))
        ratio = (ps + pi) / (self.p + pi)
        return 2.0 * self.c / (g - 1.0) * (ratio ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(L: Side, R: Side):
    """(p*, u*) of the Riemann problem."""
    def F(ps):
        return L.f(ps) + R.f(ps) + (R.u - L.u)

    lo = max(-L.pi, -R.pi) + 1e-12 * max(1.0, L.p, R.p)
    hi = 10.0 * max(L.p + L.pi, R.p + R.pi) + 1.0
    while F(hi) < 0:
        hi *= 10.0
    ps = brentq(F, lo, hi, xtol=1e-14 * hi, rtol=4 * np.finfo(float).eps, maxiter=500)
    us = 0.5 * (L.u + R.u) + 0.5 * (R.f(ps) - L.f(ps))
    return ps, us


def sample(L: Side, R: Side, xi: np.ndarray):
    """(rho, u, p, is_left_material) at similarity coordinates xi = (x-x0)/t."""
    ps, us = star_state(L, R)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    left_mat = xi < us
    for side, sgn in ((L, -1.0), (R, +1.0)):
        g, pi = side.g, side.pi
        mask = left_mat if sgn < 0 else ~left_mat
        s = xi[mask]
        ratio = (ps + pi) / (side.p + pi)
        if ps > side.p:   # shock
            gm = (g - 1.0) / (g + 1.0)
            rho_s = side.rho * (ratio + gm) / (gm * ratio + 1.0)
            S = side.u + sgn * side.c * math.sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))
            outside = (s < S) if sgn < 0 else (s > S)
            r = np.where(outside, side.rho, rho_s)
            uu = np.where(outside, side.u, us)
            pp = np.where(outside, side.p, ps)
        else:             # rarefaction
            rho_s = side.rho * ratio ** (1.0 / g)
            c_s = side.c * ratio ** ((g - 1.0) / (2.0 * g))
            head = side.u + sgn * side.c
            tail = us + sgn * c_s
            outside = (s < head) if sgn < 0 else (s > head)
            inside_star = (s > tail) if sgn < 0 else (s < tail)
            # inside the fan
            k = 2.0 / (g + 1.0) - sgn * (g - 1.0) / ((g + 1.0) * side.c) * (side.u - s)
            k = np.maximum(k, 0.0)
            r_fan = side.rho * k ** (2.0 / (g - 1.0))
            u_fan = 2.0 / (g + 1.0) * (-sgn * side.c + (g - 1.0) / 2.0 * side.u + s)
            p_fan = (side.p + pi) * k ** (2.0 * g / (g - 1.0)) - pi
            r = np.where(outside, side.rho, np.where(inside_star, rho_s, r_fan))
            uu = np.where(outside, side.u, np.where(inside_star, us, u_fan))
            pp = np.where(outside, side.p, np.where(inside_star, ps, p_fan))
        rho[mask] = r
        u[mask] = uu
        p[mask] = pp
    return rho, u, p, left_mat


def effective_gas(alpha1, g1, pi1, g2, pi2):
    """Single stiffened gas equivalent to the mixture at fixed alpha1: with
    Gamma = sum alpha_i/(gamma_i-1) and Pi = sum alpha_i gamma_i pi_i/(gamma_i-1),
    gamma = 1 + 1/Gamma and pi = Pi/(Gamma+1)."""
    a2 = 1.0 - alpha1
    G = alpha1 / (g1 - 1.0) + a2 / (g2 - 1.0)
    Pi = alpha1 * g1 * pi1 / (g1 - 1.0) + a2 * g2 * pi2 / (g2 - 1.0)
    return 1.0 + 1.0 / G, Pi / (G + 1.0)


def cell_average(L: Side, R: Side, x0: float, t: float, edges: np.ndarray, sub: int = 64):
    """Cell averages of (rho, u, p) over cells with the given edges, by
    midpoint sub-sampling (sub points per cell)."""
    n = len(edges) - 1
    h = np.diff(edges)
    offs = (np.arange(sub) + 0.5) / sub
    xs = (edges[:-1, None] + h[:, None] * offs[None, :]).ravel()
    r, u, p, _ = sample(L, R, (xs - x0) / t)
    return (r.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1))
