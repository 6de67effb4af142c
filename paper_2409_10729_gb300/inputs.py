"""Seeded synthetic initial conditions for the five-equation solver.

This module is the one piece shared by the CUDA path and the CPU oracle.  It
holds none of the solver's arithmetic: it lays out *primitive* fields
``w[f][z][y][x]`` (x fastest; unused dimensions have size 1) with the slots

    0: alpha1 rho1   1: alpha2 rho2   2..2+d-1: u_k   2+d: p   3+d: alpha1

and a plain ``dict`` of run parameters.  Each side converts ``w`` to the
conservative state with its own equation of state.

Fluid 1 is water (gamma 4.4, pi_inf 6e8 Pa), fluid 2 is air (gamma 1.4,
pi_inf 0), as in the stiffened-gas description of Sec. II-A.  A pure phase
carries the other phase at volume fraction 1e-6.  The 1-D tube has a sharp
interface; the 2-D/3-D material interfaces are diffuse over about one cell
(a tanh profile of the signed distance), as in a diffuse-interface method:
voxelised sharp spheres leave one- and two-cell slivers on which WENO5
overshoots alpha1 beyond [0, 1] and the mixture sound speed goes imaginary.  Shock states are the ideal-gas normal-shock (Rankine-Hugoniot)
relations for air moving into air at rest.
"""
from __future__ import annotations

import math

import numpy as np

WATER = (4.4, 6.0e8)
AIR = (1.4, 0.0)
ALPHA_EPS = 1.0e-6
TRANSMISSIVE, PERIODIC = 0, 1


def make_params(ndim, n, lo, hi, bc, gamma=(WATER[0], AIR[0]), pi_inf=(WATER[1], AIR[1]),
                weno_eps=1e-6) -> dict:
    """Plain parameter dict; n/lo/hi padded to 3 entries, bc to 3 pairs."""
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    if isinstance(bc, int):
        bc = [[bc, bc]] * ndim
    bc = [list(b) for b in bc] + [[TRANSMISSIVE, TRANSMISSIVE]] * (3 - len(bc))
    return {"ndim": int(ndim), "n": [int(v) for v in n], "lo": [float(v) for v in lo],
            "hi": [float(v) for v in hi], "bc": bc, "gamma": [float(g) for g in gamma],
            "pi_inf": [float(p) for p in pi_inf], "weno_eps": float(weno_eps)}


def nfluids_of(p: dict) -> int:
    return len(p["gamma"])


def neq_of(p: dict) -> int:
    """2N + ndim: N partial densities, ndim momenta, energy, N - 1 volume fractions."""
    return 2 * nfluids_of(p) + p["ndim"]


def shape_of(p: dict):
    """Array shape [neq, nz, ny, nx] of a state for params p."""
    n = p["n"]
    return (neq_of(p), n[2], n[1], n[0])


def cell_centres(p: dict):
    """1-D coordinate arrays (x, y, z) of cell centres."""
    out = []
    for d in range(3):
        n = p["n"][d]
        h = (p["hi"][d] - p["lo"][d]) / n
        out.append(p["lo"][d] + (np.arange(n, dtype=np.float64) + 0.5) * h)
    return out


def assemble(p: dict, alpha1, rho1, rho2, vel, pres) -> np.ndarray:
    """Primitive array from broadcastable per-cell fields.

    alpha1: volume fraction of fluid 1; rho1, rho2: phase densities;
    vel: list of ndim velocity components; pres: pressure."""
    shp = shape_of(p)
    w = np.empty(shp, dtype=np.float64)
    d = p["ndim"]
    a1 = np.broadcast_to(alpha1, shp[1:])
    w[0] = a1 * rho1
    w[1] = (1.0 - a1) * rho2
    for k in range(d):
        w[2 + k] = vel[k]
    w[2 + d] = pres
    w[3 + d] = a1
    return w


def assemble_n(p: dict, alphas, rhos, vel, pres) -> np.ndarray:
    """Primitive array of an N-fluid state (N = len(rhos)): alphas holds the
    volume fractions of fluids 1 .. N-1 (fluid N takes the rest), rhos the N
    phase densities, vel the ndim velocity components, pres the pressure."""
    shp = shape_of(p)
    nf = nfluids_of(p)
    assert len(rhos) == nf and len(alphas) == nf - 1
    w = np.empty(shp, dtype=np.float64)
    d = p["ndim"]
    a = [np.broadcast_to(x, shp[1:]) for x in alphas]
    rest = 1.0 - sum(a)
    for i in range(nf):
        w[i] = (a[i] if i < nf - 1 else rest) * rhos[i]
    for k in range(d):
        w[nf + k] = vel[k]
    w[nf + d] = pres
    for i in range(nf - 1):
        w[nf + d + 1 + i] = a[i]
    return w


def diffuse_alpha(dist, width):
    """Volume fraction of fluid 1 across a diffuse interface: an algebraic
    sigmoid H = (1 - x/(1 + x^4)^(1/4))/2 of x = dist/width (dist is the
    signed distance, negative inside fluid 1), bounded to
    [ALPHA_EPS, 1 - ALPHA_EPS].  A width of zero gives the sharp cell-centre
    interface.  Only +, *, / and sqrt are used, which IEEE 754 rounds exactly,
    so the profile is bit-identical on every platform."""
    if width <= 0.0:
        return np.where(dist < 0.0, 1.0 - ALPHA_EPS, ALPHA_EPS)
    x = dist / width
    x2 = x * x
    h = 0.5 * (1.0 - x / np.sqrt(np.sqrt(1.0 + x2 * x2)))
    return ALPHA_EPS + (1.0 - 2.0 * ALPHA_EPS) * h


def unit_vectors(rng, count):
    """`count` directions uniform on the circle, as (cos, sin) pairs, drawn by
    rejection from the unit square (uniform draws, * and sqrt only)."""
    out = []
    while len(out) < count:
        c, s = rng.uniform(-1.0, 1.0, size=2)
        r2 = c * c + s * s
        if 1e-6 < r2 <= 1.0:
            r = math.sqrt(r2)
            out.append((c / r, s / r))
    return np.array(out)


def normal_shock(gamma: float, rho1: float, p1: float, mach: float):
    """Ideal-gas shock of Mach number `mach` moving in +x into gas at rest.

    Returns (rho2, u2, p2, s): post-shock density, velocity, pressure and the
    shock speed s = mach * c1."""
    g = gamma
    m2 = mach * mach
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (m2 - 1.0))
    rho2 = rho1 * (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    s = mach * math.sqrt(g * p1 / rho1)
    u2 = s * (1.0 - rho1 / rho2)
    return rho2, u2, p2, s


# ---------------------------------------------------------------------------
# one-dimensional cases
# ---------------------------------------------------------------------------

def air_water_shock_tube(n: int = 1000):
    """Two-fluid shock tube on [0,1]: water (p 1e9) for x < 0.7, air (rho 50,
    p 1e5) for x >= 0.7, at rest; transmissive ends."""
    p = make_params(1, [n], [0.0], [1.0], TRANSMISSIVE)
    x, _, _ = cell_centres(p)
    water = x < 0.7
    a1 = np.where(water, 1.0 - ALPHA_EPS, ALPHA_EPS)[None, None, :]
    pres = np.where(water, 1.0e9, 1.0e5)[None, None, :]
    return p, assemble(p, a1, 1000.0, 50.0, [0.0], pres)


def sod(n: int):
    """Sod's problem for one ideal gas (gamma 1.4): (rho,u,p) = (1,0,1) for
    x < 0.5 and (0.125,0,0.1) beyond; alpha1 = 1 everywhere."""
    p = make_params(1, [n], [0.0], [1.0], TRANSMISSIVE, gamma=(1.4, 1.4), pi_inf=(0.0, 0.0))
    x, _, _ = cell_centres(p)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)[None, None, :]
    pres = np.where(left, 1.0, 0.1)[None, None, :]
    return p, assemble(p, 1.0, rho, 0.0, [0.0], pres)


def smooth_density_wave(n: int, amp: float = 0.2):
    """Periodic density wave rho = 1 + amp sin(2 pi x) (exact cell averages),
    u = 1, p = 1, two identical ideal gases at alpha1 = 1/2."""
    p = make_params(1, [n], [0.0], [1.0], PERIODIC, gamma=(1.4, 1.4), pi_inf=(0.0, 0.0))
    x, _, _ = cell_centres(p)
    h = 1.0 / n
    rho = 1.0 + amp * np.sin(2.0 * math.pi * x) * (math.sin(math.pi * h) / (math.pi * h))
    rho = rho[None, None, :]
    return p, assemble(p, 0.5, rho, rho, [1.0], 1.0)


def air_shock_1d(n: int, mach: float = 2.0, x_shock: float = 0.25):
    """A single Mach-`mach` shock in air (rho 1.2, p 1e5) at x_shock moving in
    +x; fluid 1 absent (alpha1 = 1e-6)."""
    p = make_params(1, [n], [0.0], [1.0], TRANSMISSIVE)
    x, _, _ = cell_centres(p)
    rho2, u2, p2, _ = normal_shock(AIR[0], 1.2, 1.0e5, mach)
    post = x < x_shock
    rho = np.where(post, rho2, 1.2)[None, None, :]
    u = np.where(post, u2, 0.0)[None, None, :]
    pres = np.where(post, p2, 1.0e5)[None, None, :]
    return p, assemble(p, ALPHA_EPS, 1000.0, rho, [u], pres)


# ---------------------------------------------------------------------------
# multi-dimensional cases
# ---------------------------------------------------------------------------

def air_water_slab(ndim: int, n: int, u0: float = 100.0, axis: int = 0):
    """Periodic box [0,1]^ndim at uniform p = 1e5 and velocity u0 along `axis`
    with a water slab 0.3 <= x_axis < 0.6 (rho 1000) in air (rho 1.2)."""
    p = make_params(ndim, [n] * ndim, [0.0] * ndim, [1.0] * ndim, PERIODIC)
    c = cell_centres(p)
    xa = c[axis]
    inside = (xa >= 0.3) & (xa < 0.6)
    shp = [1, 1, 1]
    shp[2 - axis] = len(xa)
    a1 = np.where(inside, 1.0 - ALPHA_EPS, ALPHA_EPS).reshape(shp)
    vel = [0.0] * ndim
    vel[axis] = u0
    return p, assemble(p, a1, 1000.0, 1.2, vel, 1.0e5)


def random_periodic(ndim: int, n, seed: int = 0):
    """Periodic box with smooth random fields plus a two-fluid interface: a
    few random Fourier modes in density, velocity and pressure, and a water
    blob of radius 0.25 (alpha1 ~ 1, tanh profile about 1.5 cells wide) in
    air.  Used for conservation and parity checks."""
    rng = np.random.default_rng(seed)
    ns = [n] * ndim if np.isscalar(n) else list(n)
    p = make_params(ndim, ns, [0.0] * ndim, [1.0] * ndim, PERIODIC)
    c = cell_centres(p)
    grids = np.meshgrid(*c[:ndim][::-1], indexing="ij")[::-1]   # x, y, z broadcast [nz,ny,nx]
    shp = shape_of(p)[1:]
    grids = [g.reshape(shp) for g in grids]

    def modes(scale):
        f = np.zeros(shp)
        for _ in range(3):
            k = rng.integers(1, 3, size=ndim)
            ph = rng.uniform(0, 2 * math.pi)
            arg = sum(2 * math.pi * k[d] * grids[d] for d in range(ndim)) + ph
            f = f + scale * rng.uniform(0.3, 1.0) * np.sin(arg)
        return f

    r = np.sqrt(sum((grids[d] - 0.5) ** 2 for d in range(ndim)))
    width = 1.5 / min(ns)
    a1 = np.clip(0.5 * (1.0 + np.tanh((0.25 - r) / width)), ALPHA_EPS, 1.0 - ALPHA_EPS)
    rho1 = 1000.0 * (1.0 + 0.01 * modes(1.0))
    rho2 = 1.2 * (1.0 + 0.2 * modes(1.0))
    vel = [20.0 * modes(1.0) for _ in range(ndim)]
    pres = 1.0e7 * (1.0 + 0.2 * modes(1.0))
    return p, assemble(p, a1, rho1, rho2, vel, pres)


def shock_water_column(nx: int = 1024, ny: int = 512, seed: int = 2409, mach: float = 1.47,
                       gap: float = 0.03, smear: float = 1.5):
    """Mach-1.47 shock in air (rho 1.2, p 1e5) approaching a water column of
    radius 0.1 centred at (0.5, 0.5) on [0,2]x[0,1] (transmissive sides).

    The interface radius is r(theta) = 0.1 [1 + 0.01 sum_{k=2..9} a_k
    cos(k theta + phi_k)] with a_k ~ U[-1,1] scaled to sum |a_k| = 1 and
    phi_k uniform on the circle, from `seed`; cos(k theta + phi_k) is formed
    by rotations, without library trigonometry, so the state is bit-identical
    on every platform.  The interface is diffuse over about
    `smear` cells (see diffuse_alpha).  The shock starts `gap` upstream of
    the column's leftmost point so that it reaches the column within the run."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, size=8)
    a = a / np.abs(a).sum()
    phase = unit_vectors(rng, 8)                 # (cos phi_k, sin phi_k)
    p = make_params(2, [nx, ny], [0.0, 0.0], [2.0, 1.0], TRANSMISSIVE)
    x, y, _ = cell_centres(p)
    X = x[None, :]
    Y = y[:, None]
    cx, cy, r0 = 0.5, 0.5, 0.1
    dx, dy = X - cx, Y - cy
    r = np.sqrt(dx * dx + dy * dy)
    rs = np.where(r > 0.0, r, 1.0)
    c1 = np.where(r > 0.0, dx / rs, 1.0)         # cos(theta)
    s1 = np.where(r > 0.0, dy / rs, 0.0)         # sin(theta)
    # cos(k theta), sin(k theta) by repeated rotation, k = 1..9
    ck, sk = c1, s1
    pert = np.zeros_like(r)
    for k in range(2, 10):
        ck, sk = ck * c1 - sk * s1, sk * c1 + ck * s1
        cphi, sphi = phase[k - 2]
        pert = pert + a[k - 2] * (ck * cphi - sk * sphi)   # a_k cos(k theta + phi_k)
    rad = r0 * (1.0 + 0.01 * pert)
    dist = r - rad                                         # signed, > 0 in air
    a1 = diffuse_alpha(dist, smear * (1.0 / ny))
    xs = cx - r0 * 1.01 - gap                              # 1.01 r0 bounds the interface radius
    rho2, u2, p2, _ = normal_shock(AIR[0], 1.2, 1.0e5, mach)
    post = np.broadcast_to(X < xs, a1.shape)
    a1 = a1[None]
    rho_air = np.where(post, rho2, 1.2)[None]
    u = np.where(post, u2, 0.0)[None]
    pres = np.where(post, p2, 1.0e5)[None]
    return p, assemble(p, a1, 1000.0, rho_air, [u, 0.0], pres)


def droplet_layout(seed: int = 2409, count: int = 8, gap: float = 0.01):
    """Non-overlapping droplets: radii U[0.05, 0.1], centres uniform over
    [0.3,0.9] x [0.15,0.85]^2, rejection-sampled so that centre distances
    exceed r_i + r_j + gap.  Returns an array [count, 4] of (cx, cy, cz, r)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        r = rng.uniform(0.05, 0.1)
        c = np.array([rng.uniform(0.3, 0.9), rng.uniform(0.15, 0.85), rng.uniform(0.15, 0.85)])
        if all(np.linalg.norm(c - o[:3]) >= r + o[3] + gap for o in out):
            out.append(np.array([c[0], c[1], c[2], r]))
    return np.stack(out)


def shock_droplets(n: int = 256, seed: int = 2409, mach: float = 2.0, gap: float = 0.01,
                   count: int = 8, smear: float = 1.5):
    """Mach-2 shock in air (rho 1.2, p 1e5) over `count` water droplets on
    [0,1]^3 (transmissive sides).  Droplets from `droplet_layout(seed)`, with
    interfaces diffuse over about `smear` cells; the shock starts `gap`
    upstream of the leftmost droplet surface."""
    drops = droplet_layout(seed, count)
    p = make_params(3, [n, n, n], [0.0] * 3, [1.0] * 3, TRANSMISSIVE)
    x, y, z = cell_centres(p)
    a1 = np.full((n, n, n), ALPHA_EPS)
    h = 1.0 / n
    for cx, cy, cz, r in drops:
        # only the bounding box of each droplet (plus the profile's tail) is touched
        lo = [max(0, int((c - r) / h) - 8) for c in (cx, cy, cz)]
        hi = [min(n, int((c + r) / h) + 9) for c in (cx, cy, cz)]
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        d2 = (x[None, None, lo[0]:hi[0]] - cx) ** 2 + (y[None, lo[1]:hi[1], None] - cy) ** 2
        d2 = d2 + (z[lo[2]:hi[2], None, None] - cz) ** 2
        a1[sl] = np.maximum(a1[sl], diffuse_alpha(np.sqrt(d2) - r, smear * h))
    xs = float(np.min(drops[:, 0] - drops[:, 3])) - gap
    rho2, u2, p2, _ = normal_shock(AIR[0], 1.2, 1.0e5, mach)
    post = (x < xs)[None, None, :]
    rho_air = np.where(post, rho2, 1.2)
    u = np.where(post, u2, 0.0)
    pres = np.where(post, p2, 1.0e5)
    return p, assemble(p, a1, 1000.0, rho_air, [u, 0.0, 0.0], pres)


OIL = (2.35, 1.0e9)   # a third stiffened gas (a generic liquid) for the N-fluid cases
GLYCOL = (1.8, 2.0e8)


def random_periodic_n(ndim: int, n, nfluids: int = 3, seed: int = 0):
    """N-fluid counterpart of random_periodic: smooth random fields and N - 1
    liquid blobs (water, oil, glycol-like) in air on a periodic box; every
    volume fraction stays within [ALPHA_EPS, 1]."""
    rng = np.random.default_rng(seed)
    ns = [n] * ndim if np.isscalar(n) else list(n)
    fl = [WATER, OIL, GLYCOL][:nfluids - 1] + [AIR]
    p = make_params(ndim, ns, [0.0] * ndim, [1.0] * ndim, PERIODIC, gamma=[f[0] for f in fl],
                    pi_inf=[f[1] for f in fl])
    c = cell_centres(p)
    grids = np.meshgrid(*c[:ndim][::-1], indexing="ij")[::-1]
    shp = shape_of(p)[1:]
    grids = [g.reshape(shp) for g in grids]

    def modes(scale):
        f = np.zeros(shp)
        for _ in range(3):
            k = rng.integers(1, 3, size=ndim)
            ph = rng.uniform(0, 2 * math.pi)
            arg = sum(2 * math.pi * k[d] * grids[d] for d in range(ndim)) + ph
            f = f + scale * rng.uniform(0.3, 1.0) * np.sin(arg)
        return f

    width = 1.5 / min(ns)
    raw = []
    for i in range(nfluids - 1):
        centre = rng.uniform(0.25, 0.75, size=ndim)
        r = np.sqrt(sum((grids[d] - centre[d]) ** 2 for d in range(ndim)))
        raw.append(np.clip(0.5 * (1.0 + np.tanh((0.18 - r) / width)), ALPHA_EPS, 1.0))
    raw.append(np.full(shp, 0.3))          # air everywhere, diluted where liquids are
    tot = sum(raw)
    alphas = [np.maximum(a / tot, ALPHA_EPS) for a in raw[:-1]]
    rhos = [1000.0 * (1.0 + 0.01 * modes(1.0)), 900.0 * (1.0 + 0.01 * modes(1.0)),
            1100.0 * (1.0 + 0.01 * modes(1.0))][:nfluids - 1] + [1.2 * (1.0 + 0.2 * modes(1.0))]
    vel = [20.0 * modes(1.0) for _ in range(ndim)]
    pres = 1.0e7 * (1.0 + 0.2 * modes(1.0))
    return p, assemble_n(p, alphas, rhos, vel, pres)


def shock_droplets_3fluid(n: int = 256, seed: int = 2409, mach: float = 2.0, gap: float = 0.01,
                          count: int = 8, smear: float = 1.5):
    """The shock-droplet array with three fluids: droplets alternate between
    water (fluid 1) and oil (fluid 2), in air (fluid 3)."""
    drops = droplet_layout(seed, count)
    p = make_params(3, [n, n, n], [0.0] * 3, [1.0] * 3, TRANSMISSIVE, gamma=[WATER[0], OIL[0], AIR[0]],
                    pi_inf=[WATER[1], OIL[1], AIR[1]])
    x, y, z = cell_centres(p)
    a = [np.full((n, n, n), ALPHA_EPS), np.full((n, n, n), ALPHA_EPS)]
    h = 1.0 / n
    for k, (cx, cy, cz, r) in enumerate(drops):
        lo = [max(0, int((c - r) / h) - 8) for c in (cx, cy, cz)]
        hi = [min(n, int((c + r) / h) + 9) for c in (cx, cy, cz)]
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        d2 = (x[None, None, lo[0]:hi[0]] - cx) ** 2 + (y[None, lo[1]:hi[1], None] - cy) ** 2
        d2 = d2 + (z[lo[2]:hi[2], None, None] - cz) ** 2
        prof = diffuse_alpha(np.sqrt(d2) - r, smear * h)
        a[k % 2][sl] = np.maximum(a[k % 2][sl], np.minimum(prof, 1.0 - 2 * ALPHA_EPS))
    xs = float(np.min(drops[:, 0] - drops[:, 3])) - gap
    rho2, u2, p2, _ = normal_shock(AIR[0], 1.2, 1.0e5, mach)
    post = (x < xs)[None, None, :]
    rho_air = np.where(post, rho2, 1.2)
    u = np.where(post, u2, 0.0)
    pres = np.where(post, p2, 1.0e5)
    return p, assemble_n(p, a, [1000.0, 900.0, rho_air], [u, 0.0, 0.0], pres)


def embed_1d(p1d: dict, w1d: np.ndarray, axis: int, m: int = 4):
    """Lay a 1-D case along `axis` of a 3-D box with m cells in the other two
    directions (transmissive there).  Velocity goes to component `axis`."""
    n = p1d["n"][0]
    ns = [m, m, m]
    ns[axis] = n
    lo = [0.0] * 3
    hi = [1.0] * 3
    lo[axis] = p1d["lo"][0]
    hi[axis] = p1d["hi"][0]
    bc = [[TRANSMISSIVE, TRANSMISSIVE] for _ in range(3)]
    bc[axis] = list(p1d["bc"][0])
    p = make_params(3, ns, lo, hi, bc, p1d["gamma"], p1d["pi_inf"], p1d["weno_eps"])
    shp = [1, 1, 1]
    shp[2 - axis] = n
    line = {k: w1d[k, 0, 0, :].reshape(shp) for k in range(5)}
    vel = [0.0, 0.0, 0.0]
    vel[axis] = line[2]
    a1 = line[4]
    w = np.empty(shape_of(p))
    w[0] = line[0]
    w[1] = line[1]
    for k in range(3):
        w[2 + k] = vel[k]
    w[5] = line[3]
    w[6] = a1
    return p, w


def tanh_edges(n: int, lo: float, hi: float, centre: float, strength: float = 10.0, refine: float = 0.5):
    """Cell edges of a grid refined around x = centre with a hyperbolic
    tangent (Sec. III-A's local mesh refinement): the width is proportional to
    1 - refine sech^2(strength (xi - xi_c)) in the uniform index coordinate
    xi, so cells near the centre are (1 - refine) times the far cells and the
    transition is smooth.  Integrated in closed form:
        s(xi) = xi - (refine/strength) (tanh(strength (xi - xi_c)) + tanh(strength xi_c)),
    normalised to [lo, hi]; the end edges are exactly lo and hi."""
    xi_c = (centre - lo) / (hi - lo)
    xi = np.arange(n + 1) / n

    def s(x):
        return x - (refine / strength) * (np.tanh(strength * (x - xi_c)) + np.tanh(strength * xi_c))

    e = lo + (hi - lo) * s(xi) / s(1.0)
    e[0], e[-1] = lo, hi
    return e
