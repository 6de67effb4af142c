"""Serial FP64 CPU oracle for the five-equation RHS -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
path (``paper_2409_10729_gb300``) never imports it and fails loudly when its
own CUDA library is missing.

The arithmetic lives in ``mfc5_oracle.c`` (plain C, ``-O2 -ffp-contract=off``),
a step-by-step statement of arXiv 2409.10729 Sec. II (model, stiffened-gas
EOS, finite-volume RHS with WENO5-JS + HLLC) plus the SSP-RK3 / CFL reading,
and in ``mlp_oracle.c`` (FP64 forward/backward/Adam of the troubled-cell
network of the gated-WENO extension).  This module only builds the shared
library and marshals numpy arrays.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, exact Riemann solutions, convergence order, conservation,
equilibrium, symmetry); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "mfc5_oracle.c"), os.path.join(_HERE, "mlp_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle_mfc5.so")
# Test hook: the mutation test points this at a deliberately broken build.
_LIB_OVERRIDE = os.environ.get("MFC5_ORACLE_LIB")

OK, EINVAL, ENOMEM, ENONPHYSICAL = 0, -1, -2, -4


_CMD = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _key() -> str:
    """SHA-256 of the sources, the compile command and the compiler version."""
    import hashlib
    h = hashlib.sha256(" ".join(_CMD).encode())
    for f in _SRCS:
        with open(f, "rb") as fh:
            h.update(fh.read())
    try:
        h.update(subprocess.run(["gcc", "--version"], capture_output=True, text=True).stdout.encode())
    except OSError:
        pass
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction).  The
    build is keyed on a hash of the sources, command and compiler (stored in
    liboracle_mfc5.so.key): a library whose key differs is rebuilt."""
    key = _key()
    try:
        with open(_LIB + ".key") as fh:
            stored = fh.read().strip()
    except OSError:
        stored = ""
    if force or not os.path.exists(_LIB) or stored != key:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run([*_CMD, "-o", tmp, *_SRCS, "-lm"], check=True)
        os.replace(tmp, _LIB)
        with open(_LIB + f".key.tmp{os.getpid()}", "w") as fh:
            fh.write(key + "\n")
        os.replace(_LIB + f".key.tmp{os.getpid()}", _LIB + ".key")
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("gamma", ctypes.c_double * 4),
        ("pi_inf", ctypes.c_double * 4),
        ("weno_eps", ctypes.c_double),
        ("weno_order", ctypes.c_int),
        ("edges", ctypes.POINTER(ctypes.c_double) * 3),
        ("nfluids", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_LIB_OVERRIDE or build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OrcParams)
        lp = ctypes.POINTER(ctypes.c_long)
        sig = {
            "orc_neq": ([pp], ctypes.c_int),
            "orc_prim_to_cons": ([pp, dp, dp], ctypes.c_int),
            "orc_cons_to_prim": ([pp, dp, dp], ctypes.c_int),
            "orc_rhs": ([pp, dp, dp], ctypes.c_int),
            "orc_rhs_points": ([pp, dp, lp, ctypes.c_long, dp], ctypes.c_int),
            "orc_rhs_gated": ([pp, dp, dp, ctypes.c_double, dp, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
            "orc_max_wavespeed": ([pp, dp, dp], ctypes.c_int),
            "orc_step_dt": ([pp, dp, ctypes.c_double], ctypes.c_int),
            "orc_run_cfl": ([pp, dp, ctypes.c_double, ctypes.c_int, dp], ctypes.c_int),
            "orc_weno5_cell": ([ctypes.c_double, dp, dp, dp], None),
            "orc_weno3_cell": ([ctypes.c_double, dp, dp, dp], None),
            "orc_linear5_cell": ([dp, dp, dp], None),
            "orc_weno5_table": ([dp, dp], ctypes.c_int),
            "orc_weno5_nu_cell": ([dp, ctypes.c_double, dp, dp, dp], None),
            "orc_hllc_face": ([pp, ctypes.c_int, dp, dp, dp, dp], ctypes.c_int),
            "orc_sound_speed2": ([pp, dp, dp], ctypes.c_int),
            "orc_weno5_weights": ([ctypes.c_double, dp, dp, dp], None),
            "mlp_nparams": ([], ctypes.c_int),
            "mlp_forward": ([dp, dp, ctypes.c_long, dp], None),
            "mlp_loss_grad": ([dp, dp, dp, ctypes.c_long, ctypes.c_double, dp], ctypes.c_double),
            "mlp_adam": ([dp, dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double], None),
            "mlp_normalise": ([dp, ctypes.c_double, dp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = res
    return _lib


def params(p: dict) -> OrcParams:
    """OrcParams from the plain dict produced by the input generators."""
    s = OrcParams()
    s.ndim = int(p["ndim"])
    for d in range(3):
        s.n[d] = int(p["n"][d])
        s.lo[d] = float(p["lo"][d])
        s.hi[d] = float(p["hi"][d])
        s.bc[d][0] = int(p["bc"][d][0])
        s.bc[d][1] = int(p["bc"][d][1])
    nf = len(p["gamma"])
    if nf < 2 or nf > 4 or len(p["pi_inf"]) != nf:
        raise ValueError("2 to 4 fluids, one gamma and one pi_inf each")
    s.nfluids = nf
    for i in range(nf):
        s.gamma[i] = float(p["gamma"][i])
        s.pi_inf[i] = float(p["pi_inf"][i])
    s.weno_eps = float(p.get("weno_eps", 1e-6))
    s.weno_order = int(p.get("weno_order", 5))
    edges = p.get("edges") or [None, None, None]
    keep = []
    for d in range(3):
        if d < s.ndim and edges[d] is not None:
            e = np.ascontiguousarray(edges[d], dtype=np.float64)
            if e.shape != (s.n[d] + 1,):
                raise ValueError(f"edges[{d}] must hold n[{d}] + 1 values")
            keep.append(e)
            s.edges[d] = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s._keep = keep   # the edge arrays live as long as the struct
    return s


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, what: str, allow_nonphysical: bool = False) -> int:
    if st == OK or (allow_nonphysical and st == ENONPHYSICAL):
        return st
    raise RuntimeError(f"oracle {what} failed with status {st}")


def neq(p: dict) -> int:
    n = lib().orc_neq(ctypes.byref(params(p)))
    if n < 0:
        raise RuntimeError(f"oracle rejected params with status {n}")
    return n


def prim_to_cons(p: dict, w: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.empty_like(w)
    _check(lib().orc_prim_to_cons(ctypes.byref(params(p)), _dptr(w), _dptr(q)), "prim_to_cons")
    return q


def cons_to_prim(p: dict, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    w = np.empty_like(q)
    _check(lib().orc_cons_to_prim(ctypes.byref(params(p)), _dptr(q), _dptr(w)), "cons_to_prim")
    return w


def rhs(p: dict, q: np.ndarray, allow_nonphysical: bool = False) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.empty_like(q)
    _check(lib().orc_rhs(ctypes.byref(params(p)), _dptr(q), _dptr(out)), "rhs", allow_nonphysical)
    return out


GATE_INFO = 8   # z_rho, z_p, flat ratios of both sensors; rho, alpha1, 1 - alpha1, c^2 margins of the linear faces


def rhs_gated(p: dict, q: np.ndarray, theta, delta: float, allow_nonphysical: bool = False):
    """L(q) of the gated form (network parameters theta, round-off floor
    delta): returns (L, decisions [ndim][nz][ny][nx] (0 WENO, 1 linear,
    2 fallback), info [ndim][nz][ny][nx][GATE_INFO])."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.empty_like(q)
    nd = int(p["ndim"])
    dec = np.zeros((nd,) + q.shape[1:], dtype=np.int8)
    info = np.zeros((nd,) + q.shape[1:] + (GATE_INFO,))
    st = lib().orc_rhs_gated(ctypes.byref(params(p)), _dptr(q), _dptr(th), float(delta), _dptr(out),
                             dec.ctypes.data_as(ctypes.c_void_p), info.ctypes.data_as(ctypes.c_void_p))
    _check(st, "rhs_gated", allow_nonphysical)
    return out, dec, info


def rhs_points(p: dict, q: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """L(q) at flat cell indices ``cells``; returns [len(cells), neq]."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    ne = int(p["ndim"]) + 4
    out = np.empty((len(cells), ne), dtype=np.float64)
    st = lib().orc_rhs_points(ctypes.byref(params(p)), _dptr(q),
                              cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                              len(cells), _dptr(out))
    _check(st, "rhs_points")
    return out


def max_wavespeed(p: dict, q: np.ndarray) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    s = ctypes.c_double()
    _check(lib().orc_max_wavespeed(ctypes.byref(params(p)), _dptr(q), ctypes.byref(s)), "wavespeed")
    return s.value


def step_dt(p: dict, q: np.ndarray, dt: float) -> np.ndarray:
    """One RK3 step of size dt; returns a new array."""
    q = np.array(q, dtype=np.float64, copy=True, order="C")
    _check(lib().orc_step_dt(ctypes.byref(params(p)), _dptr(q), float(dt)), "step_dt")
    return q


def run_cfl(p: dict, q: np.ndarray, cfl: float, nsteps: int):
    """nsteps CFL steps; returns (new state, time advanced)."""
    q = np.array(q, dtype=np.float64, copy=True, order="C")
    t = ctypes.c_double()
    _check(lib().orc_run_cfl(ctypes.byref(params(p)), _dptr(q), float(cfl), int(nsteps),
                             ctypes.byref(t)), "run_cfl")
    return q, t.value


def weno5_cell(v5, eps: float = 1e-6):
    v = np.ascontiguousarray(v5, dtype=np.float64)
    vm, vp = ctypes.c_double(), ctypes.c_double()
    lib().orc_weno5_cell(float(eps), _dptr(v), ctypes.byref(vm), ctypes.byref(vp))
    return vm.value, vp.value


def linear5_cell(v5):
    """Linear-weight face values (v_{i+1/2}^-, v_{i-1/2}^+) of the middle cell of v5."""
    v = np.ascontiguousarray(v5, dtype=np.float64)
    vm, vp = ctypes.c_double(), ctypes.c_double()
    lib().orc_linear5_cell(_dptr(v), ctypes.byref(vm), ctypes.byref(vp))
    return vm.value, vp.value


def weno3_cell(v5, eps: float = 1e-6):
    """WENO3-JS face values (v_{i+1/2}^-, v_{i-1/2}^+) of the middle cell of v5
    (only v5[1:4] enter)."""
    v = np.ascontiguousarray(v5, dtype=np.float64)
    vm, vp = ctypes.c_double(), ctypes.c_double()
    lib().orc_weno3_cell(float(eps), _dptr(v), ctypes.byref(vm), ctypes.byref(vp))
    return vm.value, vp.value


NU_TABLE = 42   # doubles per cell of a non-uniform WENO5 table


def weno5_table(widths5):
    """Non-uniform WENO5 table of a cell from the widths of cells i-2..i+2:
    dict with cp, cm (3x3 face-value functionals at i+1/2, i-1/2 per stencil),
    B, C (3x3 functionals of b = h p'(0), c = h^2 p''(0)/2), dp, dm (linear weights)."""
    w = np.ascontiguousarray(widths5, dtype=np.float64)
    T = np.empty(NU_TABLE)
    if lib().orc_weno5_table(_dptr(w), _dptr(T)):
        raise ValueError("degenerate widths")
    return {"raw": T, "cp": T[0:9].reshape(3, 3), "cm": T[9:18].reshape(3, 3), "B": T[18:27].reshape(3, 3),
            "C": T[27:36].reshape(3, 3), "dp": T[36:39], "dm": T[39:42]}


def weno5_nu_cell(table, v5, eps: float = 1e-6):
    """Non-uniform WENO5 face values (v_{i+1/2}^-, v_{i-1/2}^+) from a cell table."""
    T = np.ascontiguousarray(table["raw"], dtype=np.float64)
    v = np.ascontiguousarray(v5, dtype=np.float64)
    vm, vp = ctypes.c_double(), ctypes.c_double()
    lib().orc_weno5_nu_cell(_dptr(T), float(eps), _dptr(v), ctypes.byref(vm), ctypes.byref(vp))
    return vm.value, vp.value


def hllc_face(p: dict, direction: int, wL, wR):
    """HLLC flux between primitive face states; returns (F[neq], u_face, status)."""
    wl = np.ascontiguousarray(wL, dtype=np.float64)
    wr = np.ascontiguousarray(wR, dtype=np.float64)
    F = np.empty_like(wl)
    uf = ctypes.c_double()
    st = lib().orc_hllc_face(ctypes.byref(params(p)), int(direction), _dptr(wl), _dptr(wr),
                             _dptr(F), ctypes.byref(uf))
    return F, uf.value, st


def sound_speed2(p: dict, w) -> float:
    wv = np.ascontiguousarray(w, dtype=np.float64)
    c2 = ctypes.c_double()
    _check(lib().orc_sound_speed2(ctypes.byref(params(p)), _dptr(wv), ctypes.byref(c2)), "c2")
    return c2.value


# ---- troubled-cell network (mlp_oracle.c) ----------------------------------

def mlp_nparams() -> int:
    return lib().mlp_nparams()


def mlp_forward(theta, x) -> np.ndarray:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 5)
    z = np.empty(len(xx))
    lib().mlp_forward(_dptr(th), _dptr(xx), len(xx), _dptr(z))
    return z


def mlp_loss_grad(theta, x, y, pos_weight: float = 1.0):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 5)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    g = np.empty_like(th)
    loss = lib().mlp_loss_grad(_dptr(th), _dptr(xx), _dptr(yy), len(yy), float(pos_weight), _dptr(g))
    return loss, g


def mlp_adam(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns new (theta, m, v)."""
    th = np.array(theta, dtype=np.float64)
    mm = np.array(m, dtype=np.float64)
    vv = np.array(v, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    lib().mlp_adam(_dptr(th), _dptr(gg), _dptr(mm), _dptr(vv), int(t), lr, b1, b2, eps)
    return th, mm, vv


GATE_FLOOR = 1e-4   # the gated form's relative round-off floor (the library's MFC_GATE_FLOOR)


def mlp_normalise(v5, delta: float = GATE_FLOOR) -> np.ndarray:
    """Normalised sensor stencil (v_k - v_2)/max_j |v_j - v_2|; zeros when the
    stencil is flat (variation at most delta |v_2|)."""
    v = np.ascontiguousarray(v5, dtype=np.float64)
    x = np.empty(5)
    lib().mlp_normalise(_dptr(v), float(delta), _dptr(x))
    return x


def is_flat(v5, delta: float = GATE_FLOOR) -> bool:
    v = np.ascontiguousarray(v5, dtype=np.float64)
    x = np.empty(5)
    return lib().mlp_normalise(_dptr(v), float(delta), _dptr(x)) == 0


def weno5_weights(v5, eps: float = 1e-6):
    v = np.ascontiguousarray(v5, dtype=np.float64)
    wm, wp = np.empty(3), np.empty(3)
    lib().orc_weno5_weights(float(eps), _dptr(v), _dptr(wm), _dptr(wp))
    return wm, wp


def troubled(w5, eps: float = 1e-6, tau: float = 0.1, delta: float = GATE_FLOOR) -> bool:
    """Troubled-cell label of one cell from its primitive stencils w5[f][5]:
    some field whose stencil is not flat (variation above delta of its
    centre value) has a nonlinear WENO weight departing from its linear
    weight by more than tau (relative) at either face."""
    dm, dp = np.array([0.1, 0.6, 0.3]), np.array([0.3, 0.6, 0.1])
    for v in np.asarray(w5):
        if is_flat(v, delta):
            continue
        wm, wp = weno5_weights(v, eps)
        if max(np.max(np.abs(wm - dm) / dm), np.max(np.abs(wp - dp) / dp)) > tau:
            return True
    return False
