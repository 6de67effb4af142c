"""ctypes binding of libmfc5 (include/mfc.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Host arrays are numpy float64 C-contiguous arrays; device
arrays are torch CUDA float64 contiguous tensors (torch also supplies the CUDA
stream).  If the library has not been built this module raises on use; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmfc5.so")

MFC_OK, MFC_EINVAL, MFC_ENOMEM, MFC_ECUDA, MFC_ENONPHYSICAL, MFC_ESTATE, MFC_ETOOBIG = 0, -1, -2, -3, -4, -5, -6
MFC_NOALLOC_MAX_DOUBLES = 2 * 1024 * 1024
MFC_GATE_FLOOR = 1e-4
MFC_FP64, MFC_MIXED, MFC_GATED, MFC_FP64_FAST = 0, 1, 2, 3
PRECISIONS = {"fp64": MFC_FP64, "mixed": MFC_MIXED, "gated": MFC_GATED, "fp64_fast": MFC_FP64_FAST}


class MfcParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("gamma", ctypes.c_double * 4),
        ("pi_inf", ctypes.c_double * 4),
        ("weno_eps", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("weno_order", ctypes.c_int),
        ("nfluids", ctypes.c_int),
    ]


class MfcBlock(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("n", ctypes.c_int * 3)]


class MfcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libmfc5.so (raises if it is missing: build it with build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmfc5 is not built ({LIB_PATH} missing); run paper_2409_10729_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        sig = {
            "mfc_create": ([ctypes.POINTER(MfcParams), vp, ctypes.POINTER(vp)], ip),
            "mfc_destroy": ([vp], ip),
            "mfc_set_state": ([vp, vp, ip], ip),
            "mfc_set_state_prim": ([vp, vp, ip], ip),
            "mfc_get_state": ([vp, vp, ip], ip),
            "mfc_rhs": ([vp, vp, ip], ip),
            "mfc_max_wavespeed": ([vp, dp], ip),
            "mfc_step_rk3": ([vp, ctypes.c_double, ip, dp], ip),
            "mfc_step_rk3_dt": ([vp, ctypes.c_double, ip], ip),
            "mfc_launches_per_step": ([vp, ctypes.POINTER(ip)], ip),
            "mfc_set_timing": ([vp, ip], ip),
            "mfc_kernel_time": ([vp, ip, ctypes.POINTER(ctypes.c_char_p), dp,
                                 ctypes.POINTER(ctypes.c_longlong)], ip),
            "mfc_alu_peak": ([ip, dp], ip),
            "mfc_selfcheck_conversions": ([ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)],
                                          ip),
            "mfc_selfcheck_exact_ops": ([ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)],
                                        ip),
            "mfc_rhs_noalloc": ([ctypes.POINTER(MfcParams), vp, vp, vp], ip),
            "mfc_set_mlp_weights": ([vp, ctypes.POINTER(ctypes.c_float), ip], ip),
            "mfc_gate_stats": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong)], ip),
            "mfc_gate_flat": ([vp, ctypes.POINTER(ctypes.c_longlong)], ip),
            "mfc_gate_rhs": ([vp, vp, vp, ip], ip),
            "mfc_set_grid": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ip),
            "mfc_gate_samples": ([vp, vp, vp, ctypes.c_longlong, ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_longlong)], ip),
            "mfc_mlp_nparams": ([], ip),
            "mfc_mlp_loss_grad": ([vp, vp, ctypes.c_longlong, vp, ctypes.c_float, vp, vp, vp], ip),
            "mfc_mlp_adam": ([vp, vp, vp, vp, ip, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              vp], ip),
            "mfc_mlp_forward": ([vp, ctypes.c_longlong, vp, vp, vp], ip),
            "mfc_mlp_forward_tc": ([vp, ctypes.c_longlong, vp, vp, vp], ip),
            "mfc_create_block": ([ctypes.POINTER(MfcParams), ctypes.POINTER(MfcBlock), vp, ctypes.POINTER(vp)], ip),
            "mfc_halo_layout": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ip)], ip),
            "mfc_block_pack": ([vp, ip, vp], ip),
            "mfc_block_begin_step": ([vp, ctypes.c_double], ip),
            "mfc_block_stage": ([vp, ip, vp], ip),
            "mfc_block_wavespeed": ([vp, dp], ip),
            "mfc_block_rhs": ([vp, vp, vp, ip], ip),
            "mfc_strerror": ([ip], ctypes.c_char_p),
            "mfc_last_cuda_error": ([vp], ip),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().mfc_strerror(int(status)).decode()


def alu_peak(fp64: bool) -> float:
    """Measured FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    st = lib().mfc_alu_peak(int(bool(fp64)), ctypes.byref(t))
    if st != MFC_OK:
        raise MfcError(st, "mfc_alu_peak")
    return t.value


def make_params(p: dict, precision="fp64") -> MfcParams:
    s = MfcParams()
    s.ndim = int(p["ndim"])
    for d in range(3):
        s.n[d] = int(p["n"][d])
        s.lo[d] = float(p["lo"][d])
        s.hi[d] = float(p["hi"][d])
        s.bc[d][0] = int(p["bc"][d][0])
        s.bc[d][1] = int(p["bc"][d][1])
    nf = len(p["gamma"])
    s.nfluids = nf
    for i in range(nf):
        s.gamma[i] = float(p["gamma"][i])
        s.pi_inf[i] = float(p["pi_inf"][i])
    s.weno_eps = float(p.get("weno_eps", 1e-6))
    s.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    s.weno_order = int(p.get("weno_order", 5))
    return s


def _ptr(a, ncells_neq: int):
    """(pointer, on_device) for a numpy host array or a torch CUDA tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        if a.size != ncells_neq:
            raise ValueError(f"array has {a.size} elements, expected {ncells_neq}")
        return ctypes.c_void_p(a.ctypes.data), 0
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("device arrays must be contiguous float64 CUDA tensors")
    if a.numel() != ncells_neq:
        raise ValueError(f"tensor has {a.numel()} elements, expected {ncells_neq}")
    return ctypes.c_void_p(a.data_ptr()), 1


class Solver:
    """One mfc_ctx: a problem (params dict as produced by ``inputs``) on the
    current CUDA device, bound to torch's current stream unless given one.
    With ``block`` = (lo, n) the context is one block of the global grid
    ``p`` (mfc_create_block)."""

    def __init__(self, p: dict, precision="fp64", stream=None, block=None):
        import torch
        self.p = p
        self.neq = 2 * len(p["gamma"]) + int(p["ndim"])
        n = list(p["n"]) if block is None else [int(block[1][d]) if d < p["ndim"] else 1 for d in range(3)]
        self.shape = (self.neq, int(n[2]) if p["ndim"] > 2 else 1, int(n[1]) if p["ndim"] > 1 else 1, int(n[0]))
        self.size = int(np.prod(self.shape))
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        handle = ctypes.c_void_p()
        if block is None:
            st = lib().mfc_create(ctypes.byref(make_params(p, precision)), ctypes.c_void_p(stream.cuda_stream),
                                  ctypes.byref(handle))
        else:
            b = MfcBlock()
            for d in range(3):
                b.lo[d] = int(block[0][d]) if d < p["ndim"] else 0
                b.n[d] = int(block[1][d]) if d < p["ndim"] else 1
            st = lib().mfc_create_block(ctypes.byref(make_params(p, precision)), ctypes.byref(b),
                                        ctypes.c_void_p(stream.cuda_stream), ctypes.byref(handle))
        if st != MFC_OK:
            raise MfcError(st, "mfc_create_block" if block is not None else "mfc_create")
        self.ctx = handle
        # non-uniform directions given as cell edges in the params dict
        for d, e in enumerate(p.get("edges") or []):
            if e is not None and d < int(p["ndim"]):
                self.set_grid(d, e)

    def close(self):
        if getattr(self, "ctx", None):
            lib().mfc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str, allow=()):
        if st != MFC_OK and st not in allow:
            raise MfcError(st, what)
        return st

    # -- state -------------------------------------------------------------
    def set_grid(self, direction: int, edges):
        """Non-uniform cell edges (n[direction] + 1, strictly increasing) for one direction."""
        e = np.ascontiguousarray(edges, dtype=np.float64)
        self._check(lib().mfc_set_grid(self.ctx, int(direction), e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "mfc_set_grid")

    def set_state(self, q):
        ptr, dev = _ptr(q, self.size)
        return self._check(lib().mfc_set_state(self.ctx, ptr, dev), "mfc_set_state")

    def set_state_prim(self, w):
        ptr, dev = _ptr(w, self.size)
        return self._check(lib().mfc_set_state_prim(self.ctx, ptr, dev), "mfc_set_state_prim")

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, dev = _ptr(out, self.size)
        self._check(lib().mfc_get_state(self.ctx, ptr, dev), "mfc_get_state")
        return out

    # -- compute -----------------------------------------------------------
    def rhs(self, out=None, allow_nonphysical=False):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, dev = _ptr(out, self.size)
        allow = (MFC_ENONPHYSICAL,) if allow_nonphysical else ()
        self.last_status = self._check(lib().mfc_rhs(self.ctx, ptr, dev), "mfc_rhs", allow)
        return out

    def max_wavespeed(self) -> float:
        s = ctypes.c_double()
        self._check(lib().mfc_max_wavespeed(self.ctx, ctypes.byref(s)), "mfc_max_wavespeed")
        return s.value

    def step_rk3(self, cfl: float, nsteps: int, allow_nonphysical=False) -> float:
        t = ctypes.c_double()
        allow = (MFC_ENONPHYSICAL,) if allow_nonphysical else ()
        self.last_status = self._check(lib().mfc_step_rk3(self.ctx, float(cfl), int(nsteps), ctypes.byref(t)),
                                       "mfc_step_rk3", allow)
        return t.value

    def set_mlp_weights(self, w):
        """Gate weights (1281 floats) of a gated context."""
        arr = np.ascontiguousarray(w, dtype=np.float32)
        return self._check(lib().mfc_set_mlp_weights(self.ctx, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                     arr.size), "mfc_set_mlp_weights")

    def gate_stats(self):
        """(gated, fallback, cells) of the last rhs/step call."""
        g, f, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        self._check(lib().mfc_gate_stats(self.ctx, ctypes.byref(g), ctypes.byref(f), ctypes.byref(c)),
                    "mfc_gate_stats")
        return g.value, f.value, c.value

    def gate_flat(self) -> int:
        """Cell reconstructions of the last rhs/step call whose warp step had
        all-flat stencils (network output taken at zero input)."""
        f = ctypes.c_longlong()
        self._check(lib().mfc_gate_flat(self.ctx, ctypes.byref(f)), "mfc_gate_flat")
        return f.value

    def gate_rhs(self, allow_nonphysical=False):
        """(L(q^n), decisions [ndim][nz][ny][nx] int8: 0 WENO, 1 linear, 2 fallback)."""
        out = np.empty(self.shape, dtype=np.float64)
        dec = np.empty((int(self.p["ndim"]),) + self.shape[1:], dtype=np.int8)
        ptr, dev = _ptr(out, self.size)
        allow = (MFC_ENONPHYSICAL,) if allow_nonphysical else ()
        self.last_status = self._check(lib().mfc_gate_rhs(self.ctx, ptr, ctypes.c_void_p(dec.ctypes.data), dev),
                                       "mfc_gate_rhs", allow)
        return out, dec

    def gate_samples(self, tau: float = 0.1):
        """Labelled samples (X [n,5], Y [n]) of the current state as torch CUDA tensors."""
        import torch
        n = 2 * int(self.p["ndim"]) * int(np.prod(self.shape[1:]))
        X = torch.empty((n, 5), dtype=torch.float32, device="cuda")
        Y = torch.empty(n, dtype=torch.float32, device="cuda")
        cnt = ctypes.c_longlong()
        self._check(lib().mfc_gate_samples(self.ctx, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                           n, float(tau), ctypes.byref(cnt)), "mfc_gate_samples")
        return X, Y

    def step_rk3_dt(self, dt: float, nsteps: int):
        return self._check(lib().mfc_step_rk3_dt(self.ctx, float(dt), int(nsteps)), "mfc_step_rk3_dt")

    # -- block decomposition -----------------------------------------------
    def halo_layout(self):
        """(offsets of the six sides, -1 where none; total elements; element bytes)."""
        off = (ctypes.c_longlong * 6)()
        tot, el = ctypes.c_longlong(), ctypes.c_int()
        self._check(lib().mfc_halo_layout(self.ctx, off, ctypes.byref(tot), ctypes.byref(el)), "mfc_halo_layout")
        return list(off), tot.value, el.value

    def block_pack(self, stage: int, out):
        """Boundary layers of stage `stage`'s input into the device tensor `out`."""
        return self._check(lib().mfc_block_pack(self.ctx, int(stage), ctypes.c_void_p(out.data_ptr())),
                           "mfc_block_pack")

    def block_begin_step(self, dt: float):
        return self._check(lib().mfc_block_begin_step(self.ctx, float(dt)), "mfc_block_begin_step")

    def block_stage(self, stage: int, halo):
        ptr = ctypes.c_void_p(halo.data_ptr() if halo is not None and halo.numel() else None)
        return self._check(lib().mfc_block_stage(self.ctx, int(stage), ptr), "mfc_block_stage")

    def block_wavespeed(self, allow_nonphysical=False):
        """(S of the block's current state, status)."""
        s = ctypes.c_double()
        allow = (MFC_ENONPHYSICAL,) if allow_nonphysical else ()
        st = self._check(lib().mfc_block_wavespeed(self.ctx, ctypes.byref(s)), "mfc_block_wavespeed", allow)
        return s.value, st

    def block_rhs(self, halo, out=None, allow_nonphysical=False):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, dev = _ptr(out, self.size)
        hp = ctypes.c_void_p(halo.data_ptr() if halo is not None and halo.numel() else None)
        allow = (MFC_ENONPHYSICAL,) if allow_nonphysical else ()
        self.last_status = self._check(lib().mfc_block_rhs(self.ctx, hp, ptr, dev), "mfc_block_rhs", allow)
        return out

    # -- instrumentation ---------------------------------------------------
    def launches_per_step(self) -> int:
        n = ctypes.c_int()
        self._check(lib().mfc_launches_per_step(self.ctx, ctypes.byref(n)), "mfc_launches_per_step")
        return n.value

    def set_timing(self, enable: bool):
        return self._check(lib().mfc_set_timing(self.ctx, int(bool(enable))), "mfc_set_timing")

    def kernel_times(self) -> dict:
        out = {}
        i = 0
        while True:
            name, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_longlong()
            st = lib().mfc_kernel_time(self.ctx, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt))
            if st != MFC_OK:
                break
            out[name.value.decode()] = (ms.value, cnt.value)
            i += 1
        return out


# ---- training kernels of the gate network (device tensors) ----------------

def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def mlp_loss_grad(X, Y, theta, grad, loss, pos_weight: float = 1.0):
    st = lib().mfc_mlp_loss_grad(_dev(X), _dev(Y), int(Y.numel()), _dev(theta), float(pos_weight), _dev(grad),
                                 _dev(loss), _stream())
    if st != MFC_OK:
        raise MfcError(st, "mfc_mlp_loss_grad")


def mlp_adam(theta, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    st = lib().mfc_mlp_adam(_dev(theta), _dev(grad), _dev(m), _dev(v), int(t), float(lr), float(beta1), float(beta2),
                            float(eps), _stream())
    if st != MFC_OK:
        raise MfcError(st, "mfc_mlp_adam")


def mlp_forward(X, theta, z):
    st = lib().mfc_mlp_forward(_dev(X), int(X.shape[0]), _dev(theta), _dev(z), _stream())
    if st != MFC_OK:
        raise MfcError(st, "mfc_mlp_forward")


def mlp_forward_tc(X, theta, z):
    """Logits with the gated sweep's tensor-core evaluation (fp16 operands)."""
    st = lib().mfc_mlp_forward_tc(_dev(X), int(X.shape[0]), _dev(theta), _dev(z), _stream())
    if st != MFC_OK:
        raise MfcError(st, "mfc_mlp_forward_tc")
