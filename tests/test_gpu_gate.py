"""GPU tests of the gated form and of the gate network's own training kernels.

* The FP32 loss/gradient, Adam and forward kernels against the FP64 oracle
  (gradients to 1e-5 relative, Adam to 1e-6, logits to 1e-5).
* Training samples: normalised stencils and WENO-weight labels against the
  oracle's weights, cell by cell.
* The gated sweep: a gate that never fires reproduces the mixed form on a
  state without flat stencils (to FP32 round-off; the same WENO code in
  another kernel); a gate that always fires gives the linear-weight WENO5
  RHS (the oracle with a huge epsilon) on smooth data; on a sharp interface
  the non-physical linear faces fall back to WENO; stencils below the
  round-off floor are smooth without the network.
* The fused network (split-f16 tensor-core operands) against the FP64
  oracle network: logits to 1e-5, decisions equal away from 0.
* Parity of the whole gate: decisions and RHS of the fused gate against the
  oracle's gated RHS on an oracle-advanced 96^3 shock/droplet state.
* Training on the GPU lowers the loss; and the trained network's gain over
  the trivial (floor-only) gate: fraction of reconstructions gated, time,
  and per-field error against the FP64 path (the plain-WENO judge).
"""
import json
import os
import time

import numpy as np
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10729_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def _rand_batch(n, seed):
    rng = np.random.default_rng(seed)
    th = rng.normal(0, 0.4, 1281)
    x = rng.uniform(-1, 1, (n, 5))
    y = (rng.uniform(size=n) < 0.3).astype(float)
    return th, x, y


def test_gradient_matches_oracle():
    import torch
    from paper_2409_10729_gb300 import mfc
    th, x, y = _rand_batch(1000, 1)          # not a multiple of the block's 128 samples
    th32, x32 = th.astype(np.float32), x.astype(np.float32)
    grad = torch.empty(1281, device="cuda")
    loss = torch.empty(1, device="cuda")
    mfc.mlp_loss_grad(_cuda(x32), _cuda(y), _cuda(th32), grad, loss, pos_weight=2.5)
    lo, go = O.mlp_loss_grad(th32.astype(np.float64), x32.astype(np.float64), y, 2.5)
    g = grad.cpu().numpy()
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(g - go)) <= 1e-5 * np.max(np.abs(go))


def test_adam_matches_oracle():
    import torch
    from paper_2409_10729_gb300 import mfc
    rng = np.random.default_rng(2)
    th = rng.normal(0, 0.4, 1281).astype(np.float32)
    g = rng.normal(0, 1e-2, 1281).astype(np.float32)
    m = rng.normal(0, 1e-3, 1281).astype(np.float32)
    v = np.abs(rng.normal(0, 1e-4, 1281)).astype(np.float32)
    T, M, V = _cuda(th), _cuda(m), _cuda(v)
    mfc.mlp_adam(T, _cuda(g), M, V, 5, lr=2e-3)
    # the oracle gets the same (FP32-rounded) hyper-parameters the kernel uses
    f = lambda c: float(np.float32(c))
    to, mo, vo = O.mlp_adam(th.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                            v.astype(np.float64), 5, lr=f(2e-3), b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    # the step to 1e-6 of its size, plus the FP32 rounding of storing theta
    tg = T.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(tg - to) <= 1e-6 * np.abs(th - to) + 2.0 ** -24 * np.abs(th) + 1e-30)
    # first moment: b1 m + (1 - b1) g may cancel; bound relative to its terms
    mg = M.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(mg - mo) <= 1e-6 * np.abs(mo) + 2.0 ** -22 * (0.9 * np.abs(m) + 0.1 * np.abs(g)))
    np.testing.assert_allclose(V.cpu().numpy(), vo, rtol=1e-6, atol=1e-14)


def test_forward_matches_oracle():
    import torch
    from paper_2409_10729_gb300 import mfc
    th, x, _ = _rand_batch(777, 3)
    th32, x32 = th.astype(np.float32), x.astype(np.float32)
    z = torch.empty(777, device="cuda")
    mfc.mlp_forward(_cuda(x32), _cuda(th32), z)
    zo = O.mlp_forward(th32.astype(np.float64), x32.astype(np.float64))
    assert np.max(np.abs(z.cpu().numpy() - zo)) <= 1e-5 * max(1.0, np.max(np.abs(zo)))


def test_samples_match_oracle_labels():
    """Normalised stencils and labels of every cell and direction of a 2-D
    state (diffuse interface + shock) advanced by the oracle, recomputed with
    the oracle's normalisation, weights and round-off floor."""
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_water_column(48, 24)
    q, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 20)
    s = mfc.Solver(p, "fp64")
    s.set_state(q)
    X, Y = s.gate_samples(0.1)
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    W = O.cons_to_prim(p, q)[:, 0]            # [6, ny, nx]
    ny, nx = W.shape[1:]
    checked = flat = 0
    for d in range(2):
        for c in range(nx * ny):
            y0, x0 = divmod(c, nx)
            idx = [min(max((x0 if d == 0 else y0) + k, 0), (nx if d == 0 else ny) - 1) for k in range(-2, 3)]
            st = W[:, y0, idx] if d == 0 else W[:, idx, x0]
            # labels: departures of the non-flat fields; skip labels within
            # round-off of the threshold or of the floor
            dev, near = 0.0, False
            for v in st:
                m = np.max(np.abs(v - v[2]))
                near |= abs(m - mfc.MFC_GATE_FLOOR * abs(v[2])) <= 1e-9 * abs(v[2])
                if O.is_flat(v):
                    continue
                wm, wp = O.weno5_weights(v)
                dev = max(dev, np.max(np.abs(wm - [0.1, 0.6, 0.3]) / [0.1, 0.6, 0.3]),
                          np.max(np.abs(wp - [0.3, 0.6, 0.1]) / [0.3, 0.6, 0.1]))
            k = (d * nx * ny + c) * 2
            for sensor, v in ((0, st[0] + st[1]), (1, st[4])):
                np.testing.assert_allclose(X[k + sensor], O.mlp_normalise(v), atol=2e-6)
                if O.is_flat(v):
                    flat += 1
                    assert Y[k + sensor] == -1.0 and np.all(X[k + sensor] == 0.0)
                elif abs(dev - 0.1) > 1e-6 and not near:
                    assert Y[k + sensor] == float(dev > 0.1)
                    checked += 1
    assert checked + flat > 0.99 * 2 * 2 * nx * ny
    assert 0 < (Y > 0.5).sum() and 0 < (Y == 0).sum() and 0 < flat


def _gated(p, weights):
    from paper_2409_10729_gb300 import mfc
    s = mfc.Solver(p, "gated")
    s.set_mlp_weights(weights)
    return s


def _bias_only(b3):
    w = np.zeros(1281, np.float32)
    w[1280] = b3
    return w


def test_gate_that_never_fires_is_the_mixed_form():
    """A random periodic state has no flat stencil, so a gate whose network
    never fires reconstructs every cell with WENO5-JS: the mixed form."""
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(3, [24, 20, 18], seed=9)
    g = _gated(p, _bias_only(10.0))
    m = mfc.Solver(p, "mixed")
    for s in (g, m):
        s.set_state_prim(w)
        s.step_rk3(0.4, 4)
    # same WENO arithmetic compiled into another kernel: equal to FP32 round-off
    a, b = g.get_state().reshape(7, -1), m.get_state().reshape(7, -1)
    scale = np.abs(b).max(1)
    scale[2:5] = scale[2:5].max()
    assert (np.abs(a - b).max(1) / scale).max() <= 1e-6
    gated, fb, cells = g.gate_stats()
    assert gated == 0 and fb == 0 and cells == 4 * 3 * 3 * 24 * 20 * 18   # steps x stages x directions x cells


def test_gate_that_always_fires_is_linear_weno():
    """On smooth data every cell is reconstructed with the linear weights: the
    RHS equals the oracle's WENO5 with epsilon -> infinity (linear weights),
    to the mixed form's FP32 accuracy."""
    p, w = I.random_periodic(3, [20, 18, 16], seed=5)
    w[6] = 0.5                                     # no interface: smooth everywhere
    w[0] = 0.5 * 1000.0 * (1 + 0.01 * np.sin(np.arange(w[0].size).reshape(w[0].shape) * 0.01))
    g = _gated(p, _bias_only(-10.0))
    g.set_state_prim(w)
    L = g.rhs()
    gated, fb, cells = g.gate_stats()
    assert fb == 0 and gated == cells == 3 * 20 * 18 * 16
    plin = dict(p, weno_eps=1e30)
    q = O.prim_to_cons(p, w)
    Llin = O.rhs(plin, q)
    Lweno = O.rhs(p, q)
    S = O.max_wavespeed(p, q)
    scale = np.maximum(np.abs(Llin).reshape(7, -1).max(1), np.abs(q).reshape(7, -1).max(1) * S)
    err_lin = (np.abs(L - Llin).reshape(7, -1).max(1) / scale).max()
    err_weno = (np.abs(L - Lweno).reshape(7, -1).max(1) / scale).max()
    assert err_lin <= 2e-5
    assert err_weno > 10 * err_lin                 # and it is not the nonlinear WENO


def test_gate_falls_back_to_weno_on_sharp_interface():
    """Linear weights across the sharp water/air interface of the 1-D tube
    overshoot alpha1 out of [0, 1]; those cells are recomputed with WENO."""
    p, w = I.air_water_shock_tube(200)
    g = _gated(p, _bias_only(-10.0))
    g.set_state_prim(w)
    g.step_rk3(0.4, 5)
    gated, fb, cells = g.gate_stats()
    assert fb > 0 and gated + fb == cells
    q = g.get_state()
    assert np.all(np.isfinite(q)) and np.all(q[4] >= -1e-6) and np.all(q[0] + q[1] > 0)


def _oracle_stencils(p, q, limit=None):
    """Normalised density and pressure stencils (oracle normalisation, with
    the round-off floor) of every cell and direction of an oracle state,
    flat ones left out."""
    W = O.cons_to_prim(p, q)[:, 0]
    ny, nx = W.shape[1:]
    out = []
    for d in range(2):
        for y0 in range(ny):
            for x0 in range(nx):
                idx = [min(max((x0 if d == 0 else y0) + k, 0), (nx if d == 0 else ny) - 1) for k in range(-2, 3)]
                st = W[:, y0, idx] if d == 0 else W[:, idx, x0]
                for v in (st[0] + st[1], st[4]):
                    if not O.is_flat(v):
                        out.append(O.mlp_normalise(v))
    return np.array(out)


def test_tensor_core_logits_match_the_fp32_network():
    """The gated sweep's network (every layer on the tensor cores, operands
    split into two f16 halves) against the FP64 oracle network on the same
    FP32 inputs, to FP32 accuracy (1e-5 of the logit scale, the bar of the
    CUDA-core FP32 forward): real solver stencils of an oracle-advanced
    water-column state and random ones, with the trained weights and with
    random weights; ragged sample count.  The decisions (logit < 0) agree
    wherever the oracle logit is more than 1e-4 from 0."""
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_water_column(96, 48)
    q, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 100)
    Xs = _cuda(_oracle_stencils(p, q))
    rng = np.random.default_rng(11)
    Xr = _cuda(rng.uniform(-1, 1, (4099, 5)))
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    thetas = [rng.normal(0, 0.3, 1281).astype(np.float32)]
    if os.path.exists(wpath):
        thetas.append(np.load(wpath))
    for th in thetas:
        T = _cuda(th)
        for X in (Xs, Xr):
            X = X[:X.shape[0] - 3].contiguous()
            z32 = torch.empty(X.shape[0], device="cuda")
            ztc = torch.empty(X.shape[0], device="cuda")
            mfc.mlp_forward(X, T, z32)
            mfc.mlp_forward_tc(X, T, ztc)
            z64 = O.mlp_forward(th.astype(np.float64), X.cpu().numpy().astype(np.float64))
            a, b = ztc.cpu().numpy(), z32.cpu().numpy()
            sc = max(1.0, np.max(np.abs(z64)))
            assert np.max(np.abs(b - z64)) <= 1e-5 * sc
            assert np.max(np.abs(a - z64)) <= 1e-5 * sc
            far = np.abs(z64) > 1e-4
            assert np.array_equal(a[far] < 0, z64[far] < 0)


def test_training_on_gpu_lowers_the_loss():
    from paper_2409_10729_gb300 import train_gate as T
    rng = np.random.default_rng(0)
    X, Y, _ = T.collect([100], 128, 64, 100, 25, 2048, 0.1, rng)
    theta, hist = T.train(X, Y, epochs=24, batch=1024, lr=3e-3, pos_weight=1.0, seed=1)
    assert hist[-1] < 0.7 * hist[0]
    z, y = T.evaluate(theta, X, Y)
    acc = float(((z > 0) == (y > 0.5)).float().mean())
    assert acc > 0.85


def test_trained_gate_gain():
    """What the trained network gains over the trivial gate.  On the 3-D
    shock/droplet case (96^3, 30 steps) four runs: FP64 (plain WENO, equal to
    the oracle bit for bit: the judge), mixed (plain WENO in FP32), the gate
    with the trained network, and the trivial gate -- the same rule with a
    network that never fires, so only stencils below the round-off floor go
    linear.  Reported: fraction of cell reconstructions done with linear
    weights, time per step, and per-field error against FP64.  The network
    must gate more reconstructions than the trivial gate, at an error within
    a small factor of it and of the mixed form.  (On this state about three
    quarters of the reconstructions are below the round-off floor, and the
    network, held to a recall of 0.995 on troubled samples, adds a fraction
    of a percent: it must add something, and it must not cost accuracy.)"""
    import torch
    from paper_2409_10729_gb300 import mfc
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    if not os.path.exists(wpath):
        pytest.skip("no trained gate weights (python -m paper_2409_10729_gb300.train_gate)")
    weights = np.load(wpath)
    p, w = I.shock_droplets(96)
    steps = 30
    res = {}
    for name, form, wts in (("fp64", "fp64", None), ("mixed", "mixed", None), ("network", "gated", weights),
                            ("trivial", "gated", _bias_only(10.0))):
        s = mfc.Solver(p, form)
        if wts is not None:
            s.set_mlp_weights(wts)
        s.set_state_prim(w)
        s.step_rk3(0.4, 2)                          # warm-up (graph capture)
        s.set_state_prim(w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step_rk3(0.4, steps)
        torch.cuda.synchronize()
        res[name] = {"ms_per_step": (time.perf_counter() - t0) * 1e3 / steps, "q": s.get_state()}
        if form == "gated":
            res[name]["gate"] = s.gate_stats() + (s.gate_flat(),)
        s.close()
    ref = res["fp64"]["q"].reshape(7, -1)
    out = {}
    for name in ("mixed", "network", "trivial"):
        d = np.abs(res[name]["q"].reshape(7, -1) - ref)
        scale = np.abs(ref).max(1)
        scale[2:5] = scale[2:5].max()
        out[name] = {"ms_per_step": round(res[name]["ms_per_step"], 3),
                     "rel_linf": (d.max(1) / scale).tolist(),
                     "rel_l1": (d.sum(1) / np.abs(ref).sum(1)).tolist()}
        if "gate" in res[name]:
            gated, fb, cells, flat = res[name]["gate"]
            out[name].update(fraction_gated=gated / cells, fraction_fallback=fb / cells,
                             fraction_flat_warp_steps=flat / cells)
    print("GATE_GAIN " + json.dumps(out))
    for name in ("network", "trivial"):
        assert np.all(np.isfinite(res[name]["q"]))
    net, triv, mix = out["network"], out["trivial"], out["mixed"]
    # the network gates more than the floor alone (reconstructions above the floor)
    assert net["fraction_gated"] > triv["fraction_gated"] + 1e-3
    # at an error within a small factor of the trivial gate's and the mixed form's
    l1n, l1t, l1m = (np.array(x["rel_l1"]) for x in (net, triv, mix))
    assert np.all(l1n <= 3.0 * np.maximum(l1t, l1m) + 1e-7)


def test_flat_stencils_are_smooth_without_the_network():
    """Stencils below the round-off floor count as smooth whatever the
    network says: on a uniform state every reconstruction is such a warp
    step, a network that calls everything troubled still gates them all, and
    the RHS is exactly zero; on the shock/droplet case only part of them are,
    the same part for any network (flatness is a property of the state)."""
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_droplets(40)
    wu = np.empty_like(w)
    for f in range(w.shape[0]):
        wu[f] = w[f].reshape(-1)[0]                 # the pre-shock air state everywhere
    g = _gated(p, _bias_only(10.0))
    g.set_state_prim(wu)
    L = g.rhs()
    gated, fb, cells = g.gate_stats()
    assert g.gate_flat() == cells == gated == 3 * 40 ** 3 and fb == 0
    assert np.all(L == 0.0)
    g.set_state_prim(w)
    g.rhs()
    gated, fb, cells = g.gate_stats()
    flat = g.gate_flat()
    assert 0 < flat < cells and gated >= flat - fb
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    if os.path.exists(wpath):
        n = _gated(p, np.load(wpath))
        n.set_state_prim(w)
        n.rhs()
        assert n.gate_flat() == flat and n.gate_stats()[0] >= gated


def _lipschitz(th):
    """Upper bound of |z(x) - z(x')| / max_k |x_k - x'_k| of the network."""
    th = np.asarray(th, dtype=np.float64)
    W1 = np.abs(th[0:160].reshape(32, 5))
    W2 = np.abs(th[192:1216].reshape(32, 32))
    w3 = np.abs(th[1248:1280])
    return float(w3 @ W2 @ W1 @ np.ones(5))


def test_gated_rhs_matches_the_oracle_gate():
    """The fused gate on the tensor cores against the oracle's gated RHS
    (FP64 primitives, FP64 network, the same rule) on a 96^3 shock/droplet
    state advanced 30 steps by the oracle, with the trained weights.

    Decisions are compared cell by cell and direction by direction.  The two
    sides read the stencils in different precisions (the gated form's FP32
    state against FP64), so a decision may legitimately differ only near one
    of its thresholds: a flat ratio within 1e-3 of 1, a logit within the
    bound of what the FP32 input rounding can move it (network Lipschitz
    bound x 2^-18 (1 + 1/(floor x ratio)), plus 1e-4), or a linear face
    within FP32 rounding of admissibility (relative 1e-5 for rho and c^2,
    absolute 2^-21 for alpha1 and 1 - alpha1).  Elsewhere they must be
    equal, and the near-threshold cells must be rare.  Where a cell's decision and its
    neighbours' along every direction agree, its RHS must equal the oracle's
    to the mixed form's FP32 accuracy (1e-5 of the flux scale)."""
    from paper_2409_10729_gb300 import mfc
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    if not os.path.exists(wpath):
        pytest.skip("no trained gate weights (python -m paper_2409_10729_gb300.train_gate)")
    weights = np.load(wpath)
    p, w = I.shock_droplets(96)
    q, _ = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 30)
    Lo, deco, info = O.rhs_gated(p, q, weights.astype(np.float64), mfc.MFC_GATE_FLOOR)
    g = _gated(p, weights)
    g.set_state(q)
    L, dec = g.gate_rhs()
    g.close()

    Lnet = _lipschitz(weights)
    ratio = info[..., 2:4]
    zo = info[..., 0:2]
    with np.errstate(divide="ignore", invalid="ignore"):
        margin = Lnet * 2.0 ** -18 * (1.0 + 1.0 / (mfc.MFC_GATE_FLOOR * ratio)) + 1e-4
        near = (np.abs(ratio - 1.0) <= 1e-3).any(-1)
        near |= (~np.isnan(zo) & (np.abs(zo) <= margin)).any(-1)
        adm = info[..., 4:8]
        near |= (np.abs(adm[..., 0]) <= 1e-5) | (np.abs(adm[..., 3]) <= 1e-5)
        near |= (np.abs(adm[..., 1]) <= 2.0 ** -21) | (np.abs(adm[..., 2]) <= 2.0 ** -21)
    mismatch = dec != deco
    assert not np.any(mismatch & ~near), f"{int((mismatch & ~near).sum())} decisions differ away from thresholds"
    # the logit bound is wide for stencils just above the floor (their FP32
    # inputs carry up to 2^-19 / floor of rounding): a few percent of cells
    assert near.mean() < 0.05
    assert np.all(np.isin(dec, [0, 1, 2])) and (dec == 1).any() and (dec == 0).any()

    # cells whose reconstructions (own, and both neighbours along each
    # direction) were decided alike on both sides
    agree = ~mismatch                                 # [3, z, y, x]
    ok = np.ones(agree.shape[1:], dtype=bool)
    for d in range(3):
        a = agree[d]
        ax = 2 - d                                    # array axis of direction d
        ok &= a & np.roll(a, 1, axis=ax) & np.roll(a, -1, axis=ax)
    S = O.max_wavespeed(p, q)
    scale = np.maximum(np.abs(Lo).reshape(7, -1).max(1), np.abs(q).reshape(7, -1).max(1) * S)
    err = np.abs(L - Lo).reshape(7, -1)[:, ok.reshape(-1)].max(1) / scale
    assert ok.mean() > 0.99
    assert err.max() <= 1e-5, err
    assert np.all(np.isfinite(L))
    print("GATE_PARITY " + json.dumps({"cells": int(dec[0].size), "near_threshold": float(near.mean()),
                                       "mismatch": int(mismatch.sum()), "compared_rhs": float(ok.mean()),
                                       "rhs_err": err.tolist(),
                                       "fractions": [float((dec == k).mean()) for k in (0, 1, 2)]}))
