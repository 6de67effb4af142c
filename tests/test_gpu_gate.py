"""GPU tests of the gated form and of the gate network's own training kernels.

* The FP32 loss/gradient, Adam and forward kernels against the FP64 oracle
  (gradients to 1e-5 relative, Adam to 1e-6, logits to 1e-5).
* Training samples: normalised stencils and WENO-weight labels against the
  oracle's weights, cell by cell.
* The gated sweep: a gate that never fires reproduces the mixed form (to
  FP32 round-off; the same WENO code in another kernel); a gate that always fires gives the linear-weight WENO5 RHS (the
  oracle with a huge epsilon) on smooth data; on a sharp interface the
  non-physical linear faces fall back to WENO.
* Training on the GPU lowers the loss; and the trained network's gain: the
  fraction of cell reconstructions it gates, its time against the mixed form
  without the gate, and its error against the FP64 path (the plain-WENO
  judge), stated per field.
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
    state (diffuse interface + shock), recomputed with the oracle's weights."""
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_water_column(48, 24)
    s = mfc.Solver(p, "fp64")
    s.set_state_prim(w)
    s.step_rk3(0.4, 20)
    q = s.get_state()
    X, Y = s.gate_samples(0.1)
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    W = O.cons_to_prim(p, q)[:, 0]            # [6, ny, nx]
    ny, nx = W.shape[1:]
    checked = 0
    for d in range(2):
        for c in range(nx * ny):
            y0, x0 = divmod(c, nx)
            idx = [min(max((x0 if d == 0 else y0) + k, 0), (nx if d == 0 else ny) - 1) for k in range(-2, 3)]
            st = W[:, y0, idx] if d == 0 else W[:, idx, x0]
            # skip labels within round-off of the threshold
            dev = 0.0
            for v in st:
                wm, wp = O.weno5_weights(v)
                dev = max(dev, np.max(np.abs(wm - [0.1, 0.6, 0.3]) / [0.1, 0.6, 0.3]),
                          np.max(np.abs(wp - [0.3, 0.6, 0.1]) / [0.3, 0.6, 0.1]))
            k = (d * nx * ny + c) * 2
            np.testing.assert_allclose(X[k], O.mlp_normalise(st[0] + st[1]), atol=2e-6)
            np.testing.assert_allclose(X[k + 1], O.mlp_normalise(st[4]), atol=2e-6)
            if abs(dev - 0.1) > 1e-6:
                assert Y[k] == Y[k + 1] == float(dev > 0.1)
                checked += 1
    assert checked > 0.99 * 2 * nx * ny
    assert 0 < Y.sum() < len(Y)


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
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_droplets(40)
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
    assert gated == 0 and fb == 0 and cells == 4 * 3 * 3 * 40 ** 3   # steps x stages x directions x cells


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


def test_tensor_core_logits_match_fp32_network():
    """The gated sweep's network (hidden layers on the tensor cores, fp16
    operands, FP32 accumulation) against the FP32 network and the FP64
    oracle on the same inputs: real solver stencils and random ones, with the
    trained weights and with random weights; ragged sample count."""
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_water_column(96, 48)
    s = mfc.Solver(p, "fp64")
    s.set_state_prim(w)
    s.step_rk3(0.4, 100)
    Xs, _ = s.gate_samples(0.1)
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
            assert np.max(np.abs(b - z64)) <= 1e-4 * max(1.0, np.max(np.abs(z64)))
            # fp16 operands: a few 1e-3 of the logit scale
            assert np.max(np.abs(a - z64)) <= 2e-2 * max(1.0, np.max(np.abs(z64)))
            assert np.mean((a < 0) == (z64 < 0)) > 0.99


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
    """The committed trained network on the 3-D shock/droplet case (96^3,
    30 steps): fraction of cell reconstructions gated linear, time per step
    against the ungated mixed form, and per-field error against the FP64
    (plain WENO, oracle-exact) result, next to the mixed form's own error."""
    import torch
    from paper_2409_10729_gb300 import mfc
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    if not os.path.exists(wpath):
        pytest.skip("no trained gate weights (python -m paper_2409_10729_gb300.train_gate)")
    weights = np.load(wpath)
    p, w = I.shock_droplets(96)
    steps = 30
    res = {}
    for form in ("fp64", "mixed", "gated"):
        s = mfc.Solver(p, form)
        if form == "gated":
            s.set_mlp_weights(weights)
        s.set_state_prim(w)
        s.step_rk3(0.4, 2)                          # warm-up (graph capture)
        s.set_state_prim(w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step_rk3(0.4, steps)
        torch.cuda.synchronize()
        res[form] = {"ms_per_step": (time.perf_counter() - t0) * 1e3 / steps, "q": s.get_state()}
        if form == "gated":
            res[form]["gate"] = s.gate_stats()
        s.close()
    ref = res["fp64"]["q"].reshape(7, -1)
    out = {}
    for form in ("mixed", "gated"):
        d = np.abs(res[form]["q"].reshape(7, -1) - ref)
        scale = np.abs(ref).max(1)
        scale[2:5] = scale[2:5].max()
        out[form] = {"ms_per_step": round(res[form]["ms_per_step"], 3),
                     "rel_linf": (d.max(1) / scale).tolist(),
                     "rel_l1": (d.sum(1) / np.abs(ref).sum(1)).tolist()}
    gated, fb, cells = res["gated"]["gate"]
    out["gated"]["fraction_gated"] = gated / cells
    out["gated"]["fraction_fallback"] = fb / cells
    print("GATE_GAIN " + json.dumps(out))
    assert out["gated"]["fraction_gated"] > 0.5
    mix_l1 = np.array(out["mixed"]["rel_l1"])
    gat_l1 = np.array(out["gated"]["rel_l1"])
    assert np.all(gat_l1 <= 20 * mix_l1 + 1e-6)
    assert np.all(np.isfinite(res["gated"]["q"]))


def test_flat_warps_take_the_logit_at_zero_input():
    """Warp steps whose 32 density and pressure stencils are all exactly flat
    take the network's output at zero input (their exact input) from one
    evaluation: on a uniform state every reconstruction is such a step, the
    trained network calls them smooth, and the RHS is exactly zero; on the
    shock/droplet case only part of them are."""
    import torch
    from paper_2409_10729_gb300 import mfc
    wpath = os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")
    if not os.path.exists(wpath):
        pytest.skip("no trained gate weights (python -m paper_2409_10729_gb300.train_gate)")
    weights = np.load(wpath)
    z0 = torch.empty(64, device="cuda")
    mfc.mlp_forward_tc(torch.zeros(64, 5, device="cuda"), torch.from_numpy(weights).cuda(), z0)
    p, w = I.shock_droplets(40)
    wu = np.empty_like(w)
    for f in range(w.shape[0]):
        wu[f] = w[f].reshape(-1)[0]                 # the pre-shock air state everywhere
    g = _gated(p, weights)
    g.set_state_prim(wu)
    L = g.rhs()
    gated, fb, cells = g.gate_stats()
    assert g.gate_flat() == cells == 3 * 40 ** 3
    if float(z0[0]) < 0:
        assert gated == cells and fb == 0
    assert np.all(L == 0.0)
    g.set_state_prim(w)
    g.rhs()
    gated, fb, cells = g.gate_stats()
    flat = g.gate_flat()
    assert 0 < flat < cells
    # flatness is a property of the state: a never-firing gate sees the same
    # flat steps on the same state, and still never fires
    n = _gated(p, _bias_only(10.0))
    n.set_state_prim(w)
    n.rhs()
    assert n.gate_stats()[0] == 0 and n.gate_flat() == flat
