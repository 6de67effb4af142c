"""Pins for the oracle's troubled-cell network (FP64 forward/backward/Adam).

The backward pass is pinned by central finite differences of the loss; the
forward pass by a direct numpy evaluation of the network; Adam by its
closed-form first step; the weights used for labels by the WENO5-JS
smooth/discontinuous limits.
"""
import numpy as np
import pytest

import oracle as O

NP = 1281


def _theta(seed=0, scale=0.4):
    return np.random.default_rng(seed).normal(0.0, scale, NP)


def _unpack(th):
    W1 = th[:160].reshape(32, 5)
    b1 = th[160:192]
    W2 = th[192:1216].reshape(32, 32)
    b2 = th[1216:1248]
    w3 = th[1248:1280]
    return W1, b1, W2, b2, w3, th[1280]


def test_parameter_count():
    assert O.mlp_nparams() == NP == 5 * 32 + 32 + 32 * 32 + 32 + 32 + 1


def test_forward_matches_numpy_network():
    rng = np.random.default_rng(1)
    th = _theta(1)
    x = rng.uniform(-1, 1, (200, 5))
    W1, b1, W2, b2, w3, b3 = _unpack(th)
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    z = h2 @ w3 + b3
    np.testing.assert_allclose(O.mlp_forward(th, x), z, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("wp", [1.0, 3.5])
def test_gradient_matches_central_differences(wp):
    rng = np.random.default_rng(2)
    th = _theta(2)
    x = rng.uniform(-1, 1, (64, 5))
    y = (rng.uniform(size=64) < 0.3).astype(float)
    loss, g = O.mlp_loss_grad(th, x, y, wp)
    h = 1e-6
    idx = list(range(0, 160, 7)) + list(range(160, 1281, 13)) + [1280]
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (O.mlp_loss_grad(tp, x, y, wp)[0] - O.mlp_loss_grad(tm, x, y, wp)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(g[k]), k


def test_loss_is_weighted_bce():
    th = _theta(3)
    x = np.random.default_rng(3).uniform(-1, 1, (10, 5))
    y = np.array([0, 1] * 5, float)
    z = O.mlp_forward(th, x)
    sp = lambda t: np.log1p(np.exp(t))
    ref = np.mean(2.0 * y * sp(-z) + (1 - y) * sp(z))
    assert O.mlp_loss_grad(th, x, y, 2.0)[0] == pytest.approx(ref, rel=1e-12)


def test_adam_first_step_is_lr_sign():
    """With zero moments, the bias-corrected first step is lr * g/(|g| + eps)."""
    th = _theta(4)
    g = np.random.default_rng(4).normal(size=NP)
    t2, m, v = O.mlp_adam(th, g, np.zeros(NP), np.zeros(NP), 1, lr=1e-3)
    np.testing.assert_allclose(th - t2, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_normalised_stencil():
    x = O.mlp_normalise([1.0, 2.0, 3.0, 5.0, 3.5])
    assert np.array_equal(x, [-1.0, -0.5, 0.0, 1.0, 0.25])       # exact: divisions by 2
    assert np.all(O.mlp_normalise([7.0] * 5) == 0.0)
    # the round-off floor: variation 0.9e-4 of the centre value is flat, 1.1e-4 is not
    s = 1e5 * np.array([1.0, 1.0, 1.0, 1.0 + 0.9e-4, 1.0])
    assert O.is_flat(s) and np.all(O.mlp_normalise(s) == 0.0)
    s = 1e5 * np.array([1.0, 1.0, 1.0, 1.0 + 1.1e-4, 1.0])
    assert not O.is_flat(s)
    np.testing.assert_allclose(O.mlp_normalise(s), [0.0, 0.0, 0.0, 1.0, 0.0], atol=1e-12)
    assert O.is_flat(s, delta=2e-4)


def test_labels_from_weno_weights():
    """Smooth stencils keep the linear weights (not troubled); a jump makes the
    stencil crossing it lose its weight (troubled)."""
    xs = np.linspace(0, 0.4, 5)
    smooth = [np.sin(xs) + 2.0, np.full(5, 1e5)]
    assert not O.troubled(smooth)
    jump = [np.array([1.0, 1.0, 1.0, 5.0, 5.0]), np.full(5, 1e5)]
    assert O.troubled(jump)
    # a pressure stencil wiggling at round-off (1e-9 of 1e5: WENO's absolute
    # epsilon reads it as non-smooth) is below the floor and not troubled
    wiggle = [np.full(5, 1.2), 1e5 * (1.0 + 1e-9 * np.array([1.0, -1.0, 1.0, -1.0, 1.0]))]
    wm, _ = O.weno5_weights(wiggle[1])
    assert np.max(np.abs(wm - [0.1, 0.6, 0.3]) / [0.1, 0.6, 0.3]) > 0.1
    assert not O.troubled(wiggle)
    assert O.troubled(wiggle, delta=0.0)
    wm, wp = O.weno5_weights(np.array([1.0, 1.0, 1.0, 5.0, 5.0]))
    assert wm[0] > 0.99 and wp[0] > 0.99
