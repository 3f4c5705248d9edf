"""Pins for the float64 tile-net oracle: library correlation and finite differences."""

import numpy as np
import pytest

from oracle import tcnn


def test_conv_matches_scipy_correlation():
    from scipy import signal

    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 16, 16))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    out = tcnn.conv_s2(x, W, b)
    for n in range(2):
        for o in range(4):
            full = sum(signal.correlate2d(np.pad(x[n, c], 1), W[o, c], mode="valid") for c in range(3))
            np.testing.assert_allclose(out[n, o], full[::2, ::2] + b[o], rtol=1e-12, atol=1e-12)


def test_forward_shapes_and_layout():
    assert tcnn.NP == 3585
    p = np.arange(tcnn.NP, dtype=np.float64)
    assert np.array_equal(tcnn.pack(tcnn.unpack(p)), p)
    z, (x0, a1, a2, a3, g) = tcnn.forward(np.zeros((3, 64, 64), np.uint8), p * 1e-4)
    assert z.shape == (3,) and a1.shape == (3, 8, 32, 32) and a2.shape == (3, 16, 16, 16)
    assert a3.shape == (3, 16, 8, 8) and g.shape == (3, 16)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    tiles = rng.integers(0, 256, (4, 64, 64)).astype(np.uint8)
    labels = np.array([1, 0, 1, 0], np.float64)
    p = rng.normal(scale=0.2, size=tcnn.NP)
    L, g = tcnn.loss_grad(tiles, labels, p, pos_weight=3.0)
    assert L == pytest.approx(tcnn.loss(tiles, labels, p, pos_weight=3.0), rel=1e-12)
    idx = np.concatenate([rng.choice(tcnn.NP, 60, replace=False), [tcnn.NP - 1, tcnn.NP - 2, 0, 72]])
    h = 1e-6
    for i in idx:
        e = np.zeros(tcnn.NP)
        e[i] = h
        fd = (tcnn.loss(tiles, labels, p + e, 3.0) - tcnn.loss(tiles, labels, p - e, 3.0)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=2e-4, abs=1e-9), i


def test_adam_closed_form_first_step():
    # First bias-corrected step moves every weight by lr * sign(g) (for |g| >> eps).
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    q, m, v = tcnn.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(q, p - 0.01 * np.sign(g), rtol=1e-9)
