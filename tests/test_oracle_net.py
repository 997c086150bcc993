"""Pins of the FP64 reference of the proposal network: its convolution
against scipy's correlation, its gradients against central finite
differences."""
import numpy as np
import pytest

from oracle import conv_net as cn


def test_conv3x3_matches_scipy_correlate():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(0)
    x = rng.normal(size=(7, 9, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cn.conv3x3(x, W, b)
    for o in range(4):
        ref = b[o] + sum(correlate2d(x[..., c], W[o, :, :, c], mode="same", boundary="fill") for c in range(3))
        assert np.abs(y[..., o] - ref).max() < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    T = 1
    params = cn.he_init(T, seed=3).astype(np.float64)
    params += rng.normal(0, 0.05, size=params.shape)      # non-zero biases, no dead ReLUs at 0
    x = rng.normal(size=(5, 6, 2 * T))
    target = np.stack([rng.normal(size=(5, 6)), rng.uniform(0, 1, size=(5, 6))], -1)
    target[0, 0, 0] = np.nan                              # a skipped pixel
    loss, g = cn.loss_and_grads(params, x, target, T, lam_r=0.7)
    idx = rng.choice(len(params), size=60, replace=False)
    eps = 1e-6
    for i in idx:
        p = params.copy()
        p[i] += eps
        lp, _ = cn.loss_and_grads(p, x, target, T, lam_r=0.7)
        p[i] -= 2 * eps
        lm, _ = cn.loss_and_grads(p, x, target, T, lam_r=0.7)
        fd = (lp - lm) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-4, abs=1e-8)


def test_layout_counts():
    assert cn.num_params(8) == len(cn.he_init(8))
    assert cn.num_params(8) == 42210
