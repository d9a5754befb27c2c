"""Pins for the oracle's FP64 MLP (12-64-64-64-1, ReLU hidden layers, sigmoid output) used
by the learned segment proposal.  The paper has no counterpart; the checks are the
mathematics itself: special cases and central finite differences."""
import math

import numpy as np

import oracle


def _rand_params(rng, scale=0.3):
    return [rng.normal(0.0, scale, size=s) for s in oracle.MLP_SHAPES]


def test_zero_network_is_half_and_log2_loss():
    ps = [np.zeros(s) for s in oracle.MLP_SHAPES]
    x = np.random.default_rng(0).normal(size=(7, 12))
    np.testing.assert_array_equal(oracle.mlp_forward(ps, x), np.full(7, 0.5))
    t = np.linspace(0, 1, 7)
    loss, g = oracle.mlp_loss_grad(ps, x, t)
    assert abs(loss - math.log(2.0)) < 1e-15
    # only the output bias sees a gradient: mean(y - t)
    assert abs(g[7][0] - np.mean(0.5 - t)) < 1e-15
    for k in range(7):
        assert np.all(g[k] == 0)


def test_pass_through_network():
    ps = [np.zeros(s) for s in oracle.MLP_SHAPES]
    ps[0][0, 3] = 1.0  # hidden unit 0 of layer 1 copies feature 3
    ps[2][0, 0] = 1.0
    ps[4][0, 0] = 1.0
    ps[6][0, 0] = 2.0
    ps[7][0] = -1.0
    x = np.zeros((4, 12))
    x[:, 3] = [-2.0, 0.0, 0.5, 3.0]
    want = 1.0 / (1.0 + np.exp(-(2.0 * np.maximum(x[:, 3], 0.0) - 1.0)))
    np.testing.assert_allclose(oracle.mlp_forward(ps, x), want, rtol=0, atol=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    ps = _rand_params(rng)
    x = rng.normal(size=(16, 12))
    t = rng.uniform(size=16)
    loss, g = oracle.mlp_loss_grad(ps, x, t)
    eps = 1e-6
    worst = 0.0
    for k, p in enumerate(ps):
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 40), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = oracle.mlp_loss_grad(ps, x, t)
            flat[i] = old - eps
            lm, _ = oracle.mlp_loss_grad(ps, x, t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            # central differences carry ~eps^2 truncation and ~1e-16/eps rounding error
            err = abs(fd - an) / (1e-8 + 1e-6 * abs(an))
            worst = max(worst, err)
    assert worst < 1.0, worst


def test_loss_is_bce_of_forward():
    rng = np.random.default_rng(2)
    ps = _rand_params(rng)
    x = rng.normal(size=(9, 12))
    t = rng.uniform(size=9)
    y = oracle.mlp_forward(ps, x)
    want = -np.mean(t * np.log(y) + (1 - t) * np.log(1 - y))
    loss, _ = oracle.mlp_loss_grad(ps, x, t)
    assert abs(loss - want) < 1e-10 * abs(want)  # log(y) near 0 or 1 loses a few digits
