"""Pins for the router's CPU oracle (oracle/mlp.py): its analytic gradient of
the expectile loss against central finite differences in fp64."""
import numpy as np

from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, size=mlp.NPARAM)
    X = rng.normal(size=(40, mlp.NIN))
    y = rng.normal(size=40)
    for q in (0.5, 0.9):
        L, g = mlp.loss_and_grad(theta, X, y, q)
        h = 1e-6
        for k in rng.choice(mlp.NPARAM, 60, replace=False):
            tp = theta.copy(); tp[k] += h
            tm = theta.copy(); tm[k] -= h
            fd = (mlp.loss_and_grad(tp, X, y, q)[0] - mlp.loss_and_grad(tm, X, y, q)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k]))


def test_expectile_weights_bias_upward():
    # with q > 1/2 the loss-minimising constant exceeds the mean
    rng = np.random.default_rng(1)
    y = rng.normal(size=2000)
    cs = np.linspace(-1, 1, 2001)
    loss = [np.mean(np.where(y - c > 0, 0.9, 0.1) * (y - c) ** 2) for c in cs]
    assert cs[int(np.argmin(loss))] > np.mean(y) + 0.3
