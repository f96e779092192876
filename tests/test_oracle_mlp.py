"""Pins of the oracle's POD + MLP warm-start model (FP64).

* Back-propagated gradients equal central finite differences of the loss (every parameter
  array checked on random entries).
* The tanh form of GELU stays within its known distance (< 1e-3) of x Phi(x) (erf form) and
  has the right limits.
* POD: orthonormal basis; the truncated projection reproduces snapshots whose span it captures.
* Adam drives a quadratic to its minimum; the trained MLP fits a smooth coefficient curve.
"""
import math

import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(6, hidden=16, seed=1)
    U = rng.uniform(0, 1, size=(7, 2))
    Y = rng.standard_normal((7, 6))
    _, g = mlp.loss_and_grads(p, U, Y)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, U, Y)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, U, Y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_gelu_tanh_form():
    x = np.linspace(-6, 6, 241)
    exact = 0.5 * x * (1 + np.array([math.erf(v / math.sqrt(2)) for v in x]))
    assert np.abs(mlp.gelu(x) - exact).max() < 1e-3
    assert abs(mlp.gelu(np.array([0.0]))[0]) == 0.0
    assert abs(mlp.gelu(np.array([20.0]))[0] - 20.0) < 1e-12


def test_pod_basis():
    rng = np.random.default_rng(2)
    basis = np.linalg.qr(rng.standard_normal((50, 4)) + 1j * rng.standard_normal((50, 4)))[0]
    X = basis @ (rng.standard_normal((4, 9)) + 1j * rng.standard_normal((4, 9)))
    Phi = mlp.pod(X)
    assert Phi.shape == (50, 4)
    assert np.allclose(Phi.conj().T @ Phi, np.eye(4), atol=1e-12)
    assert np.abs(Phi @ (Phi.conj().T @ X) - X).max() < 1e-12 * np.abs(X).max()


def test_adam_and_training():
    p = {"w": np.array([0.0])}
    opt = mlp.Adam(p, lr=0.1)
    for _ in range(500):
        opt.step(p, {"w": p["w"] - 3.0})
    assert abs(p["w"][0] - 3.0) < 1e-3
    # fit a smooth 2-output curve of the frequency
    s = 250 + 1j * np.linspace(0, 2000, 40)
    U = mlp.features(s, 2000.0)
    Y = np.stack([np.cos(2 * U[:, 1]), np.sin(3 * U[:, 1])], axis=1)
    prm = mlp.init_params(2, hidden=32, seed=3)
    opt = mlp.Adam(prm, lr=3e-3)
    for _ in range(3000):
        _, g = mlp.loss_and_grads(prm, U, Y)
        opt.step(prm, g)
    y, _ = mlp.forward(prm, U)
    assert np.abs(y - Y).max() < 0.05
