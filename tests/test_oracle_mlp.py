"""Pins of the oracle's POD + MLP warm-start model (FP64).

* Back-propagated gradients equal central finite differences of the loss (every parameter
  array checked on random entries).
* The tanh form of GELU stays within its known distance (< 1e-3) of x Phi(x) (erf form) and
  has the right limits.
* POD: orthonormal basis; the truncated projection reproduces snapshots whose span it captures;
  the energy cut keeps exactly the modes a known spectrum calls for.
* Targets depend only on each snapshot's direction (invariant under x_j -> gamma_j x_j), have unit
  norm and a real non-negative leading entry.
* The minimal-residual scale leaves a residual orthogonal to A x^, never larger than |b|, and
  recovers x exactly when x is a multiple of x^.
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


def _orthonormal(rng, n, k):
    return np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))[0]


def test_pod_energy_cut():
    rng = np.random.default_rng(8)
    U, V = _orthonormal(rng, 40, 4), _orthonormal(rng, 6, 4)
    X = U @ np.diag([1.0, 1e-3, 1e-6, 1e-9]) @ V.conj().T
    # energies 1, 1e-6, 1e-12, 1e-18: the tail after two modes (~1e-12) is the first below 1e-10
    assert mlp.pod(X, energy_tol=1e-10).shape[1] == 2
    assert mlp.pod(X, energy_tol=1e-5).shape[1] == 1
    assert mlp.pod(X, energy_tol=1e-15).shape[1] == 3
    assert mlp.pod(X, r_max=1, energy_tol=1e-15).shape[1] == 1
    Phi = mlp.pod(X, energy_tol=1e-10)
    sv = np.linalg.svd(Phi.conj().T @ U[:, :2], compute_uv=False)
    assert sv.min() > 1 - 1e-12


def test_targets_are_directions():
    rng = np.random.default_rng(9)
    Phi = _orthonormal(rng, 30, 3)
    C = rng.standard_normal((3, 5)) + 1j * rng.standard_normal((3, 5))
    X = Phi @ C
    T = mlp.targets(Phi, X)
    gamma = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    assert np.allclose(mlp.targets(Phi, X * gamma), T, atol=1e-12)
    Ct = T[:, :3] + 1j * T[:, 3:]
    assert np.allclose(np.linalg.norm(Ct, axis=1), 1.0)
    assert np.allclose(Ct[:, 0].imag, 0.0, atol=1e-14) and (Ct[:, 0].real > 0).all()
    # the direction itself is unchanged: Ct is C up to one complex factor per snapshot
    for j in range(5):
        ratio = Ct[j] / C[:, j]
        assert np.allclose(ratio, ratio[0])


def test_min_residual_scale():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    b = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    xh = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    x0 = mlp.min_residual_scale(A, b, xh)
    r = b - A @ x0
    assert abs(np.vdot(A @ xh, r)) <= 1e-12 * np.linalg.norm(A @ xh) * np.linalg.norm(b)
    assert np.linalg.norm(r) <= np.linalg.norm(b)
    g = 0.3 - 2.1j
    assert np.allclose(mlp.min_residual_scale(A, A @ (g * xh), xh), g * xh)
    assert np.all(mlp.min_residual_scale(A, b, np.zeros(12)) == 0)
