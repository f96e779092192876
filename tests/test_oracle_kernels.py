"""Pins of the oracle's fundamental solutions against the mathematics they must satisfy.

U must solve the Laplace-domain Navier equation away from the load, tend to Kelvin's solution
as s -> 0 and to plane P/S waves far away; T must be the traction of U by Hooke's law.  None of
these checks re-types the oracle's formula: a dropped term, wrong sign or swapped index in U or
T fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import kernels as K

MAT = (1e9, 0.25, 2000.0)
S_CASES = [250.0 + 0.0j, 250.0 + 5000.0j, 10.0 + 10.0j, 250.0 + 20000.0j]


def _points(n=6, seed=1):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * rng.uniform(0.3, 2.0, size=(n, 1))


def _U(d, s):
    return K.fundamental_U(d, s, *MAT)


def _navier_residual(d, s, h):
    mu, nu, rho = MAT
    lam = K.lame_lambda(mu, nu)
    E = np.eye(3) * h
    D2 = np.zeros((3, 3, 3, 3), dtype=complex)   # D2[k, l, i, j] = d2 U_ij / dy_k dy_l
    for k in range(3):
        for l in range(3):
            D2[k, l] = (_U(d + E[k] + E[l], s) - _U(d + E[k] - E[l], s)
                        - _U(d - E[k] + E[l], s) + _U(d - E[k] - E[l], s)) / (4 * h * h)
    lap = sum(D2[k, k] for k in range(3))
    grad_div = np.einsum("jkik->ij", D2)          # d_j d_k U_ik
    return mu * lap + (lam + mu) * grad_div - rho * s * s * _U(d, s), mu * np.abs(lap).max()


@pytest.mark.parametrize("s", S_CASES)
def test_U_solves_navier_equation(s):
    """mu lap u + (lam+mu) grad div u - rho s^2 u = 0 for u_j = U_ij (central differences,
    Richardson-extrapolated in the step so the O(h^2) truncation error drops out)."""
    for d in _points():
        r1, scale = _navier_residual(d, s, 1e-3)
        r2, _ = _navier_residual(d, s, 5e-4)
        res = (4.0 * r2 - r1) / 3.0
        assert np.abs(res).max() / scale < 1e-6


@pytest.mark.parametrize("s", S_CASES)
def test_T_is_hooke_traction_of_U(s):
    """T_ij = sigma^{(i)}_jk n_k with sigma from the strain of u_j = U_ij (central differences)."""
    mu, nu, rho = MAT
    lam = K.lame_lambda(mu, nu)
    rng = np.random.default_rng(7)
    h = 1e-5
    for d in _points(seed=3):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        grad = np.zeros((3, 3, 3), dtype=complex)   # grad[i, j, k] = d U_ij / d y_k
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            grad[:, :, k] = (_U(d + e, s) - _U(d - e, s)) / (2 * h)
        eps = 0.5 * (grad + grad.transpose(0, 2, 1))
        div = np.einsum("ikk->i", grad)
        sigma = lam * div[:, None, None] * np.eye(3) + 2 * mu * eps
        T_fd = np.einsum("ijk,k->ij", sigma, n)
        T = K.fundamental_T(d, n, s, *MAT)
        assert np.abs(T - T_fd).max() / np.abs(T).max() < 1e-7


def test_static_limit_is_kelvin():
    mu, nu, rho = MAT
    rng = np.random.default_rng(5)
    for d in _points(seed=9):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        U = K.fundamental_U(d, 1e-6, *MAT)
        T = K.fundamental_T(d, n, 1e-6, *MAT)
        assert np.allclose(U, K.kelvin_U(d, mu, nu), rtol=1e-8, atol=0)
        assert np.abs(T - K.kelvin_T(d, n, nu)).max() < 1e-8 * np.abs(T).max()


def test_far_field_plane_waves():
    """|z| >> 1: U -> [E_s/r (delta - rh rh)/mu + E_p/r rh rh/(lam+2mu)] / (4 pi)."""
    mu, nu, rho = MAT
    lam = K.lame_lambda(mu, nu)
    cs, cp = K.wave_speeds(mu, nu, rho)
    s = 250.0 + 2.0e5j
    for d in _points(seed=11):
        r = np.linalg.norm(d)
        rh = d / r
        Es, Ep = np.exp(-s * r / cs), np.exp(-s * r / cp)
        ff = (Es / (mu * r) * (np.eye(3) - np.outer(rh, rh)) + Ep / ((lam + 2 * mu) * r)
              * np.outer(rh, rh)) / (4 * math.pi)
        U = _U(d, s)
        assert np.abs(U - ff).max() / np.abs(ff).max() < 5.0 / abs(s * r / cs)


def test_symmetry_and_reciprocity():
    for s in S_CASES:
        for d in _points(seed=13):
            U = _U(d, s)
            assert np.allclose(U, U.T, rtol=1e-14, atol=0)
            assert np.allclose(U, _U(-d, s), rtol=1e-14, atol=0)


def test_h_series_matches_closed_form_at_switch():
    """The two branches of h(z) agree across |z| = Z_SERIES (no jump at the switch)."""
    for ang in np.linspace(-1.5, 1.5, 7):
        z0 = K.Z_SERIES * np.exp(1j * ang)
        zin, zout = z0 * (1 - 1e-9), z0 * (1 + 1e-9)
        a = K.h_of_z(np.array([zin]))[0]          # series branch
        b = K.h_of_z(np.array([zout]))[0]         # closed-form branch
        assert abs(a - ((1 + zin) * np.exp(-zin) - 1) / zin ** 2) < 1e-13
        assert abs(b - a) < 1e-9 * abs(zout - zin) / 1e-9 + 1e-13
    assert abs(K.h_of_z(np.array([1e-12 + 0j]))[0] + 0.5) < 1e-11


def test_wave_speeds():
    cs, cp = K.wave_speeds(1e9, 0.25, 2000.0)
    assert abs(cs - math.sqrt(5e5)) < 1e-9
    assert abs(cp - math.sqrt(3.0) * cs) < 1e-9   # nu = 1/4: lambda = mu, cp^2 = 3 cs^2
