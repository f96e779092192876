"""Laplace-domain elastodynamic fundamental solutions (oracle, FP64, test infrastructure only).

The boundary integral equation of Sec. 2.1, Eq. (bie), needs the displacement and traction
fundamental solutions U_ij(x, y; s) and T_ij(x, y; s); the paper states that they are found in
text books and omits them.  They are written out here from the Laplace transform of the
classical Stokes solution for a point force in an unbounded isotropic elastic solid
(Laplace variable s, time factor e^{st}, transform f(s) = int_0^inf f(t) e^{-st} dt).

Notation (r = y - x, r = |r|, rh = r / r, n = unit normal at y, dr/dn = rh . n):
    z_s = s r / c_s,  z_p = s r / c_p,  E_s = e^{-z_s},  E_p = e^{-z_p},  beta2 = c_s^2 / c_p^2
    I(r, s) = [(1 + z_p) E_p - (1 + z_s) E_s] / s^2
    psi  = E_s / r - c_s^2 I / r^3
    chi  = E_s / r - beta2 E_p / r - 3 c_s^2 I / r^3
    U_ij = (psi delta_ij - chi rh_i rh_j) / (4 pi mu)
and T_ij (traction component j at y, on the surface with normal n, due to a unit point load in
direction i at x) follows from Hooke's law applied to U:
    T_ij = 1/(4 pi) [ (psi' - chi/r)(delta_ij dr/dn + rh_j n_i)
                      - (2 chi / r)(n_j rh_i - 2 rh_i rh_j dr/dn)
                      - 2 chi' rh_i rh_j dr/dn
                      + (c_p^2/c_s^2 - 2)(psi' - chi' - 2 chi / r) rh_i n_j ]
with psi' = d psi / dr and chi' = d chi / dr written out below.

I suffers from cancellation when |z| is small (its O(1) and O(z) terms cancel), so it is
evaluated through h(z) = ((1 + z) e^{-z} - 1) / z^2, for which I = r^2 (h(z_p)/c_p^2 -
h(z_s)/c_s^2) exactly; h uses its Taylor series sum_{n>=2} (-1)^n (1-n)/n! z^{n-2} for
|z| < Z_SERIES and the closed form otherwise.
"""
from __future__ import annotations

import math

import numpy as np

Z_SERIES = 0.5
N_SERIES = 26  # terms n = 2 .. 27; |z|^25/27! < 1e-30 at |z| = 0.5


def lame_lambda(mu, nu):
    """Lame's first parameter from shear modulus and Poisson's ratio."""
    return 2.0 * mu * nu / (1.0 - 2.0 * nu)


def wave_speeds(mu, nu, rho):
    """S- and P-wave speeds, Sec. 2.1: c_s = sqrt(mu/rho), c_p = sqrt((lambda+2mu)/rho).

    The paper prints c_p = sqrt(lambda + 2 mu / rho); the dimensionally consistent reading,
    (lambda + 2 mu) / rho under the root, is used.
    """
    lam = lame_lambda(mu, nu)
    return math.sqrt(mu / rho), math.sqrt((lam + 2.0 * mu) / rho)


def _h_series_coeffs():
    return np.array([(-1.0) ** n * (1.0 - n) / math.factorial(n) for n in range(2, 2 + N_SERIES)])


_HC = _h_series_coeffs()


def h_of_z(z):
    """h(z) = ((1+z) e^{-z} - 1) / z^2, elementwise, accurate for all z with Re z >= 0."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty_like(z)
    small = np.abs(z) < Z_SERIES
    zs = z[small]
    acc = np.zeros_like(zs)
    for c in _HC[::-1]:
        acc = acc * zs + c
    out[small] = acc
    zl = z[~small]
    out[~small] = ((1.0 + zl) * np.exp(-zl) - 1.0) / zl ** 2
    return out


def radial_functions(r, s, mu, nu, rho):
    """psi, chi, dpsi/dr, dchi/dr at distances r (array) and complex frequency s."""
    cs, cp = wave_speeds(mu, nu, rho)
    r = np.asarray(r, dtype=np.float64)
    zs = s * r / cs
    zp = s * r / cp
    Es = np.exp(-zs)
    Ep = np.exp(-zp)
    beta2 = cs ** 2 / cp ** 2
    I = r ** 2 * (h_of_z(zp) / cp ** 2 - h_of_z(zs) / cs ** 2)
    psi = Es / r - cs ** 2 * I / r ** 3
    chi = Es / r - beta2 * Ep / r - 3.0 * cs ** 2 * I / r ** 3
    dpsi = -(s / cs) * Es / r - 2.0 * Es / r ** 2 + beta2 * Ep / r ** 2 + 3.0 * cs ** 2 * I / r ** 4
    dchi = (-(s / cs) * Es / r - 4.0 * Es / r ** 2 + beta2 * (s / cp) * Ep / r
            + 4.0 * beta2 * Ep / r ** 2 + 9.0 * cs ** 2 * I / r ** 4)
    return psi, chi, dpsi, dchi


def fundamental_U(d, s, mu, nu, rho):
    """U_ij for separation vectors d = y - x of shape (..., 3); returns (..., 3, 3) complex."""
    d = np.asarray(d, dtype=np.float64)
    r = np.linalg.norm(d, axis=-1)
    rh = d / r[..., None]
    psi, chi, _, _ = radial_functions(r, s, mu, nu, rho)
    eye = np.eye(3)
    U = psi[..., None, None] * eye - chi[..., None, None] * rh[..., :, None] * rh[..., None, :]
    return U / (4.0 * math.pi * mu)


def fundamental_T(d, n, s, mu, nu, rho):
    """T_ij for separations d = y - x (..., 3) and unit normals n at y (..., 3)."""
    d = np.asarray(d, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), d.shape)
    cs, cp = wave_speeds(mu, nu, rho)
    r = np.linalg.norm(d, axis=-1)
    rh = d / r[..., None]
    drdn = np.einsum("...k,...k->...", rh, n)
    psi, chi, dpsi, dchi = radial_functions(r, s, mu, nu, rho)
    eye = np.eye(3)
    A = (dpsi - chi / r)[..., None, None]
    B = (2.0 * chi / r)[..., None, None]
    C = (2.0 * dchi)[..., None, None]
    D = ((cp ** 2 / cs ** 2 - 2.0) * (dpsi - dchi - 2.0 * chi / r))[..., None, None]
    dn = drdn[..., None, None]
    rr = rh[..., :, None] * rh[..., None, :]          # rh_i rh_j
    n_i_rh_j = n[..., :, None] * rh[..., None, :]     # n_i rh_j
    rh_i_n_j = rh[..., :, None] * n[..., None, :]     # rh_i n_j
    T = (A * (eye * dn + n_i_rh_j) - B * (rh_i_n_j - 2.0 * rr * dn) - C * rr * dn + D * rh_i_n_j)
    return T / (4.0 * math.pi)


def kelvin_U(d, mu, nu):
    """Static Kelvin solution (s -> 0 limit of U), for pins."""
    d = np.asarray(d, dtype=np.float64)
    r = np.linalg.norm(d, axis=-1)
    rh = d / r[..., None]
    c = 1.0 / (16.0 * math.pi * mu * (1.0 - nu) * r)
    return c[..., None, None] * ((3.0 - 4.0 * nu) * np.eye(3) + rh[..., :, None] * rh[..., None, :])


def kelvin_T(d, n, nu):
    """Static Kelvin traction kernel (s -> 0 limit of T):
    T0_ij = -1/(8 pi (1-nu) r^2) [dr/dn ((1-2nu) delta_ij + 3 rh_i rh_j)
                                  + (1-2nu)(n_i rh_j - n_j rh_i)]."""
    d = np.asarray(d, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), d.shape)
    r = np.linalg.norm(d, axis=-1)
    rh = d / r[..., None]
    dn = np.einsum("...k,...k->...", rh, n)[..., None, None]
    c = (-1.0 / (8.0 * math.pi * (1.0 - nu) * r ** 2))[..., None, None]
    rr = rh[..., :, None] * rh[..., None, :]
    anti = n[..., :, None] * rh[..., None, :] - rh[..., :, None] * n[..., None, :]
    return c * (dn * ((1.0 - 2.0 * nu) * np.eye(3) + 3.0 * rr) + (1.0 - 2.0 * nu) * anti)
