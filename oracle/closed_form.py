"""Closed-form solutions used as pins for the oracle (FP64, test infrastructure only).

1. Pressurised spherical cavity in a full space.

Radially symmetric field outside a cavity of radius a in an unbounded isotropic solid, driven
by a pressure P(s) on the wall (Laplace domain, Re s > 0).  With the outgoing potential
phi = A e^{-s r / c_p} / r, u_r = d phi / dr and the wall condition sigma_rr(a) = -P(s):
    u_r(a, s) = P(s) a (1 + s a / c_p) / (rho s^2 a^2 + 4 mu (1 + s a / c_p)).
For a step pressure P(s) = p0 / s this is rational in s with poles at 0 and at the roots of
rho a^2 c_p s^2 + 4 mu a s + 4 mu c_p = 0, so the time response follows from residues.

2. Prismatic rod with Poisson's ratio 0 (the rod of Sec. 4, Example 1): fixed at x = 0, axial
traction P(s) = P0 / s on the end x = L, lateral faces free.  With nu = 0 the 1-D bar field
u = u(x, t) e_x is an exact solution of the 3-D equations (no lateral coupling), with
c = sqrt(E / rho).  Laplace domain: u(x, s) = A sinh(s x / c) with E u_x(L) = P0 / s, so
    u(L, s) = P0 c tanh(s L / c) / (E s^2).
Expanding tanh z = 1 + 2 sum_{n>=1} (-1)^n e^{-2 n z} and inverting term by term:
    u(L, t) = (P0 c / E) [t + 2 sum_{n>=1} (-1)^n (t - 2 n L / c) H(t - 2 n L / c)],
a triangle wave between 0 and 2 P0 L / E of period 4 L / c.
"""
from __future__ import annotations

import numpy as np

from .kernels import wave_speeds


def cavity_ur(s, a, mu, nu, rho, p0):
    """u_r(a, s) for the step pressure p0 H(t)."""
    _, cp = wave_speeds(mu, nu, rho)
    s = np.asarray(s, dtype=np.complex128)
    k = 1.0 + s * a / cp
    return (p0 / s) * a * k / (rho * s ** 2 * a ** 2 + 4.0 * mu * k)


def cavity_poles_residues(a, mu, nu, rho, p0):
    """Poles and residues of u_r(a, s) = p0 a (c_p + s a) / (s (rho a^2 c_p s^2 + 4 mu a s +
    4 mu c_p)) -- a proper rational function with three simple poles."""
    _, cp = wave_speeds(mu, nu, rho)
    num = np.array([p0 * a * a, p0 * a * cp])                       # p0 a (a s + c_p)
    den = np.polymul([1.0, 0.0], [rho * a * a * cp, 4.0 * mu * a, 4.0 * mu * cp])
    poles = np.roots(den)
    dden = np.polyder(den)
    res = np.polyval(num, poles) / np.polyval(dden, poles)
    return poles, res


def cavity_ur_time(t, a, mu, nu, rho, p0):
    """u_r(a, t) = sum over poles of residue * e^{pole t}, t >= 0 (real)."""
    poles, res = cavity_poles_residues(a, mu, nu, rho, p0)
    t = np.asarray(t, dtype=np.float64)
    return np.real(np.sum(res[:, None] * np.exp(poles[:, None] * t[None, :]), axis=0))


def rod_end_displacement_s(s, L, E, rho, P0):
    """u(L, s) of the nu = 0 rod (Laplace domain)."""
    c = np.sqrt(E / rho)
    s = np.asarray(s, dtype=np.complex128)
    return P0 * c * np.tanh(s * L / c) / (E * s * s)


def rod_end_displacement_t(t, L, E, rho, P0):
    """u(L, t) of the nu = 0 rod (time domain, the reflection series)."""
    c = np.sqrt(E / rho)
    t = np.asarray(t, dtype=np.float64)
    u = t.copy()
    n_max = int(np.ceil(t.max() * c / (2 * L))) + 1 if t.size else 0
    for n in range(1, n_max + 1):
        tn = t - 2 * n * L / c
        u += 2 * (-1) ** n * np.where(tn > 0, tn, 0.0)
    return P0 * c / E * u
