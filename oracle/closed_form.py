"""Closed-form pressurised spherical cavity in a full space (pin for the oracle; FP64).

Radially symmetric field outside a cavity of radius a in an unbounded isotropic solid, driven
by a pressure P(s) on the wall (Laplace domain, Re s > 0).  With the outgoing potential
phi = A e^{-s r / c_p} / r, u_r = d phi / dr and the wall condition sigma_rr(a) = -P(s):
    u_r(a, s) = P(s) a (1 + s a / c_p) / (rho s^2 a^2 + 4 mu (1 + s a / c_p)).
For a step pressure P(s) = p0 / s this is rational in s with poles at 0 and at the roots of
rho a^2 c_p s^2 + 4 mu a s + 4 mu c_p = 0, so the time response follows from residues.
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
