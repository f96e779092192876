"""Fourier series method (FSM) inverse Laplace transform (oracle, FP64, test infrastructure).

Sec. 2.2: the Bromwich integral, Eq. (invLap), h(t) = 1/(2 pi i) int h(s) e^{st} ds along
Re s = eta, is truncated and evaluated by the trapezoidal rule on the equally spaced frequencies
s_k = eta + i k dw, dw = 2 pi / P (P = the period of the time window), k = 0 .. N_s/2,
N_c = N_s/2 + 1 solves; the remaining N_s/2 - 1 samples follow from conjugate symmetry
h(s_{N_s-k}) = conj(h(s_k)).  Eq. (IDFT-MFT) writes the result on the grid t_n = n dt,
dt = P / N_s, with the Hanning window W_k = (1 + cos(2 pi k / N_s)) / 2.

Readings (the printed formula is garbled):
  * the trapezoidal rule carries the factor dw / (2 pi) = 1 / P, which Eq. (IDFT-MFT) omits;
  * the symmetric form below is used, valid for any t (not only t = n dt) and equal to the
    N_s-term sum of Eq. (IDFT-MFT) on the grid:
        h(t) = e^{eta t} / P [ W_0 Re h_0 + 2 Re sum_{k=1}^{N_s/2-1} W_k h_k e^{i k dw t}
                               + W_{N_s/2} Re(h_{N_s/2} e^{i (N_s/2) dw t}) ];
  * eta = kappa ln(10) / T with kappa in [2, 3] is the paper's recommendation; the benchmark
    configuration gives eta (sigma) and the spacing pi / T directly, i.e. P = 2 T.
"""
from __future__ import annotations

import math

import numpy as np


def eta_from_kappa(kappa, T):
    """Damping abscissa eta = kappa ln(10) / T (Sec. 2.2)."""
    return kappa * math.log(10.0) / T


def frequencies(eta, P, Ns):
    """s_k = eta + i k 2 pi / P, k = 0 .. Ns/2 (N_c = Ns/2 + 1 values)."""
    assert Ns % 2 == 0
    k = np.arange(Ns // 2 + 1)
    return eta + 1j * k * 2.0 * math.pi / P


def hanning(Ns):
    """W_k = (1 + cos(2 pi k / Ns)) / 2 for k = 0 .. Ns/2."""
    k = np.arange(Ns // 2 + 1)
    return 0.5 * (1.0 + np.cos(2.0 * math.pi * k / Ns))


def invert(h, eta, P, t, window=True):
    """Time response at times t from samples h (N_c, ...) at s_k = eta + i k 2pi/P.

    h's first axis runs over k = 0 .. Ns/2 with Ns = 2 (N_c - 1).  Returns (len(t), ...)."""
    h = np.asarray(h, dtype=np.complex128)
    Nc = h.shape[0]
    Ns = 2 * (Nc - 1)
    W = hanning(Ns) if window else np.ones(Nc)
    dw = 2.0 * math.pi / P
    t = np.asarray(t, dtype=np.float64)
    k = np.arange(Nc)
    coef = np.full(Nc, 2.0)
    coef[0] = 1.0
    coef[-1] = 1.0                                   # Nyquist term counted once
    ph = np.exp(1j * dw * np.outer(t, k))            # (nt, Nc)
    wh = (W * coef)[:, None] * h.reshape(Nc, -1)     # (Nc, m)
    out = np.real(ph @ wh)                           # (nt, m)
    out *= (np.exp(eta * t) / P)[:, None]
    return out.reshape((len(t),) + h.shape[1:])
