"""Pins of the oracle's FSM inverse Laplace transform.

Exact discrete pairs: for a real sequence g_n sampled at t_n = n dt, the samples
h(s_k) = dt sum_n g_n e^{-s_k t_n} are inverted back to g exactly without a window, and to the
closed-form three-point smoothing 1/2 g_n + 1/4 e^{-eta dt} g_{n+1} + 1/4 e^{eta dt} g_{n-1}
(circular in e^{-eta t} g) with the Hanning window.  Continuous pairs are inverted within the
method's aliasing / truncation error.
"""
import math

import numpy as np

import workloads as W
from oracle import closed_form as CF
from oracle import fsm


def _discrete_pair(Ns=126, P=0.04, eta=250.0, seed=0):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(Ns)
    dt = P / Ns
    s = fsm.frequencies(eta, P, Ns)
    n = np.arange(Ns)
    h = dt * np.exp(-np.outer(s, n * dt)) @ g
    return g, h, n * dt, eta, P, dt


def test_exact_discrete_pair_without_window():
    g, h, t, eta, P, _ = _discrete_pair()
    out = fsm.invert(h, eta, P, t, window=False)
    assert np.abs(out - g).max() < 1e-12 * np.abs(g).max() * math.exp(eta * P)


def test_exact_discrete_pair_with_hanning():
    g, h, t, eta, P, dt = _discrete_pair(seed=1)
    Ns = len(g)
    gt = g * np.exp(-eta * t)                      # e^{-eta t} g, periodic
    ref = np.exp(eta * t) * (0.5 * gt + 0.25 * np.roll(gt, -1) + 0.25 * np.roll(gt, 1))
    out = fsm.invert(h, eta, P, t, window=True)
    assert np.abs(out - ref).max() < 1e-12 * np.abs(g).max() * math.exp(eta * P)


def test_conjugate_symmetry_real_response():
    """Off-grid times give a real response that equals the full N_s-term sum with
    h(s_{N_s-k}) = conj(h(s_k)) only on the grid; check the grid equality."""
    g, h, t, eta, P, dt = _discrete_pair(seed=2)
    Ns = len(g)
    hk = np.concatenate([h, np.conj(h[1:-1][::-1])])      # k = 0 .. Ns-1
    Wk = 0.5 * (1 + np.cos(2 * math.pi * np.arange(Ns) / Ns))
    n = np.arange(Ns)
    full = np.exp(eta * n * dt) / P * (np.exp(2j * math.pi * np.outer(n, np.arange(Ns)) / Ns)
                                      @ (Wk * hk))
    assert np.abs(full.imag).max() < 1e-9 * np.abs(full.real).max()
    out = fsm.invert(h, eta, P, n * dt)
    assert np.abs(out - full.real).max() < 1e-12 * np.abs(full.real).max()


def test_continuous_pair_exponential():
    """1/(s+a) -> e^{-a t}: FSM error on [1, 10] ms with the benchmark grid (P = 40 ms)."""
    a = 300.0
    s = W.fsm_frequencies(0.02, 250.0, 64)
    t = np.linspace(1e-3, 1e-2, 50)
    out = fsm.invert(1.0 / (s + a), 250.0, 0.04, t)
    assert np.abs(out - np.exp(-a * t)).max() < 1e-2


def test_cavity_closed_form_round_trip():
    """FSM of the exact cavity u_r(a, s) reproduces the exact u_r(a, t) on the 200 output times
    (0..10 ms) within the FSM's own truncation error (the step is smoothed by the window)."""
    m = W.CAVITY_MATERIAL
    s = W.fsm_frequencies(0.02, 250.0, 64)
    t = np.linspace(0.0, 0.01, 200)
    h = CF.cavity_ur(s, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    out = fsm.invert(h, 250.0, 0.04, t)
    ex = CF.cavity_ur_time(t, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    final = W.CAVITY_P0 / (4 * m.mu)
    assert abs(ex[-1] - final) < 0.2 * final           # approaches the static value p0 a/(4 mu)
    assert np.abs(out[t > 1e-3] - ex[t > 1e-3]).max() < 0.05 * final
    assert np.abs(out[t > 5e-3] - ex[t > 5e-3]).max() < 0.005 * final


def test_cavity_closed_form_poles():
    m = W.CAVITY_MATERIAL
    poles, res = CF.cavity_poles_residues(1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    order = np.argsort(poles.imag)
    poles, res = poles[order], res[order]
    assert abs(poles[1]) < 1e-9                         # the step's pole at s = 0
    cp = math.sqrt(3.0 * m.mu / m.rho)
    # rho a^2 s^2 + 4 mu a s / c_p + 4 mu = 0  ->  s = (-2 mu/cp +- i sqrt(...)) / (rho a^2)
    re = -2.0 * m.mu / (cp * m.rho)
    im = math.sqrt(4.0 * m.mu * m.rho - 4.0 * m.mu ** 2 / cp ** 2) / m.rho
    assert abs(poles[0] - complex(re, -im)) < 1e-6 and abs(poles[2] - complex(re, im)) < 1e-6
    assert abs(res[1] - W.CAVITY_P0 / (4 * m.mu)) < 1e-18


def test_rod_closed_form_laplace_and_time_agree():
    """The nu = 0 rod: the Laplace-domain end displacement P0 c tanh(sL/c)/(E s^2), inverted by
    the FSM on the rod example's grid (kappa = 3, Hanning, N_c = 110 over T = 0.0155 s), matches
    the reflection-series time response away from its kinks; the series is a triangle wave of
    period 4L/c between 0 and 2 P0 L / E."""
    import numpy as np
    from oracle import closed_form as CF, fsm
    L, E, rho, P0, T = 3.0, 2.11e11, 7.85e3, -1e6, 0.0155
    c = np.sqrt(E / rho)
    t = np.linspace(0.0, T * 0.6, 400)
    u = CF.rod_end_displacement_t(t, L, E, rho, P0)
    ext = CF.rod_end_displacement_t(np.array([0.0, 2 * L / c, 4 * L / c, 6 * L / c]), L, E, rho, P0)
    assert np.allclose(ext, [0.0, 2 * P0 * L / E, 0.0, 2 * P0 * L / E], atol=1e-12 * abs(P0 * L / E))
    assert u.min() >= 2 * P0 * L / E * (1 + 1e-12) and u.max() <= 1e-18
    tp = 4 * L / c
    assert np.allclose(CF.rod_end_displacement_t(t[t < T * 0.6 - tp] + tp, L, E, rho, P0),
                       u[t < T * 0.6 - tp], atol=1e-18)
    eta = fsm.eta_from_kappa(3.0, T)
    s = fsm.frequencies(eta, T, 218)
    h = CF.rod_end_displacement_s(s, L, E, rho, P0)
    inv = fsm.invert(h, eta, T, t, window=True)
    # away from the kinks (every 2L/c) the windowed inversion follows the triangle wave
    kink = 2 * L / c
    far = np.abs(((t + kink / 2) % kink) - kink / 2) > 0.15 * kink
    err = np.abs(inv - u)[far].max() / np.abs(u).max()
    assert err < 0.05, err


def test_fsm_grid_matches_the_rod_example_printed_values():
    """Sec. 4, Example 1 prints, for T = 0.0155 s: dt = pi / Omega_s = 7.11e-5 s,
    N_s = ceil(T / dt) = 218 and N_c = 110 (tests/golden/rod_example1_fsm_grid.txt).  The oracle's
    grid s_k = eta + i k 2 pi / T, k = 0 .. N_s/2, reproduces them: N_c = N_s/2 + 1 and
    Omega_s = (N_c - 1) 2 pi / T with pi / Omega_s = dt to the printed digits."""
    import math
    import os
    import numpy as np
    from oracle import fsm
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "rod_example1_fsm_grid.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    T, Ns = vals["T_s"], int(vals["N_s"])
    s = fsm.frequencies(fsm.eta_from_kappa(vals["kappa"], T), T, Ns)
    assert len(s) == int(vals["N_c"])
    omega = s[-1].imag
    assert abs(math.pi / omega - vals["dt_s"]) < 0.005e-5
    assert round(T / (math.pi / omega)) == Ns                    # N_s = T / dt on this grid
    assert np.allclose(np.diff(s.imag), 2 * math.pi / T)
