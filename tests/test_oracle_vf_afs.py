"""Pins of the oracle's vector fitting (Sec. 2.3) and adaptive frequency sampling (Sec. 3).

* VF recovers the poles and residues of a known rational function exactly (to rounding) and an
  over-ordered fit reproduces the data; the time response of r/(s - a) is r e^{a t} (the sign of
  Eq. (vf-td) is read this way) -- checked on 1/(s + a) = L{e^{-a t}}.
* VF on the closed-form spherical-cavity response finds its physical pole pair.
* AFS on a rational response converges with fewer samples than the poles' FSM grid would need
  and returns the exact transient; on the cavity closed form it returns the exact u_r(t).
* The Chebyshev initial set and the fit orders follow their formulas.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import afs, closed_form as CF, fsm, vf

MODES = np.array([-40 + 400j, -60 + 1100j, -90 + 2300j, -120 + 3700j, -150 + 5200j])


def _rational(K=6, seed=1, real_pole=0.0):
    rng = np.random.default_rng(seed)
    poles = np.concatenate([MODES, np.conj(MODES), [real_pole + 0j]])
    R = rng.standard_normal((K, len(MODES))) + 1j * rng.standard_normal((K, len(MODES)))
    Rf = np.hstack([R, np.conj(R), rng.standard_normal((K, 1)) + 0j])
    return poles, Rf


def test_vf_recovers_known_poles_and_residues():
    poles, R = _rational(real_pole=-300.0)
    s = 250 + 1j * np.linspace(0, 6000, 60)
    F = vf.evaluate(s, poles, R)
    p, Rr = vf.fit(s, F[:, :3], 11, 6000.0)
    order = np.argsort(p.imag + 1e-9 * p.real)
    ref = np.argsort(poles.imag + 1e-9 * poles.real)
    assert np.abs(p[order] - poles[ref]).max() < 1e-8 * np.abs(poles).max()
    # residues of all six responses with the poles identified from the first three
    pairs = p[p.imag > 0]
    reals = p[np.abs(p.imag) == 0].real
    p2, R2 = vf.residues(s, F, pairs, reals)
    assert np.abs(vf.evaluate(s, p2, R2) - F).max() < 1e-10 * np.abs(F).max()


def test_vf_overordered_fit_reproduces_data():
    poles, R = _rational(real_pole=-300.0)
    s = 250 + 1j * np.linspace(0, 6000, 60)
    F = vf.evaluate(s, poles, R)
    p, Rr = vf.fit(s, F, 17, 6000.0)
    assert np.abs(vf.evaluate(s, p, Rr) - F).max() < 1e-9 * np.abs(F).max()


def test_time_response_sign():
    a = 300.0
    t = np.linspace(0, 0.01, 11)
    h = vf.time_response(t, np.array([-a + 0j]), np.array([[1.0 + 0j]]))
    assert np.abs(h[:, 0] - np.exp(-a * t)).max() < 1e-15


def test_vf_on_cavity_closed_form():
    m = W.CAVITY_MATERIAL
    s = W.fsm_frequencies(0.02, 250.0, 64)
    F = CF.cavity_ur(s, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)[:, None]
    p, Rr = vf.fit(s, F, 5, s[-1].imag)
    true_p, _ = CF.cavity_poles_residues(1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    pair = true_p[true_p.imag > 0][0]
    assert np.abs(p - pair).min() < 1e-8 * abs(pair)
    assert np.abs(vf.evaluate(s, p, Rr) - F).max() < 1e-10 * np.abs(F).max()


def test_chebyshev_initial_set_and_fit_orders():
    s = afs.chebyshev_frequencies(250.0, 1000.0, 16)
    assert np.allclose(s.real, 250.0)
    assert abs(s[0].imag) < 1e-12 and abs(s[-1].imag - 1000.0) < 1e-9
    assert np.all(np.diff(s.imag) > 0)
    assert afs.fit_orders(30) == (15, 13)
    assert afs.fit_orders(16) == (8, 6)


def test_afs_on_rational_response_is_exact():
    poles, R = _rational()
    T = 0.04
    eta = 3 * math.log(10) / T
    res = afs.run(lambda s: vf.evaluate(s, poles, R), eta, 6000.0, T, orf=[0, 1, 2, 3],
                  test=[4, 5], J0=8)
    exact = vf.time_response(res.t, poles, R)
    assert np.abs(res.h - exact).max() < 1e-9 * np.abs(exact).max()
    # an FSM of the same band with the same period needs Omega T / pi + 1 = 77 solves
    assert len(res.s) < 6000.0 * T / math.pi + 1
    assert res.E1[-1] < 1e-4 and res.E2[-1] < 2e-3


def test_afs_on_cavity_closed_form():
    m = W.CAVITY_MATERIAL
    ur = lambda s: np.repeat(CF.cavity_ur(s, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)[:, None], 2, axis=1)
    res = afs.run(ur, 250.0, 63 * math.pi / 0.02, 0.02, orf=[0], test=[1], J0=8)
    ex = CF.cavity_ur_time(res.t, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    assert np.abs(res.h[:, 1] - ex).max() < 1e-8 * np.abs(ex).max()
    assert len(res.s) < 64


def test_pick_new_several_frequencies():
    """The batch variant's selection: the first pick is the paper's s_new (argmax away from
    samples); further picks mask +-Omega/(2J) around earlier ones and stop below 0.1 of the first."""
    omega = 1000.0
    grid = 10.0 + 1j * np.linspace(0.0, omega, 1001)
    w = grid.imag
    d = (1.0 * np.exp(-((w - 300) / 20) ** 2) + 0.5 * np.exp(-((w - 700) / 20) ** 2)
         + 0.3 * np.exp(-((w - 320) / 5) ** 2) + 0.05 * np.exp(-((w - 900) / 20) ** 2))
    s = 10.0 + 1j * np.array([0.0, 500.0, 1000.0, 300.0])      # a sample sits on the top peak
    one = afs.pick_new(grid, d, s, omega, batch=1)
    # the top peak at 300 sits on a sample (skipped within 1.5 spacings): the argmax elsewhere
    assert len(one) == 1
    ref = d.copy()
    ref[np.abs(w[:, None] - s.imag[None, :]).min(axis=1) < 1.5] = -1
    assert one == [int(np.argmax(ref))]
    many = afs.pick_new(grid, d, s, omega, batch=4)
    assert many[0] == one[0]
    half = omega / (2 * len(s))
    for a in range(len(many)):
        assert d[many[a]] >= 0.1 * d[many[0]]
        for b in range(a):
            assert abs(w[many[a]] - w[many[b]]) > half
    assert not any(abs(w[g] - 900) < 50 for g in many)          # below 0.1 of the first pick


@pytest.mark.parametrize("batch", [2, 4])
def test_afs_several_new_frequencies_per_step(batch):
    poles, R = _rational()
    T = 0.04
    eta = 3 * math.log(10) / T
    res = afs.run(lambda s: vf.evaluate(s, poles, R), eta, 6000.0, T, orf=[0, 1, 2, 3],
                  test=[4, 5], J0=8, batch=batch)
    exact = vf.time_response(res.t, poles, R)
    assert np.abs(res.h - exact).max() < 1e-9 * np.abs(exact).max()
    assert len(res.s) < 6000.0 * T / math.pi + 1
    assert len(np.unique(np.round(res.s.imag, 9))) == len(res.s)
    m = W.CAVITY_MATERIAL
    ur = lambda s: np.repeat(CF.cavity_ur(s, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)[:, None], 2, axis=1)
    res = afs.run(ur, 250.0, 63 * math.pi / 0.02, 0.02, orf=[0], test=[1], J0=8, batch=batch)
    ex = CF.cavity_ur_time(res.t, 1.0, m.mu, m.nu, m.rho, W.CAVITY_P0)
    assert np.abs(res.h[:, 1] - ex).max() < 1e-8 * np.abs(ex).max()
    assert len(res.s) < 64


# ---------------------------------------------------------------------------------------------
# A finite elastic body: undamped modes (poles on the imaginary axis) and the step pole at 0.
# Sec. 2.2 sets the sampling abscissa eta = kappa ln(10) / T with kappa in [2, 3] (kappa = 3 in
# Sec. 4); the fitted time response of Eq. (vf-td) carries e^{a t} for every pole left of the
# line, so a pole misplaced by the data's noise at 0 < Re a < eta grows by up to e^{eta T} over
# the window.  With kappa = 3 (e^{eta T} = 1e3) AFS converges on data with 1e-7 relative noise;
# with eta T = 25 (e^{eta T} ~ 7e10) the same data keep E1 large and AFS reaches its cap.
UNDAMPED = np.array([1760.0, 2090.0, 3390.0, 3850.0, 5200.0, 6100.0])


def _undamped_body(seed=3):
    rng = np.random.default_rng(seed)
    rm = (rng.standard_normal((len(UNDAMPED), 3)) + 1j * rng.standard_normal((len(UNDAMPED), 3))) * 0.1
    r0 = rng.standard_normal(3)

    def f_s(s):
        s = np.asarray(s)[:, None]
        out = r0[None, :] / s + 0j
        for w, r in zip(UNDAMPED, rm):
            out = out + r[None, :] / (s - 1j * w) + np.conj(r)[None, :] / (s + 1j * w)
        return out

    def f_t(t):
        t = np.asarray(t)[:, None]
        out = np.repeat(r0[None, :], len(t), 0)
        for w, r in zip(UNDAMPED, rm):
            out = out + 2.0 * np.real(r[None, :] * np.exp(1j * w * t))
        return out

    return f_s, f_t


def _noisy(f_s, level, seed=5):
    rng = np.random.default_rng(seed)

    def solve(sl):
        f = f_s(sl)
        return f * (1.0 + level * (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)))

    return solve


def test_afs_on_undamped_body_needs_the_papers_damping():
    f_s, f_t = _undamped_body()
    P, omega = 0.1, 63 * math.pi / 0.05
    t = np.linspace(0.0, P, 400)
    eta = fsm.eta_from_kappa(3.0, P)
    res = afs.run(_noisy(f_s, 1e-7), eta, omega, P, orf=[0, 1, 2], test=[0, 1, 2], J0=8, max_samples=60)
    assert len(res.s) < 60 and res.E1[-1] < 1e-4 and res.E2[-1] < 2e-3
    h = vf.time_response(t, res.poles, res.R, eta)
    assert np.abs(h - f_t(t)).max() < 5e-3 * np.abs(f_t(t)).max()
    # eta T = 25: same data model, no convergence within the cap, a transient off by far more
    res2 = afs.run(_noisy(f_s, 1e-7), 250.0, omega, P, orf=[0, 1, 2], test=[0, 1, 2], J0=8, max_samples=60)
    assert len(res2.s) == 60 and res2.E1[-1] > 1e-4
    h2 = vf.time_response(t, res2.poles, res2.R, 250.0)
    assert np.abs(h2 - f_t(t)).max() > 10 * np.abs(h - f_t(t)).max()


def test_relocated_pole_is_kept_off_the_samples():
    s = 69.0 + 1j * np.linspace(0.0, 4000.0, 9)
    gap = vf.SAMPLE_GAP * 4000.0
    pairs, reals = vf.keep_off_samples(s, np.array([s[3] + 0.1 * gap, 10.0 + 700j]),
                                       np.array([69.0 - 0.3 * gap, -5.0]), 4000.0)
    assert pairs[0] == s[3] - gap and pairs[1] == 10.0 + 700j
    assert reals[0] == 69.0 - gap and reals[1] == -5.0
