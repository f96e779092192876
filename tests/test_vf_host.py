"""The library's host vector fitting (C++, FP64: fast per-response QR elimination, Householder
least squares, Hessenberg + Francis QR eigenvalues) against the oracle's vector fitting
(full least squares with numpy, numpy eigenvalues).  Runs on the CPU: VF is host code.

Poles are compared directly where the data are exactly rational (they are then unique); on other
data only the fitted responses are compared (poles of an approximate fit are not unique)."""
import numpy as np
import pytest

import workloads as W
from oracle import closed_form as CF, vf

MODES = np.array([-40 + 400j, -60 + 1100j, -90 + 2300j, -120 + 3700j, -150 + 5200j])


def _P():
    import paper_1511_04355_gb300 as P
    try:
        P.load_library()
    except ImportError:
        pytest.skip("library not built")
    return P


def _rational(K=5, seed=2):
    rng = np.random.default_rng(seed)
    poles = np.concatenate([MODES, np.conj(MODES), [-300.0 + 0j]])
    R = rng.standard_normal((K, 5)) + 1j * rng.standard_normal((K, 5))
    return poles, np.hstack([R, np.conj(R), rng.standard_normal((K, 1)) + 0j])


def _sorted(p):
    return p[np.lexsort((p.real, p.imag))]


def test_host_vf_recovers_rational_poles():
    P = _P()
    poles, R = _rational()
    s = 250 + 1j * np.linspace(0, 6000, 50)
    F = vf.evaluate(s, poles, R)
    p, Rr = P.bem_vf_fit(s, F, 11, 6000.0, fit_cols=[0, 1, 2])
    assert np.abs(_sorted(p) - _sorted(poles)).max() < 1e-8 * np.abs(poles).max()
    assert np.abs(P.bem_vf_eval(p, Rr, s) - F).max() < 1e-10 * np.abs(F).max()
    po, Ro = vf.fit(s, F[:, :3], 11, 6000.0)
    assert np.abs(_sorted(p) - _sorted(po)).max() < 1e-8 * np.abs(poles).max()


def test_host_vf_matches_oracle_responses_on_cavity():
    P = _P()
    m = W.CAVITY_MATERIAL
    s = W.fsm_frequencies(0.02, 250.0, 40)
    F = np.stack([CF.cavity_ur(s, a, m.mu, m.nu, m.rho, W.CAVITY_P0) for a in (1.0, 0.7)], axis=1)
    for M in (4, 9):
        p, Rr = P.bem_vf_fit(s, F, M, s[-1].imag)
        po, Ro = vf.fit(s, F, M, s[-1].imag)
        grid = 250 + 1j * np.linspace(0, s[-1].imag, 300)
        fa, fb = P.bem_vf_eval(p, Rr, grid), vf.evaluate(grid, po, Ro)
        assert np.abs(fa - fb).max() < 1e-7 * np.abs(fb).max(), M
        t = np.linspace(0, 0.01, 50)
        ha, hb = P.bem_vf_time(p, Rr, t), vf.time_response(t, po, Ro)
        assert np.abs(ha - hb).max() < 1e-6 * np.abs(hb).max(), M


def test_host_vf_errors():
    P = _P()
    with pytest.raises(P.BemError):
        P.bem_vf_fit(np.array([250 + 0j, 250 + 1j]), np.ones((2, 1)), 5, 10.0)   # M > J


def test_host_vf_threaded_size_recovers_poles_and_is_deterministic():
    """A fit large enough for the per-response eliminations to run on host threads
    (160 samples, 6 responses, 49 poles): exact pole recovery on rational data, the oracle's
    poles, and bit-identical results on a repeat."""
    P = _P()
    rng = np.random.default_rng(5)
    modes = -(30 + 120 * rng.random(24)) + 1j * np.sort(rng.uniform(200, 7800, 24))
    poles = np.concatenate([modes, np.conj(modes), [-400.0 + 0j]])
    R = rng.standard_normal((6, 24)) + 1j * rng.standard_normal((6, 24))
    R = np.hstack([R, np.conj(R), rng.standard_normal((6, 1)) + 0j])
    s = 250 + 1j * np.linspace(0, 8000, 160)
    F = vf.evaluate(s, poles, R)
    p1, R1 = P.bem_vf_fit(s, F, 49, 8000.0)
    p2, R2 = P.bem_vf_fit(s, F, 49, 8000.0)
    assert np.array_equal(p1, p2) and np.array_equal(R1, R2)
    assert np.abs(_sorted(p1) - _sorted(poles)).max() < 1e-6 * np.abs(poles).max()
    assert np.abs(P.bem_vf_eval(p1, R1, s) - F).max() < 1e-9 * np.abs(F).max()
    po, _ = vf.fit(s, F, 49, 8000.0)
    assert np.abs(_sorted(p1) - _sorted(po)).max() < 1e-6 * np.abs(poles).max()
