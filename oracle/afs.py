"""Adaptive frequency sampling (oracle, FP64, test infrastructure only).

Sec. 3 of the paper (Algorithm AFS), written over a callback `solve(s_list) -> responses`
(the BEM solve restricted to the observed unknowns; a rational test function in the pins):

  initialisation  J0 Chebyshev frequencies s_j = eta + i Omega [1 - cos(j pi / (2 (J0 - 1)))]
                  (the printed cosine argument lacks the pi; read as above), solved;
  each step       fits of orders M_H = floor(J / alpha_H), M_L = floor(J / alpha_L)
                  (Eq. (fit-ords)) to the observation responses (ORFs); residues of every
                  observed unknown with the common poles; the relative discrepancy
                  e_k = max |f_kH - f_kL| / max |f_kH| over s in [0, Omega] (Eq. (ferr));
                  s_new = argmax |f_kmax,H - f_kmax,L| for the ORF with the largest e_k
                  (Eqs. (snew), (snew1));
                  E1 = max_k int (f^(i) - f^(i-1))^2 dt / int (f^(i))^2 dt over the test
                  unknowns (Eq. (stop-E1), E1^(0) = inf) with the time responses of the M_H fit;
                  E2 = max_k e_k over the test unknowns (Eq. (stop-E2));
  convergence     stop once E1 < E1bar and E2 < E2bar hold at a step and at the J_c steps that
                  follow (Eq. (converge) with the validation stage);
  post-processing time responses by Eq. (vf-td) with the final M_H fit.
Time responses (for E1 and the output) sum Eq. (vf-td) over the fitted poles left of the
sampling line Re s = eta only (the Bromwich contour of Eq. (invLap)); see vf.time_response.
Readings where the paper is silent: the search for s_new runs over n_grid uniform frequencies in
[0, Omega] and skips grid points within 1.5 grid spacings of an existing sample; each ORF is
scaled by its largest sampled magnitude before pole identification; the integrals of E1 are
trapezoidal sums on a uniform grid of nt times in [0, T].

Several new frequencies per step (batch > 1; a variant, not the paper's algorithm, which adds
one): the first is the paper's s_new; each further one is the argmax of the same discrepancy
curve after masking +-Omega / (2 J) around every frequency already picked this step (J = the
number of samples before the step), kept only while its discrepancy is at least 0.1 of the first
pick's; all of them are solved together.  batch = 1 is the paper's algorithm.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import vf


def chebyshev_frequencies(eta, omega_max, J0):
    j = np.arange(J0)
    return eta + 1j * omega_max * (1.0 - np.cos(j * math.pi / (2.0 * (J0 - 1))))


def fit_orders(J, alpha_H=2.0, alpha_L=2.3):
    return int(math.floor(J / alpha_H)), int(math.floor(J / alpha_L))


@dataclasses.dataclass
class AFSResult:
    s: np.ndarray            # sampled frequencies (N_c,)
    F: np.ndarray            # sampled responses (N_c, n_obs)
    poles: np.ndarray        # final M_H poles
    R: np.ndarray            # residues (n_obs, M_H)
    E1: list
    E2: list
    t: np.ndarray
    h: np.ndarray            # time responses (nt, n_obs) of the final fit


def _step(s, F, orf, eta, omega_max, grid, t, alpha_H, alpha_L, n_iter):
    J = len(s)
    MH, ML = fit_orders(J, alpha_H, alpha_L)
    scale = np.abs(F[:, orf]).max(axis=0)
    scale[scale == 0] = 1.0
    Fo = F[:, orf] / scale
    pH, _ = vf.fit(s, Fo, MH, omega_max, n_iter=n_iter)
    pL, _ = vf.fit(s, Fo, ML, omega_max, n_iter=n_iter)
    pairsH = pH[(pH.imag > 0)]
    realsH = pH[np.abs(pH.imag) == 0].real
    pairsL = pL[(pL.imag > 0)]
    realsL = pL[np.abs(pL.imag) == 0].real
    polesH, RH = vf.residues(s, F, pairsH, realsH)
    polesL, RL = vf.residues(s, F, pairsL, realsL)
    fH = vf.evaluate(grid, polesH, RH)
    fL = vf.evaluate(grid, polesL, RL)
    diff = np.abs(fH - fL)
    e = diff.max(axis=0) / np.maximum(np.abs(fH).max(axis=0), 1e-300)
    h = vf.time_response(t, polesH, RH, eta)
    return polesH, RH, e, diff, h


def pick_new(grid, d, s, omega_max, batch=1):
    """Indices of the new frequencies on the search grid from the discrepancy curve d of the
    ORF with the largest e_k: the argmax over grid points more than 1.5 spacings from every
    sample, then (batch > 1) further argmaxes after masking +-Omega/(2J) around each pick."""
    dgrid = omega_max / (len(grid) - 1)
    d = np.array(d, dtype=float)
    taken = np.abs(grid.imag[:, None] - np.asarray(s).imag[None, :]).min(axis=1) < 1.5 * dgrid
    d[taken] = -1.0
    picks = [int(np.argmax(d))]
    first = d[picks[0]]
    half = omega_max / (2.0 * len(s))
    while len(picks) < batch:
        d[np.abs(grid.imag - grid.imag[picks[-1]]) <= half] = -1.0
        g = int(np.argmax(d))
        if d[g] < 0.1 * first or d[g] < 0:
            break
        picks.append(g)
    return picks


def run(solve, eta, omega_max, T, orf, test, J0=16, alpha_H=2.0, alpha_L=2.3, E1bar=1e-4,
        E2bar=2e-3, Jc=3, n_grid=4096, nt=512, max_samples=400, n_iter=20, batch=1):
    """orf, test: column indices into the responses returned by solve."""
    orf = np.asarray(orf)
    test = np.asarray(test)
    s = chebyshev_frequencies(eta, omega_max, J0)
    F = np.asarray(solve(s))
    grid = eta + 1j * np.linspace(0.0, omega_max, n_grid)
    t = np.linspace(0.0, T, nt)
    E1s, E2s = [], []
    h_prev = None
    ok_run = 0
    while True:
        polesH, RH, e, diff, h = _step(s, F, orf, eta, omega_max, grid, t, alpha_H, alpha_L, n_iter)
        if h_prev is None:
            E1 = math.inf
        else:
            num = np.trapezoid((h[:, test] - h_prev[:, test]) ** 2, t, axis=0)
            den = np.trapezoid(h[:, test] ** 2, t, axis=0)
            E1 = float(np.max(num / np.maximum(den, 1e-300)))
        E2 = float(np.max(e[test]))
        E1s.append(E1)
        E2s.append(E2)
        h_prev = h
        ok_run = ok_run + 1 if (E1 < E1bar and E2 < E2bar) else 0
        if ok_run >= Jc + 1 or len(s) >= max_samples:
            return AFSResult(s=s, F=F, poles=polesH, R=RH, E1=E1s, E2=E2s, t=t, h=h)
        kmax = orf[np.argmax(e[orf])]
        picks = pick_new(grid, diff[:, kmax], s, omega_max, min(batch, max_samples - len(s)))
        s_new = grid[picks]
        s = np.append(s, s_new)
        F = np.vstack([F, np.asarray(solve(s_new))])
