"""Vector fitting (oracle, FP64, test infrastructure only).

Sec. 2.3, Eq. (vf-f): the K sampled responses f_k(s_j), j = 1..J, are approximated by partial
fractions with common poles, f_k(s) = sum_m r_{k,m} / (s - a_m) (no constant or linear term, as
in the paper), by the two steps the paper describes:

* pole identification: with the current poles abar_m, the linear least-squares problem
      sum_m c_{k,m}/(s_j - abar_m) - f_k(s_j) sum_m ct_m/(s_j - abar_m) = f_k(s_j)   (all j, k)
  is solved for the c_k and the shared ct; the zeros of sigma(s) = 1 + sum_m ct_m/(s - abar_m)
  become the new poles (the eigenvalues of A - b ct^T in a real realisation of sigma), and this
  is repeated;
* residue identification: with the poles fixed, f_k(s_j) = sum_m r_{k,m}/(s_j - a_m) is a
  linear least-squares problem per response.
Real coefficients: a complex pole pair (a, conj a) uses the real basis
  1/(s-a) + 1/(s-conj a),  i/(s-a) - i/(s-conj a)
with real coefficients (c', c'') = residue c' + i c'' on a and its conjugate on conj a; the
real and imaginary parts of every equation are stacked, which is equivalent to fitting the
samples and their conjugates.  Unstable poles are kept (not flipped).  Initial poles: pairs
-beta/100 +- i beta with beta equally spaced over (0, Omega] (plus one real pole -Omega/100 when
M is odd).  Columns are scaled to unit norm before each least-squares solve.

Time response, Eq. (vf-td): the inverse Laplace transform of r/(s - a) is r e^{a t}, so
h(t) = sum_m r_m e^{a_m t} (the paper prints e^{-a_m t}; the sign is read as a misprint).
"""
from __future__ import annotations

import numpy as np


def initial_poles(M, omega_max):
    """M poles as (complex pair representatives with Im > 0, real poles)."""
    npair = M // 2
    beta = omega_max * np.arange(1, npair + 1) / max(npair, 1)
    pairs = -beta / 100.0 + 1j * beta
    reals = np.array([-omega_max / 100.0]) if M % 2 else np.zeros(0)
    return pairs, reals


def _basis(s, pairs, reals):
    """Real-coefficient basis Phi (J, M): per pair two columns, per real pole one."""
    s = np.asarray(s)[:, None]
    cols = []
    for a in pairs:
        cols.append(1.0 / (s - a) + 1.0 / (s - np.conj(a)))
        cols.append(1j / (s - a) - 1j / (s - np.conj(a)))
    for a in reals:
        cols.append(1.0 / (s - a))
    return np.hstack(cols) if cols else np.zeros((len(s), 0), complex)


def _ri(A):
    """Stack real and imaginary parts of the rows (complex equations -> real ones)."""
    return np.vstack([A.real, A.imag])


def _lstsq_scaled(M, rhs):
    nrm = np.linalg.norm(M, axis=0)
    nrm[nrm == 0] = 1.0
    x = np.linalg.lstsq(M / nrm, rhs, rcond=None)[0]
    return x / (nrm[:, None] if x.ndim == 2 else nrm)


def _split_poles(z, tol=1e-12):
    """Eigenvalues of a real matrix -> (pairs with Im > 0, real poles)."""
    z = np.asarray(z)
    scale = max(np.abs(z).max(), 1.0)
    real = np.abs(z.imag) <= tol * scale
    reals = np.sort(z[real].real)
    pairs = z[(~real) & (z.imag > 0)]
    return pairs[np.argsort(pairs.imag)], reals


def pole_identification(s, F, pairs, reals):
    """One relocation step: returns the new (pairs, reals)."""
    s = np.asarray(s)
    F = np.asarray(F).reshape(len(s), -1)
    J, K = F.shape
    Phi = _basis(s, pairs, reals)
    M = Phi.shape[1]
    rows = []
    rhs = []
    for k in range(K):
        blk = np.zeros((J, (K + 1) * M), complex)
        blk[:, k * M:(k + 1) * M] = Phi
        blk[:, K * M:] = -F[:, k:k + 1] * Phi
        rows.append(_ri(blk))
        rhs.append(np.concatenate([F[:, k].real, F[:, k].imag]))
    x = _lstsq_scaled(np.vstack(rows), np.concatenate(rhs))
    ct = x[K * M:]
    # real realisation of sigma(s) = 1 + ct^T (sI - A)^{-1} b
    A = np.zeros((M, M))
    b = np.zeros(M)
    c = 0
    for a in pairs:
        A[c:c + 2, c:c + 2] = [[a.real, a.imag], [-a.imag, a.real]]
        b[c] = 2.0
        c += 2
    for a in reals:
        A[c, c] = a
        b[c] = 1.0
        c += 1
    return _split_poles(np.linalg.eigvals(A - np.outer(b, ct)))


def residues(s, F, pairs, reals):
    """Residue identification: complex residues per response for the expanded pole list
    (each pair as a, conj a).  Returns (poles (M,), R (K, M))."""
    s = np.asarray(s)
    F = np.asarray(F).reshape(len(s), -1)
    Phi = _basis(s, pairs, reals)
    X = _lstsq_scaled(_ri(Phi), np.vstack([F.real, F.imag]))   # (M, K) real coefficients
    poles, R = [], []
    c = 0
    for a in pairs:
        poles += [a, np.conj(a)]
        R += [X[c] + 1j * X[c + 1], X[c] - 1j * X[c + 1]]
        c += 2
    for a in reals:
        poles.append(a + 0j)
        R.append(X[c] + 0j)
        c += 1
    return np.array(poles), np.array(R).T


SAMPLE_GAP = 1e-6   # relocated poles keep at least this fraction of Omega from every sample


def keep_off_samples(s, pairs, reals, omega_max):
    """A relocated pole closer than SAMPLE_GAP * Omega to a sample s_j is moved to s_j - SAMPLE_GAP
    * Omega (the same imaginary part, left of the sampling line): the samples lie to the right of
    the physical poles (Re s = eta > 0) and unstable poles are kept, so with noisy data an extra
    pole can settle on a sample, where the basis 1/(s - a) of the next step is infinite.  The paper
    is silent on this case."""
    s = np.asarray(s)
    gap = SAMPLE_GAP * omega_max

    def fix(a):
        sj = s[np.argmin(np.abs(s - a))]
        return sj - gap if abs(sj - a) < gap else a

    return (np.array([fix(a) for a in pairs], dtype=complex),
            np.array([np.real(fix(a)) for a in reals], dtype=float))


def fit(s, F, M, omega_max, n_iter=20, tol=1e-10, init=None):
    """Vector fit of order M: (poles (M,), residues (K, M)) with pairs expanded."""
    pairs, reals = init if init is not None else initial_poles(M, omega_max)
    for _ in range(n_iter):
        p2, r2 = pole_identification(s, F, pairs, reals)
        p2, r2 = keep_off_samples(s, p2, r2, omega_max)
        if len(p2) == len(pairs) and len(r2) == len(reals):
            change = max(np.abs(p2 - pairs).max(initial=0.0), np.abs(r2 - reals).max(initial=0.0))
            pairs, reals = p2, r2
            if change <= tol * omega_max:
                break
        else:
            pairs, reals = p2, r2
    return residues(s, F, pairs, reals)


def evaluate(s, poles, R):
    """f(s) for the fit: (len(s), K)."""
    s = np.asarray(s)[:, None]
    return (1.0 / (s - poles[None, :])) @ R.T


def time_response(t, poles, R, eta=None):
    """Eq. (vf-td): h(t) = sum_m r_m e^{a_m t}, real part (conjugate pairs sum to real).

    With eta given, the sum runs over the poles left of the sampling line Re s = eta only: the
    Bromwich integral of Eq. (invLap) along that line -- the contour the samples lie on, which
    Sec. 2.2 places to the right of every singularity -- picks up exactly those residues; a
    fitted pole right of the line lies outside the region the data describe."""
    t = np.asarray(t)[:, None]
    if eta is not None:
        keep = poles.real < eta
        poles, R = poles[keep], R[:, keep]
    return np.real(np.exp(t * poles[None, :]) @ R.T)
