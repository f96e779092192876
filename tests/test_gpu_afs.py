"""GPU AFS (Sec. 3, Algorithm AFS) through the C ABI.

* On the 80-triangle cavity, the library's AFS (host driver, host VF, batched GPU solves) and
  the oracle's AFS (numpy VF, dense-LU BEM) sample almost the same number of frequencies and
  return the same transients (the two VF implementations differ only in rounding, but the
  greedy frequency choice can take another branch on ties, so N_c is compared within a margin),
  with one new frequency per step (the paper's algorithm) and with four.
* On the 320-triangle cavity, the AFS transient of the radial displacement agrees with the FSM
  transient of the same discretisation (64 frequencies) away from the step.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import afs as OA, bem as OB

pytestmark = pytest.mark.gpu


def _P():
    import paper_1511_04355_gb300 as P
    return P


def _ctx(level):
    P = _P()
    prob = W.spherical_cavity(level=level)
    m = prob.material
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    c.set_options(precision=P.BEM_PREC_MIXED, tol=1e-9)
    return c, prob


@pytest.mark.parametrize("batch", [1, 4])
def test_afs_matches_oracle_afs(batch):
    """batch = 1 is the paper's algorithm; batch = 4 the variant that adds up to four
    frequencies per step, solved in one batch (the same rule in both implementations)."""
    P = _P()
    c, prob = _ctx(1)
    T, eta = 0.02, 250.0
    omega = 32 * math.pi / T
    orf = [0, 4, 100, 161]
    test = [50, 230]
    cap = 60 if batch == 1 else 150
    prm = P.bem_default_afs_params(eta=eta, omega_max=omega, T=T, J0=8, max_samples=cap, batch=batch)
    t = np.linspace(0, 0.01, 100)
    out, info = c.afs(prm, orf, test, t)
    g = OB.geometry(prob.verts, prob.tris)
    m = prob.material
    dofs = orf + test

    def solve(s):
        return np.stack([OB.solve(g, sk, m, prob.bc_type, prob.bc_value)[0][dofs] for sk in s])

    ref = OA.run(solve, eta, omega, T, orf=[0, 1, 2, 3], test=[4, 5], J0=8, max_samples=cap, batch=batch)
    print("AFS samples (library, oracle), batch", batch, ":", info["n_samples"], len(ref.s))
    if batch == 1:
        assert abs(info["n_samples"] - len(ref.s)) <= 4, (info["n_samples"], len(ref.s))
    else:
        # several picks per step make the sample sequence sensitive to rounding-level differences
        # between the two VF implementations: both must converge below the cap, N_c is reported
        assert info["n_samples"] < cap and len(ref.s) < cap, (info["n_samples"], len(ref.s))
        assert ref.E1[-1] < 1e-4 and ref.E2[-1] < 2e-3
    from oracle import vf
    h_ref = vf.time_response(t, ref.poles, ref.R, eta)
    if batch == 1:
        scale = np.abs(h_ref).max(axis=0)
        assert (np.abs(out - h_ref).max(axis=0) / scale).max() < 2e-3
    else:
        # different sample sets: compare in the L2 sense AFS controls (E1-type, thresholds
        # 1e-4 on the squared ratio -> 1e-2 on the ratio)
        rel = np.sqrt(np.trapezoid((out - h_ref) ** 2, t, axis=0) / np.trapezoid(h_ref ** 2, t, axis=0))
        assert rel.max() < 1e-2, rel
    assert info["E1"][-1] < 1e-4 and info["E2"][-1] < 2e-3


def test_afs_agrees_with_fsm_on_small_configuration():
    P = _P()
    c, prob = _ctx(2)
    T = prob.T
    ne = len(prob.tris)
    dofs = np.array([0, 1, 2, 3 * 100, 3 * 200 + 1, 3 * 319 + 2])
    t = np.linspace(0, 0.01, 200)
    fsm_out, _ = c.fsm(2 * T, prob.sigma, 64, t, dofs)
    prm = P.bem_default_afs_params(eta=prob.sigma, omega_max=63 * math.pi / T, T=2 * T, J0=8,
                                   max_samples=60)
    afs_out, info = c.afs(prm, dofs[:4], dofs[4:], t)
    late = t > 2e-3
    scale = np.abs(fsm_out).max(axis=0)
    err = (np.abs(afs_out[late] - fsm_out[late]).max(axis=0) / scale).max()
    assert err < 0.02, err
    assert info["n_samples"] < 64
