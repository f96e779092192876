"""The warm start inside AFS (Sec. 3, Algorithm AFS: each adaptive step solves one new frequency
next to the frequencies already solved), through bem_afs.

For each workload bem_afs runs four times, with the context's warm_start set to ZERO (GMRES
from x0 = 0), NEAREST (the stored solution at the nearest sampled frequency), MLP (the POD +
MLP prediction, retrained every 4 samples, combined with the nearest solution by minimal
residual) and VF (the rational prediction of every unknown from the step's fitted poles,
combined with the nearest solution the same way).
The warm start may change the GMRES iterations only: every run must sample the same number of
frequencies (within 2, since the greedy choice can take another branch on rounding-level
differences of the solutions) and return the same transients (within 2e-3 of the largest
response), and each must converge.  The per-solve iterations and times of the adaptive stage
are printed; the test asserts that the warm starts do not cost iterations in that stage.

Workloads: the 320-triangle cavity (mixed path, tol 1e-9) and the prismatic rod of Example 1
(1792 triangles, mixed path, tol 1e-6, GMRES(200)), whose upper frequencies need hundreds of
iterations from a zero start.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fsm as OF

pytestmark = pytest.mark.gpu


def _P():
    import paper_1511_04355_gb300 as P
    return P


def _cavity():
    P = _P()
    prob = W.spherical_cavity(level=2)
    m = prob.material
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    opts = dict(precision=P.BEM_PREC_MIXED, tol=1e-9)
    dofs = np.array([0, 1, 2, 3 * 100, 3 * 200 + 1, 3 * 319 + 2])
    T = prob.T
    prm = dict(eta=prob.sigma, omega_max=63 * math.pi / T, T=2 * T, J0=8, max_samples=60)
    return c, opts, dofs[:4], dofs[4:], prm, np.linspace(0, 0.01, 200)


def _rod():
    P = _P()
    rod = W.prismatic_rod()
    m = rod["material"]
    c = P.Context(0)
    c.set_mesh(rod["verts"], rod["tris"])
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(rod["bc_type"], rod["bc_value"], P.BEM_PROFILE_STEP)
    opts = dict(precision=P.BEM_PREC_MIXED, tol=1e-6, restart=200, max_iters=4000, max_refine=20)
    face = rod["face"]
    end = np.flatnonzero(face == 1)
    side = np.flatnonzero(face == 2)
    orf = [int(3 * end[len(end) // 2]), int(3 * side[len(side) // 3]), int(3 * side[len(side) // 2] + 1),
           int(3 * end[0] + 1), int(3 * side[2 * len(side) // 3])]
    test = [int(3 * end[len(end) // 4]), int(3 * side[len(side) // 4])]
    T = 0.0155
    prm = dict(eta=OF.eta_from_kappa(3.0, T), omega_max=109 * 2 * math.pi / T, T=T, J0=16, max_samples=110)
    return c, opts, orf, test, prm, np.linspace(0.0, 0.6 * T, 300)


@pytest.mark.parametrize("case", ["cavity320", "rod1792"])
def test_afs_warm_start_modes(case):
    P = _P()
    c, opts, orf, test, prm, t = _cavity() if case == "cavity320" else _rod()
    runs = {}
    for name, mode in (("zero", P.BEM_WARM_ZERO), ("nearest", P.BEM_WARM_NEAREST), ("mlp", P.BEM_WARM_MLP),
                       ("vf", P.BEM_WARM_VF)):
        c.set_options(warm_start=mode, **opts)
        p = P.bem_default_afs_params(**prm)
        out, info = c.afs(p, orf, test, t)
        runs[name] = (out, info)
        J0 = p.J0
        it = info["gmres_iters"]
        print(f"{case} {name}: N_c {info['n_samples']}, GMRES iterations initial {int(it[:J0].sum())} "
              f"adaptive {int(it[J0:].sum())} (mean {it[J0:].mean():.1f}), solve {info['seconds_solve']:.2f} s, "
              f"fit {info['seconds_fit']:.2f} s, train {info['seconds_train']:.2f} s "
              f"({info['warm_trainings']} trainings, {info['warm_learned_gains']} solves where the network's "
              f"direction helped)")
        print(f"{case} {name} per-solve iterations: {it.tolist()}")
        assert info["E1"][-1] < prm.get("E1bar", 1e-4) and info["E2"][-1] < 2e-3
        assert info["n_samples"] < prm["max_samples"]
    out0, info0 = runs["zero"]
    scale = np.abs(out0).max(axis=0)
    for name in ("nearest", "mlp", "vf"):
        out, info = runs[name]
        assert abs(info["n_samples"] - info0["n_samples"]) <= 2, (name, info["n_samples"], info0["n_samples"])
        err = (np.abs(out - out0).max(axis=0) / scale).max()
        assert err < 2e-3, (name, err)
    # the warm starts exist to save iterations in the adaptive stage: per adaptive solve they must
    # not cost more than the zero start
    J0 = prm["J0"]
    per = {k: runs[k][1]["gmres_iters"][J0:].mean() for k in runs}
    print(f"{case} mean adaptive-stage iterations per solve: {per}")
    assert per["nearest"] <= per["zero"] and per["mlp"] <= per["zero"] and per["vf"] <= per["zero"], per
    assert runs["mlp"][1]["warm_trainings"] >= 2
