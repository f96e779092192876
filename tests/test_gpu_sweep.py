"""The two-pass frequency sweep (warm_start = BEM_WARM_SWEEP) of bem_solve_frequencies: every
other frequency from a zero start, a vector fit (Sec. 2.3, Eq. (vf-f)) of order J/2 to 8
unknowns of those solutions, then the other frequencies from the fit's rational prediction of
every unknown combined with the nearest solved frequency.

The sweep changes the starting vectors only: every frequency is still certified by its FP64-class
residual at the tolerance, so the solutions agree with the zero-start batch and with the
oracle's dense LU to the accuracy that tolerance gives (elementwise, against the largest entry),
and the second pass needs fewer GMRES iterations."""
import numpy as np
import pytest

import workloads as W
from _parity import max_rel_err
from oracle import bem as OB

pytestmark = pytest.mark.gpu


def test_sweep_matches_zero_start_and_saves_iterations():
    import paper_1511_04355_gb300 as P
    prob = W.spherical_cavity(level=3, n_freq=64)
    m = prob.material
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    out = {}
    for name, mode in (("zero", P.BEM_WARM_ZERO), ("sweep", P.BEM_WARM_SWEEP)):
        c.set_options(precision=P.BEM_PREC_MIXED, tol=1e-9, warm_start=mode)
        x, info = c.solve(prob.s)
        assert (info["status"] == 0).all() and (info["residual"] <= 1e-9).all()
        out[name] = (x, info)
    xz, iz = out["zero"]
    xs, isw = out["sweep"]
    print("GMRES iterations zero / sweep:", int(iz["iterations"].sum()), int(isw["iterations"].sum()),
          "; odd frequencies:", int(iz["iterations"][1::2].sum()), int(isw["iterations"][1::2].sum()))
    for k in range(len(prob.s)):
        assert max_rel_err(xs[k], xz[k], prob.bc_type) < 1e-7, k
    # even frequencies: the same zero-start solve; odd ones: warm
    assert int(isw["iterations"][1::2].sum()) < int(iz["iterations"][1::2].sum())
    g = OB.geometry(prob.verts, prob.tris)
    for k in (1, 33, 63):
        A, b = OB.assemble(g, prob.s[k], m, prob.bc_type, prob.bc_value)
        assert max_rel_err(xs[k], np.linalg.solve(A, b), prob.bc_type) < 1e-7, k


def test_sweep_short_list_is_one_batch():
    import paper_1511_04355_gb300 as P
    prob = W.spherical_cavity(level=1, n_freq=5)
    m = prob.material
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    c.set_options(precision=P.BEM_PREC_MIXED, tol=1e-9, warm_start=P.BEM_WARM_SWEEP)
    x, info = c.solve(prob.s)
    assert (info["status"] == 0).all()
    g = OB.geometry(prob.verts, prob.tris)
    xr = OB.solve_frequencies(prob.verts, prob.tris, m, prob.bc_type, prob.bc_value, prob.s)
    for k in range(5):
        assert max_rel_err(x[k], xr[k], prob.bc_type) < 1e-6, k
