"""GPU parity on a small porous block (the porous-solid workloads' recipe at test size): a unit
box surface of 108 triangles with two level-1 spherical voids (268 triangles), traction on
z = 0, z = 1 fixed (displacement given), every other surface traction-free, so traction- and
displacement-given columns, box edges and corners, and several disjoint surfaces all appear.

* plain FP64 path at tol 1e-12 == the oracle's dense LU to 1e-10, elementwise (each entry
  against the largest LU entry of its kind: displacement or traction unknown);
* mixed path at tol 1e-9 == LU to 1e-6 in the same sense; at the benchmark tolerance 1e-6 the
  FP64-class residual the solver reports agrees with the oracle's dense residual of the
  returned solution.
"""
import functools

import numpy as np
import pytest

import workloads as W
from _parity import max_rel_err
from oracle import bem as OB

pytestmark = pytest.mark.gpu

S_SET = 250.0 + 1j * np.array([0.0, 2513.3, 9424.8])


def _P():
    import paper_1511_04355_gb300 as P
    return P


@functools.lru_cache(maxsize=None)
def _case():
    pb = W.porous_block(L=(1.0, 1.0, 1.0), n=(3, 3, 3), n_voids=2, void_level=1)
    g = OB.geometry(pb["verts"], pb["tris"])
    sols = []
    for s in S_SET:
        A, b = OB.assemble(g, s, pb["material"], pb["bc_type"], pb["bc_value"])
        sols.append((np.linalg.solve(A, b), A, b))
    return pb, sols


def _ctx(**opt):
    P = _P()
    pb, _ = _case()
    m = pb["material"]
    c = P.Context(0)
    c.set_mesh(pb["verts"], pb["tris"])
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(pb["bc_type"], pb["bc_value"], P.BEM_PROFILE_STEP)
    c.set_options(**opt)
    return c


def test_porous_block_size():
    pb, _ = _case()
    assert len(pb["tris"]) == 268 and (pb["bc_type"] == 1).sum() == 18


def test_fp64_solve_matches_lu():
    P = _P()
    _, sols = _case()
    x, info = _ctx(precision=P.BEM_PREC_FP64, tol=1e-12).solve(S_SET)
    assert (info["status"] == 0).all()
    for f, (xr, _, _) in enumerate(sols):
        assert max_rel_err(x[f], xr, _case()[0]["bc_type"]) <= 1e-10, f


def test_mixed_solve_matches_lu():
    P = _P()
    _, sols = _case()
    x, info = _ctx(precision=P.BEM_PREC_MIXED, tol=1e-9).solve(S_SET)
    assert (info["status"] == 0).all()
    for f, (xr, _, _) in enumerate(sols):
        # every entry against the largest of its kind (displacement or traction unknowns)
        assert max_rel_err(x[f], xr, _case()[0]["bc_type"]) <= 1e-6, f
    x, info = _ctx(precision=P.BEM_PREC_MIXED, tol=1e-6).solve(S_SET)
    for f, (_, A, b) in enumerate(sols):
        rel = np.linalg.norm(b - A @ x[f]) / np.linalg.norm(b)
        assert rel <= 1e-6 and abs(rel - info["residual"][f]) <= 1e-9, (f, rel, info["residual"][f])
