"""GPU parity of the H-matrix far field (csrc/hmatrix.cu) against the FP64 oracle.

The fast operator approximates the 4-point far-field part of the FP32 operator; its result is
the operator A(s) x, which has a plain definition: the oracle's dense assembly.  Checks:
  * the device partition statistics equal the host partition (bit-exact against the oracle in
    the CPU tests);
  * y = A x with the H-matrix far field against the oracle's dense A rows, elementwise
    (every entry against the largest |y|), and against the direct FP32 far kernel in the
    2-norm within 10 eps, on a porous block with traction- and displacement-given columns, at
    about 480, 1760 and 5920 triangles (blocks of up to 512 elements, ragged leaves);
  * a mixed solve whose inner operator is the H-matrix, certified by the exact float-float
    residual: the same discrete solution as the oracle's dense LU (1e-6 elementwise per kind of
    unknown at tol 1e-9);
  * frequency chunking (max_freqs) gives the same solutions as one batch.
"""
import functools
import math

import numpy as np
import pytest

import workloads as W
from _parity import max_rel_err
from oracle import bem as OB

pytestmark = pytest.mark.gpu

PERIOD = 0.04
ETA = 3.0 * math.log(10.0) / PERIOD
S_LOW = ETA + 1j * np.array([0.0, 3.0, 7.0]) * 2.0 * math.pi / PERIOD


def _P():
    import paper_1511_04355_gb300 as P
    return P


@functools.lru_cache(maxsize=None)
def _block(n=4, voids=2):
    return W.porous_block(L=(2.0, 1.0, 1.0), n=(2 * n, n, n), n_voids=voids, radii=(0.08, 0.1), void_level=1)


def _ctx(pb, **opt):
    P = _P()
    m = pb["material"]
    c = P.Context(0)
    c.set_mesh(pb["verts"], pb["tris"])
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(pb["bc_type"], pb["bc_value"], P.BEM_PROFILE_STEP)
    if opt:
        c.set_options(**opt)
    return c


def _x(pb, ns, seed=11):
    rng = np.random.default_rng(seed)
    ne = len(pb["tris"])
    x = rng.standard_normal((ns, 3 * ne)) + 1j * rng.standard_normal((ns, 3 * ne))
    # traction unknowns (displacement-given elements) at the scale of the stresses that the
    # displacement unknowns cause (mu times a unit strain)
    return x * np.repeat(np.where(pb["bc_type"] == 1, pb["material"].mu, 1.0), 3)


def test_partition_statistics_match_the_host_partition():
    P = _P()
    pb = _block(8, 6)
    c = _ctx(pb)
    c.set_hmatrix(True, leaf=16, eta=2.0, max_block=512)
    info = c.hmatrix_info()
    perm, cl, lr, dn = P.bem_hmatrix_partition(pb["verts"], pb["tris"],
                                               P.bem_default_hmatrix_params(leaf=16, eta=2.0, max_block=512))
    assert info["clusters"] == len(cl) and info["lowrank_blocks"] == len(lr) and info["dense_blocks"] == len(dn)
    sizes = cl[:, 1].astype(np.int64)
    assert info["lowrank_pairs"] + info["dense_pairs"] == len(pb["tris"]) ** 2
    assert info["lowrank_pairs"] == int((sizes[lr[:, 0]] * sizes[lr[:, 1]]).sum())


@pytest.mark.parametrize("n,voids,eps", [(4, 2, 1e-4), (8, 6, 1e-4), (8, 6, 1e-5), (16, 10, 1e-4)])
def test_hmatrix_apply_matches_the_oracle_operator(n, voids, eps):
    P = _P()
    pb = _block(n, voids)
    ne = len(pb["tris"])
    x = _x(pb, len(S_LOW))
    c = _ctx(pb)
    y32 = c.apply(S_LOW, x, precision=P.BEM_PREC_FP32)
    c.set_hmatrix(True, leaf=16, eta=2.0, max_block=512, eps=eps, max_rank=128)
    yh = c.apply(S_LOW, x, precision=P.BEM_PREC_FP32)
    info = c.hmatrix_info()
    assert info["builds"] == 1 and info["frequencies"] == len(S_LOW) and info["capped"] == 0
    assert 0 < info["rank_max"] <= 128 and info["factor_bytes"] > 0
    # against the direct FP32 far kernel: only the far-field approximation differs
    for f in range(len(S_LOW)):
        assert np.linalg.norm(yh[f] - y32[f]) <= (10 * eps + 2e-6) * np.linalg.norm(y32[f]), f
    # against the oracle's dense operator rows, elementwise
    g = OB.geometry(pb["verts"], pb["tris"])
    rows = np.unique(np.concatenate([np.arange(0, ne, max(1, ne // 24)), [ne - 1]]))
    for f, s in enumerate(S_LOW):
        A, _ = OB.operators(g, s, pb["material"], pb["bc_type"], rows=rows)
        yr = A @ x[f]
        got = yh[f].reshape(ne, 3)[rows].reshape(-1)
        err = np.abs(got - yr).max() / np.abs(yr).max()
        assert err <= 20 * eps + 1e-5, (f, err)


def test_mixed_solve_with_hmatrix_inner_operator_matches_lu():
    P = _P()
    pb = _block(4, 2)
    g = OB.geometry(pb["verts"], pb["tris"])
    S = S_LOW[[0, 2]]
    c = _ctx(pb, precision=P.BEM_PREC_MIXED, tol=1e-9, max_refine=20)
    c.set_hmatrix(True, leaf=16, eta=2.0, max_block=512, eps=1e-4)
    x, info = c.solve(S)
    assert (info["status"] == 0).all() and (info["residual"] <= 1e-9).all()
    for f, s in enumerate(S):
        A, b = OB.assemble(g, s, pb["material"], pb["bc_type"], pb["bc_value"])
        xr = np.linalg.solve(A, b)
        assert max_rel_err(x[f], xr, pb["bc_type"]) <= 1e-6, f
    assert c.hmatrix_info()["builds"] >= 1


def test_frequency_chunks_give_the_batch_solution():
    P = _P()
    pb = _block(8, 6)
    S = ETA + 1j * np.arange(4) * 2.0 * math.pi / PERIOD
    c = _ctx(pb, precision=P.BEM_PREC_MIXED, tol=1e-8, max_refine=20)
    c.set_hmatrix(True, leaf=16, eta=2.0, max_block=512, eps=1e-4)
    x1, i1 = c.solve(S)
    assert c.hmatrix_info()["frequencies"] == 4
    c.set_hmatrix(True, leaf=16, eta=2.0, max_block=512, eps=1e-4, max_freqs=2)
    x2, i2 = c.solve(S)
    info = c.hmatrix_info()
    assert info["frequencies"] == 2 and info["builds"] == 2
    assert (i1["status"] == 0).all() and (i2["status"] == 0).all()
    for f in range(4):
        assert max_rel_err(x2[f], x1[f], pb["bc_type"]) <= 1e-6, f


def test_disabling_restores_the_direct_operator():
    P = _P()
    pb = _block(4, 2)
    x = _x(pb, 1)
    c = _ctx(pb)
    y0 = c.apply(S_LOW[:1], x, precision=P.BEM_PREC_FP32)
    c.set_hmatrix(True, leaf=16, eps=1e-2)
    yh = c.apply(S_LOW[:1], x, precision=P.BEM_PREC_FP32)
    c.set_hmatrix(False)
    y1 = c.apply(S_LOW[:1], x, precision=P.BEM_PREC_FP32)
    # the direct kernel sums with FP64 atomics: equal up to the order of those additions
    assert np.linalg.norm(y1 - y0) <= 1e-6 * np.linalg.norm(y0)
    assert np.linalg.norm(yh - y0) > 1e-5 * np.linalg.norm(y0)
