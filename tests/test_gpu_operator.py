"""GPU parity of the operator-level steps (geometry, near lists, element blocks, A x, K x, RHS,
preconditioner) against the FP64 CPU oracle, through the C ABI.

Sizes: 80 and 320 triangles (ragged against the 128-target and 64/32-source tiles), 5
frequencies (ragged against the 12- and 4-frequency tiles) including s = sigma (|z| small, the
series branch) and the top of the benchmark band; traction-given and mixed boundary conditions.
Tolerances: FP64 path 1e-10 relative (the two sides differ only in rounding order and in the
|z| threshold of the Taylor branch); FP32 operator 2e-6 elementwise against the largest entry
(float-float distances and phases, single-precision kernel algebra), the bound the benchmark-size
test uses.
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import bem as OB

pytestmark = pytest.mark.gpu

S_SET = 250.0 + 1j * np.array([0.0, 157.08, 1570.8, 4712.4, 9896.0])


def _P():
    import paper_1511_04355_gb300 as P
    return P


@functools.lru_cache(maxsize=None)
def _case(level, mixed_bc):
    v, f = W.icosphere(level, 1.0)
    m = W.CAVITY_MATERIAL
    rng = np.random.default_rng(level)
    if mixed_bc:
        bc = (rng.random(len(f)) < 0.3).astype(np.int8)
        val = rng.standard_normal((len(f), 3))
    else:
        bc = np.zeros(len(f), np.int8)
        val = W.pressure_pattern(v, f)
    g = OB.geometry(v, f)
    ops = [OB.operators(g, s, m, bc) for s in S_SET]
    return v, f, m, bc, val, g, ops


def _ctx(level, mixed_bc):
    P = _P()
    v, f, m, bc, val, g, ops = _case(level, mixed_bc)
    c = P.Context(0)
    c.set_mesh(v, f)
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(bc, val, P.BEM_PROFILE_STEP)
    return c


@pytest.mark.parametrize("level", [1, 2])
def test_geometry_and_near_lists(level):
    v, f, m, bc, val, g, _ = _case(level, False)
    c = _ctx(level, False)
    geo = c.geometry()
    assert np.abs(geo[:, 0:3] - g.centroid).max() < 1e-15
    assert np.abs(geo[:, 3:6] - g.normal).max() < 1e-15
    assert np.abs(geo[:, 6] - g.area).max() < 1e-15 * g.area.max()
    assert np.abs(geo[:, 7] - g.h).max() < 1e-15
    rp, cols = c.near_lists()
    orp, ocols = OB.near_lists(g)
    assert np.array_equal(rp, orp) and np.array_equal(cols, ocols)   # bit-exact integer work


@pytest.mark.parametrize("level", [1, 2])
def test_element_blocks_fp64(level):
    v, f, m, bc, val, g, _ = _case(level, False)
    c = _ctx(level, False)
    near = OB.near_mask(g)
    rng = np.random.default_rng(4)
    rows = rng.integers(0, len(f), 12)
    rows = np.concatenate([rows, rows, np.nonzero(near)[0][:6]])
    cols = np.concatenate([rows[:12], rng.integers(0, len(f), 12), np.nonzero(near)[1][:6]])
    for s in S_SET[[0, 3]]:
        H, G = c.element_blocks(s, rows, cols)
        Ho, Go = OB.element_blocks(g, s, m, rows=np.unique(rows))
        idx = {r: k for k, r in enumerate(np.unique(rows))}
        for k, (i, e) in enumerate(zip(rows, cols)):
            hr, gr = Ho[idx[i], e], Go[idx[i], e]
            # scale: the row's largest block (a self block of a near-equilateral element can be
            # ~1e-16, pure rounding noise on both sides)
            hs, gs = np.abs(Ho[idx[i]]).max(), np.abs(Go[idx[i]]).max()
            assert np.abs(H[k] - hr).max() <= 1e-10 * hs, (i, e, s)
            assert np.abs(G[k] - gr).max() <= 1e-10 * gs, (i, e, s)


@pytest.mark.parametrize("level,mixed_bc", [(1, False), (2, False), (1, True), (2, True)])
@pytest.mark.parametrize("which", [0, 1])
def test_apply_fp64_and_fp32(level, mixed_bc, which):
    P = _P()
    v, f, m, bc, val, g, ops = _case(level, mixed_bc)
    c = _ctx(level, mixed_bc)
    x = W.random_complex_vectors(len(S_SET), 3 * len(f), seed=level)
    ref = np.stack([ops[k][which] @ x[k] for k in range(len(S_SET))])
    y64 = c.apply(S_SET, x, P.BEM_PREC_FP64, which)
    y32 = c.apply(S_SET, x, P.BEM_PREC_FP32, which)
    for k in range(len(S_SET)):
        scale = np.abs(ref[k]).max()
        assert np.abs(y64[k] - ref[k]).max() <= 1e-10 * scale, k
        # FP32 operator: elementwise, against the largest entry (as at the benchmark size)
        e32 = np.abs(y32[k] - ref[k]).max() / scale
        print(f"level {level} mixed {mixed_bc} which {which} k {k}: FP32 elementwise {e32:.2e}")
        assert e32 < 2e-6, (k, e32)


@pytest.mark.parametrize("level,mixed_bc", [(2, False), (1, True)])
def test_rhs_and_preconditioner(level, mixed_bc):
    v, f, m, bc, val, g, ops = _case(level, mixed_bc)
    c = _ctx(level, mixed_bc)
    b = c.rhs(S_SET)
    x = W.random_complex_vectors(len(S_SET), 3 * len(f), seed=9)
    y = c.precond(S_SET, x)
    for k, s in enumerate(S_SET):
        A, Kn = ops[k]
        bref = Kn @ OB.known_data(val, s)
        assert np.abs(b[k] - bref).max() <= 1e-10 * np.abs(bref).max()
        yref = np.concatenate([np.linalg.solve(A[3 * i:3 * i + 3, 3 * i:3 * i + 3], x[k, 3 * i:3 * i + 3])
                               for i in range(len(f))])
        assert np.abs(y[k] - yref).max() <= 1e-10 * np.abs(yref).max()


def test_invalid_arguments_are_errors():
    P = _P()
    c = _ctx(1, False)
    with pytest.raises(P.BemError) as e:
        c.apply(np.array([-1.0 + 2j]), np.zeros((1, 240), complex))
    assert e.value.code == P.BEM_ERR_INVALID_ARG
    with pytest.raises(P.BemError):
        c.element_blocks(250.0, [0], [80])
    with pytest.raises(P.BemError):
        c.set_mesh(np.zeros((3, 3)), np.array([[0, 1, 2]]))       # zero-area triangle
    c3 = _ctx(1, False)   # the rejected mesh above leaves c without one
    for call in (lambda: c3.solve(np.zeros(0, complex)),            # empty frequency lists
                 lambda: c3.apply(np.zeros(0, complex), np.zeros((0, 240), complex)),
                 lambda: c3.residual(np.zeros(0, complex), np.zeros((0, 240), complex))):
        with pytest.raises(P.BemError) as e:
            call()
        assert e.value.code == P.BEM_ERR_INVALID_ARG
    c2 = P.Context(0)
    with pytest.raises(P.BemError) as e:
        c2.rhs(np.array([250.0]))
    assert e.value.code in (P.BEM_ERR_NO_MESH, P.BEM_ERR_INVALID_ARG)


@pytest.mark.parametrize("level,mixed_bc", [(1, False), (2, False), (2, True)])
def test_refinement_residual_df64_and_fp64(level, mixed_bc):
    """r = b - A x: the float-float far field (default in the mixed solver) and the native FP64
    one both match the oracle's dense b - A x; at a near-solution x (residual ~1e-6 ||b||, the
    regime the refinement certifies) the float-float residual stays within 5e-10 ||b|| (measured
    2.4e-10 with lazily renormalised float-float pairs: float-float precision times the
    cancellation of the sum), 2e3 below the 1e-6 tolerance it certifies."""
    P = _P()
    v, f, m, bc, val, g, ops = _case(level, mixed_bc)
    c = _ctx(level, mixed_bc)
    x = W.random_complex_vectors(len(S_SET), 3 * len(f), seed=21) * 1e-6
    for mode, bound in ((P.BEM_RESID_DF64, 5e-10), (P.BEM_RESID_FP64, 1e-10)):
        r = c.residual(S_SET, x, mode)
        for k, s in enumerate(S_SET):
            A, Kn = ops[k]
            b = Kn @ OB.known_data(val, s)
            ref = b - A @ x[k]
            assert np.abs(r[k] - ref).max() <= bound * np.abs(ref).max(), (mode, k)
    # near-solution: x = A^{-1} b (1 + 1e-6 noise)
    rng = np.random.default_rng(3)
    xs = []
    for k, s in enumerate(S_SET):
        A, Kn = ops[k]
        b = Kn @ OB.known_data(val, s)
        xe = np.linalg.solve(A, b)
        # entrywise relative noise: the unknowns mix displacements and tractions
        xs.append(xe * (1 + 1e-6 * (rng.standard_normal(len(xe)) + 1j * rng.standard_normal(len(xe)))))
    xs = np.array(xs)
    r = c.residual(S_SET, xs, P.BEM_RESID_DF64)
    for k, s in enumerate(S_SET):
        A, Kn = ops[k]
        b = Kn @ OB.known_data(val, s)
        ref = b - A @ xs[k]
        assert np.linalg.norm(r[k] - ref) <= 5e-10 * np.linalg.norm(b), k
