"""Pins of the H-matrix oracle (oracle/hmatrix.py) and the library's host-side cluster tree and
block partition against it (CPU only).

What pins the oracle, independently of itself:
  * far4_operator against the dense assembly of oracle.bem on the far pairs (an independent
    loop over rows), zero own blocks, and the 4-point rule on the near pairs;
  * the cluster tree's invariants: a permutation, children splitting their parent's range at
    size // 2, the median property along the split axis, leaves of at most `leaf` elements;
  * the partition by brute force: every (target, source) element pair covered exactly once,
    every low-rank block admissible for the true vertex sets (max diameter <= eta x minimum
    distance), dense blocks only between leaves;
  * ACA: exact recovery of random rank-r matrices at rank r, the singular values of a smooth
    kernel matrix (its rank within a small factor of the SVD's at the same tolerance), and a
    three-class block whose third class a plain cross approximation misses;
  * the H-matrix product against the dense A4 on a porous block with mixed boundary conditions,
    within 10 eps relative.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import bem as B
from oracle import hmatrix as HM


def _small_block():
    pb = W.porous_block(L=(2.0, 1.0, 1.0), n=(8, 4, 4), n_voids=2, radii=(0.08, 0.1), void_level=1)
    return pb["verts"], pb["tris"], pb["material"], pb["bc_type"]


def test_far4_operator_is_the_far_part_of_the_dense_assembly():
    cav = W.spherical_cavity(level=1, n_freq=4)
    g = B.geometry(cav.verts, cav.tris)
    bc = np.zeros(len(cav.tris), dtype=np.int8)
    bc[::3] = B.DIRICHLET
    s = cav.s[2]
    A4 = HM.far4_operator(g, s, cav.material, bc)
    A, _ = B.operators(g, s, cav.material, bc)
    ne = len(cav.tris)
    near = B.near_mask(g)
    far = ~near
    np.fill_diagonal(far, False)
    A4b = A4.reshape(ne, 3, ne, 3)
    Ab = A.reshape(ne, 3, ne, 3)
    ii, ee = np.nonzero(far)
    assert np.allclose(A4b[ii, :, ee, :], Ab[ii, :, ee, :], rtol=0, atol=1e-14 * np.abs(Ab).max())
    assert np.all(A4b[np.arange(ne), :, np.arange(ne), :] == 0)
    # near pairs: the 4-point rule, not the 7-point one the assembly uses there
    ii, ee = np.nonzero(near)
    blk = HM.element_pair_blocks(g, s, cav.material, bc, ii, ee)
    assert np.allclose(A4b[ii, :, ee, :], blk, rtol=0, atol=1e-14 * np.abs(blk).max())
    assert not np.allclose(A4b[ii, :, ee, :], Ab[ii, :, ee, :], rtol=0, atol=1e-6 * np.abs(blk).max())


@pytest.mark.parametrize("leaf", [1, 7, 32])
def test_cluster_tree_invariants(leaf):
    v, f, _, _ = _small_block()
    t = HM.cluster_tree(v, f, leaf)
    ne = len(f)
    assert np.array_equal(np.sort(t.perm), np.arange(ne))
    c = HM.element_centroids(v, f)
    p = np.asarray(v)[np.asarray(f)]
    for k in range(len(t.begin)):
        b, n = t.begin[k], t.size[k]
        idx = t.perm[b:b + n]
        assert np.all(p[idx].min(axis=(0, 1)) >= t.lo[k]) and np.all(p[idx].max(axis=(0, 1)) <= t.hi[k])
        l, r = t.child[k]
        if l < 0:
            assert n <= leaf
            continue
        assert n > leaf
        assert t.begin[l] == b and t.size[l] == n // 2 and t.begin[r] == b + n // 2 and t.size[r] == n - n // 2
        ext = c[idx].max(axis=0) - c[idx].min(axis=0)
        ax = int(np.argmax(ext))
        left, right = t.perm[b:b + n // 2], t.perm[b + n // 2:b + n]
        assert c[left, ax].max() <= c[right, ax].min()


@pytest.mark.parametrize("eta,max_block", [(1.0, 64), (2.0, 512)])
def test_partition_covers_every_pair_once_and_low_rank_blocks_are_admissible(eta, max_block):
    v, f, _, _ = _small_block()
    leaf = 16
    t = HM.cluster_tree(v, f, leaf)
    part = HM.block_partition(t, eta, max_block)
    ne = len(f)
    cover = np.zeros((ne, ne), dtype=np.int32)
    p = np.asarray(v)[np.asarray(f)]

    def elems(k):
        return t.perm[t.begin[k]:t.begin[k] + t.size[k]]

    for a, b in part.lowrank:
        ta, tb = elems(a), elems(b)
        cover[np.ix_(ta, tb)] += 1
        assert t.size[a] <= max_block and t.size[b] <= max_block
        pa, pb_ = p[ta].reshape(-1, 3), p[tb].reshape(-1, 3)
        da = np.linalg.norm(pa[:, None] - pa[None], axis=-1).max()
        db = np.linalg.norm(pb_[:, None] - pb_[None], axis=-1).max()
        dist = np.linalg.norm(pa[:, None] - pb_[None], axis=-1).min()
        assert dist > 0 and max(da, db) <= eta * dist * (1 + 1e-12)
    for a, b in part.dense:
        assert t.child[a, 0] < 0 and t.child[b, 0] < 0
        cover[np.ix_(elems(a), elems(b))] += 1
    assert np.all(cover == 1)


def test_aca_recovers_exact_low_rank_matrices():
    rng = np.random.default_rng(3)
    for m, n, r in [(30, 45, 1), (60, 40, 5), (90, 90, 12)]:
        A = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ \
            (rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
        U, V = HM.aca(lambda i: A[i], lambda j: A[:, j], m, n, 1e-10, 64, classes=3)
        assert U.shape[1] == r
        assert np.linalg.norm(A - U @ V.T) <= 1e-10 * np.linalg.norm(A)


def test_aca_rank_is_close_to_the_svd_rank_on_a_smooth_kernel():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (120, 3))
    y = rng.uniform(0, 1, (150, 3)) + np.array([3.0, 0.5, 0.0])
    r = np.linalg.norm(x[:, None] - y[None], axis=-1)
    A = np.exp(-0.3j * r) / r
    sv = np.linalg.svd(A, compute_uv=False)
    tail = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1] / np.linalg.norm(sv)
    for eps in (1e-4, 1e-6):
        U, V = HM.aca(lambda i: A[i], lambda j: A[:, j], 120, 150, eps, 100)
        err = np.linalg.norm(A - U @ V.T) / np.linalg.norm(A)
        r_svd = int(np.argmax(tail <= eps))
        assert err <= 10 * eps
        assert U.shape[1] <= 2 * r_svd + 4


def test_aca_trial_steps_find_a_class_the_pivots_never_reach():
    # rows of classes 0 and 1 couple only to the even columns, rows of class 2 only to the odd
    # ones: a plain cross approximation from row 0 never pivots on an odd column
    rng = np.random.default_rng(5)
    m, n = 60, 40
    X = rng.standard_normal((m, 2)) @ rng.standard_normal((2, n))
    Y = rng.standard_normal((m, 2)) @ rng.standard_normal((2, n))
    A = np.zeros((m, n), dtype=np.complex128)
    rows2 = np.arange(m) % 3 == 2
    A[np.ix_(~rows2, np.arange(0, n, 2))] = X[np.ix_(~rows2, np.arange(0, n, 2))]
    A[np.ix_(rows2, np.arange(1, n, 2))] = Y[np.ix_(rows2, np.arange(1, n, 2))]
    U1, V1 = HM.aca(lambda i: A[i], lambda j: A[:, j], m, n, 1e-8, 40, classes=1)
    U3, V3 = HM.aca(lambda i: A[i], lambda j: A[:, j], m, n, 1e-8, 40, classes=3)
    assert np.linalg.norm(A - U1 @ V1.T) > 0.1 * np.linalg.norm(A)
    assert np.linalg.norm(A - U3 @ V3.T) <= 1e-8 * np.linalg.norm(A)


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_hmatrix_product_matches_the_dense_far_field(eps):
    v, f, mat, bc = _small_block()
    assert (bc == B.DIRICHLET).any() and (bc == B.NEUMANN).any()
    g = B.geometry(v, f)
    period = 0.04
    s = 3 * math.log(10) / period + 1j * 5 * 2 * math.pi / period
    A4 = HM.far4_operator(g, s, mat, bc)
    H = HM.build_hmatrix(v, f, g, s, mat, bc, leaf=16, eta=2.0, max_block=512, eps=eps, kmax=96)
    assert len(H.U) > 0 and len(H.D) > 0
    rng = np.random.default_rng(6)
    x = rng.standard_normal(3 * len(f)) + 1j * rng.standard_normal(3 * len(f))
    x *= np.repeat(np.where(bc == B.DIRICHLET, mat.mu, 1.0), 3)   # tractions ~ mu x displacements
    y = A4 @ x
    yh = HM.hmatvec(H, x)
    assert np.linalg.norm(yh - y) <= 10 * eps * np.linalg.norm(y)
    lr, dn, full = HM.storage(H)
    if eps >= 1e-3:   # on 480 elements the blocks are small: compression shows at the looser tolerance
        assert lr < 0.8 * (full - dn)


def _lib_or_skip():
    import paper_1511_04355_gb300 as P
    try:
        P.load_library()
    except ImportError:
        pytest.skip("library not built (run __graft_entry__.build())")
    return P


def test_library_partition_is_the_oracles():
    P = _lib_or_skip()
    cav = W.spherical_cavity(level=3, n_freq=2)
    v1, f1, _, _ = _small_block()
    rod = W.prismatic_rod(n=(12, 4, 4))
    for v, f in [(cav.verts, cav.tris), (v1, f1), (rod["verts"], rod["tris"])]:
        for leaf, eta, mb in [(32, 2.0, 512), (16, 1.0, 64), (7, 3.0, 1024)]:
            p = P.bem_default_hmatrix_params(leaf=leaf, eta=eta, max_block=mb)
            perm, cl, lr, dn = P.bem_hmatrix_partition(v, f, p)
            t = HM.cluster_tree(v, f, leaf)
            part = HM.block_partition(t, eta, mb)
            assert np.array_equal(perm, t.perm)
            assert np.array_equal(cl[:, 0], t.begin) and np.array_equal(cl[:, 1], t.size)
            assert np.array_equal(lr, part.lowrank) and np.array_equal(dn, part.dense)


def test_library_partition_refuses_bad_arguments():
    P = _lib_or_skip()
    v, f, _, _ = _small_block()
    for kw in (dict(leaf=0), dict(leaf=200), dict(max_block=8, leaf=16), dict(eta=0.0), dict(eps=1.5),
               dict(max_rank=0), dict(max_rank=300), dict(max_freqs=-1)):
        with pytest.raises(P.BemError):
            P.bem_hmatrix_partition(v, f, P.bem_default_hmatrix_params(**kw))
    bad = np.array(f, dtype=np.int32).copy()
    bad[0, 0] = len(v)
    with pytest.raises(P.BemError):
        P.bem_hmatrix_partition(v, bad)
