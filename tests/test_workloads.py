"""Checks of the seeded input generators (no method arithmetic): closed, consistently oriented
surfaces with normals out of the elastic domain, and the porous-block recipe (voids inside the
block, disjoint, with the requested clearance; load and support faces as specified)."""
import numpy as np

import workloads as W


def _edge_counts(tris):
    """Directed-edge bookkeeping: on a closed, consistently oriented surface every undirected
    edge appears exactly twice, once in each direction."""
    fwd = {}
    for a, b, c in tris:
        for u, v in ((a, b), (b, c), (c, a)):
            fwd[(u, v)] = fwd.get((u, v), 0) + 1
    return fwd


def _closed_and_oriented(tris):
    fwd = _edge_counts(tris)
    return all(n == 1 for n in fwd.values()) and all(fwd.get((v, u), 0) == 1 for (u, v) in fwd)


def _signed_volume(verts, tris):
    p0, p1, p2 = (verts[tris[:, k]] for k in range(3))
    return np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0


def test_icosphere_closed_inward():
    v, f = W.icosphere(2, 1.0)
    assert len(f) == 320 and _closed_and_oriented(f)
    # inward normals: the divergence theorem gives minus the enclosed volume
    assert _signed_volume(v, f) < 0
    assert abs(-_signed_volume(v, f) - 4 / 3 * np.pi) < 0.05 * 4 / 3 * np.pi   # inscribed polyhedron


def test_box_surface_closed_outward():
    L = (1.0, 2.0, 1.5)
    v, f, face = W.box_surface(L, (3, 4, 2))
    assert _closed_and_oriented(f)
    assert abs(_signed_volume(v, f) - 3.0) < 1e-12          # outward: + volume
    n = W.unit_normals(v, f)
    expect = {0: (-1, 0, 0), 1: (1, 0, 0), 2: (0, -1, 0), 3: (0, 1, 0), 4: (0, 0, -1), 5: (0, 0, 1)}
    for k, e in expect.items():
        assert np.allclose(n[face == k], e)


def test_porous_block_recipe():
    pb = W.porous_block(L=(1.0, 1.0, 1.0), n=(4, 4, 4), n_voids=6, radii=(0.08, 0.15), void_level=1)
    v, f, face = pb["verts"], pb["tris"], pb["face"]
    c, r = pb["centres"], pb["radii"]
    assert len(c) == 6 and ((r >= 0.08) & (r <= 0.15)).all()
    # voids inside the block with clearance, pairwise disjoint with clearance
    assert ((c - r[:, None] >= 0.02 - 1e-12) & (c + r[:, None] <= 1.0 - 0.02 + 1e-12)).all()
    for a in range(len(c)):
        for b in range(a + 1, len(c)):
            assert np.linalg.norm(c[a] - c[b]) > r[a] + r[b] + 0.02
    # every component closed and oriented; total signed volume = block minus voids (polyhedral)
    assert _closed_and_oriented(f)
    vol = _signed_volume(v, f)
    void_vol = sum(-_signed_volume(*W.icosphere(1, rr, cc)) for cc, rr in zip(c, r))
    assert abs(vol - (1.0 - void_vol)) < 1e-12
    # loads: +p0 e_z traction on z = 0, z = 1 fixed, everything else traction-free
    assert (pb["bc_type"][face == 5] == 1).all() and (pb["bc_type"][face != 5] == 0).all()
    assert np.allclose(pb["bc_value"][face == 4], [0.0, 0.0, W.CAVITY_P0])
    assert np.allclose(pb["bc_value"][face != 4], 0.0)


def test_porous_block_size_of_the_large_recipe():
    # 27 voids with radii in [0.08, 0.15] fit in the unit block (the ~30000-triangle recipe with
    # level-2 voids and a 42 x 42 grid on each face)
    pb = W.porous_block(n=(42, 42, 42), n_voids=27, void_level=2)
    assert len(pb["centres"]) == 27
    assert 25000 < len(pb["tris"]) < 35000


def test_example3_block_recipe():
    """The third example's block: 1 x 1 x 1.5 m, 98 identical cavities of radius 0.072 m inside it,
    disjoint, fixed on z = 1.5, step traction on z = 0."""
    pb = W.example3_block(n=(4, 4, 6), void_level=1)
    v, f, face = pb["verts"], pb["tris"], pb["face"]
    c, r = pb["centres"], pb["radii"]
    assert len(c) == 98 and np.allclose(r, 0.072)
    assert ((c - 0.072 > 0.0) & (c + 0.072 < np.array([1.0, 1.0, 1.5]))).all()
    d = np.linalg.norm(c[:, None] - c[None], axis=-1) + np.eye(98)
    assert d.min() > 2 * 0.072
    # equally spaced layers along z, 14 cavities each
    assert len(np.unique(np.round(c[:, 2], 9))) == 7
    assert all((np.round(c[:, 2], 9) == z).sum() == 14 for z in np.unique(np.round(c[:, 2], 9)))
    assert _closed_and_oriented(f)
    vol = _signed_volume(v, f)
    void_vol = sum(-_signed_volume(*W.icosphere(1, 0.072, cc)) for cc in c)
    assert abs(vol - (1.5 - void_vol)) < 1e-12
    assert (pb["bc_type"][face == 5] == 1).all() and (pb["bc_type"][face != 5] == 0).all()
    assert np.allclose(pb["bc_value"][face == 4], [0.0, 0.0, W.CAVITY_P0])
    assert abs(pb["material"].mu - 69e9 / 2.6) < 1.0 and pb["material"].nu == 0.3


def test_large_porous_recipe_size():
    # the large porous solid: 2 x 1 x 1 m, 200 voids with radii in [0.05, 0.1], ~100000 triangles
    pb = W.porous_block(L=(2.0, 1.0, 1.0), n=(84, 42, 42), n_voids=200, radii=(0.05, 0.1), void_level=2)
    assert len(pb["centres"]) == 200 and len(pb["tris"]) == 99280
