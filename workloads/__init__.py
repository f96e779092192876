"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only builds inputs: triangle meshes, materials, boundary-condition patterns and
frequency lists.  It holds none of the boundary-element arithmetic (no kernels, no quadrature,
no solver, no transform), so that the CPU oracle and the CUDA library can both consume its
output without sharing any of the method's code.

Mesh convention (the one the library and the oracle both expect): triangles are listed with
their vertices counter-clockwise about the unit normal n = (v1-v0) x (v2-v0) / |...|, and that
normal points OUT OF THE ELASTIC DOMAIN (into a cavity, or out of a finite body).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 20151113


# ----------------------------------------------------------------------------------------------
# icosphere
# ----------------------------------------------------------------------------------------------
def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((a, b, 0.0))
            v.append((0.0, a, b))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    # faces: triples of mutually adjacent vertices (edge length 2 in these coordinates)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=-1)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    faces = np.array(faces, dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, _orient_outward(v, faces)


def _orient_outward(v, f):
    """Reorder each face so that its right-hand normal points away from the origin."""
    f = f.copy()
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", nrm, p0 + p1 + p2) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0), inward: bool = True):
    """Icosphere with 20*4**level flat triangles, vertices on the sphere of `radius`.

    inward=True orients the faces so their normals point to the centre: the convention for a
    spherical cavity in an unbounded elastic medium (normal out of the elastic domain).
    """
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(nf, dtype=np.int64)
    v = np.array(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    if inward:
        f = f[:, [0, 2, 1]]
    return v, f.astype(np.int32)


def ellipsoid(level: int, semi_axes, center=(0.0, 0.0, 0.0), inward: bool = True):
    """Icosphere scaled to an ellipsoid with the given semi-axes (orientation preserved)."""
    v, f = icosphere(level, 1.0, (0.0, 0.0, 0.0), inward)
    v = v * np.asarray(semi_axes, dtype=np.float64) + np.asarray(center, dtype=np.float64)
    return v, f


# ----------------------------------------------------------------------------------------------
# materials, loads, frequency lists
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Material:
    mu: float  # shear modulus [Pa]
    nu: float  # Poisson's ratio [-]
    rho: float  # mass density [kg/m^3]


CAVITY_MATERIAL = Material(mu=1e9, nu=0.25, rho=2000.0)
CAVITY_P0 = 1e6  # step pressure amplitude [Pa]


def unit_normals(verts, tris):
    """Right-hand unit normals of the triangles (input convention check, no BEM arithmetic)."""
    p0, p1, p2 = (verts[tris[:, k]] for k in range(3))
    n = np.cross(p1 - p0, p2 - p0)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def pressure_pattern(verts, tris, p0=CAVITY_P0):
    """Traction pattern of a uniform pressure p0 acting on the wall of a cavity.

    The pressure pushes the medium away from the cavity, i.e. against the normal that points out
    of the medium: t = -p0 * n.  Returned as an (ne, 3) float64 array (to be multiplied by the
    Laplace-domain time profile, 1/s for a step).
    """
    return -p0 * unit_normals(verts, tris)


def fsm_frequencies(T: float, sigma: float, n: int):
    """The benchmark frequency list s_k = sigma + i*k*pi/T, k = 0..n-1 (complex128)."""
    k = np.arange(n, dtype=np.float64)
    return sigma + 1j * k * math.pi / T


@dataclasses.dataclass
class CavityProblem:
    verts: np.ndarray
    tris: np.ndarray
    material: Material
    bc_type: np.ndarray  # int8 per triangle: 0 traction given, 1 displacement given
    bc_value: np.ndarray  # (ne, 3) float64 spatial pattern
    s: np.ndarray  # complex128 frequency list
    T: float
    sigma: float
    radius: float


def spherical_cavity(level: int = 2, n_freq: int = 64, T: float = 0.02, sigma: float = 250.0,
                     radius: float = 1.0):
    """Pressurised spherical cavity in a full space (the small and the single-mesh batched
    workloads): icosphere of `radius`, mu=1e9 Pa, nu=0.25, rho=2000 kg/m^3, step pressure 1e6 Pa,
    frequencies sigma + i*k*pi/T."""
    v, f = icosphere(level, radius, inward=True)
    ne = len(f)
    return CavityProblem(
        verts=v, tris=f, material=CAVITY_MATERIAL,
        bc_type=np.zeros(ne, dtype=np.int8),
        bc_value=pressure_pattern(v, f),
        s=fsm_frequencies(T, sigma, n_freq), T=T, sigma=sigma, radius=radius)


def random_complex_vectors(n_freq: int, n: int, seed: int = SEED):
    """Seeded complex test vectors (n_freq, n) for operator parity tests."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_freq, n)) + 1j * rng.standard_normal((n_freq, n))


def uneven_instances(n_inst: int = 16, seed: int = SEED, levels=(2, 3, 4, 5)):
    """Seeded batch of ellipsoidal cavities of uneven size with random materials.

    Semi-axes uniform in [0.5, 2] m, nu uniform in [0.2, 0.35], mu log-uniform in [1e8, 1e10] Pa,
    rho uniform in [1500, 3000] kg/m^3; icosphere level drawn from `levels`.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        lvl = int(rng.choice(levels))
        axes = rng.uniform(0.5, 2.0, size=3)
        mat = Material(mu=float(10 ** rng.uniform(8.0, 10.0)), nu=float(rng.uniform(0.2, 0.35)),
                       rho=float(rng.uniform(1500.0, 3000.0)))
        v, f = ellipsoid(lvl, axes)
        out.append((v, f, mat))
    return out


# ----------------------------------------------------------------------------------------------
# porous block
# ----------------------------------------------------------------------------------------------
def box_surface(L=(1.0, 1.0, 1.0), n=(8, 8, 8)):
    """Surface of the box [0,Lx]x[0,Ly]x[0,Lz], each face split into squares of the grid n and
    each square into two triangles; normals point out of the box (out of the solid).
    Returns (verts, tris, face_id) with face_id in {0: x=0, 1: x=Lx, 2: y=0, 3: y=Ly, 4: z=0,
    5: z=Lz}."""
    L = np.asarray(L, dtype=np.float64)
    verts, tris, fid = [], [], []
    index = {}

    def vid(p):
        key = tuple(np.round(p, 12))
        if key not in index:
            index[key] = len(verts)
            verts.append(p)
        return index[key]

    for axis in range(3):
        a1, a2 = [d for d in range(3) if d != axis]
        for side in (0, 1):
            for i in range(n[a1]):
                for j in range(n[a2]):
                    corner = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = np.zeros(3)
                        p[axis] = side * L[axis]
                        p[a1] = (i + di) * L[a1] / n[a1]
                        p[a2] = (j + dj) * L[a2] / n[a2]
                        corner.append(vid(p))
                    for t in ((corner[0], corner[1], corner[2]), (corner[0], corner[2], corner[3])):
                        tris.append(t)
                        fid.append(2 * axis + side)
    verts = np.array(verts)
    tris = np.array(tris, dtype=np.int64)
    # orient outward: the normal must point away from the box centre
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", nrm, (p0 + p1 + p2) / 3 - L / 2) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris.astype(np.int32), np.array(fid, dtype=np.int32)


def porous_block(L=(1.0, 1.0, 1.0), n=(8, 8, 8), n_voids=27, radii=(0.08, 0.15), void_level=2,
                 clearance=0.02, seed=SEED, p0=CAVITY_P0, material=CAVITY_MATERIAL):
    """Block with seeded non-overlapping spherical voids (the porous-solid workloads): step
    traction p0 (compressive, along +z into the block) on the face z = 0, the face z = Lz fixed,
    every other face and every void traction-free.  Returns a CavityProblem-like record."""
    rng = np.random.default_rng(seed)
    L = np.asarray(L, dtype=np.float64)
    bv, bt, fid = box_surface(L, n)
    centres, rad = [], []
    tries = 0
    while len(centres) < n_voids and tries < 100000:
        tries += 1
        r = rng.uniform(*radii)
        c = rng.uniform(r + clearance, L - r - clearance)
        if all(np.linalg.norm(c - c2) > r + r2 + clearance for c2, r2 in zip(centres, rad)):
            centres.append(c)
            rad.append(r)
    verts = [bv]
    tris = [bt]
    off = len(bv)
    for c, r in zip(centres, rad):
        v, f = icosphere(void_level, r, c, inward=True)
        verts.append(v)
        tris.append(f + off)
        off += len(v)
    verts = np.vstack(verts)
    tris = np.vstack(tris).astype(np.int32)
    ne = len(tris)
    face = np.full(ne, -1, dtype=np.int32)
    face[:len(bt)] = fid
    bc_type = np.zeros(ne, dtype=np.int8)
    bc_value = np.zeros((ne, 3))
    bc_value[face == 4, 2] = p0            # traction +p0 e_z on z = 0 (pushes into the block)
    bc_type[face == 5] = 1                 # z = Lz fixed (zero displacement)
    return dict(verts=verts, tris=tris, face=face, material=material, bc_type=bc_type,
                bc_value=bc_value, centres=np.array(centres), radii=np.array(rad))


# ----------------------------------------------------------------------------------------------
# block with 98 spherical cavities (the paper's third example)
# ----------------------------------------------------------------------------------------------
ALUMINIUM = Material(mu=69e9 / (2.0 * 1.3), nu=0.3, rho=2.7e3)   # E = 69 GPa, nu = 0.3


def example3_cavity_centres(L=(1.0, 1.0, 1.5), layers=7):
    """Centres of the 98 identical cavities: `layers` equally spaced layers along z, each with
    14 cavities in four staggered rows of 4, 3, 4 and 3 (rows at y = 1/8, 3/8, 5/8, 7/8 of Ly;
    rows of 4 at x = 1/8 .. 7/8 of Lx, rows of 3 at x = 1/4, 1/2, 3/4).  The paper states 98
    identical cavities equally distributed in the block; its figure is not available, so this
    arrangement is a reading of that sentence."""
    L = np.asarray(L, dtype=np.float64)
    cs = []
    for k in range(layers):
        z = (k + 0.5) * L[2] / layers
        for row, y in enumerate((0.125, 0.375, 0.625, 0.875)):
            xs = (0.125, 0.375, 0.625, 0.875) if row % 2 == 0 else (0.25, 0.5, 0.75)
            for x in xs:
                cs.append((x * L[0], y * L[1], z))
    return np.array(cs)


def example3_block(n=(12, 12, 18), void_level=1, radius=0.072, p0=CAVITY_P0, material=ALUMINIUM):
    """The elastic block of the paper's third example: 1 x 1 x 1.5 m with 98 identical spherical
    cavities of radius 0.072 m (example3_cavity_centres), fixed on z = 1.5, uniform step traction
    p0 along +z (into the block) on z = 0, every other surface and every cavity traction-free;
    aluminium.  The box faces are split into the squares of the grid n, two triangles each; each
    cavity is an icosphere of 20 * 4**void_level triangles.  Returns a porous_block-like record."""
    L = np.array([1.0, 1.0, 1.5])
    bv, bt, fid = box_surface(L, n)
    centres = example3_cavity_centres(L)
    verts, tris, off = [bv], [bt], len(bv)
    for c in centres:
        v, f = icosphere(void_level, radius, c, inward=True)
        verts.append(v)
        tris.append(f + off)
        off += len(v)
    verts = np.vstack(verts)
    tris = np.vstack(tris).astype(np.int32)
    ne = len(tris)
    face = np.full(ne, -1, dtype=np.int32)
    face[:len(bt)] = fid
    bc_type = np.zeros(ne, dtype=np.int8)
    bc_value = np.zeros((ne, 3))
    bc_value[face == 4, 2] = p0
    bc_type[face == 5] = 1
    return dict(verts=verts, tris=tris, face=face, material=material, bc_type=bc_type,
                bc_value=bc_value, centres=centres, radii=np.full(len(centres), radius))


# ----------------------------------------------------------------------------------------------
# prismatic rod
# ----------------------------------------------------------------------------------------------
ROD_MATERIAL = Material(mu=2.11e11 / 2.0, nu=0.0, rho=7.85e3)   # E = 2.11e11 Pa, nu = 0
ROD_P0 = -1e6                                                   # axial step traction [Pa]


def prismatic_rod(L=(3.0, 1.0, 1.0), n=(24, 8, 8), p0=ROD_P0, material=ROD_MATERIAL):
    """The prismatic rod (box [0,Lx]x[0,Ly]x[0,Lz]) fixed at x = 0, axial step traction p0 e_x on
    x = Lx, lateral faces free; each face split into the squares of the grid n, two triangles
    each, normals out of the rod.  Returns (verts, tris, face, material, bc_type, bc_value)."""
    verts, tris, face = box_surface(L, n)
    ne = len(tris)
    bc_type = np.zeros(ne, dtype=np.int8)
    bc_value = np.zeros((ne, 3))
    bc_type[face == 0] = 1                    # x = 0 fixed (zero displacement)
    bc_value[face == 1, 0] = p0               # x = Lx: traction p0 e_x
    return dict(verts=verts, tris=tris, face=face, material=material, bc_type=bc_type,
                bc_value=bc_value)
