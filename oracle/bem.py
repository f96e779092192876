"""Dense constant-element collocation BEM for the Laplace-domain BIE (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Discretisation of Sec. 2.1, Eq. (bie), with flat triangles and one collocation point (the
centroid x_i) and one constant displacement / traction vector per element:
    1/2 u_i + sum_e H_ie u_e = sum_e G_ie t_e,
    H_ie = int_e T(x_i, y; s) dA_y,   G_ie = int_e U(x_i, y; s) dA_y   (3 x 3 complex blocks),
the free term c_ij = delta_ij / 2 holding at the centroid of a flat element.  Columns are
arranged by boundary condition (Sec. 2.1, Eq. (Aa_b)): where the traction is given, the
unknown is u_e and the column is 1/2 delta_ie I + H_ie; where the displacement is given, the
unknown is t_e and the column is -G_ie; the known data go to the right-hand side b(s).

Element integrals:
  * far   (|x_i - c_e| >= 2 h_e, h_e = longest edge of e):  4-point degree-3 rule
  * near  (|x_i - c_e| <  2 h_e, e != i):                   7-point degree-5 rule
  * self  (e == i): G_ii by 13 x 13 Gauss-Legendre on the three Duffy squares around x_i;
    H_ii = CPV of the static (Kelvin) part + the bounded dynamic remainder T - T0 by the same
    Duffy rule.  On a flat element dr/dn = 0, so the static part reduces to
    -(1-2nu)/(8 pi (1-nu)) (n_i C_j - n_j C_i) with C_k = CPV int_e rh_k / r^2 dA, and by the
    divergence theorem in the element plane C_k = - sum_edges nu_k int_edge ds / r (nu = the
    in-plane outward normal of the edge; the small circle around x_i contributes nothing),
    each edge integral being asinh(t2/p) - asinh(t1/p).
The system is solved by dense LU with partial pivoting (numpy.linalg.solve).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kernels as K
from . import quadrature as Q

NEUMANN = 0    # traction given, displacement unknown
DIRICHLET = 1  # displacement given, traction unknown

PROFILE_STEP = 0      # Laplace factor 1/s
PROFILE_CONSTANT = 1  # Laplace factor 1

NEAR_FACTOR = 2.0
DUFFY_N = 13


@dataclasses.dataclass
class Geometry:
    p: np.ndarray        # (ne, 3, 3) vertices
    centroid: np.ndarray  # (ne, 3)
    normal: np.ndarray   # (ne, 3) unit, right-hand from vertex order
    area: np.ndarray     # (ne,)
    h: np.ndarray        # (ne,) longest edge
    q4: np.ndarray       # (ne, 4, 3) 4-point rule points
    w4: np.ndarray       # (ne, 4) weights * area
    q7: np.ndarray       # (ne, 7, 3)
    w7: np.ndarray       # (ne, 7)


def geometry(verts, tris) -> Geometry:
    """Per-element centroid, unit normal, area, longest edge and quadrature points."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    p = verts[tris]                                   # (ne, 3, 3)
    e1 = p[:, 1] - p[:, 0]
    e2 = p[:, 2] - p[:, 0]
    cr = np.cross(e1, e2)
    a2 = np.linalg.norm(cr, axis=1)
    normal = cr / a2[:, None]
    area = 0.5 * a2
    edges = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 1], p[:, 0] - p[:, 2]], axis=1)
    h = np.linalg.norm(edges, axis=2).max(axis=1)
    centroid = p.mean(axis=1)
    b4, w4 = Q.rule_4pt()
    b7, w7 = Q.rule_7pt()
    q4 = np.einsum("qk,ekd->eqd", b4, p)
    q7 = np.einsum("qk,ekd->eqd", b7, p)
    return Geometry(p=p, centroid=centroid, normal=normal, area=area, h=h,
                    q4=q4, w4=w4[None, :] * area[:, None], q7=q7, w7=w7[None, :] * area[:, None])


def near_mask(g: Geometry):
    """Boolean (ne, ne): source e is near collocation point i (|x_i - c_e| < 2 h_e, e != i)."""
    d = np.linalg.norm(g.centroid[:, None, :] - g.centroid[None, :, :], axis=-1)
    m = d < NEAR_FACTOR * g.h[None, :]
    np.fill_diagonal(m, False)
    return m


def near_lists(g: Geometry):
    """CSR (row_ptr, cols) of the near-source lists, columns ascending."""
    m = near_mask(g)
    cols = [np.nonzero(m[i])[0] for i in range(m.shape[0])]
    row_ptr = np.zeros(m.shape[0] + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in cols])
    return row_ptr, (np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64))


def _rule_blocks(xi, pts, wts, normals, s, mat):
    """sum_q w_q T(x_i, y_q), sum_q w_q U(x_i, y_q) for a batch of pairs.

    xi (n, 3); pts (n, q, 3); wts (n, q); normals (n, 3).  Returns H, G of shape (n, 3, 3)."""
    d = pts - xi[:, None, :]
    nq = np.broadcast_to(normals[:, None, :], d.shape)
    T = K.fundamental_T(d, nq, s, mat.mu, mat.nu, mat.rho)
    U = K.fundamental_U(d, s, mat.mu, mat.nu, mat.rho)
    return np.einsum("nq,nqij->nij", wts, T), np.einsum("nq,nqij->nij", wts, U)


def edge_inverse_distance(x0, a, b):
    """int over the segment a->b of ds / |y - x0| (closed form)."""
    L = np.linalg.norm(b - a)
    t = (b - a) / L
    t1 = np.dot(a - x0, t)
    perp = (a - x0) - t1 * t
    p = np.linalg.norm(perp)
    return math.asinh((t1 + L) / p) - math.asinh(t1 / p)


def cpv_rh_over_r2(x0, tri, normal):
    """C_k = CPV int_tri rh_k / r^2 dA for x0 inside the flat triangle (closed form)."""
    C = np.zeros(3)
    for k in range(3):
        a, b = tri[k], tri[(k + 1) % 3]
        L = np.linalg.norm(b - a)
        nu_edge = np.cross(b - a, normal) / L     # in-plane outward edge normal
        C -= nu_edge * edge_inverse_distance(x0, a, b)
    return C


def self_blocks(g: Geometry, i, s, mat, n=DUFFY_N):
    """(H_ii, G_ii) for element i (3 x 3 complex each)."""
    x0 = g.centroid[i]
    tri = g.p[i]
    nrm = g.normal[i]
    pts, wts = [], []
    for k in range(3):
        p, w = Q.duffy_points(x0, tri[k], tri[(k + 1) % 3], n)
        pts.append(p)
        wts.append(w)
    pts = np.concatenate(pts)
    wts = np.concatenate(wts)
    d = pts - x0
    U = K.fundamental_U(d, s, mat.mu, mat.nu, mat.rho)
    G = np.einsum("q,qij->ij", wts, U)
    T = K.fundamental_T(d, nrm, s, mat.mu, mat.nu, mat.rho)
    T0 = K.kelvin_T(d, nrm, mat.nu)
    H_dyn = np.einsum("q,qij->ij", wts, T - T0)
    C = cpv_rh_over_r2(x0, tri, nrm)
    H_static = -(1.0 - 2.0 * mat.nu) / (8.0 * math.pi * (1.0 - mat.nu)) * (
        np.outer(nrm, C) - np.outer(C, nrm))
    return H_dyn + H_static, G


def element_blocks(g: Geometry, s, mat, rows=None):
    """H, G blocks for the rows `rows` (default all): arrays (nr, ne, 3, 3) complex."""
    ne = len(g.area)
    rows = np.arange(ne) if rows is None else np.asarray(rows)
    near = near_mask(g)
    H = np.zeros((len(rows), ne, 3, 3), dtype=np.complex128)
    G = np.zeros_like(H)
    for a, i in enumerate(rows):
        far_e = np.nonzero(~near[i])[0]
        far_e = far_e[far_e != i]
        near_e = np.nonzero(near[i])[0]
        for es, pts, wts in ((far_e, g.q4, g.w4), (near_e, g.q7, g.w7)):
            if len(es):
                xi = np.broadcast_to(g.centroid[i], (len(es), 3))
                h, gg = _rule_blocks(xi, pts[es], wts[es], g.normal[es], s, mat)
                H[a, es] = h
                G[a, es] = gg
        H[a, i], G[a, i] = self_blocks(g, i, s, mat)
    return H, G


def profile_factor(profile, s):
    """Laplace-domain factor of the time profile (step -> 1/s, constant -> 1)."""
    if profile == PROFILE_STEP:
        return 1.0 / s
    if profile == PROFILE_CONSTANT:
        return 1.0
    raise ValueError(f"unknown time profile {profile}")


def operators(g: Geometry, s, mat, bc_type, rows=None):
    """Dense A(s) and K(s) (rows x N): A acts on the unknowns, K on the known boundary data,
    so that b(s) = K(s) (profile(s) * pattern).  Eq. (Aa_b) with the BC column swap."""
    ne = len(g.area)
    rows = np.arange(ne) if rows is None else np.asarray(rows)
    H, G = element_blocks(g, s, mat, rows=rows)
    H = H + 0.5 * np.eye(3)[None, None] * (rows[:, None] == np.arange(ne)[None, :])[:, :, None, None]
    neu = np.asarray(bc_type) == NEUMANN
    A_blk = np.where(neu[None, :, None, None], H, -G)
    K_blk = np.where(neu[None, :, None, None], G, -H)
    A = A_blk.transpose(0, 2, 1, 3).reshape(3 * len(rows), 3 * ne)
    Kn = K_blk.transpose(0, 2, 1, 3).reshape(3 * len(rows), 3 * ne)
    return A, Kn


def known_data(bc_value, s, profile=PROFILE_STEP):
    """profile(s) * pattern, flattened (N,)."""
    return (np.asarray(bc_value, dtype=np.float64) * profile_factor(profile, s)).reshape(-1)


def assemble(g: Geometry, s, mat, bc_type, bc_value, profile=PROFILE_STEP):
    """Dense A(s) (N x N) and b(s) (N) with N = 3 ne, Eq. (Aa_b)."""
    A, Kn = operators(g, s, mat, bc_type)
    return A, Kn @ known_data(bc_value, s, profile)


def solve(g: Geometry, s, mat, bc_type, bc_value, profile=PROFILE_STEP):
    """Solution vector a(s) of A(s) a = b(s) by LU (per element: u_e or t_e)."""
    A, b = assemble(g, s, mat, bc_type, bc_value, profile)
    return np.linalg.solve(A, b), A, b


def solve_frequencies(verts, tris, mat, bc_type, bc_value, s_list, profile=PROFILE_STEP):
    """Dense LU solutions for every frequency in s_list: (ns, N) complex."""
    g = geometry(verts, tris)
    return np.stack([solve(g, s, mat, bc_type, bc_value, profile)[0] for s in s_list])
