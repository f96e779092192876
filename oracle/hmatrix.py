"""Hierarchical low-rank far field of the BEM operator (oracle, FP64, test infrastructure only).

The paper accelerates the matrix-vector product of its iterative BEM solve with a fast
multipole method (Sec. 2.1, the paragraph on the fast solver: a kernel-independent FMM).  The
fast operator of this build is a hierarchical matrix instead: a cluster tree of the elements, a
block partition by the standard admissibility condition, and adaptive cross approximation (ACA)
of the admissible blocks (Hackbusch 1999, "A sparse matrix arithmetic based on H-matrices";
Bebendorf 2000, "Approximation of boundary element matrices", Numer. Math. 86).  What it
approximates has a plain definition: the 4-point-rule far-field part A4 of the system matrix,
    A4[i, e] = sum_q w_q K_col(e)(x_i, y_q)  for every pair e != i,  A4[i, i] = 0,
with K_col(e) = T for a traction-given column and -U for a displacement-given column (the
column swap of Sec. 2.1, Eq. (Aa_b)); the near and own-element corrections stay exact.  This
module writes out
  * far4_operator   the dense A4 (the definition the fast operator is measured against);
  * cluster_tree    recursive median bisection of the elements along the longest side of
                    their centroids' bounding box, ties broken by element index;
  * block_partition recursive subdivision of (root, root): a pair of clusters is a low-rank
                    block when max(diam) <= eta dist of their vertex bounding boxes and both
                    hold at most max_block elements, a dense block when both are leaves;
  * aca             partially pivoted ACA with the Frobenius-norm stopping rule and trial steps
                    per row class;
  * HMatrix         the blocks of one frequency and the product y = A_H x.
A low-rank block (3 m x 3 n, element-major) is approximated by one cross approximation whose
rows fall into three classes, the components c of the 3 x 3 element blocks.  On the planar
faces of a box the T kernel has structural zeros (T_cd = 0 for in-plane c, d when targets and
sources are coplanar), and a plain partially pivoted cross approximation, whose pivots never
visited the rows of the normal component, stopped with 70 % error on such blocks; the trial
steps per class (see aca) find that part.  Columns of displacement-given elements (U kernel,
entries ~1 / (4 pi mu r)) are scaled by mu / D (D the bounding-box diagonal of the mesh) inside
the cross approximation, so that the block-relative stopping rule weighs them like the columns
of traction-given elements (T kernel, ~1 / (4 pi r^2)); the stored factors undo the scaling.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import bem as B


# ----------------------------------------------------------------------------- the definition
def far4_operator(g: B.Geometry, s, mat, bc_type):
    """Dense A4 (3 ne x 3 ne complex): 4-point rule over every pair e != i, zero own blocks."""
    ne = len(g.area)
    neu = np.asarray(bc_type) == B.NEUMANN
    A = np.zeros((ne, 3, ne, 3), dtype=np.complex128)
    for i in range(ne):
        es = np.array([e for e in range(ne) if e != i], dtype=np.int64)
        xi = np.broadcast_to(g.centroid[i], (len(es), 3))
        H, G = B._rule_blocks(xi, g.q4[es], g.w4[es], g.normal[es], s, mat)
        A[i, :, es, :] = np.where(neu[es][:, None, None], H, -G)
    return A.reshape(3 * ne, 3 * ne)


def element_pair_blocks(g: B.Geometry, s, mat, bc_type, targets, sources):
    """A4 blocks (3 x 3) of the pairs (targets[k], sources[k]); zero where they coincide."""
    targets = np.asarray(targets, dtype=np.int64)
    sources = np.asarray(sources, dtype=np.int64)
    neu = np.asarray(bc_type) == B.NEUMANN
    with np.errstate(divide="ignore", invalid="ignore"):   # r = 0 on coinciding pairs
        H, G = B._rule_blocks(g.centroid[targets], g.q4[sources], g.w4[sources], g.normal[sources], s, mat)
    blk = np.where(neu[sources][:, None, None], H, -G)
    blk[targets == sources] = 0.0
    return blk


# ----------------------------------------------------------------------------- cluster tree
@dataclasses.dataclass
class ClusterTree:
    perm: np.ndarray      # tree order -> element index
    begin: np.ndarray     # per cluster: first position in perm
    size: np.ndarray      # per cluster: number of elements
    child: np.ndarray     # per cluster: (left, right) cluster ids, -1 for a leaf
    lo: np.ndarray        # per cluster: vertex bounding box, lower corner (3,)
    hi: np.ndarray        # per cluster: upper corner
    diam: np.ndarray      # per cluster: bounding-box diagonal


def element_centroids(verts, tris):
    """(p0 + p1 + p2) / 3 per triangle, summed in that order."""
    p = np.asarray(verts, dtype=np.float64)[np.asarray(tris, dtype=np.int64)]
    return ((p[:, 0] + p[:, 1]) + p[:, 2]) / 3.0


def cluster_tree(verts, tris, leaf):
    """Clusters in depth-first order (a cluster, then its left subtree, then its right one).

    A cluster of more than `leaf` elements is split at the median along the longest side of its
    centroids' bounding box (lowest axis on ties): its elements sorted by that coordinate,
    equal coordinates by element index, the first half (size // 2) going left."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    c = element_centroids(verts, tris)
    vlo = verts[tris].min(axis=1)
    vhi = verts[tris].max(axis=1)
    ne = len(tris)
    perm = np.arange(ne, dtype=np.int64)
    begin, size, child, lo, hi = [], [], [], [], []

    def build(b, n):
        cid = len(begin)
        begin.append(b)
        size.append(n)
        child.append([-1, -1])
        idx = perm[b:b + n]
        lo.append(vlo[idx].min(axis=0))
        hi.append(vhi[idx].max(axis=0))
        if n <= leaf:
            return cid
        ext = c[idx].max(axis=0) - c[idx].min(axis=0)
        ax = int(np.argmax(ext))            # first maximum: lowest axis on ties
        order = np.lexsort((idx, c[idx, ax]))
        perm[b:b + n] = idx[order]
        h = n // 2
        left = build(b, h)
        right = build(b + h, n - h)
        child[cid] = [left, right]
        return cid

    build(0, ne)
    lo = np.array(lo)
    hi = np.array(hi)
    d = hi - lo
    diam = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    return ClusterTree(perm=perm, begin=np.array(begin), size=np.array(size),
                       child=np.array(child, dtype=np.int64), lo=lo, hi=hi, diam=diam)


def box_distance(t: ClusterTree, a, b):
    """Euclidean distance between the bounding boxes of clusters a and b (0 if they meet)."""
    g = np.maximum(0.0, np.maximum(t.lo[b] - t.hi[a], t.lo[a] - t.hi[b]))
    return math.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])


def admissible(t: ClusterTree, a, b, eta):
    """max(diam a, diam b) <= eta dist(a, b), with dist > 0."""
    d = box_distance(t, a, b)
    return d > 0.0 and max(t.diam[a], t.diam[b]) <= eta * d


@dataclasses.dataclass
class Partition:
    lowrank: np.ndarray   # (nl, 2) cluster ids (target, source)
    dense: np.ndarray     # (nd, 2)


def block_partition(t: ClusterTree, eta, max_block):
    """Blocks in the order of a depth-first recursion from (root, root); a pair that is neither
    a block is split on both sides (on the non-leaf side when one is a leaf), children in
    (left, right) order, target children outer."""
    lr, dn = [], []

    def rec(a, b):
        if t.size[a] <= max_block and t.size[b] <= max_block and admissible(t, a, b, eta):
            lr.append((a, b))
            return
        la, lb = t.child[a, 0] < 0, t.child[b, 0] < 0
        if la and lb:
            dn.append((a, b))
            return
        ta = [a] if la else list(t.child[a])
        tb = [b] if lb else list(t.child[b])
        for x in ta:
            for y in tb:
                rec(x, y)

    rec(0, 0)
    return Partition(lowrank=np.array(lr, dtype=np.int64).reshape(-1, 2),
                     dense=np.array(dn, dtype=np.int64).reshape(-1, 2))


# ----------------------------------------------------------------------------- ACA
def aca(row, col, m, n, eps, kmax, classes=1):
    """Partially pivoted adaptive cross approximation of an m x n matrix given by its rows and
    columns: row(i) -> (n,), col(j) -> (m,).  Returns U (m, k), V (n, k), A ~ U V^T.

    Step k: the residual of the pivot row i (entries minus the current approximation) picks the
    pivot column j of largest modulus (first on ties); v = residual row / its pivot entry,
    u = residual column j; with the update the squared Frobenius norm of the approximation would be
        |S_k|^2 = |S_{k-1}|^2 + 2 Re sum_{l<k} <u_l, u><v_l, v> + |u|^2 |v|^2,
    and the step is small when |u| |v| <= eps |S_k|.  A step that is not small is appended and
    the next pivot row is the unused row of largest |u| (first on ties); a small step is not
    appended (its term is below the tolerance; appending it only adds rank, and after an exact
    approximation its pivot is rounding noise).  A residual row that vanishes before the first
    update moves to the next unused row.
    Rows fall into `classes` interleaved classes (row i in class i % classes: the components of
    a vector kernel).  A small step does not end the approximation by itself: one trial step is
    then taken from each class in turn, its pivot row the unused row of that class with the
    largest |u| of the last step, and the approximation ends when every trial step is small
    (a vanishing residual row counts as small).  A trial step that is not small resumes the
    ordinary iteration.  Without the trials, a block whose rows of one class meet only columns
    that the pivots never reached stops with that part missing."""
    U = np.zeros((m, 0), dtype=np.complex128)
    V = np.zeros((n, 0), dtype=np.complex128)
    used = np.zeros(m, dtype=bool)
    cls = np.arange(m) % classes
    i = 0
    norm2 = 0.0
    trial = -1          # class of the current trial step, -1 outside the trials
    ulast = None
    while U.shape[1] < kmax:
        r = row(i) - U[i, :] @ V.T
        used[i] = True
        j = int(np.argmax(np.abs(r)))
        if np.abs(r[j]) == 0.0:
            small = True
            if U.shape[1] == 0 and trial < 0:
                rest = np.flatnonzero(~used)
                if rest.size == 0:
                    break
                i = int(rest[0])
                continue
        else:
            v = r / r[j]
            u = col(j) - U @ V[j, :]
            cross = (U.conj().T @ u) * (V.conj().T @ v)
            nu2 = float(np.vdot(u, u).real)
            nv2 = float(np.vdot(v, v).real)
            grown = max(norm2 + 2.0 * float(np.sum(cross).real) + nu2 * nv2, 0.0)
            ulast = u
            small = math.sqrt(nu2 * nv2) <= eps * math.sqrt(grown)
            if not small:
                norm2 = grown
                U = np.concatenate([U, u[:, None]], axis=1)
                V = np.concatenate([V, v[:, None]], axis=1)
        if small:
            # the next trial class with an unused row; none left: done
            nxt = -1
            c = trial + 1
            while c < classes:
                cand = np.flatnonzero((~used) & (cls == c))
                if cand.size:
                    nxt = int(cand[np.argmax(np.abs(ulast[cand]))]) if ulast is not None else int(cand[0])
                    break
                c += 1
            if nxt < 0:
                break
            trial = c
            i = nxt
        else:
            trial = -1
            au = np.abs(ulast)
            au[used] = -1.0
            if au.max() < 0.0:
                break
            i = int(np.argmax(au))
    return U, V


# ----------------------------------------------------------------------------- H-matrix
def column_scale(verts, mat):
    """mu / D, D the bounding-box diagonal of the mesh: the factor on displacement-given columns."""
    v = np.asarray(verts, dtype=np.float64)
    e = v.max(axis=0) - v.min(axis=0)
    return mat.mu / math.sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2])


@dataclasses.dataclass
class HMatrix:
    tree: ClusterTree
    part: Partition
    U: list               # per low-rank block: (3 m, k), rows element-major in tree order
    V: list               # per low-rank block: (3 n, k)
    D: list               # per dense block: (3 m, 3 n)
    ne: int


def build_hmatrix(verts, tris, g: B.Geometry, s, mat, bc_type, leaf=32, eta=2.0, max_block=512,
                  eps=1e-4, kmax=96):
    """The H-matrix of A4 at one frequency: each low-rank block (3 m x 3 n, rows and columns
    element-major in tree order) by one cross approximation with three row classes."""
    tree = cluster_tree(verts, tris, leaf)
    part = block_partition(tree, eta, max_block)
    bc = np.asarray(bc_type)
    cscale = np.where(bc == B.DIRICHLET, column_scale(verts, mat), 1.0)   # per element
    Us, Vs, Ds = [], [], []
    for a, b in part.lowrank:
        te = tree.perm[tree.begin[a]:tree.begin[a] + tree.size[a]]
        se = tree.perm[tree.begin[b]:tree.begin[b] + tree.size[b]]
        csc = np.repeat(cscale[se], 3)

        def row(i, te=te, se=se, csc=csc):
            blk = element_pair_blocks(g, s, mat, bc, np.full(len(se), te[i // 3]), se)
            return blk[:, i % 3, :].reshape(-1) * csc

        def col(j, te=te, se=se, csc=csc):
            blk = element_pair_blocks(g, s, mat, bc, te, np.full(len(te), se[j // 3]))
            return blk[:, :, j % 3].reshape(-1) * csc[j]

        Uk, Vk = aca(row, col, 3 * len(te), 3 * len(se), eps, kmax, classes=3)
        Us.append(Uk)
        Vs.append(Vk / csc[:, None])
    for a, b in part.dense:
        te = tree.perm[tree.begin[a]:tree.begin[a] + tree.size[a]]
        se = tree.perm[tree.begin[b]:tree.begin[b] + tree.size[b]]
        tt, ss = np.meshgrid(te, se, indexing="ij")
        blk = element_pair_blocks(g, s, mat, bc, tt.reshape(-1), ss.reshape(-1))
        Ds.append(blk.reshape(len(te), len(se), 3, 3).transpose(0, 2, 1, 3).reshape(3 * len(te), 3 * len(se)))
    return HMatrix(tree=tree, part=part, U=Us, V=Vs, D=Ds, ne=len(tris))


def hmatvec(H: HMatrix, x):
    """y = A_H x for x of length 3 ne (element-major, original element order)."""
    t = H.tree
    xe = np.asarray(x).reshape(H.ne, 3)
    y = np.zeros((H.ne, 3), dtype=np.complex128)

    def rng(c):
        return t.perm[t.begin[c]:t.begin[c] + t.size[c]]

    for (a, b), Uk, Vk in zip(H.part.lowrank, H.U, H.V):
        te, se = rng(a), rng(b)
        y[te] += (Uk @ (Vk.T @ xe[se].reshape(-1))).reshape(-1, 3)
    for (a, b), Dk in zip(H.part.dense, H.D):
        te, se = rng(a), rng(b)
        y[te] += (Dk @ xe[se].reshape(-1)).reshape(-1, 3)
    return y.reshape(-1)


def storage(H: HMatrix):
    """(complex entries of the low-rank factors, of the dense blocks, of the dense matrix)."""
    lr = sum(u.size + v.size for u, v in zip(H.U, H.V))
    dn = sum(d.size for d in H.D)
    return lr, dn, (3 * H.ne) ** 2
