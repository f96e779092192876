"""Quadrature rules used by the oracle (FP64, test infrastructure only).

The discretisation is constant-element collocation on flat triangles (the paper's Sec. 2.1
uses a 6-point Gauss rule on curved quadratic elements; this build uses a 4-point rule for
regular source elements, a 7-point rule for near sources and a Duffy-mapped Gauss-Legendre
rule on the collocation point's own element).  Readings:
  * "4-point" = the degree-3 rule with the centroid (weight -27/48) and the three points of
    barycentric coordinates (3/5, 1/5, 1/5) (weight 25/48 each);
  * "7-point" = Radon's degree-5 rule: centroid (9/40) plus the orbits (a, a, 1-2a) with
    a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200;
  * "13-point Duffy" = 13 x 13 Gauss-Legendre points on each of the three Duffy squares the
    element splits into around the collocation point.
Weights are normalised to sum to 1 (multiply by the element area).
"""
from __future__ import annotations

import math

import numpy as np


def rule_4pt():
    """(barycentric (4,3), weights (4,)) of the degree-3 four-point rule."""
    bary = np.array([[1 / 3, 1 / 3, 1 / 3], [0.6, 0.2, 0.2], [0.2, 0.6, 0.2], [0.2, 0.2, 0.6]])
    w = np.array([-27 / 48, 25 / 48, 25 / 48, 25 / 48])
    return bary, w


def rule_7pt():
    """(barycentric (7,3), weights (7,)) of Radon's degree-5 seven-point rule."""
    s15 = math.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    bary = [[1 / 3, 1 / 3, 1 / 3]]
    w = [9.0 / 40.0]
    for a, wa in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        bary += [[b, a, a], [a, b, a], [a, a, b]]
        w += [wa] * 3
    return np.array(bary), np.array(w)


def gauss_legendre_01(n):
    """n-point Gauss-Legendre nodes and weights on [0, 1] (library routine on [-1, 1])."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def duffy_points(x0, va, vb, n):
    """Duffy map of the triangle (x0, va, vb) from the unit square, n x n Gauss-Legendre.

    y(u, v) = x0 + u (va - x0) + u v (vb - va); dA = 2 |T| u du dv, so a 1/r singularity at x0
    is cancelled by the factor u.  Returns points (n*n, 3) and weights (n*n,) that integrate
    over the triangle's area.
    """
    g, gw = gauss_legendre_01(n)
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(gw, gw, indexing="ij")
    u, v, wu, wv = u.ravel(), v.ravel(), wu.ravel(), wv.ravel()
    area2 = np.linalg.norm(np.cross(va - x0, vb - va))
    pts = x0 + u[:, None] * (va - x0) + (u * v)[:, None] * (vb - va)
    w = wu * wv * u * area2
    return pts, w
