"""Elementwise comparison of solution vectors, per kind of unknown.

A solution vector holds, per element, the displacement (traction given) or the traction
(displacement given), three complex components each.  The two kinds differ in size by many
orders of magnitude, so a norm over the whole vector can hide a large error on the smaller
kind: every entry is compared with the largest entry of its own kind instead.
"""
import numpy as np


def max_rel_err(x, x_ref, bc_type):
    """max over the two kinds of unknowns of max_n |x_n - xref_n| / max_n |xref_n| (n of that
    kind); x, x_ref: (..., 3 ne) complex, bc_type: (ne,) with 0 = displacement unknown."""
    x = np.asarray(x)
    x_ref = np.asarray(x_ref)
    kind = np.repeat(np.asarray(bc_type), 3)
    worst = 0.0
    for k in (0, 1):
        sel = kind == k
        if not sel.any():
            continue
        scale = np.abs(x_ref[..., sel]).max()
        if scale == 0.0:
            continue
        worst = max(worst, float(np.abs(x[..., sel] - x_ref[..., sel]).max() / scale))
    return worst
