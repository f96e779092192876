"""The launch-shape autotuner of the FP32 far-field operator (bem_autotune, bem_set_tuning,
bem_load_tuning, bem_launch_shape).

* Every launch shape (ft in {1, 4, 8, 12}, tiles in {1, 2, 4}, waves in {2, 4, 8}) computes the same
  operator: on the 1280-triangle cavity, for an equally spaced frequency run (the recurrence
  kernel) and an irregular list (the direct kernel), the FP32 product A x with the shape forced by
  a one-entry table matches the FP64 product elementwise to 2e-6 of its largest entry (the FP32
  operator's accuracy at full size), and so does its difference from the fixed shape's product
  (other summation orders and recurrence chain lengths round differently).
* bem_autotune returns valid entries for the requested launch sizes, installs them, and the
  lookup rule (smallest ne_max >= ne, then smallest nfl_max >= nfl, else the largest) picks them;
  a table read from a file and the empty table (the fixed shape) are honoured.
"""
import itertools
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(level):
    import paper_1511_04355_gb300 as P
    prob = W.spherical_cavity(level=level, n_freq=20)
    c = P.Context(0)
    c.set_mesh(prob.verts, prob.tris)
    m = prob.material
    c.set_material(m.mu, m.nu, m.rho)
    c.set_bc(prob.bc_type, prob.bc_value)
    return P, c, prob


def test_every_launch_shape_gives_the_same_operator():
    P, c, prob = _ctx(3)
    ne = len(prob.tris)
    lists = {"equally spaced": prob.s,
             "irregular": 250.0 + 1j * np.array([0.0, 333.3, 1234.5, 2500.0, 4321.0, 7777.7, 9000.1])}
    for name, s in lists.items():
        x = W.random_complex_vectors(len(s), 3 * ne, seed=7)
        y64 = c.apply(s, x, P.BEM_PREC_FP64)
        P.bem_set_tuning(c.h, [])
        y_fixed = c.apply(s, x, P.BEM_PREC_FP32)
        scale = np.abs(y64).max(axis=1, keepdims=True)
        for ft, tiles, waves in itertools.product((1, 4, 8, 12), (1, 2, 4), (2, 4, 8)):
            P.bem_set_tuning(c.h, [dict(ne_max=10 ** 9, nfl_max=10 ** 6, ft=ft, tiles=tiles, waves=waves)])
            assert P.bem_launch_shape(c.h, len(s)) == (ft, tiles, waves)
            y = c.apply(s, x, P.BEM_PREC_FP32)
            e64 = (np.abs(y - y64) / scale).max()
            ef = (np.abs(y - y_fixed) / scale).max()
            assert e64 <= 2e-6 and ef <= 2e-6, (name, ft, tiles, waves, e64, ef)
    P.bem_set_tuning(c.h, [])
    assert P.bem_launch_shape(c.h, 5) == (12, 2, 4)


def test_autotune_table_and_lookup(tmp_path):
    P, c, prob = _ctx(2)
    ent = P.bem_autotune(c.h, prob.s, [1, 8, 20])
    assert [e["nfl_max"] for e in ent] == [1, 8, 20]
    for e in ent:
        assert e["ne_max"] == len(prob.tris) and e["ft"] in (1, 4, 8, 12) and e["ms"] > 0
        assert 0 < e["ms"] <= e["ms_fixed"] * (1 + 1e-6)
    assert P.bem_launch_shape(c.h, 1)[0] == ent[0]["ft"]
    assert P.bem_launch_shape(c.h, 5) == (ent[1]["ft"], ent[1]["tiles"], ent[1]["waves"])
    assert P.bem_launch_shape(c.h, 100) == (ent[2]["ft"], ent[2]["tiles"], ent[2]["waves"])
    # file table: the bucket with the smallest ne_max >= ne, then the smallest nfl_max >= nfl
    path = os.path.join(tmp_path, "table.txt")
    with open(path, "w") as fh:
        fh.write("# ne_max nfl_max ft tiles waves ms ms_fixed\n"
                 "100 1000 4 1 2\n"
                 "400 4 8 4 8 1.0 2.0\n"
                 "400 1000 4 2 2\n"
                 "99999 1000 12 1 8\n")
    P.bem_load_tuning(c.h, path)
    assert P.bem_launch_shape(c.h, 3) == (8, 4, 8)
    assert P.bem_launch_shape(c.h, 50) == (4, 2, 2)
    with open(path, "w") as fh:
        fh.write("400 4 5 4 8\n")
    with pytest.raises(P.BemError):
        P.bem_load_tuning(c.h, path)
