"""Several meshes of uneven size in one call (the uneven-instance workload's recipe at test
size): four ellipsoidal cavities with their own materials (icosphere levels 1-2, 80-320
triangles), each at its own frequencies, solved by bem_solve_batch with concurrent workers.

* every instance matches the oracle's dense LU to 1e-6 (mixed path at tol 1e-9);
* the batched results equal those of solving each instance alone (1e-8: only the order of the
  FP64 atomic additions may differ between runs);
* a repeated context is refused before anything runs.
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import bem as OB

pytestmark = pytest.mark.gpu


def _P():
    import paper_1511_04355_gb300 as P
    return P


@functools.lru_cache(maxsize=None)
def _cases():
    out = []
    for k, (v, f, mat) in enumerate(W.uneven_instances(n_inst=4, levels=(1, 2))):
        s = W.fsm_frequencies(0.02, 250.0, 64)[k::16]          # 4 frequencies, offset per instance
        bc = np.zeros(len(f), np.int8)
        val = W.pressure_pattern(v, f)
        g = OB.geometry(v, f)
        ref = [np.linalg.solve(*OB.assemble(g, sk, mat, bc, val)) for sk in s]
        out.append((v, f, mat, bc, val, s, np.array(ref)))
    return out


def _contexts(P):
    ctxs = []
    for v, f, mat, bc, val, s, _ in _cases():
        c = P.Context(0)
        c.set_mesh(v, f)
        c.set_material(mat.mu, mat.nu, mat.rho)
        c.set_bc(bc, val, P.BEM_PROFILE_STEP)
        c.set_options(precision=P.BEM_PREC_MIXED, tol=1e-9)
        ctxs.append(c)
    return ctxs


def test_instances_are_uneven():
    sizes = sorted(len(c[1]) for c in _cases())
    assert sizes[0] < sizes[-1]
    assert len({c[2] for c in _cases()}) == 4


def test_batch_matches_lu_and_single_solves():
    P = _P()
    cases = _cases()
    ctxs = _contexts(P)
    probs = [(c.h, case[5], np.zeros((len(case[5]), 3 * c.ne), np.complex128)) for c, case in zip(ctxs, cases)]
    res = P.bem_solve_batch(probs)
    for k, ((x, info), case, c) in enumerate(zip(res, cases, ctxs)):
        ref = case[6]
        assert (info["status"] == 0).all() and info["rc"] == 0, k
        err = np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 1e-6, (k, err)
        alone, _ = c.solve(case[5])
        d = np.linalg.norm(x - alone, axis=1) / np.linalg.norm(alone, axis=1)
        assert d.max() <= 1e-8, (k, d)


def test_batch_one_worker_and_repeated_context():
    P = _P()
    cases = _cases()
    ctxs = _contexts(P)
    probs = [(c.h, case[5], np.zeros((len(case[5]), 3 * c.ne), np.complex128)) for c, case in zip(ctxs, cases)]
    res = P.bem_solve_batch(probs, max_workers=1)
    for (x, info), case in zip(res, cases):
        err = np.linalg.norm(x - case[6], axis=1) / np.linalg.norm(case[6], axis=1)
        assert err.max() <= 1e-6
    with pytest.raises(P.BemError) as e:
        P.bem_solve_batch([probs[0], probs[0]])
    assert e.value.code == P.BEM_ERR_INVALID_ARG
