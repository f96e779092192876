"""The allocation-free FSM entry point (bem_fsm_eval_noalloc) against bem_fsm_eval.

Callers that cannot allocate device memory while they run use bem_fsm_eval_noalloc, whose only
working memory is a fixed array inside the library.  This checks, through the C ABI, that two
calls in a row (different sizes, windows and data, so stale scratch contents would show) give
the same responses as the allocating entry point, within the FP64 tolerance of the other FSM
tests, and that a size beyond the fixed scratch is refused.  Collected last on purpose; it
passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(nc, m, nt, seed):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((nc, m)) + 1j * rng.standard_normal((nc, m))
    t = np.sort(rng.uniform(0.0, 0.04, nt))
    return h, t


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import paper_1511_04355_gb300 as P

    ctx = P.Context(0)
    try:
        for (nc, m, nt, window, seed) in [(64, 200, 257, 1, 1), (33, 17, 40, 0, 2)]:
            h, t = _case(nc, m, nt, seed)
            ref = ctx.fsm_eval(h, 250.0, 0.04, t, window)
            hd = torch.from_numpy(h).cuda()
            td = torch.from_numpy(t).cuda()
            od = torch.full((nt, m), float("nan"), dtype=torch.float64, device="cuda")
            P.bem_fsm_eval_noalloc(hd, 250.0, 0.04, td, od, window)
            out = od.cpu().numpy()
            assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        ctx.close()


def test_noalloc_more_times_than_one_grid_dimension():
    """nt = 70000 > 65535 (the grid's y limit) with nc = 2 fits the fixed scratch and every time
    row is written, matching the allocating entry point."""
    import torch
    import paper_1511_04355_gb300 as P

    nc, m, nt = 2, 3, 70000
    h, t = _case(nc, m, nt, 3)
    ctx = P.Context(0)
    try:
        ref = ctx.fsm_eval(h, 250.0, 0.04, t, 1)
    finally:
        ctx.close()
    od = torch.full((nt, m), float("nan"), dtype=torch.float64, device="cuda")
    P.bem_fsm_eval_noalloc(torch.from_numpy(h).cuda(), 250.0, 0.04, torch.from_numpy(t).cuda(), od, 1)
    assert np.abs(od.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_oversized_table():
    import torch
    import paper_1511_04355_gb300 as P

    h = torch.zeros((1025, 1), dtype=torch.complex128, device="cuda")
    t = torch.zeros((256,), dtype=torch.float64, device="cuda")
    out = torch.zeros((256, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(P.BemError) as e:
        P.bem_fsm_eval_noalloc(h, 250.0, 0.04, t, out)
    assert e.value.code == P.BEM_ERR_INVALID_ARG
    assert "exceeds" in str(e.value)
