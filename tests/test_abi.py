"""CPU checks of the C ABI: the library loads without a GPU, exports every function that
include/bem.h declares, the binding's table matches the header, and calls fail cleanly (an
error code, no crash) when no CUDA device is present."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(bem_[a-z_0-9]+)\s*\(", src, re.M)))


def _lib():
    import paper_1511_04355_gb300 as P
    try:
        return P.load_library()
    except ImportError:
        pytest.skip("library not built (run __graft_entry__.build())")


def test_header_declares_functions():
    names = _declared()
    assert "bem_solve_frequencies" in names and "bem_fsm_eval" in names and len(names) >= 20


def test_library_exports_every_declared_symbol():
    lib = _lib()
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_table_matches_header():
    import paper_1511_04355_gb300 as P
    assert sorted(P.declared_symbols()) == _declared()


def test_calls_without_gpu_return_error_codes():
    import paper_1511_04355_gb300 as P
    lib = _lib()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = lib.bem_create(ctypes.byref(h), 0, None)
    assert rc == P.BEM_ERR_CUDA
    assert lib.bem_last_error(None)
    assert lib.bem_solve_frequencies(None, None, 0, None, None) == P.BEM_ERR_INVALID_ARG
    opt = P.bem_options()
    assert lib.bem_default_options(ctypes.byref(opt)) == 0 and opt.tol == 1e-6 and opt.restart == 50
    # batch driver: argument checks happen before any worker starts or any CUDA call
    assert lib.bem_solve_batch(None, 1, 0) == P.BEM_ERR_INVALID_ARG
    items = (P.bem_batch_item * 2)()
    assert lib.bem_solve_batch(items, 2, 0) == P.BEM_ERR_INVALID_ARG       # null contexts
    assert lib.bem_solve_batch(items, 0, 0) == P.BEM_ERR_INVALID_ARG


def test_afs_defaults_are_the_papers_printed_values():
    """bem_default_afs_params and the oracle's AFS defaults carry the parameters the paper prints
    (tests/golden/afs_parameters.txt)."""
    import inspect
    import os
    import paper_1511_04355_gb300 as P
    from oracle import afs as OA
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "afs_parameters.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    p = P.bem_default_afs_params()
    for k in ("J0", "alpha_H", "alpha_L", "E1bar", "E2bar", "Jc"):
        assert getattr(p, k) == vals[k], k
    d = {n: v.default for n, v in inspect.signature(OA.run).parameters.items()}
    for k in ("J0", "alpha_H", "alpha_L", "E1bar", "E2bar", "Jc"):
        assert d[k] == vals[k], k


def test_noalloc_binding_refuses_bad_tensors_before_calling_the_library():
    """The allocation-free FSM wrapper checks dtypes, shapes and devices itself: the library can
    only see that it was handed device pointers, not how large the buffers behind them are."""
    torch = pytest.importorskip("torch")
    import paper_1511_04355_gb300 as P

    nc, m, nt = 8, 5, 7
    h = torch.zeros((nc, m), dtype=torch.complex128)
    t = torch.zeros((nt,), dtype=torch.float64)
    out = torch.zeros((nt, m), dtype=torch.float64)
    bad = [
        (h.real.contiguous(), t, out, "dtype"),                            # real h: half the bytes
        (h, t.float(), out, "dtype"),
        (h, t, torch.zeros((nt, m + 1), dtype=torch.float64), "shape"),    # out too wide
        (h, t, torch.zeros((nt - 1, m), dtype=torch.float64), "shape"),    # out too short
        (h, t, out, "device"),                                             # host tensors
        (h[None], t, out, "2-D"),
        (h, t[None], out, "1-D"),
    ]
    for hh, tt, oo, word in bad:
        with pytest.raises(ValueError) as e:
            P.bem_fsm_eval_noalloc(hh, 250.0, 0.04, tt, oo)
        assert word in str(e.value), (word, str(e.value))


def test_hmatrix_defaults_and_null_arguments_without_gpu():
    import paper_1511_04355_gb300 as P
    lib = _lib()
    p = P.bem_hmatrix_params()
    assert lib.bem_default_hmatrix_params(ctypes.byref(p)) == 0
    assert (p.enable, p.leaf, p.max_block, p.max_rank, p.eta, p.eps, p.max_freqs) == (0, 32, 512, 96, 2.0, 1e-4, 0)
    assert lib.bem_default_hmatrix_params(None) == P.BEM_ERR_INVALID_ARG
    counts = (ctypes.c_int64 * 3)()
    assert lib.bem_hmatrix_partition(None, 0, None, 0, ctypes.byref(p), None, None, 0, None, 0, None, 0,
                                     counts) == P.BEM_ERR_INVALID_ARG
    assert lib.bem_last_error(None)
    assert lib.bem_set_hmatrix(None, ctypes.byref(p)) == P.BEM_ERR_INVALID_ARG
