"""Thin ctypes binding of the C ABI declared in include/bem.h (argument marshalling only).

Every computation runs in the CUDA library libbem_gb300.so; this module converts Python
arguments (numpy arrays for host memory, or torch tensors, host or CUDA) to the pointers and
sizes the C functions take, and raises BemError for a negative return code.  There is no
Python or CPU fallback: if the library is missing the import of a function fails loudly.

Function names are those of the C ABI.  `Context` is a convenience wrapper over them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbem_gb300.so")

BEM_OK = 0
BEM_ERR_INVALID_ARG = -1
BEM_ERR_CUDA = -2
BEM_ERR_NOT_CONVERGED = -3
BEM_ERR_OOM = -4
BEM_ERR_BREAKDOWN = -5
BEM_ERR_NO_MESH = -6
BEM_BC_TRACTION = 0
BEM_BC_DISPLACEMENT = 1
BEM_PROFILE_STEP = 0
BEM_PROFILE_CONSTANT = 1
BEM_PREC_FP64 = 0
BEM_PREC_MIXED = 1
BEM_PREC_FP32 = 2
BEM_APPLY_A = 0
BEM_APPLY_K = 1
BEM_RESID_DF64 = 0
BEM_RESID_FP64 = 1
BEM_WARM_ZERO = 0
BEM_WARM_NEAREST = 1
BEM_WARM_MLP = 2
BEM_WARM_VF = 3
BEM_WARM_SWEEP = 4
BEM_KERNEL_FAR32 = 0
BEM_KERNEL_FAR64 = 1
BEM_KERNEL_NEAR32 = 2
BEM_KERNEL_NEAR64 = 3
BEM_KERNEL_SELF = 4
BEM_KERNEL_VEC = 5
BEM_KERNEL_RES64 = 6
BEM_KERNEL_HAPPLY = 7
BEM_KERNEL_HBUILD = 8
BEM_PEAK_FP32 = 0
BEM_PEAK_FP64 = 1
BEM_PEAK_FP32X2 = 2
KERNEL_NAMES = {0: "far32", 1: "far64", 2: "near32", 3: "near64", 4: "self", 5: "gmres_vec",
                6: "res64", 7: "happly", 8: "hbuild"}


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class bem_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("restart", C.c_int32), ("max_iters", C.c_int32),
                ("max_refine", C.c_int32), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("warm_start", C.c_int32), ("reserved0", C.c_int32 * 2),
                ("residual_mode", C.c_int32), ("reserved", C.c_int32 * 6)]


class bem_solve_stats(C.Structure):
    _fields_ = [("iterations", C.POINTER(C.c_int32)), ("refinements", C.POINTER(C.c_int32)),
                ("residual", C.POINTER(C.c_double)), ("status", C.POINTER(C.c_int32)),
                ("seconds", C.c_double), ("fp32_operator_applies", C.c_int64),
                ("fp64_operator_applies", C.c_int64), ("kernel_launches", C.c_int64)]


class bem_afs_params(C.Structure):
    _fields_ = [("eta", C.c_double), ("omega_max", C.c_double), ("T", C.c_double),
                ("alpha_H", C.c_double), ("alpha_L", C.c_double), ("E1bar", C.c_double),
                ("E2bar", C.c_double), ("J0", C.c_int32), ("Jc", C.c_int32), ("n_grid", C.c_int32),
                ("nt", C.c_int32), ("max_samples", C.c_int32), ("vf_iters", C.c_int32),
                ("batch", C.c_int32), ("warm_retrain", C.c_int32), ("reserved", C.c_int32 * 4)]


class bem_afs_stats(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("s", C.POINTER(C.c_double)),
                ("gmres_iters", C.POINTER(C.c_int32)), ("E1", C.POINTER(C.c_double)),
                ("E2", C.POINTER(C.c_double)), ("poles", C.POINTER(C.c_double)),
                ("n_samples", C.c_int64), ("n_steps", C.c_int64), ("n_poles", C.c_int32),
                ("seconds_solve", C.c_double), ("seconds_fit", C.c_double),
                ("seconds_train", C.c_double), ("warm_trainings", C.c_int32),
                ("warm_learned_gains", C.c_int32)]


class bem_warm_params(C.Structure):
    _fields_ = [("r_max", C.c_int32), ("energy_tol", C.c_double), ("steps", C.c_int32),
                ("lr", C.c_double), ("seed", C.c_uint64), ("reserved", C.c_int32 * 4)]


class bem_warm_stats(C.Structure):
    _fields_ = [("r", C.c_int32), ("n_snapshots", C.c_int32), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("seconds", C.c_double)]


class bem_tune_entry(C.Structure):
    _fields_ = [("ne_max", C.c_int64), ("nfl_max", C.c_int32), ("ft", C.c_int32),
                ("tiles", C.c_int32), ("waves", C.c_int32), ("ms", C.c_double),
                ("ms_fixed", C.c_double)]


class bem_hmatrix_params(C.Structure):
    _fields_ = [("enable", C.c_int32), ("leaf", C.c_int32), ("max_block", C.c_int32),
                ("max_rank", C.c_int32), ("eta", C.c_double), ("eps", C.c_double),
                ("max_freqs", C.c_int32), ("reserved", C.c_int32 * 5)]


class bem_hmatrix_info(C.Structure):
    _fields_ = [("clusters", C.c_int64), ("lowrank_blocks", C.c_int64), ("dense_blocks", C.c_int64),
                ("lowrank_pairs", C.c_int64), ("dense_pairs", C.c_int64), ("frequencies", C.c_int64),
                ("factor_bytes", C.c_int64), ("rank_sum", C.c_int64), ("rank_max", C.c_int32),
                ("capped", C.c_int32), ("seconds_build", C.c_double), ("builds", C.c_int64),
                ("reserved", C.c_int64 * 4)]


class bem_batch_item(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("s", C.c_void_p), ("ns", C.c_int64), ("x_out", C.c_void_p),
                ("stats", C.POINTER(bem_solve_stats)), ("status", C.c_int32)]


_P = C.c_void_p
_I64 = C.c_int64
_SIGS = {
    "bem_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "bem_destroy": (C.c_int, [_P]),
    "bem_last_error": (C.c_char_p, [_P]),
    "bem_default_options": (C.c_int, [C.POINTER(bem_options)]),
    "bem_set_options": (C.c_int, [_P, C.POINTER(bem_options)]),
    "bem_set_mesh": (C.c_int, [_P, _P, _I64, _P, _I64]),
    "bem_set_material": (C.c_int, [_P, C.c_double, C.c_double, C.c_double]),
    "bem_set_bc": (C.c_int, [_P, _P, _P, C.c_int]),
    "bem_solve_frequencies": (C.c_int, [_P, _P, _I64, _P, C.POINTER(bem_solve_stats)]),
    "bem_geometry": (C.c_int, [_P, _P]),
    "bem_near_lists": (C.c_int, [_P, _P, _P, _I64, C.POINTER(_I64)]),
    "bem_element_blocks": (C.c_int, [_P, C.c_double, C.c_double, _P, _P, _I64, _P, _P]),
    "bem_apply": (C.c_int, [_P, _P, _I64, _P, _P, C.c_int, C.c_int]),
    "bem_rhs": (C.c_int, [_P, _P, _I64, _P]),
    "bem_precond_apply": (C.c_int, [_P, _P, _I64, _P, _P]),
    "bem_residual": (C.c_int, [_P, _P, _I64, _P, _P, C.c_int]),
    "bem_profile": (C.c_int, [_P, C.c_int]),
    "bem_default_warm_params": (C.c_int, [C.POINTER(bem_warm_params)]),
    "bem_warm_store": (C.c_int, [_P, _P, _I64, _P]),
    "bem_warm_clear": (C.c_int, [_P]),
    "bem_warm_train": (C.c_int, [_P, C.POINTER(bem_warm_params), C.POINTER(bem_warm_stats)]),
    "bem_warm_basis": (C.c_int, [_P, _P, C.POINTER(C.c_int32)]),
    "bem_solve_batch": (C.c_int, [C.POINTER(bem_batch_item), C.c_int32, C.c_int32]),
    "bem_warm_predict": (C.c_int, [_P, C.c_int32, _P, _I64, _P]),
    "bem_mlp_eval": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32, _P, _P, _P, C.POINTER(C.c_double)]),
    "bem_vf_fit": (C.c_int, [_P, _I64, _P, _I64, _P, C.c_int32, C.c_int32, C.c_double, C.c_int32, _P, _P]),
    "bem_vf_eval": (C.c_int, [_P, C.c_int32, _P, _I64, _P, _I64, _P]),
    "bem_vf_time": (C.c_int, [_P, C.c_int32, _P, _I64, _P, _I64, C.c_double, _P]),
    "bem_default_afs_params": (C.c_int, [C.POINTER(bem_afs_params)]),
    "bem_afs": (C.c_int, [_P, C.POINTER(bem_afs_params), _P, _I64, _P, _I64, _P, _I64, _P,
                          C.POINTER(bem_afs_stats)]),
    "bem_fsm_eval": (C.c_int, [_P, _P, _I64, _I64, C.c_double, C.c_double, _P, _I64, C.c_int, _P]),
    "bem_fsm_eval_noalloc": (C.c_int, [_P, _I64, _I64, C.c_double, C.c_double, _P, _I64, C.c_int,
                                       _P, _P]),
    "bem_noalloc_last_error": (C.c_char_p, []),
    "bem_fsm": (C.c_int, [_P, C.c_double, C.c_double, _I64, _P, _I64, _P, _I64, _P,
                          C.POINTER(bem_solve_stats)]),
    "bem_kernel_time": (C.c_int, [_P, C.c_int, C.POINTER(_I64), C.POINTER(C.c_double),
                                  C.POINTER(_I64)]),
    "bem_measure_peak": (C.c_int, [_P, C.c_int, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "bem_autotune": (C.c_int, [_P, _P, _I64, _P, C.c_int32, C.POINTER(bem_tune_entry)]),
    "bem_set_tuning": (C.c_int, [_P, C.POINTER(bem_tune_entry), C.c_int32]),
    "bem_load_tuning": (C.c_int, [_P, C.c_char_p]),
    "bem_launch_shape": (C.c_int, [_P, _I64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "bem_default_hmatrix_params": (C.c_int, [C.POINTER(bem_hmatrix_params)]),
    "bem_set_hmatrix": (C.c_int, [_P, C.POINTER(bem_hmatrix_params)]),
    "bem_get_hmatrix_info": (C.c_int, [_P, C.POINTER(bem_hmatrix_info)]),
    "bem_hmatrix_partition": (C.c_int, [_P, _I64, _P, _I64, C.POINTER(bem_hmatrix_params), _P, _P, _I64,
                                        _P, _I64, _P, _I64, _P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbem_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_1511_04355_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    """Names of the functions the header declares (the binding's table)."""
    return sorted(_SIGS)


# ------------------------------------------------------------------------------ marshalling
def _ptr(a):
    """Pointer of a numpy array (host) or torch tensor (host or CUDA); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, rc, what):
    if rc != BEM_OK:
        msg = load_library().bem_last_error(ctx)
        raise BemError(rc, f"{what}: {msg.decode() if msg else ''}")


def _cplx_as_pairs(s):
    """Frequency list as interleaved doubles: numpy (host) or a complex128 torch tensor (any
    device, passed by pointer)."""
    if hasattr(s, "data_ptr"):
        if str(s.dtype) != "torch.complex128" or not s.is_contiguous():
            raise TypeError("frequency tensors must be contiguous complex128")
        return s, s.numel()
    s = np.ascontiguousarray(np.asarray(s, dtype=np.complex128).reshape(-1))
    return s, len(s)


# ------------------------------------------------------------------------------ functions
def bem_create(device: int = 0, stream=None):
    lib = load_library()
    h = _P()
    rc = lib.bem_create(C.byref(h), device, stream)
    _check(None, rc, "bem_create")
    return h


def bem_destroy(ctx):
    load_library().bem_destroy(ctx)


def bem_default_options():
    o = bem_options()
    load_library().bem_default_options(C.byref(o))
    return o


def bem_set_options(ctx, opt: bem_options):
    _check(ctx, load_library().bem_set_options(ctx, C.byref(opt)), "bem_set_options")


def bem_set_mesh(ctx, verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    _check(ctx, load_library().bem_set_mesh(ctx, _ptr(v), len(v), _ptr(t), len(t)), "bem_set_mesh")


def bem_set_material(ctx, mu, nu, rho):
    _check(ctx, load_library().bem_set_material(ctx, mu, nu, rho), "bem_set_material")


def bem_set_bc(ctx, bc_type, bc_value, profile=BEM_PROFILE_STEP):
    t = np.ascontiguousarray(bc_type, dtype=np.int8)
    v = np.ascontiguousarray(bc_value, dtype=np.float64)
    _check(ctx, load_library().bem_set_bc(ctx, _ptr(t), _ptr(v), profile), "bem_set_bc")


def bem_solve_frequencies(ctx, s, x_out=None, allow_not_converged=False):
    """Returns (x_out, stats dict).  x_out: None -> a new (ns, 3ne) complex128 numpy array;
    else a caller array/tensor (host or CUDA, complex128, ns*3ne entries) written in place."""
    s, ns = _cplx_as_pairs(s)
    stats = bem_solve_stats()
    it = np.zeros(ns, np.int32)
    rf = np.zeros(ns, np.int32)
    res = np.zeros(ns, np.float64)
    st = np.zeros(ns, np.int32)
    stats.iterations = it.ctypes.data_as(C.POINTER(C.c_int32))
    stats.refinements = rf.ctypes.data_as(C.POINTER(C.c_int32))
    stats.residual = res.ctypes.data_as(C.POINTER(C.c_double))
    stats.status = st.ctypes.data_as(C.POINTER(C.c_int32))
    rc = load_library().bem_solve_frequencies(ctx, _ptr(s), ns, _ptr(x_out), C.byref(stats))
    if not (allow_not_converged and rc == BEM_ERR_NOT_CONVERGED):
        _check(ctx, rc, "bem_solve_frequencies")
    info = dict(iterations=it, refinements=rf, residual=res, status=st, seconds=stats.seconds,
                fp32_operator_applies=stats.fp32_operator_applies,
                fp64_operator_applies=stats.fp64_operator_applies,
                kernel_launches=stats.kernel_launches, rc=rc)
    return x_out, info


def bem_solve_batch(problems, max_workers=0, allow_not_converged=False):
    """problems: list of (ctx handle, s, x_out) with x_out as in bem_solve_frequencies (None:
    a new host array; the context's element count is then needed, so pass an array).  Returns
    a list of (x_out, stats dict) in the order given."""
    n = len(problems)
    items = (bem_batch_item * n)()
    keep = []
    outs = []
    for k, (ctx, s, x_out) in enumerate(problems):
        s, ns = _cplx_as_pairs(s)
        stats = bem_solve_stats()
        arrs = dict(iterations=np.zeros(ns, np.int32), refinements=np.zeros(ns, np.int32),
                    residual=np.zeros(ns, np.float64), status=np.zeros(ns, np.int32))
        stats.iterations = arrs["iterations"].ctypes.data_as(C.POINTER(C.c_int32))
        stats.refinements = arrs["refinements"].ctypes.data_as(C.POINTER(C.c_int32))
        stats.residual = arrs["residual"].ctypes.data_as(C.POINTER(C.c_double))
        stats.status = arrs["status"].ctypes.data_as(C.POINTER(C.c_int32))
        keep += [s, stats, arrs]
        items[k].ctx = ctx
        items[k].s = _ptr(s)
        items[k].ns = ns
        items[k].x_out = _ptr(x_out)
        items[k].stats = C.pointer(stats)
        outs.append((x_out, stats, arrs))
    rc = load_library().bem_solve_batch(items, n, max_workers)
    if rc != BEM_OK and not (allow_not_converged and rc == BEM_ERR_NOT_CONVERGED):
        bad = [k for k in range(n) if items[k].status != BEM_OK]
        k = bad[0] if bad else 0
        msg = load_library().bem_last_error(problems[k][0])
        raise BemError(rc, f"bem_solve_batch: item {k} failed with {items[k].status}: "
                           f"{msg.decode() if msg else ''}")
    res = []
    for k, (x_out, stats, arrs) in enumerate(outs):
        info = dict(arrs, seconds=stats.seconds, fp32_operator_applies=stats.fp32_operator_applies,
                    fp64_operator_applies=stats.fp64_operator_applies,
                    kernel_launches=stats.kernel_launches, rc=items[k].status)
        res.append((x_out, info))
    return res


def bem_geometry(ctx, ne):
    out = np.zeros((ne, 8), np.float64)
    _check(ctx, load_library().bem_geometry(ctx, _ptr(out)), "bem_geometry")
    return out


def bem_near_lists(ctx, ne):
    lib = load_library()
    nnz = _I64()
    rp = np.zeros(ne + 1, np.int64)
    _check(ctx, lib.bem_near_lists(ctx, _ptr(rp), None, 0, C.byref(nnz)), "bem_near_lists")
    cols = np.zeros(max(nnz.value, 1), np.int32)
    _check(ctx, lib.bem_near_lists(ctx, None, _ptr(cols), len(cols), C.byref(nnz)), "bem_near_lists")
    return rp, cols[:nnz.value]


def bem_element_blocks(ctx, s, rows, cols):
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    H = np.zeros((len(r), 3, 3), np.complex128)
    G = np.zeros((len(r), 3, 3), np.complex128)
    s = complex(s)
    _check(ctx, load_library().bem_element_blocks(ctx, s.real, s.imag, _ptr(r), _ptr(c), len(r),
                                                  _ptr(H), _ptr(G)), "bem_element_blocks")
    return H, G


def bem_apply(ctx, s, x, y=None, precision=BEM_PREC_FP64, which=BEM_APPLY_A):
    s, ns = _cplx_as_pairs(s)
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        if y is None:
            y = np.zeros_like(x)
    _check(ctx, load_library().bem_apply(ctx, _ptr(s), ns, _ptr(x), _ptr(y), precision, which),
           "bem_apply")
    return y


def bem_rhs(ctx, s, ne, b_out=None):
    s, ns = _cplx_as_pairs(s)
    if b_out is None:
        b_out = np.zeros((ns, 3 * ne), np.complex128)
    _check(ctx, load_library().bem_rhs(ctx, _ptr(s), ns, _ptr(b_out)), "bem_rhs")
    return b_out


def bem_residual(ctx, s, x, r=None, mode=BEM_RESID_DF64):
    """r = b(s) - A(s) x (FP64-class refinement residual)."""
    s, ns = _cplx_as_pairs(s)
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        if r is None:
            r = np.zeros_like(x)
    _check(ctx, load_library().bem_residual(ctx, _ptr(s), ns, _ptr(x), _ptr(r), mode), "bem_residual")
    return r


def bem_precond_apply(ctx, s, x, y=None):
    s, ns = _cplx_as_pairs(s)
    x = np.ascontiguousarray(x, dtype=np.complex128) if isinstance(x, np.ndarray) else x
    if y is None:
        y = np.zeros_like(x)
    _check(ctx, load_library().bem_precond_apply(ctx, _ptr(s), ns, _ptr(x), _ptr(y)),
           "bem_precond_apply")
    return y


def bem_fsm_eval(ctx, h, eta, period, t, window=1, out=None):
    """h: (nc, m) complex samples at eta + i k 2 pi / period; t: (nt,) -> (nt, m) response."""
    h = np.ascontiguousarray(h, dtype=np.complex128) if isinstance(h, np.ndarray) else h
    t = np.ascontiguousarray(t, dtype=np.float64) if isinstance(t, np.ndarray) else t
    nc, m = h.shape
    nt = t.shape[0]
    if out is None:
        out = np.zeros((nt, m), np.float64)
    _check(ctx, load_library().bem_fsm_eval(ctx, _ptr(h), nc, m, eta, period, _ptr(t), nt, window,
                                            _ptr(out)), "bem_fsm_eval")
    return out


def _require_tensors(specs):
    """ValueError unless every (name, x, dtype, shape) in specs is a contiguous CUDA tensor of
    the current device with that dtype and shape (dtypes and shapes are checked for all of them
    before devices): the C side can only check that it was given device pointers, not how many
    bytes lie behind them."""
    import torch

    for name, x, dtype, shape in specs:
        if not isinstance(x, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if x.dtype != dtype:
            raise ValueError(f"{name} must have dtype {dtype}, got {x.dtype}")
        if tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, x, _, _ in specs:
        if x.device.type != "cuda" or x.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device, got {x.device}")


def bem_fsm_eval_noalloc(h, eta, period, t, out, window=1, stream=None):
    """Allocation-free FSM inversion: h (nc, m) complex128, t (nt,) float64 and out (nt, m)
    float64 must be contiguous CUDA tensors of the current device; stream: a cudaStream_t handle
    or None.  Dtypes and shapes are checked here (ValueError) before the library is called."""
    import torch

    if not isinstance(h, torch.Tensor) or h.dim() != 2:
        raise ValueError("h must be a 2-D torch tensor (nc, m)")
    if not isinstance(t, torch.Tensor) or t.dim() != 1:
        raise ValueError("t must be a 1-D torch tensor (nt,)")
    nc, m = h.shape
    nt = t.shape[0]
    _require_tensors([("h", h, torch.complex128, (nc, m)), ("t", t, torch.float64, (nt,)),
                      ("out", out, torch.float64, (nt, m))])
    rc = load_library().bem_fsm_eval_noalloc(_ptr(h), nc, m, eta, period, _ptr(t), nt, window,
                                             _ptr(out), stream)
    if rc != BEM_OK:
        msg = load_library().bem_noalloc_last_error()
        raise BemError(rc, f"bem_fsm_eval_noalloc: {msg.decode() if msg else ''}")
    return out


def _stats_arrays(n):
    stats = bem_solve_stats()
    arr = dict(iterations=np.zeros(n, np.int32), refinements=np.zeros(n, np.int32),
               residual=np.zeros(n, np.float64), status=np.zeros(n, np.int32))
    stats.iterations = arr["iterations"].ctypes.data_as(C.POINTER(C.c_int32))
    stats.refinements = arr["refinements"].ctypes.data_as(C.POINTER(C.c_int32))
    stats.residual = arr["residual"].ctypes.data_as(C.POINTER(C.c_double))
    stats.status = arr["status"].ctypes.data_as(C.POINTER(C.c_int32))
    return stats, arr


def bem_fsm(ctx, period, eta, nc, t, dofs, allow_not_converged=False):
    """Solve at eta + i k 2 pi / period (k < nc) and return (nt, ndofs) time responses."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    d = np.ascontiguousarray(dofs, dtype=np.int64)
    out = np.zeros((len(t), len(d)), np.float64)
    stats, arr = _stats_arrays(nc)
    rc = load_library().bem_fsm(ctx, period, eta, nc, _ptr(t), len(t), _ptr(d), len(d), _ptr(out),
                                C.byref(stats))
    if not (allow_not_converged and rc == BEM_ERR_NOT_CONVERGED):
        _check(ctx, rc, "bem_fsm")
    arr.update(kernel_launches=stats.kernel_launches, rc=rc)
    return out, arr


def _check_global(rc, what):
    if rc != BEM_OK:
        msg = load_library().bem_last_error(None)
        raise BemError(rc, f"{what}: {msg.decode() if msg else ''}")


def bem_vf_fit(s, F, M, omega_max, n_iter=20, fit_cols=None):
    """Vector fit (host, FP64).  s (J,), F (J, K) complex -> (poles (M,), residues (K, M))."""
    s = np.ascontiguousarray(s, dtype=np.complex128).reshape(-1)
    F = np.ascontiguousarray(F, dtype=np.complex128).reshape(len(s), -1)
    K = F.shape[1]
    cols = None if fit_cols is None else np.ascontiguousarray(fit_cols, dtype=np.int32)
    poles = np.zeros(M, np.complex128)
    R = np.zeros((K, M), np.complex128)
    rc = load_library().bem_vf_fit(_ptr(s), len(s), _ptr(F), K, _ptr(cols),
                                   0 if cols is None else len(cols), M, omega_max, n_iter,
                                   _ptr(poles), _ptr(R))
    _check_global(rc, "bem_vf_fit")
    return poles, R


def bem_vf_eval(poles, R, s):
    poles = np.ascontiguousarray(poles, dtype=np.complex128)
    R = np.ascontiguousarray(R, dtype=np.complex128)
    s = np.ascontiguousarray(s, dtype=np.complex128).reshape(-1)
    out = np.zeros((len(s), R.shape[0]), np.complex128)
    _check_global(load_library().bem_vf_eval(_ptr(poles), len(poles), _ptr(R), R.shape[0], _ptr(s),
                                             len(s), _ptr(out)), "bem_vf_eval")
    return out


def bem_vf_time(poles, R, t, eta=float("inf")):
    poles = np.ascontiguousarray(poles, dtype=np.complex128)
    R = np.ascontiguousarray(R, dtype=np.complex128)
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.zeros((len(t), R.shape[0]), np.float64)
    _check_global(load_library().bem_vf_time(_ptr(poles), len(poles), _ptr(R), R.shape[0], _ptr(t),
                                             len(t), eta, _ptr(out)), "bem_vf_time")
    return out


def bem_default_afs_params(**kw):
    p = bem_afs_params()
    load_library().bem_default_afs_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def bem_afs(ctx, params, orf, test, t_out, capacity=1024):
    """Adaptive frequency sampling; returns (responses (nt, K + Kt), stats dict)."""
    orf = np.ascontiguousarray(orf, dtype=np.int64)
    test = np.ascontiguousarray(test, dtype=np.int64)
    t_out = np.ascontiguousarray(t_out, dtype=np.float64)
    out = np.zeros((len(t_out), len(orf) + len(test)), np.float64)
    st = bem_afs_stats()
    st.capacity = capacity
    arr = dict(s=np.zeros(capacity, np.complex128), gmres_iters=np.zeros(capacity, np.int32),
               E1=np.zeros(capacity), E2=np.zeros(capacity), poles=np.zeros(capacity, np.complex128))
    st.s = arr["s"].ctypes.data_as(C.POINTER(C.c_double))
    st.gmres_iters = arr["gmres_iters"].ctypes.data_as(C.POINTER(C.c_int32))
    st.E1 = arr["E1"].ctypes.data_as(C.POINTER(C.c_double))
    st.E2 = arr["E2"].ctypes.data_as(C.POINTER(C.c_double))
    st.poles = arr["poles"].ctypes.data_as(C.POINTER(C.c_double))
    rc = load_library().bem_afs(ctx, C.byref(params), _ptr(orf), len(orf), _ptr(test), len(test),
                                _ptr(t_out), len(t_out), _ptr(out), C.byref(st))
    _check(ctx, rc, "bem_afs")
    n, ns, npol = st.n_samples, st.n_steps, st.n_poles
    info = dict(s=arr["s"][:n], gmres_iters=arr["gmres_iters"][:n], E1=arr["E1"][:ns],
                E2=arr["E2"][:ns], poles=arr["poles"][:npol], n_samples=n,
                seconds_solve=st.seconds_solve, seconds_fit=st.seconds_fit,
                seconds_train=st.seconds_train, warm_trainings=st.warm_trainings,
                warm_learned_gains=st.warm_learned_gains)
    return out, info


def bem_default_warm_params(**kw):
    p = bem_warm_params()
    load_library().bem_default_warm_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def bem_warm_store(ctx, s, x):
    s, ns = _cplx_as_pairs(s)
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.complex128)
    _check(ctx, load_library().bem_warm_store(ctx, _ptr(s), ns, _ptr(x)), "bem_warm_store")


def bem_warm_clear(ctx):
    _check(ctx, load_library().bem_warm_clear(ctx), "bem_warm_clear")


def bem_warm_train(ctx, params=None):
    params = params or bem_default_warm_params()
    st = bem_warm_stats()
    _check(ctx, load_library().bem_warm_train(ctx, C.byref(params), C.byref(st)), "bem_warm_train")
    return dict(r=st.r, n_snapshots=st.n_snapshots, loss_first=st.loss_first, loss_last=st.loss_last,
                seconds=st.seconds)


def bem_warm_basis(ctx, n_unknowns):
    r = C.c_int32()
    _check(ctx, load_library().bem_warm_basis(ctx, None, C.byref(r)), "bem_warm_basis")
    phi = np.zeros((r.value, n_unknowns), np.complex128)
    _check(ctx, load_library().bem_warm_basis(ctx, _ptr(phi), C.byref(r)), "bem_warm_basis")
    return phi


def bem_warm_predict(ctx, mode, s, n_unknowns):
    """Warm-start directions x^(s), (len(s), n_unknowns) complex, host."""
    s, ns = _cplx_as_pairs(s)
    x = np.zeros((ns, n_unknowns), np.complex128)
    _check(ctx, load_library().bem_warm_predict(ctx, mode, _ptr(s), ns, _ptr(x)), "bem_warm_predict")
    return x


def bem_mlp_eval(ctx, r, params, U, T=None):
    """(y, grads, loss) of one MLP pass with the given flat float32 parameters."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    U = np.ascontiguousarray(U, dtype=np.float32)
    B = U.shape[0]
    y = np.zeros((B, 2 * r), np.float32)
    grads = None
    loss = C.c_double(0.0)
    if T is not None:
        T = np.ascontiguousarray(T, dtype=np.float32)
        grads = np.zeros_like(params)
    _check(ctx, load_library().bem_mlp_eval(ctx, r, _ptr(params), _ptr(U), B, _ptr(T), _ptr(y),
                                            _ptr(grads), C.byref(loss)), "bem_mlp_eval")
    return y, grads, loss.value


def bem_profile(ctx, enable=True):
    _check(ctx, load_library().bem_profile(ctx, 1 if enable else 0), "bem_profile")


def bem_kernel_time(ctx, kind):
    """(launches, milliseconds, frequency-launches) of a kernel class since bem_profile."""
    n = _I64()
    ms = C.c_double()
    fl = _I64()
    _check(ctx, load_library().bem_kernel_time(ctx, kind, C.byref(n), C.byref(ms), C.byref(fl)),
           "bem_kernel_time")
    return n.value, ms.value, fl.value


TUNING_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "far32_tuning.txt")


def bem_autotune(ctx, s, nfl):
    """Time every FP32 far-field launch shape for launches of the first nfl[j] frequencies of s on
    the context's mesh; returns the chosen entries as dicts (also installed in the context)."""
    s, ns = _cplx_as_pairs(s)
    n = np.ascontiguousarray(nfl, dtype=np.int32)
    out = (bem_tune_entry * len(n))()
    _check(ctx, load_library().bem_autotune(ctx, _ptr(s), ns, _ptr(n), len(n), out), "bem_autotune")
    return [dict(ne_max=e.ne_max, nfl_max=e.nfl_max, ft=e.ft, tiles=e.tiles, waves=e.waves, ms=e.ms,
                 ms_fixed=e.ms_fixed) for e in out]


def bem_set_tuning(ctx, entries):
    """Install a list of entry dicts (ne_max, nfl_max, ft, tiles, waves[, ms]); [] = fixed shape."""
    arr = (bem_tune_entry * max(len(entries), 1))()
    for a, e in zip(arr, entries):
        a.ne_max, a.nfl_max, a.ft, a.tiles, a.waves = (e["ne_max"], e["nfl_max"], e["ft"], e["tiles"],
                                                        e["waves"])
        a.ms = e.get("ms", 0.0)
        a.ms_fixed = e.get("ms_fixed", 0.0)
    _check(ctx, load_library().bem_set_tuning(ctx, arr, len(entries)), "bem_set_tuning")


def bem_load_tuning(ctx, path=TUNING_TABLE):
    _check(ctx, load_library().bem_load_tuning(ctx, path.encode()), "bem_load_tuning")


def bem_launch_shape(ctx, nfl):
    ft, tiles, waves = C.c_int32(), C.c_int32(), C.c_int32()
    _check(ctx, load_library().bem_launch_shape(ctx, nfl, C.byref(ft), C.byref(tiles), C.byref(waves)),
           "bem_launch_shape")
    return ft.value, tiles.value, waves.value


def bem_measure_peak(ctx, kind, iters=2048, reps=5):
    """(TFLOP/s of the best launch, its milliseconds, SM count) of the FMA-chain peak kernel."""
    tf = C.c_double()
    ms = C.c_double()
    sm = C.c_int32()
    _check(ctx, load_library().bem_measure_peak(ctx, kind, iters, reps, C.byref(tf), C.byref(ms),
                                                C.byref(sm)), "bem_measure_peak")
    return tf.value, ms.value, sm.value


def bem_default_hmatrix_params(**kw):
    p = bem_hmatrix_params()
    _check_global(load_library().bem_default_hmatrix_params(C.byref(p)), "bem_default_hmatrix_params")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"bem_hmatrix_params has no field {k}")
        setattr(p, k, v)
    return p


def bem_set_hmatrix(ctx, params=None):
    _check(ctx, load_library().bem_set_hmatrix(ctx, C.byref(params) if params is not None else None),
           "bem_set_hmatrix")


def bem_get_hmatrix_info(ctx):
    out = bem_hmatrix_info()
    _check(ctx, load_library().bem_get_hmatrix_info(ctx, C.byref(out)), "bem_get_hmatrix_info")
    return {name: getattr(out, name) for name, _ in bem_hmatrix_info._fields_ if name != "reserved"}


def bem_hmatrix_partition(verts, tris, params=None):
    """(perm, clusters (n, 2), lowrank (n, 2), dense (n, 2)) of the H-matrix tree and partition."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    p = params if params is not None else bem_default_hmatrix_params()
    lib = load_library()
    counts = np.zeros(3, np.int64)
    perm = np.zeros(len(t), np.int32)
    _check_global(lib.bem_hmatrix_partition(_ptr(v), len(v), _ptr(t), len(t), C.byref(p), _ptr(perm), None, 0,
                                            None, 0, None, 0, _ptr(counts)), "bem_hmatrix_partition")
    cl = np.zeros((max(int(counts[0]), 1), 2), np.int32)
    lr = np.zeros((max(int(counts[1]), 1), 2), np.int32)
    dn = np.zeros((max(int(counts[2]), 1), 2), np.int32)
    _check_global(lib.bem_hmatrix_partition(_ptr(v), len(v), _ptr(t), len(t), C.byref(p), _ptr(perm), _ptr(cl),
                                            int(counts[0]), _ptr(lr), int(counts[1]), _ptr(dn), int(counts[2]),
                                            _ptr(counts)), "bem_hmatrix_partition")
    return perm, cl[:counts[0]], lr[:counts[1]], dn[:counts[2]]


class Context:
    """Owns one bem_ctx (device + stream) and remembers the mesh size.  tuning: a launch-shape
    table file to load (True: the table written by paper_1511_04355_gb300.tune, when it exists;
    False: the fixed launch shape)."""

    def __init__(self, device: int = 0, stream=None, tuning=True):
        self.h = bem_create(device, stream)
        self.ne = 0
        path = TUNING_TABLE if tuning is True else tuning
        if path and os.path.exists(path):
            bem_load_tuning(self.h, path)

    def close(self):
        if self.h:
            bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mesh(self, verts, tris):
        bem_set_mesh(self.h, verts, tris)
        self.ne = len(tris)

    def set_material(self, mu, nu, rho):
        bem_set_material(self.h, mu, nu, rho)

    def set_bc(self, bc_type, bc_value, profile=BEM_PROFILE_STEP):
        bem_set_bc(self.h, bc_type, bc_value, profile)

    def set_options(self, **kw):
        o = bem_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        bem_set_options(self.h, o)
        return o

    def solve(self, s, x_out=None, allow_not_converged=False):
        s = np.asarray(s, dtype=np.complex128).reshape(-1)
        if x_out is None:
            x_out = np.zeros((len(s), 3 * self.ne), np.complex128)
        return bem_solve_frequencies(self.h, s, x_out, allow_not_converged)

    def apply(self, s, x, precision=BEM_PREC_FP64, which=BEM_APPLY_A):
        return bem_apply(self.h, s, x, None, precision, which)

    def rhs(self, s):
        return bem_rhs(self.h, s, self.ne)

    def residual(self, s, x, mode=BEM_RESID_DF64):
        return bem_residual(self.h, s, x, None, mode)

    def precond(self, s, x):
        return bem_precond_apply(self.h, s, x)

    def profile(self, enable=True):
        bem_profile(self.h, enable)

    def set_hmatrix(self, enable=True, **kw):
        """Enable (or disable) the H-matrix far field of the FP32 operator; kw: fields of
        bem_hmatrix_params (leaf, max_block, max_rank, eta, eps, max_freqs)."""
        bem_set_hmatrix(self.h, bem_default_hmatrix_params(enable=int(enable), **kw))

    def hmatrix_info(self):
        return bem_get_hmatrix_info(self.h)

    def kernel_times(self):
        """{name: (launches, milliseconds, frequency-launches)} since profile(True)."""
        return {name: bem_kernel_time(self.h, k) for k, name in KERNEL_NAMES.items()}

    def fsm_eval(self, h, eta, period, t, window=1):
        return bem_fsm_eval(self.h, h, eta, period, t, window)

    def afs(self, params, orf, test, t_out):
        return bem_afs(self.h, params, orf, test, t_out)

    def fsm(self, period, eta, nc, t, dofs, allow_not_converged=False):
        return bem_fsm(self.h, period, eta, nc, t, dofs, allow_not_converged)

    def geometry(self):
        return bem_geometry(self.h, self.ne)

    def near_lists(self):
        return bem_near_lists(self.h, self.ne)

    def element_blocks(self, s, rows, cols):
        return bem_element_blocks(self.h, s, rows, cols)
