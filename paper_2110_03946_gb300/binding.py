"""Thin ctypes binding of the dd_inpaint C ABI (include/dd_inpaint.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions carry the C names; pointers are passed as integers (e.g. a torch
CUDA tensor's ``data_ptr()``), streams as integers (``torch.cuda.Stream
.cuda_stream``) or None.  Loading fails loudly if the library is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdd_inpaint.so")

DD_OK, DD_EINVAL, DD_EEMPTYMASK, DD_ENOMEM, DD_ENOTCONVERGED, DD_ENUMERIC, DD_ECUDA, DD_ETIMEOUT, DD_EAGAIN = range(9)
DD_ML_CASCADE, DD_ML_CORRECTION = 0, 1
DD_SOLVER_ORAS, DD_SOLVER_CG = 0, 1
DD_PREC_FP32, DD_PREC_FP32_REF, DD_PREC_FP16_REF, DD_PREC_BF16_REF = 0, 1, 2, 3
DD_BATCH_GRAPH, DD_BATCH_PERSISTENT = 0, 1
DD_MAX_STAT_CHANNELS = 16
DD_MAX_LEVELS = 8

# every entry point declared in include/dd_inpaint.h
EXPORTS = (
    "dd_params_default", "dd_strerror", "dd_last_error",
    "dd_inpaint_create", "dd_inpaint_solve", "dd_inpaint_destroy", "dd_inpaint_set_data",
    "dd_inpaint_stats", "dd_inpaint_set_iterate", "dd_inpaint_get_iterate", "dd_inpaint_sweep",
    "dd_restrict", "dd_prolong", "dd_coarse_cg", "dd_residual_norms", "dd_inpaint_solve_static",
    "dd_inpaint_set_data_async", "dd_inpaint_solve_async", "dd_inpaint_query", "dd_inpaint_solve_finish",
    "dd_batch_create", "dd_batch_create_mode", "dd_batch_launch", "dd_batch_finish", "dd_batch_destroy",
    "dd_set_device_budget", "dd_device_bytes_in_use", "dd_fp32_fma_peak",
)


class dd_params(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_int), ("overlap", ctypes.c_int), ("local_cg_iters", ctypes.c_int),
        ("levels", ctypes.c_int), ("ml_mode", ctypes.c_int), ("coarse_factor", ctypes.c_int),
        ("robin_p", ctypes.c_float), ("precision", ctypes.c_int), ("max_sweeps", ctypes.c_int),
        ("inputs_on_device", ctypes.c_int), ("coarse_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
        ("max_corrections", ctypes.c_int), ("coarse_sweeps", ctypes.c_int), ("timing", ctypes.c_int),
        ("tile_warps", ctypes.c_int), ("solver", ctypes.c_int), ("correction_sweeps", ctypes.c_int),
        ("local_rtol", ctypes.c_double), ("device_loop", ctypes.c_int), ("test_stall_polls", ctypes.c_int),
        ("correction_trigger", ctypes.c_double), ("final_local_rtol", ctypes.c_double),
        ("correction_cg", ctypes.c_int), ("local_atol", ctypes.c_double),
    ]


class dd_stats(ctypes.Structure):
    _fields_ = [
        ("sweeps_total", ctypes.c_int), ("sweeps_per_level", ctypes.c_int * DD_MAX_LEVELS),
        ("corrections", ctypes.c_int), ("converged", ctypes.c_int), ("channels", ctypes.c_int),
        ("rel_residual", ctypes.c_double * DD_MAX_STAT_CHANNELS), ("ms_total", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_longlong),
        ("local_unknowns", ctypes.c_longlong), ("fine_sweep_launches", ctypes.c_int),
        ("fine_sweep_ms", ctypes.c_double),
        ("fine_cg_pixel_steps", ctypes.c_longlong), ("fine_swept_unknowns", ctypes.c_longlong),
        ("host_continued", ctypes.c_int), ("coarse_corrections", ctypes.c_int),
    ]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def load(path: str | None = None):
    """Load the CUDA library (raises OSError / RuntimeError if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"dd_inpaint CUDA library not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    sig = {
        "dd_params_default": (None, [ctypes.POINTER(dd_params)]),
        "dd_strerror": (ctypes.c_char_p, [_I]),
        "dd_last_error": (ctypes.c_char_p, []),
        "dd_inpaint_create": (_I, [_I, _I, _I, _P, _P, ctypes.POINTER(dd_params), ctypes.POINTER(_P)]),
        "dd_inpaint_solve": (_I, [_P, _P, _D, _P]),
        "dd_inpaint_destroy": (_I, [_P]),
        "dd_inpaint_set_data": (_I, [_P, _P, _P, _I]),
        "dd_inpaint_stats": (_I, [_P, ctypes.POINTER(dd_stats)]),
        "dd_inpaint_set_iterate": (_I, [_P, _P, _P]),
        "dd_inpaint_get_iterate": (_I, [_P, _P, _P]),
        "dd_inpaint_sweep": (_I, [_P, _I, _P, _P]),
        "dd_restrict": (_I, [_I, _I, _I, _P, _P, _P, _P, _P]),
        "dd_prolong": (_I, [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P]),
        "dd_coarse_cg": (_I, [_I, _I, _I, _P, _P, _P, _I, _D, _P, _P]),
        "dd_residual_norms": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P]),
        "dd_inpaint_solve_static": (_I, [_I, _I, _I, _P, _P, _P, ctypes.POINTER(dd_params), _D, _P]),
        "dd_inpaint_set_data_async": (_I, [_P, _P, _P, _I, _P]),
        "dd_inpaint_solve_async": (_I, [_P, _P, _D, _P]),
        "dd_inpaint_query": (_I, [_P]),
        "dd_inpaint_solve_finish": (_I, [_P, _P]),
        "dd_batch_create": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, ctypes.POINTER(_P),
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "dd_batch_create_mode": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(_P),
                                      ctypes.POINTER(ctypes.c_longlong)]),
        "dd_batch_launch": (_I, [_P, _P]),
        "dd_batch_finish": (_I, [_P, _P, ctypes.POINTER(_I)]),
        "dd_batch_destroy": (_I, [_P]),
        "dd_set_device_budget": (None, [ctypes.c_size_t]),
        "dd_device_bytes_in_use": (ctypes.c_size_t, []),
        "dd_fp32_fma_peak": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DDError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.dd_strerror(code).decode()
        detail = lib.dd_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}) {detail}")
        self.code = code


def check(code: int, where: str, ok=(DD_OK,)):
    if code not in ok:
        raise DDError(code, where)
    return code


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


# ---- functions with the C names -------------------------------------------------------
def dd_params_default() -> dd_params:
    p = dd_params()
    load().dd_params_default(ctypes.byref(p))
    return p


def dd_strerror(code: int) -> str:
    return load().dd_strerror(code).decode()


def dd_last_error() -> str:
    return load().dd_last_error().decode()


def dd_inpaint_create(H: int, W: int, C: int, mask_ptr: int, values_ptr: int, params: dd_params | None):
    """Returns (code, handle)."""
    h = ctypes.c_void_p()
    rc = load().dd_inpaint_create(H, W, C, mask_ptr, values_ptr,
                                  ctypes.byref(params) if params is not None else None, ctypes.byref(h))
    return rc, h


def dd_inpaint_solve(h, u_out_ptr: int, tol: float, stream=None) -> int:
    return load().dd_inpaint_solve(h, u_out_ptr, tol, _stream(stream))


def dd_inpaint_destroy(h) -> int:
    return load().dd_inpaint_destroy(h)


def dd_inpaint_set_data(h, mask_ptr: int, values_ptr: int, keep_iterate: int) -> int:
    return load().dd_inpaint_set_data(h, mask_ptr, values_ptr, int(keep_iterate))


def dd_inpaint_stats(h):
    s = dd_stats()
    rc = load().dd_inpaint_stats(h, ctypes.byref(s))
    return rc, s


def dd_inpaint_set_iterate(h, u_ptr: int, stream=None) -> int:
    return load().dd_inpaint_set_iterate(h, u_ptr, _stream(stream))


def dd_inpaint_get_iterate(h, u_out_ptr: int, stream=None) -> int:
    return load().dd_inpaint_get_iterate(h, u_out_ptr, _stream(stream))


def dd_inpaint_sweep(h, n: int, C: int | None = None, stream=None):
    """Returns (code, list of C input-iterate residual norms or None)."""
    if C is None:
        return load().dd_inpaint_sweep(h, n, None, _stream(stream)), None
    buf = (ctypes.c_double * C)()
    rc = load().dd_inpaint_sweep(h, n, buf, _stream(stream))
    return rc, list(buf)


def dd_restrict(H, W, C, mask_ptr, f_ptr, mask_c_ptr, f_c_ptr, stream=None) -> int:
    return load().dd_restrict(H, W, C, mask_ptr, f_ptr, mask_c_ptr, f_c_ptr, _stream(stream))


def dd_prolong(Hc, Wc, H, W, C, uc_ptr, mask_ptr, f_ptr, u_ptr, stream=None) -> int:
    return load().dd_prolong(Hc, Wc, H, W, C, uc_ptr, mask_ptr, f_ptr, u_ptr, _stream(stream))


def dd_coarse_cg(H, W, C, mask_ptr, g_ptr, e_ptr, max_iter: int, tol: float, stream=None):
    """Returns (code, list of C iteration counts)."""
    it = (ctypes.c_int * C)()
    rc = load().dd_coarse_cg(H, W, C, mask_ptr, g_ptr, e_ptr, int(max_iter), float(tol), it, _stream(stream))
    return rc, list(it)


def dd_inpaint_solve_static(H, W, C, mask_ptr, values_ptr, u_out_ptr, params, tol, stream=None) -> int:
    """Allocation-free one-level FP32 solve into caller buffers (all device)."""
    return load().dd_inpaint_solve_static(H, W, C, mask_ptr, values_ptr, u_out_ptr,
                                          ctypes.byref(params) if params is not None else None, tol,
                                          _stream(stream))


def dd_residual_norms(H, W, C, mask_ptr, f_ptr, u_ptr, stream=None):
    """Returns (code, norms list, ref_norms list)."""
    n = (ctypes.c_double * C)()
    r = (ctypes.c_double * C)()
    rc = load().dd_residual_norms(H, W, C, mask_ptr, f_ptr, u_ptr, n, r, _stream(stream))
    return rc, list(n), list(r)


def dd_inpaint_set_data_async(h, mask_ptr: int, values_ptr: int, keep_iterate: int, stream=None) -> int:
    return load().dd_inpaint_set_data_async(h, mask_ptr, values_ptr, int(keep_iterate), _stream(stream))


def dd_inpaint_solve_async(h, u_out_ptr: int, tol: float, stream=None) -> int:
    return load().dd_inpaint_solve_async(h, u_out_ptr, tol, _stream(stream))


def dd_inpaint_query(h) -> int:
    return load().dd_inpaint_query(h)


def dd_inpaint_solve_finish(h, stream=None) -> int:
    return load().dd_inpaint_solve_finish(h, _stream(stream))


def dd_batch_create(handles, out_ptrs, tol: float, mode: int | None = None):
    """Returns (code, batch handle, kernels per launch); mode None = the
    library's default (dd_batch_create), else dd_batch_create_mode."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    outs = (ctypes.c_void_p * n)(*out_ptrs)
    b = ctypes.c_void_p()
    k = ctypes.c_longlong(0)
    if mode is None:
        rc = load().dd_batch_create(n, hs, outs, tol, ctypes.byref(b), ctypes.byref(k))
    else:
        rc = load().dd_batch_create_mode(n, hs, outs, tol, int(mode), ctypes.byref(b), ctypes.byref(k))
    return rc, b, k.value


def dd_batch_launch(b, stream=None) -> int:
    return load().dd_batch_launch(b, _stream(stream))


def dd_batch_finish(b, n: int, stream=None):
    """Returns (code, list of n per-handle codes)."""
    st = (ctypes.c_int * n)()
    rc = load().dd_batch_finish(b, _stream(stream), st)
    return rc, list(st)


def dd_batch_destroy(b) -> int:
    return load().dd_batch_destroy(b)


def dd_set_device_budget(nbytes: int) -> None:
    load().dd_set_device_budget(int(nbytes))


def dd_device_bytes_in_use() -> int:
    return int(load().dd_device_bytes_in_use())


def dd_fp32_fma_peak(reps: int = 5, stream=None):
    """Returns (code, TFLOP/s, SM count)."""
    t = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    rc = load().dd_fp32_fma_peak(int(reps), ctypes.byref(t), ctypes.byref(n), _stream(stream))
    return rc, t.value, n.value
