"""ctypes front end of the plain C FP64 CG oracle (``cg_ref.c``).

TEST INFRASTRUCTURE ONLY.  Solves A u = b (paper Sec. 2, Eq. eq:ls) on the
unknown pixels by conjugate gradients to a relative residual ``tol`` measured
against u0 = C f.  Used where the sparse direct solve of ``inpaint_ref`` is too
slow (full-HD and 4K frames) and as the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_ref.c")
_LIB = os.path.join(_HERE, "liboracle_cg.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cg_ref.c with gcc -O2 -fopenmp into liboracle_cg.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_cg_solve.restype = ctypes.c_int
        lib.oracle_cg_solve.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_cg_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_cg_threads())


def solve_cg(f, mask, tol: float = 1e-12, max_iter: int = 200000):
    """Return (u, iters, relres): u float64 shaped like f; per-channel
    iteration counts and final true relative residuals."""
    lib = _load()
    f = np.asarray(f, dtype=np.float64)
    two_d = f.ndim == 2
    f3 = np.ascontiguousarray(f[None] if two_d else f)
    m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
    C, H, W = f3.shape
    if m.shape != (H, W):
        raise ValueError("mask shape mismatch")
    u = np.empty_like(f3)
    iters = np.zeros(C, dtype=np.int32)
    rel = np.zeros(C, dtype=np.float64)
    rc = lib.oracle_cg_solve(H, W, C, m.ctypes.data, f3.ctypes.data, u.ctypes.data,
                             float(tol), int(max_iter), iters.ctypes.data, rel.ctypes.data)
    if rc == -3:
        raise ValueError("empty mask: A is singular")
    if rc < 0:
        raise RuntimeError(f"oracle_cg_solve failed ({rc})")
    return (u[0] if two_d else u), iters, rel
