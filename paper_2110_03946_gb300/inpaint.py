"""Python convenience layer over the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and streams only; every step of the solver runs
in the CUDA library through ``binding``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

PRECISIONS = {"fp32": B.DD_PREC_FP32, "fp32_ref": B.DD_PREC_FP32_REF,
              "fp16_ref": B.DD_PREC_FP16_REF, "bf16_ref": B.DD_PREC_BF16_REF}
ML_MODES = {"cascade": B.DD_ML_CASCADE, "correction": B.DD_ML_CORRECTION}


def make_params(block=None, overlap=None, local_cg_iters=None, levels=None, ml_mode=None,
                robin_p=None, precision=None, max_sweeps=None, coarse_tol=None, inner_tol=None,
                max_corrections=None, coarse_sweeps=None, inputs_on_device=1, timing=None,
                tile_warps=None, solver=None, device_loop=None, correction_sweeps=None,
                local_rtol=None, coarse_factor=None, test_stall_polls=None,
                correction_trigger=None, final_local_rtol=None, correction_cg=None,
                local_atol=None) -> B.dd_params:
    p = B.dd_params_default()
    if block is not None: p.block = int(block)
    if overlap is not None: p.overlap = int(overlap)
    if local_cg_iters is not None: p.local_cg_iters = int(local_cg_iters)
    if levels is not None: p.levels = int(levels)
    if ml_mode is not None: p.ml_mode = ML_MODES[ml_mode] if isinstance(ml_mode, str) else int(ml_mode)
    if robin_p is not None: p.robin_p = float(robin_p)
    if precision is not None:
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if max_sweeps is not None: p.max_sweeps = int(max_sweeps)
    if coarse_tol is not None: p.coarse_tol = float(coarse_tol)
    if inner_tol is not None: p.inner_tol = float(inner_tol)
    if max_corrections is not None: p.max_corrections = int(max_corrections)
    if coarse_sweeps is not None: p.coarse_sweeps = int(coarse_sweeps)
    if timing is not None: p.timing = int(timing)
    if tile_warps is not None: p.tile_warps = int(tile_warps)
    if solver is not None:
        p.solver = {"oras": B.DD_SOLVER_ORAS, "cg": B.DD_SOLVER_CG}[solver] if isinstance(solver, str) else int(solver)
    if device_loop is not None: p.device_loop = int(device_loop)
    if correction_sweeps is not None: p.correction_sweeps = int(correction_sweeps)
    if local_rtol is not None: p.local_rtol = float(local_rtol)
    if coarse_factor is not None: p.coarse_factor = int(coarse_factor)
    if test_stall_polls is not None: p.test_stall_polls = int(test_stall_polls)
    if correction_trigger is not None: p.correction_trigger = float(correction_trigger)
    if final_local_rtol is not None: p.final_local_rtol = float(final_local_rtol)
    if correction_cg is not None: p.correction_cg = int(correction_cg)
    if local_atol is not None: p.local_atol = float(local_atol)
    p.inputs_on_device = int(inputs_on_device)
    return p


def _dev_u8(mask, device):
    t = torch.as_tensor(np.ascontiguousarray(mask) if isinstance(mask, np.ndarray) else mask)
    return (t != 0).to(device=device, dtype=torch.uint8).contiguous()


def _dev_f32(values, device):
    t = torch.as_tensor(np.ascontiguousarray(values) if isinstance(values, np.ndarray) else values)
    return t.to(device=device, dtype=torch.float32).contiguous()


class Inpainter:
    """One frame's solver state (a dd_inpaint handle).

    mask: (H, W), nonzero = known; values: (C, H, W) or (H, W).  Inputs may be
    numpy arrays or torch tensors; they are copied to the current CUDA device.
    """

    def __init__(self, mask, values, device="cuda", **params):
        self.device = torch.device(device)
        m = _dev_u8(mask, self.device)
        v = _dev_f32(values, self.device)
        if v.dim() == 2:
            v = v.unsqueeze(0)
        self.C, self.H, self.W = v.shape
        if tuple(m.shape) != (self.H, self.W):
            raise ValueError("mask shape does not match values")
        self.params = make_params(inputs_on_device=1, **params)
        with torch.cuda.device(self.device):
            rc, h = B.dd_inpaint_create(self.H, self.W, self.C, m.data_ptr(), v.data_ptr(), self.params)
        B.check(rc, "dd_inpaint_create")
        self._h = h

    def solve(self, tol: float = 1e-6, out: torch.Tensor | None = None, stream=None, allow_unconverged=False):
        if out is None:
            out = torch.empty((self.C, self.H, self.W), device=self.device, dtype=torch.float32)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        rc = B.dd_inpaint_solve(self._h, out.data_ptr(), float(tol), stream)
        ok = (B.DD_OK, B.DD_ENOTCONVERGED) if allow_unconverged else (B.DD_OK,)
        B.check(rc, "dd_inpaint_solve", ok)
        return out

    def set_data(self, mask, values, keep_iterate: bool):
        m = _dev_u8(mask, self.device)
        v = _dev_f32(values, self.device)
        torch.cuda.synchronize(self.device)
        B.check(B.dd_inpaint_set_data(self._h, m.data_ptr(), v.data_ptr(), int(keep_iterate)), "dd_inpaint_set_data")

    def set_iterate(self, u: torch.Tensor, stream=None):
        u = _dev_f32(u, self.device)
        B.check(B.dd_inpaint_set_iterate(self._h, u.data_ptr(), stream or torch.cuda.current_stream(self.device)),
                "dd_inpaint_set_iterate")
        torch.cuda.synchronize(self.device)

    def get_iterate(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.C, self.H, self.W), device=self.device, dtype=torch.float32)
        B.check(B.dd_inpaint_get_iterate(self._h, out.data_ptr(), stream or torch.cuda.current_stream(self.device)),
                "dd_inpaint_get_iterate")
        return out

    def sweep(self, n: int = 1, stream=None):
        rc, norms = B.dd_inpaint_sweep(self._h, n, self.C, stream or torch.cuda.current_stream(self.device))
        B.check(rc, "dd_inpaint_sweep")
        return norms

    def stats(self) -> dict:
        rc, s = B.dd_inpaint_stats(self._h)
        B.check(rc, "dd_inpaint_stats")
        return {
            "sweeps_total": s.sweeps_total,
            "sweeps_per_level": list(s.sweeps_per_level),
            "corrections": s.corrections,
            "converged": bool(s.converged),
            "rel_residual": list(s.rel_residual)[: min(self.C, B.DD_MAX_STAT_CHANNELS)],
            "ms_total": s.ms_total,
            "device_bytes": int(s.device_bytes),
            "kernel_launches": int(s.kernel_launches),
            "local_unknowns": int(s.local_unknowns),
            "fine_sweep_launches": int(s.fine_sweep_launches),
            "fine_sweep_ms": float(s.fine_sweep_ms),
            "fine_cg_pixel_steps": int(s.fine_cg_pixel_steps),
            "fine_swept_unknowns": int(s.fine_swept_unknowns),
            "host_continued": bool(s.host_continued),
            "coarse_corrections": int(s.coarse_corrections),
        }

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            B.dd_inpaint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def inpaint(mask, values, tol: float = 1e-6, **params) -> torch.Tensor:
    """Solve one frame and return u (C, H, W) float32 on the GPU."""
    with Inpainter(mask, values, **params) as ip:
        return ip.solve(tol)
