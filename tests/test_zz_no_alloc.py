"""The allocation-free entry point dd_inpaint_solve_static.

It serves callers that cannot allocate device memory (code inside a framework
that owns the allocator, plug-ins that may not grow the device footprint,
real-time paths).  Its answer must match the allocating entry point
dd_inpaint_solve configured the same way (one level, FP32 iterate), within the
FP32 solve tolerance used by the other parity tests, on two calls in a row:
the second call reuses the shared scratch array left by the first.  The file
is named so that pytest collects it last."""
import numpy as np
import pytest

import synth
from oracle import inpaint_ref as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300 import binding as B  # noqa: E402
from paper_2110_03946_gb300.inpaint import Inpainter, make_params  # noqa: E402

TOL_U = 0.05          # max|du| on the 0-255 scale, as in the other FP32 parity tests
DEV = torch.device("cuda:0")


def _static_solve(mask_d, vals_d, params, tol):
    C, H, W = vals_d.shape
    out = torch.full((C, H, W), float("nan"), dtype=torch.float32, device=DEV)
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), params, tol,
                                   torch.cuda.current_stream(DEV))
    B.check(rc, "dd_inpaint_solve_static")
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,seed", [(200, 330, 3, 3), (256, 256, 1, 4)])
def test_static_matches_allocating_entry_point(H, W, C, seed):
    f, m = synth.make_frame(H, W, C, 0.04, "edge", seed)
    prm = dict(block=32, overlap=6, local_cg_iters=16, levels=1, precision="fp32")
    with Inpainter(m, f, **prm) as ip:
        u_ref = ip.solve(1e-6).cpu().numpy()
    mask_d = torch.as_tensor(m).to(DEV)
    vals_d = torch.as_tensor(f).to(DEV)
    p = make_params(**prm)
    u1 = _static_solve(mask_d, vals_d, p, 1e-6)
    # the second call reuses the scratch left by the first, and allocates no
    # device memory: the output buffer is made before the free memory is read
    out = torch.full((C, H, W), float("nan"), dtype=torch.float32, device=DEV)
    torch.cuda.synchronize(DEV)
    free0, reserved0 = torch.cuda.mem_get_info(DEV)[0], torch.cuda.memory_reserved(DEV)
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), p, 1e-6,
                                   torch.cuda.current_stream(DEV))
    B.check(rc, "dd_inpaint_solve_static (second call)")
    torch.cuda.synchronize(DEV)
    assert torch.cuda.mem_get_info(DEV)[0] == free0
    assert torch.cuda.memory_reserved(DEV) == reserved0
    u2 = out.cpu().numpy()
    for u in (u1, u2):
        assert np.isfinite(u).all()
        assert np.max(np.abs(u - u_ref)) <= TOL_U
        assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
        assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))


def test_static_empty_mask():
    # no known pixel: A is singular; the call finds it from its own block-mask count
    H, W, C = 96, 130, 2
    mask_d = torch.zeros((H, W), dtype=torch.uint8, device=DEV)
    vals_d = torch.rand((C, H, W), dtype=torch.float32, device=DEV) * 255
    out = torch.empty((C, H, W), dtype=torch.float32, device=DEV)
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), None, 1e-6,
                                   torch.cuda.current_stream(DEV))
    assert rc == B.DD_EEMPTYMASK


def test_static_not_converged_still_writes_output():
    # one sweep cannot reach 1e-6: DD_ENOTCONVERGED, and u_out holds the iterate
    # reached (finite, known pixels equal to the data)
    f, m = synth.make_frame(128, 160, 3, 0.05, "uniform", 11)
    mask_d = torch.as_tensor(m).to(DEV)
    vals_d = torch.as_tensor(f).to(DEV)
    C, H, W = f.shape
    out = torch.full((C, H, W), float("nan"), dtype=torch.float32, device=DEV)
    p = make_params(block=32, overlap=6, local_cg_iters=8, levels=1, precision="fp32", max_sweeps=1)
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), p, 1e-6,
                                   torch.cuda.current_stream(DEV))
    assert rc == B.DD_ENOTCONVERGED
    u = out.cpu().numpy()
    assert np.isfinite(u).all()
    assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))
    rel = ref.rel_residual(u.astype(np.float64), f, m)
    assert np.all(rel < 1.0) and np.any(rel > 1e-6)


def test_static_rejects_bad_params():
    H, W, C = 64, 64, 1
    mask_d = torch.ones((H, W), dtype=torch.uint8, device=DEV)
    vals_d = torch.zeros((C, H, W), dtype=torch.float32, device=DEV)
    out = torch.empty((C, H, W), dtype=torch.float32, device=DEV)
    for bad in (dict(local_rtol=1.5), dict(local_cg_iters=5000), dict(solver="cg")):
        p = make_params(levels=1, precision="fp32", **bad)
        rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), p, 1e-6, None)
        assert rc == B.DD_EINVAL, bad


def test_static_rejects_oversized_input():
    H, W, C = 2048, 2049, 1                           # C*H*roundup(W,32) > 2^22
    mask_d = torch.ones((H, W), dtype=torch.uint8, device=DEV)
    vals_d = torch.zeros((C, H, W), dtype=torch.float32, device=DEV)
    out = torch.empty((C, H, W), dtype=torch.float32, device=DEV)
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), None, 1e-6, None)
    assert rc == B.DD_EINVAL
    assert "capacity" in B.dd_last_error()


def test_static_rejects_block_masks_beyond_capacity():
    # 64 x 64 blocks of eight warps at stride 16: about 15000 blocks of 256 threads, whose
    # masks (2 words per thread) exceed the 2^20 block-thread capacity of the shared array
    H, W, C = 2048, 2016, 1
    mask_d = torch.ones((H, W), dtype=torch.uint8, device=DEV)
    vals_d = torch.zeros((C, H, W), dtype=torch.float32, device=DEV)
    out = torch.empty((C, H, W), dtype=torch.float32, device=DEV)
    p = make_params(block=64, overlap=48, tile_warps=8, levels=1, precision="fp32")
    rc = B.dd_inpaint_solve_static(H, W, C, mask_d.data_ptr(), vals_d.data_ptr(), out.data_ptr(), p, 1e-6, None)
    assert rc == B.DD_EINVAL
    assert "capacity" in B.dd_last_error()
