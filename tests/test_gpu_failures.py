"""Failure paths of the C ABI, made without a GPU fault.

DD_ETIMEOUT: the test hook params.test_stall_polls makes every CTA's first wait
for a staged tile poll a barrier that no copy completes; the wait gives up
after that many polls, the kernel waits for its copies in flight and returns,
and the solve reports DD_ETIMEOUT.  The context stays usable: a normal solve on
the same device afterwards matches the oracle.  DD_ENUMERIC: NaN or Inf among
the known values.  DD_ENOMEM: a device budget smaller than a handle
(dd_set_device_budget), checked on the host before any allocation."""
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

DEV = torch.device("cuda:0")
TOL_U = 0.05


def _normal_solve_still_matches():
    f, m = synth.make_frame(96, 130, 3, 0.05, "uniform", 77)
    with Inpainter(m, f, block=32, overlap=4, levels=2, precision="fp32") as ip:
        u = ip.solve(1e-6).cpu().numpy()
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U


@pytest.mark.parametrize("params", [
    dict(levels=2, precision="fp32"),                       # device loops
    dict(levels=2, precision="fp32", device_loop=0),        # plain launches
    dict(levels=1, precision="fp32", timing=1),             # host-timed launches
    dict(levels=2, precision="fp16_ref"),                   # device correction loop
    dict(levels=2, precision="fp32_ref", device_loop=0),    # host correction loop
])
def test_stalled_wait_reports_timeout(params):
    f, m = synth.make_frame(96, 130, 3, 0.05, "uniform", 5)
    with Inpainter(m, f, block=32, overlap=4, test_stall_polls=64, **params) as ip:
        out = torch.empty((3, 96, 130), dtype=torch.float32, device=DEV)
        for _ in range(2):   # the same code every time: nothing stays stuck
            rc = B.dd_inpaint_solve(ip._h, out.data_ptr(), 1e-6, torch.cuda.current_stream(DEV))
            assert rc == B.DD_ETIMEOUT, B.dd_strerror(rc)
            assert "gave up" in B.dd_last_error()
        torch.cuda.synchronize(DEV)
    _normal_solve_still_matches()


def test_stalled_wait_in_async_and_batch_paths():
    f, m = synth.make_frame(96, 130, 3, 0.05, "uniform", 6)
    with Inpainter(m, f, block=32, overlap=4, levels=2, precision="fp32", test_stall_polls=16) as ip:
        out = torch.empty((3, 96, 130), dtype=torch.float32, device=DEV)
        s = torch.cuda.current_stream(DEV)
        B.check(B.dd_inpaint_solve_async(ip._h, out.data_ptr(), 1e-6, s), "solve_async")
        assert B.dd_inpaint_solve_finish(ip._h, s) == B.DD_ETIMEOUT
        rc, b, _ = B.dd_batch_create([ip._h], [out.data_ptr()], 1e-6)
        B.check(rc, "batch_create")
        try:
            B.check(B.dd_batch_launch(b, s), "batch_launch")
            rc, st = B.dd_batch_finish(b, 1, s)
            assert rc == B.DD_ETIMEOUT and st == [B.DD_ETIMEOUT]
        finally:
            B.dd_batch_destroy(b)
    _normal_solve_still_matches()


def test_stalled_wait_in_static_solve():
    f, m = synth.make_frame(80, 100, 2, 0.05, "uniform", 7)
    md, fd = torch.as_tensor(m).to(DEV), torch.as_tensor(f).to(DEV)
    out = torch.empty((2, 80, 100), dtype=torch.float32, device=DEV)
    p = make_params(block=32, overlap=4, levels=1, precision="fp32", test_stall_polls=32)
    rc = B.dd_inpaint_solve_static(80, 100, 2, md.data_ptr(), fd.data_ptr(), out.data_ptr(), p, 1e-6,
                                   torch.cuda.current_stream(DEV))
    assert rc == B.DD_ETIMEOUT
    p.test_stall_polls = 0
    rc = B.dd_inpaint_solve_static(80, 100, 2, md.data_ptr(), fd.data_ptr(), out.data_ptr(), p, 1e-6,
                                   torch.cuda.current_stream(DEV))
    B.check(rc, "static solve after the timeout")
    assert np.max(np.abs(out.cpu().numpy() - ref.solve_direct(f, m))) <= TOL_U


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("params", [
    dict(levels=3, precision="fp32"),
    dict(levels=2, precision="fp32", device_loop=0),
    dict(levels=2, precision="fp16_ref"),
    dict(levels=2, precision="fp32", solver="cg", max_sweeps=500),
])
def test_non_finite_known_value_reports_numeric(bad, params):
    f, m = synth.make_frame(64, 96, 3, 0.05, "uniform", 8)
    ky, kx = np.argwhere(m != 0)[3]
    f = f.copy()
    f[1, ky, kx] = bad
    with Inpainter(m, f, block=32, overlap=4, **params) as ip:
        out = torch.empty((3, 64, 96), dtype=torch.float32, device=DEV)
        rc = B.dd_inpaint_solve(ip._h, out.data_ptr(), 1e-6, torch.cuda.current_stream(DEV))
        assert rc == B.DD_ENUMERIC, B.dd_strerror(rc)
    _normal_solve_still_matches()


def test_device_budget_gives_enomem_and_frees_partial_allocations():
    f, m = synth.make_frame(256, 256, 3, 0.05, "uniform", 9)
    md, fd = torch.as_tensor(m).to(DEV), torch.as_tensor(f).to(DEV)
    p = make_params(levels=3, precision="fp32")
    held0 = B.dd_device_bytes_in_use()
    B.dd_set_device_budget(held0 + (1 << 20))   # 1 MiB more than is held: a 256 x 256 x 3 handle needs more
    try:
        rc, h = B.dd_inpaint_create(256, 256, 3, md.data_ptr(), fd.data_ptr(), p)
        assert rc == B.DD_ENOMEM and not h.value
        assert "budget" in B.dd_last_error()
        assert B.dd_device_bytes_in_use() == held0    # the partial allocations were released
    finally:
        B.dd_set_device_budget(0)
    rc, h = B.dd_inpaint_create(256, 256, 3, md.data_ptr(), fd.data_ptr(), p)
    B.check(rc, "create without a budget")
    try:
        rc, st = B.dd_inpaint_stats(h)
        assert B.dd_device_bytes_in_use() == held0 + st.device_bytes
    finally:
        B.dd_inpaint_destroy(h)
    assert B.dd_device_bytes_in_use() == held0


def test_timed_launches_are_the_full_sweeps():
    # with timing on, only launches that ran as full sweeps are timed (probes
    # and launches after the stop are not), so the timed count equals the
    # fine-level sweep count of a solve that converges within the first chunk
    f, m = synth.make_frame(192, 256, 3, 0.03, "edge", 10)
    with Inpainter(m, f, block=32, overlap=3, levels=3, precision="fp32", timing=1, local_rtol=0.05,
                   local_cg_iters=20) as ip:
        ip.solve(1e-6)
        st = ip.stats()
    assert st["converged"] and not st["host_continued"]
    assert st["fine_sweep_launches"] == st["sweeps_per_level"][0]
    assert st["fine_sweep_ms"] > 0 and st["fine_cg_pixel_steps"] > 0
