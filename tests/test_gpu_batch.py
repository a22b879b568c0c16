"""Asynchronous solves and CUDA-graph batches through the C ABI.

The asynchronous and batched paths run the same kernels with the same
parameters as dd_inpaint_solve, so their outputs must equal the synchronous
ones bit for bit, and match the oracle within the FP32 solve tolerance."""
import numpy as np
import pytest

import synth
from oracle import inpaint_ref as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300 import binding as B  # noqa: E402
from paper_2110_03946_gb300.inpaint import Inpainter  # noqa: E402

DEV = torch.device("cuda:0")
TOL_U = 0.05
PRM = dict(block=32, overlap=3, local_cg_iters=16, robin_p=0.15, levels=3, coarse_tol=3e-3, precision="fp32")
SHAPES = [(120, 170, 3, 0.05, "uniform"), (96, 64, 1, 0.08, "edge"), (257, 190, 3, 0.03, "edge"),
          (40, 300, 2, 0.06, "uniform")]


def _frames(seed0):
    return [synth.make_frame(H, W, C, d, pat, seed0 + i) for i, (H, W, C, d, pat) in enumerate(SHAPES)]


def _sync_solve(f, m):
    with Inpainter(m, f, **PRM) as ip:
        return ip.solve(1e-6).cpu().numpy()


def test_async_solves_on_several_streams_match_sync():
    frames = _frames(700)
    ips = [Inpainter(m, f, **PRM) for f, m in frames]
    streams = [torch.cuda.Stream(DEV) for _ in frames]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    dev_in = [(torch.as_tensor(m).to(DEV), torch.as_tensor(f).to(DEV)) for f, m in frames]
    torch.cuda.synchronize()
    for ip, s, (md, fd), o in zip(ips, streams, dev_in, outs):
        B.check(B.dd_inpaint_set_data_async(ip._h, md.data_ptr(), fd.data_ptr(), 0, s), "set_data_async")
        B.check(B.dd_inpaint_solve_async(ip._h, o.data_ptr(), 1e-6, s), "solve_async")
    for ip, s in zip(ips, streams):
        B.check(B.dd_inpaint_solve_finish(ip._h, s), "finish")
        assert B.dd_inpaint_query(ip._h) == B.DD_EINVAL          # nothing in flight any more
    for (f, m), o, ip in zip(frames, outs, ips):
        u = o.cpu().numpy()
        assert np.array_equal(u, _sync_solve(f, m))
        assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
        assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
        ip.close()


def test_async_empty_mask_reported_at_finish():
    f, m = synth.make_frame(64, 64, 1, 0.05, "uniform", 3)
    with Inpainter(m, f, **PRM) as ip:
        z = torch.zeros((64, 64), dtype=torch.uint8, device=DEV)
        fd = torch.as_tensor(f).to(DEV)
        out = torch.empty((1, 64, 64), dtype=torch.float32, device=DEV)
        B.check(B.dd_inpaint_set_data_async(ip._h, z.data_ptr(), fd.data_ptr(), 0, None), "set_data_async")
        B.check(B.dd_inpaint_solve_async(ip._h, out.data_ptr(), 1e-6, None), "solve_async")
        assert B.dd_inpaint_solve_finish(ip._h, None) == B.DD_EEMPTYMASK
        assert B.dd_inpaint_solve(ip._h, out.data_ptr(), 1e-6, None) == B.DD_EEMPTYMASK
        md = torch.as_tensor(m).to(DEV)
        B.check(B.dd_inpaint_set_data(ip._h, md.data_ptr(), fd.data_ptr(), 0), "set_data")
        B.check(B.dd_inpaint_solve(ip._h, out.data_ptr(), 1e-6, None), "solve")


def test_batch_graph_matches_independent_solves():
    frames_a, frames_b = _frames(800), _frames(900)
    ips = [Inpainter(m, f, **PRM) for f, m in frames_a]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames_a]
    rc, b, kernels = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6)
    B.check(rc, "dd_batch_create")
    assert kernels > len(ips)
    try:
        for frames in (frames_a, frames_b):       # second launch: new data in the same handles
            dev_in = [(torch.as_tensor(m).to(DEV), torch.as_tensor(f).to(DEV)) for f, m in frames]
            for ip, (md, fd) in zip(ips, dev_in):
                B.check(B.dd_inpaint_set_data(ip._h, md.data_ptr(), fd.data_ptr(), 0), "set_data")
            stream = torch.cuda.current_stream(DEV)
            B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
            rc, status = B.dd_batch_finish(b, len(ips), stream)
            assert rc == B.DD_OK and all(sc == B.DD_OK for sc in status)
            for (f, m), o, ip in zip(frames, outs, ips):
                u = o.cpu().numpy()
                assert np.array_equal(u, _sync_solve(f, m))
                assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
                assert ip.stats()["converged"]
    finally:
        B.dd_batch_destroy(b)
        for ip in ips:
            ip.close()


def test_batch_rejects_bad_input():
    f, m = synth.make_frame(64, 64, 1, 0.05, "uniform", 4)
    with Inpainter(m, f, precision="fp16_ref", device_loop=0) as ip16, Inpainter(m, f, **PRM) as ip:
        o = torch.empty((1, 64, 64), dtype=torch.float32, device=DEV)
        # the host-driven correction loop cannot be captured
        rc, b, _ = B.dd_batch_create([ip16._h], [o.data_ptr()], 1e-6)
        assert rc == B.DD_EINVAL and not b.value
        rc, b, _ = B.dd_batch_create([ip._h, ip._h], [o.data_ptr(), o.data_ptr()], 1e-6)
        assert rc == B.DD_EINVAL


PRM16 = dict(block=32, overlap=4, local_cg_iters=18, local_rtol=0.05, levels=3, coarse_tol=3e-3, precision="fp16_ref")


def test_mixed_precision_async_and_batch():
    """FP16 inner storage with the FP64-accurate outer correction, driven on the
    device: asynchronous solves on several streams and a batch graph give the
    synchronous solve's result bit for bit, within tolerance of the oracle."""
    frames = _frames(1000)
    sync = []
    for f, m in frames:
        with Inpainter(m, f, **PRM16) as ip:
            sync.append(ip.solve(1e-6).cpu().numpy())
            st = ip.stats()
            assert st["converged"] and st["corrections"] >= 1
    ips = [Inpainter(m, f, **PRM16) for f, m in frames]
    streams = [torch.cuda.Stream(DEV) for _ in frames]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    try:
        for ip, s, o in zip(ips, streams, outs):
            B.check(B.dd_inpaint_solve_async(ip._h, o.data_ptr(), 1e-6, s), "solve_async")
        for ip, s in zip(ips, streams):
            B.check(B.dd_inpaint_solve_finish(ip._h, s), "finish")
        for (f, m), o, u0 in zip(frames, outs, sync):
            u = o.cpu().numpy()
            assert np.array_equal(u, u0)
            assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
            assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
        rc, b, _ = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6)
        B.check(rc, "dd_batch_create")
        try:
            for o in outs:
                o.zero_()
            stream = torch.cuda.current_stream(DEV)
            B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
            rc, status = B.dd_batch_finish(b, len(ips), stream)
            assert rc == B.DD_OK and all(sc == B.DD_OK for sc in status)
            for o, u0 in zip(outs, sync):
                assert np.array_equal(o.cpu().numpy(), u0)
        finally:
            B.dd_batch_destroy(b)
    finally:
        for ip in ips:
            ip.close()


@pytest.mark.parametrize("precision", ["fp16_ref", "bf16_ref", "fp32_ref"])
def test_correction_loop_on_device_and_on_host(precision):
    """The device-driven correction loop and the host-driven one both reach the
    tolerance and the oracle's solution."""
    f, m = synth.make_frame(150, 210, 3, 0.04, "edge", 1101)
    exact = ref.solve_direct(f, m)
    for loop in (1, 0):
        with Inpainter(m, f, **dict(PRM16, precision=precision, device_loop=loop)) as ip:
            u = ip.solve(1e-6).cpu().numpy()
            st = ip.stats()
        assert st["converged"]
        assert np.max(np.abs(u - exact)) <= TOL_U
        assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
        assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))


def test_correction_mode_async_and_batch():
    """DD_ML_CORRECTION passes (fine sweep + coarse-grid correction) inside the
    device loops: asynchronous solves and a batch graph give the synchronous
    result bit for bit."""
    prm = dict(PRM, ml_mode="correction", correction_sweeps=2, levels=3)
    frames = _frames(1200)
    sync = []
    for f, m in frames:
        with Inpainter(m, f, **prm) as ip:
            sync.append(ip.solve(1e-6).cpu().numpy())
            assert ip.stats()["converged"]
    ips = [Inpainter(m, f, **prm) for f, m in frames]
    streams = [torch.cuda.Stream(DEV) for _ in frames]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    try:
        for ip, s, o in zip(ips, streams, outs):
            B.check(B.dd_inpaint_solve_async(ip._h, o.data_ptr(), 1e-6, s), "solve_async")
        for ip, s in zip(ips, streams):
            B.check(B.dd_inpaint_solve_finish(ip._h, s), "finish")
        for (f, m), o, u0 in zip(frames, outs, sync):
            u = o.cpu().numpy()
            assert np.array_equal(u, u0)
            assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
        rc, b, _ = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6)
        B.check(rc, "dd_batch_create")
        try:
            for o in outs:
                o.zero_()
            stream = torch.cuda.current_stream(DEV)
            B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
            rc, status = B.dd_batch_finish(b, len(ips), stream)
            assert rc == B.DD_OK and all(sc == B.DD_OK for sc in status)
            for o, u0 in zip(outs, sync):
                assert np.array_equal(o.cpu().numpy(), u0)
        finally:
            B.dd_batch_destroy(b)
    finally:
        for ip in ips:
            ip.close()


# ---- persistent batches: one launch per sweep over the blocks of all frames ---------------
MIXED = [(120, 170, 3, 0.05, "uniform"), (96, 64, 1, 0.08, "edge"), (257, 190, 3, 0.03, "edge"),
         (40, 300, 2, 0.06, "uniform"), (5, 6, 1, 0.3, "uniform"), (2, 40, 3, 0.2, "uniform")]


def _mixed(seed0):
    return [synth.make_frame(H, W, C, d, pat, seed0 + i) for i, (H, W, C, d, pat) in enumerate(MIXED)]


def _run_batch(ips, outs, mode):
    rc, b, kernels = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6, mode=mode)
    B.check(rc, "dd_batch_create_mode")
    try:
        stream = torch.cuda.current_stream(DEV)
        B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
        rc, status = B.dd_batch_finish(b, len(ips), stream)
    finally:
        B.dd_batch_destroy(b)
    return rc, status


@pytest.mark.parametrize("prm", [PRM, dict(PRM, overlap=4), dict(PRM, overlap=4, coarse_factor=4, levels=2),
                                 dict(PRM, block=64, overlap=4, levels=2),
                                 dict(PRM, overlap=4, local_rtol=0.05, final_local_rtol=0.35, local_atol=0.5)])
def test_persistent_batch_equals_independent_solves(prm):
    """Frames of different sizes, channel counts and level counts (the 5 x 6 and
    2 x 40 frames have fewer levels) swept level by level in single persistent
    launches: each result and each frame's sweep counts equal its solve alone,
    bit for bit (the same per-block arithmetic and exact stop sums)."""
    for seed in (1300, 1400):      # two launches of one batch, new data in the same handles
        frames = _mixed(seed)
        alone, stats = [], []
        for f, m in frames:
            with Inpainter(m, f, **prm) as ip:
                alone.append(ip.solve(1e-6).cpu().numpy())
                stats.append(ip.stats())
        if seed == 1300:
            ips = [Inpainter(m, f, **prm) for f, m in frames]
            outs = [torch.zeros(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
            rc, b, _ = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6,
                                         mode=B.DD_BATCH_PERSISTENT)
            B.check(rc, "dd_batch_create_mode")
        else:
            for ip, (f, m) in zip(ips, frames):
                md, fd = torch.as_tensor(m).to(DEV), torch.as_tensor(f).to(DEV)
                B.check(B.dd_inpaint_set_data(ip._h, md.data_ptr(), fd.data_ptr(), 0), "set_data")
        stream = torch.cuda.current_stream(DEV)
        B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
        rc, status = B.dd_batch_finish(b, len(ips), stream)
        assert rc == B.DD_OK and all(sc == B.DD_OK for sc in status)
        for (f, m), o, u0, st0, ip in zip(frames, outs, alone, stats, ips):
            u = o.cpu().numpy()
            assert np.array_equal(u, u0)
            st = ip.stats()
            assert st["converged"] and not st["host_continued"]
            assert st["sweeps_per_level"] == st0["sweeps_per_level"]
            assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
            assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
    B.dd_batch_destroy(b)
    for ip in ips:
        ip.close()


def test_persistent_batch_frame_with_nan_fails_alone():
    frames = _mixed(1500)[:4]
    f_bad, m_bad = frames[2]
    f_bad = f_bad.copy()
    ky, kx = np.argwhere(m_bad != 0)[5]
    f_bad[0, ky, kx] = float("nan")
    frames[2] = (f_bad, m_bad)
    ips = [Inpainter(m, f, **PRM) for f, m in frames]
    outs = [torch.zeros(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    try:
        rc, status = _run_batch(ips, outs, B.DD_BATCH_PERSISTENT)
        assert status[2] == B.DD_ENUMERIC and rc == B.DD_ENUMERIC
        for i in (0, 1, 3):
            f, m = frames[i]
            assert status[i] == B.DD_OK
            assert np.array_equal(outs[i].cpu().numpy(), _sync_solve(f, m))
    finally:
        for ip in ips:
            ip.close()


def test_persistent_batch_stalled_wait_reports_timeout_and_recovers():
    frames = _mixed(1600)[:4]
    ips = [Inpainter(m, f, **dict(PRM, test_stall_polls=(32 if i == 1 else 0))) for i, (f, m) in enumerate(frames)]
    outs = [torch.zeros(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    try:
        rc, status = _run_batch(ips, outs, B.DD_BATCH_PERSISTENT)
        assert rc == B.DD_ETIMEOUT and status[1] == B.DD_ETIMEOUT
        # the handles without the hook solve normally afterwards
        for i in (0, 2, 3):
            f, m = frames[i]
            u = ips[i].solve(1e-6).cpu().numpy()
            assert np.array_equal(u, _sync_solve(f, m))
    finally:
        for ip in ips:
            ip.close()


def test_persistent_batch_rejects_mixed_layouts_and_precisions():
    f, m = synth.make_frame(64, 64, 1, 0.05, "uniform", 4)
    with Inpainter(m, f, **PRM) as a, Inpainter(m, f, **dict(PRM, overlap=5)) as b_, \
            Inpainter(m, f, **dict(PRM, precision="fp16_ref")) as c:
        o = torch.empty((1, 64, 64), dtype=torch.float32, device=DEV)
        for pair in ([a, b_], [a, c]):
            rc, bb, _ = B.dd_batch_create([p._h for p in pair], [o.data_ptr(), o.data_ptr()], 1e-6,
                                          mode=B.DD_BATCH_PERSISTENT)
            assert rc == B.DD_EINVAL and not bb.value
