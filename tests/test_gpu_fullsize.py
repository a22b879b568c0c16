"""Parity at the workloads' full sizes, in the launch configuration of bench.py.

The 4K RGB workload (3840 x 2160 x 3, 3 % edge-clustered mask) runs with the
autotuned parameters the bench uses:
- in FP32, three frames in flight on three streams through the asynchronous
  C ABI, as in the bench's timed region;
- with FP16 inner storage and the FP64-accurate outer correction.
The 1080p workload (1920 x 1080 x 3, 4 % edge-clustered) runs with 64 x 64
blocks at overlap 4 and a 1/8 coarsest grid (4 dyadic levels).

Frame 0 of each is compared pixel by pixel with the oracle's FP64 CG solution
to rel-res 1e-12: max|du| <= 0.05 on the 0-255 scale, the bound for
FP32-output solves.  Every frame is also checked for properties that hold at
any size:
- the oracle-evaluated relative residual <= tol;
- known pixels reproduced exactly;
- the discrete maximum principle."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import inpaint_ref as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300 import autotune  # noqa: E402
from paper_2110_03946_gb300 import binding as B  # noqa: E402
from paper_2110_03946_gb300.inpaint import Inpainter  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-6
TOL_U = 0.05
FALLBACK = dict(block=32, overlap=6, local_cg_iters=16, robin_p=0.0, levels=3, coarse_tol=1e-2)


def _params(name, precision):
    w = synth.WORKLOADS[name]
    tuned = autotune.lookup(w.H, w.W, w.C, w.density, precision, TOL)
    return dict(tuned if tuned else FALLBACK, precision=precision)


def _check_properties(u, f, m):
    known = m != 0
    assert np.isfinite(u).all()
    assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= TOL)
    assert np.array_equal(u[:, known], f[:, known].astype(np.float32))
    for c in range(f.shape[0]):
        lo, hi = f[c][known].min(), f[c][known].max()
        assert lo - TOL_U <= u[c].min() and u[c].max() <= hi + TOL_U


@pytest.fixture(scope="module")
def frames4k():
    return [synth.workload_frame("rgb4k_edge3", j) for j in range(3)]


@pytest.fixture(scope="module")
def exact4k(frames4k):
    f, m = frames4k[0]
    u, _, rel = ocg.solve_cg(f, m, tol=1e-12)
    assert np.all(rel <= 1e-10)
    return u


def test_rgb4k_fp32_three_in_flight(frames4k, exact4k):
    prm = _params("rgb4k_edge3", "fp32")
    dm = [torch.as_tensor(m).to(DEV) for _, m in frames4k]
    dv = [torch.as_tensor(f).to(DEV) for f, _ in frames4k]
    ips = [Inpainter(dm[0], dv[0], device=DEV, **prm) for _ in frames4k]
    streams = [torch.cuda.Stream(DEV) for _ in frames4k]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames4k]
    try:
        for ip, s, md, vd, o in zip(ips, streams, dm, dv, outs):
            B.check(B.dd_inpaint_set_data_async(ip._h, md.data_ptr(), vd.data_ptr(), 0, s), "set_data_async")
            B.check(B.dd_inpaint_solve_async(ip._h, o.data_ptr(), TOL, s), "solve_async")
        for ip, s in zip(ips, streams):
            B.check(B.dd_inpaint_solve_finish(ip._h, s), "finish")
        us = [o.cpu().numpy() for o in outs]
    finally:
        for ip in ips:
            ip.close()
    assert np.max(np.abs(us[0] - exact4k)) <= TOL_U
    for u, (f, m) in zip(us, frames4k):
        _check_properties(u, f, m)


def test_rgb4k_fp16_storage_with_fp64_correction(frames4k, exact4k):
    f, m = frames4k[0]
    with Inpainter(m, f, device=DEV, **_params("rgb4k_edge3", "fp16_ref")) as ip:
        u = ip.solve(TOL).cpu().numpy()
        assert ip.stats()["corrections"] >= 1
    assert np.max(np.abs(u - exact4k)) <= TOL_U
    _check_properties(u, f, m)


def test_rgb1080p_blocks64_overlap4_eighth_coarse_grid():
    f, m = synth.workload_frame("rgb1080p_edge4", 0)
    prm = dict(block=64, overlap=4, local_cg_iters=20, local_rtol=0.05, robin_p=0.15, levels=4, coarse_tol=3e-3,
               precision="fp32")
    with Inpainter(m, f, device=DEV, **prm) as ip:
        u = ip.solve(TOL).cpu().numpy()
        assert ip.stats()["converged"]
    exact, _, rel = ocg.solve_cg(f, m, tol=1e-12)
    assert np.all(rel <= 1e-10)
    assert np.max(np.abs(u - exact)) <= TOL_U
    _check_properties(u, f, m)


def test_batch_of_48_mixed_frames_one_graph():
    """The bench's batch: 48 frames of 512x512, 1280x720, 1920x1080 and
    3840x2160 RGB (mask density U[1 %, 10 %], uniform and edge-clustered in
    turn, the same seeds) solved by one CUDA-graph launch with the 4K FP32
    parameters, first as a graph of per-frame solves, then with one persistent
    launch per sweep over the blocks of all frames (DD_BATCH_PERSISTENT), which
    gives the same images bit for bit.  Every frame converges and meets the
    properties; the 512x512 frames are also compared with the oracle's direct
    solution."""
    rng = np.random.default_rng(4000)
    sizes = [(512, 512), (720, 1280), (1080, 1920), (2160, 3840)]
    frames = []
    for j in range(48):
        H, W = sizes[rng.integers(4)]
        d = rng.uniform(0.01, 0.10)
        frames.append(synth.make_frame(H, W, 3, d, "uniform" if j % 2 == 0 else "edge", 4000 + j))
    prm = _params("rgb4k_edge3", "fp32")
    ips = [Inpainter(m, f, device=DEV, **prm) for f, m in frames]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    results = {}
    try:
        for mode in (B.DD_BATCH_GRAPH, B.DD_BATCH_PERSISTENT):
            for o in outs:
                o.zero_()
            rc, b, _ = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], TOL, mode=mode)
            B.check(rc, "dd_batch_create_mode")
            try:
                stream = torch.cuda.current_stream(DEV)
                B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
                rc, status = B.dd_batch_finish(b, len(ips), stream)
                assert rc == B.DD_OK and all(sc == B.DD_OK for sc in status)
            finally:
                B.dd_batch_destroy(b)
            for ip in ips:
                assert ip.stats()["converged"]
            results[mode] = [o.cpu().numpy() for o in outs]
    finally:
        for ip in ips:
            ip.close()
    us = results[B.DD_BATCH_PERSISTENT]
    for a, b_ in zip(results[B.DD_BATCH_GRAPH], us):
        assert np.array_equal(a, b_)
    small = 0
    for u, (f, m) in zip(us, frames):
        _check_properties(u, f, m)
        if f.shape[1:] == (512, 512):
            assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
            small += 1
    assert small > 0


def test_serving_stream_full_size_alone_and_in_the_mix():
    """The bench's serving mix at full size: Poisson arrivals at 60 requests/s,
    70 % 4K, 20 % 1080p and 10 % 720p RGB video sequences warm-started from the
    previous frame, 4K FP32 parameters, 40 GB HBM budget.  Each result equals
    the same frame solved alone (bit for bit when cold, within the FP32 bound
    when warm) and meets the residual and property checks."""
    from paper_2110_03946_gb300.serve import CudaBackend, Server, make_pool, poisson_stream
    shapes = [(2160, 3840, 3), (1080, 1920, 3), (720, 1280, 3)]
    pool = make_pool(shapes, n_frames=3, n_masks=2, density_range=(0.02, 0.08), seed=5000)
    reqs = poisson_stream(60.0, 0.4, shapes, [0.7, 0.2, 0.1], 30, 5001, pool)
    assert len(reqs) >= 8
    w = synth.WORKLOADS["rgb4k_edge3"]
    prm = autotune.lookup(w.H, w.W, w.C, w.density, "fp32", TOL) or FALLBACK
    srv = Server(CudaBackend(prm, tol=TOL, device=DEV), hbm_budget=40 << 30)
    got = {}
    try:
        _, met = srv.run(reqs, realtime=False, on_result=lambda r: got.__setitem__(r.rid, (r.output.clone(), r.warm)))
    finally:
        srv.close()
    assert met["failures"] == 0 and len(got) == len(reqs) and met["warm_starts"] > 0
    for rq in reqs:
        u, warm = got[rq.rid]
        u = u.numpy()
        f, mask = rq.values.numpy(), rq.mask.numpy()
        with Inpainter(mask, f, device=DEV, precision="fp32", **prm) as ip:
            alone = ip.solve(TOL).cpu().numpy()
        if warm:
            assert np.max(np.abs(u - alone)) <= TOL_U
        else:
            assert np.array_equal(u, alone)
        _check_properties(u, f.astype(np.float32), mask)
