"""The coarse-grid correction applied only after slow passes
(DD_ML_CORRECTION with params.correction_trigger > 0).

The cascade's fine sweeps contract fast until the residual is dominated by a
smooth error mode, e.g. in a large unsampled region, which the local solves
spread slowly (the multilevel argument of Sec. 4).  With a trigger, the fine
sweeps run alone until a pass reduces the residual by less than the trigger
factor; from the next sweep on each sweep is followed by the coarse-grid
correction.  Every result must still be the solution of Eq. eq:ls (the FP64
direct solve), within the FP32 tolerance."""
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

TOL_U = 0.05
DEV = torch.device("cuda:0")
PRM = dict(block=32, overlap=4, local_cg_iters=20, robin_p=0.15, levels=3, coarse_tol=3e-3, precision="fp32")


def _hole_frame(H=192, W=256, C=3, seed=7):
    """A uniform 3 % mask with a disc of radius 0.3 min(H, W) left unsampled."""
    f, m = synth.make_frame(H, W, C, 0.03, "uniform", seed)
    yy, xx = np.mgrid[:H, :W]
    m = m.copy()
    m[(yy - H / 2) ** 2 + (xx - W / 2) ** 2 < (0.3 * min(H, W)) ** 2] = 0
    return f, m


def _solve(f, m, **prm):
    with Inpainter(m, f, **prm) as ip:
        u = ip.solve(1e-6).cpu().numpy()
        return u, ip.stats()


def _check(u, st, f, m, exact):
    assert st["converged"]
    assert np.max(np.abs(u - exact)) <= TOL_U
    assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
    assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))


def test_trigger_fires_in_a_large_hole_and_saves_fine_sweeps():
    f, m = _hole_frame()
    exact = ref.solve_direct(f, m)
    u_c, st_c = _solve(f, m, **PRM)
    u_a, st_a = _solve(f, m, **PRM, ml_mode="correction", correction_trigger=0.5)
    print("cascade", st_c["sweeps_per_level"][:3], "adaptive", st_a["sweeps_per_level"][:3],
          "corrections", st_a["coarse_corrections"])
    _check(u_c, st_c, f, m, exact)
    _check(u_a, st_a, f, m, exact)
    assert st_c["coarse_corrections"] == 0
    assert st_a["coarse_corrections"] >= 1
    assert st_a["sweeps_per_level"][0] < st_c["sweeps_per_level"][0]


def test_trigger_that_never_fires_gives_the_cascade_bit_for_bit():
    # a frame that contracts fast on every pass: the gate and the conditional
    # node change nothing
    f, m = synth.make_frame(200, 330, 3, 0.04, "edge", 314)
    u_c, st_c = _solve(f, m, **PRM)
    u_a, st_a = _solve(f, m, **PRM, ml_mode="correction", correction_trigger=0.95)
    assert st_a["coarse_corrections"] == 0
    assert st_a["sweeps_per_level"] == st_c["sweeps_per_level"]
    assert np.array_equal(u_a, u_c)


@pytest.mark.parametrize("trigger", [0.0, 0.5])
def test_launches_and_device_loop_agree(trigger):
    """The gate decides the same on plain launches (kernels that return when
    the gate says skip) and in the device loops (a plain-phase loop, then a
    corrected-phase loop that runs only if the trigger fired)."""
    f, m = _hole_frame(160, 224, 3, 8)
    prm = dict(PRM, ml_mode="correction", correction_trigger=trigger)
    u_l, st_l = _solve(f, m, **prm, device_loop=1)
    u_p, st_p = _solve(f, m, **prm, device_loop=0)
    exact = ref.solve_direct(f, m)
    _check(u_l, st_l, f, m, exact)
    _check(u_p, st_p, f, m, exact)
    if st_p["sweeps_per_level"][0] <= 16 and not st_p["host_continued"]:   # no host-side continuation
        assert st_l["coarse_corrections"] == st_p["coarse_corrections"]
        assert np.array_equal(u_l, u_p)


@pytest.mark.parametrize("coarse_cg", [0, 300])
def test_adaptive_correction_in_a_batch_graph_equals_solves_alone(coarse_cg):
    frames = [_hole_frame(192, 256, 3, 7), synth.make_frame(144, 200, 3, 0.05, "edge", 9)]
    prm = dict(PRM, ml_mode="correction", correction_trigger=0.5, correction_cg=coarse_cg)
    alone = [_solve(f, m, **prm) for f, m in frames]
    ips = [Inpainter(m, f, **prm) for f, m in frames]
    outs = [torch.zeros(f.shape, dtype=torch.float32, device=DEV) for f, _ in frames]
    try:
        rc, b, _ = B.dd_batch_create([ip._h for ip in ips], [o.data_ptr() for o in outs], 1e-6)
        B.check(rc, "dd_batch_create")
        try:
            stream = torch.cuda.current_stream(DEV)
            for _ in range(2):   # a replay starts again from the data in the handles
                for o in outs:
                    o.zero_()
                B.check(B.dd_batch_launch(b, stream), "dd_batch_launch")
                rc, status = B.dd_batch_finish(b, len(ips), stream)
                B.check(rc, "dd_batch_finish")
                for ip, o, (u0, st0) in zip(ips, outs, alone):
                    assert np.array_equal(o.cpu().numpy(), u0)
                    assert ip.stats()["coarse_corrections"] == st0["coarse_corrections"]
        finally:
            B.dd_batch_destroy(b)
    finally:
        for ip in ips:
            ip.close()
