"""The small-grid coarse solve (dd_coarse_cg) and the coarse-grid correction
that uses it (DD_ML_CORRECTION with params.correction_cg > 0).

dd_coarse_cg solves A e = g with e = 0 on known pixels (the operator of
Eq. eq:ls on a coarse grid, Sec. 4) by CG in one CTA per channel.  It is
checked against the oracle's sparse direct solve of the same system."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import inpaint_ref as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300 import binding as B  # noqa: E402
from paper_2110_03946_gb300.inpaint import Inpainter  # noqa: E402

DEV = torch.device("cuda:0")


def _coarse_problem(H, W, C, seed, hole=True):
    rng = np.random.default_rng(seed)
    m = (rng.random((H, W)) < 0.3).astype(np.uint8)
    if hole:
        yy, xx = np.mgrid[:H, :W]
        m[(yy - H / 2) ** 2 + (xx - W / 2) ** 2 < (0.3 * min(H, W)) ** 2] = 0
    if not m.any():
        m[0, 0] = 1
    g = rng.normal(0.0, 50.0, size=(C, H, W)).astype(np.float32)
    return m, g


def _direct(m, g):
    """e* = A^-1 g on unknown pixels, e* = 0 on known ones (oracle assembly)."""
    lu = spla.splu(ref.assemble_A(m).tocsc())
    rhs = np.where(m[None] != 0, 0.0, g.astype(np.float64)).reshape(g.shape[0], -1)
    return np.stack([lu.solve(rhs[c]) for c in range(g.shape[0])]).reshape(g.shape)


def _run(m, g, max_iter, tol):
    C, H, W = g.shape
    md = torch.as_tensor(m).to(DEV)
    gd = torch.as_tensor(g).to(DEV)
    ed = torch.full_like(gd, float("nan"))
    rc, iters = B.dd_coarse_cg(H, W, C, md.data_ptr(), gd.data_ptr(), ed.data_ptr(), max_iter, tol,
                               torch.cuda.current_stream(DEV))
    return rc, iters, ed.cpu().numpy()


@pytest.mark.parametrize("H,W,C", [(68, 120, 3), (45, 80, 2), (96, 128, 1), (1, 37, 1), (3, 3, 2)])
def test_coarse_cg_matches_direct_solve(H, W, C):
    m, g = _coarse_problem(H, W, C, H * 1000 + W)
    rc, iters, e = _run(m, g, 5000, 1e-6)
    B.check(rc, "dd_coarse_cg")
    es = _direct(m, g)
    assert np.all(e[:, m != 0] == 0.0)
    assert all(0 <= i < 5000 for i in iters)
    # relative residual of the returned e, evaluated in FP64 by the oracle's operator
    A = ref.assemble_A(m)
    for c in range(C):
        rhs = np.where(m != 0, 0.0, g[c].astype(np.float64)).ravel()
        res = rhs - A @ e[c].astype(np.float64).ravel()
        assert np.linalg.norm(res) <= 1e-4 * np.linalg.norm(rhs)
    scale = max(1.0, float(np.max(np.abs(es))))
    assert np.max(np.abs(e - es)) <= 1e-3 * scale


def test_coarse_cg_trivial_cases_and_limits():
    m, g = _coarse_problem(40, 50, 2, 5)
    rc, iters, e = _run(m, np.zeros_like(g), 100, 1e-3)   # g = 0: nothing to solve
    B.check(rc, "dd_coarse_cg")
    assert iters == [0, 0] and np.all(e == 0.0)
    rc, iters, e = _run(m, g, 0, 1e-3)                     # no iteration allowed: e = 0
    B.check(rc, "dd_coarse_cg")
    assert iters == [0, 0] and np.all(e == 0.0)
    rc, iters, e = _run(m, g, 3, 1e-12)                    # the iteration cap holds
    B.check(rc, "dd_coarse_cg")
    assert iters == [3, 3] and np.all(np.isfinite(e))
    big = np.ones((100, 123), dtype=np.uint8)               # 12300 > 12288 pixels
    rc, _, _ = _run(big, np.zeros((1, 100, 123), dtype=np.float32), 10, 1e-3)
    assert rc == B.DD_EINVAL


def test_correction_with_coarse_cg_on_a_large_hole():
    """A 480 x 640 frame with an unsampled disc of radius 144 px: the cascade
    alone needs many fine sweeps; the triggered correction whose coarse
    equation is solved by the small-grid CG needs few, and both give the
    solution of Eq. eq:ls."""
    H, W = 480, 640
    f, m = synth.make_frame(H, W, 3, 0.03, "uniform", 17)
    yy, xx = np.mgrid[:H, :W]
    m = m.copy()
    m[(yy - H / 2) ** 2 + (xx - W / 2) ** 2 < (0.3 * min(H, W)) ** 2] = 0
    prm = dict(block=32, overlap=4, local_cg_iters=20, local_rtol=0.05, robin_p=0.15, levels=4, coarse_tol=3e-3,
               precision="fp32", max_sweeps=400)
    exact = ref.solve_direct(f, m)
    out = {}
    for name, extra in [("cascade", {}),
                        ("cg", dict(ml_mode="correction", correction_trigger=0.5, correction_cg=500))]:
        with Inpainter(m, f, **prm, **extra) as ip:
            u = ip.solve(1e-6, allow_unconverged=True).cpu().numpy()
            out[name] = (u, ip.stats())
    u, st = out["cg"]
    print("cascade", out["cascade"][1]["sweeps_per_level"][:4], "cg", st["sweeps_per_level"][:4],
          "corrections", st["coarse_corrections"])
    assert st["converged"] and st["coarse_corrections"] >= 1
    assert np.max(np.abs(u - exact)) <= 0.05
    assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)
    assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))
    assert st["sweeps_per_level"][0] < out["cascade"][1]["sweeps_per_level"][0]


def test_correction_cg_below_a_shallow_cascade():
    """A 2-level cascade on 480 x 640: its coarsest level (240 x 320) is too
    large for the small-grid CG, so the correction restricts on through
    correction-only levels down to 60 x 80; the cascade itself keeps 2 levels."""
    H, W = 480, 640
    f, m = synth.make_frame(H, W, 3, 0.03, "uniform", 17)
    yy, xx = np.mgrid[:H, :W]
    m = m.copy()
    m[(yy - H / 2) ** 2 + (xx - W / 2) ** 2 < (0.3 * min(H, W)) ** 2] = 0
    with Inpainter(m, f, block=32, overlap=4, local_cg_iters=20, local_rtol=0.05, robin_p=0.15, levels=2,
                   coarse_tol=3e-3, precision="fp32", max_sweeps=400, ml_mode="correction", correction_trigger=0.5,
                   correction_cg=500) as ip:
        u = ip.solve(1e-6).cpu().numpy()
        st = ip.stats()
    assert st["converged"] and st["coarse_corrections"] >= 1
    assert st["sweeps_per_level"][1] > 0 and all(n == 0 for n in st["sweeps_per_level"][2:])
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= 0.05
    assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)


def test_correction_cg_rejects_a_frame_with_no_small_level():
    # 3 x 60000: the restriction stops at 2 rows, every level keeps more than 12288 pixels
    f, m = synth.make_frame(3, 60000, 1, 0.05, "uniform", 3)
    with pytest.raises(B.DDError) as ei:
        Inpainter(m, f, levels=2, precision="fp32", ml_mode="correction", correction_cg=100)
    assert ei.value.code == B.DD_EINVAL
