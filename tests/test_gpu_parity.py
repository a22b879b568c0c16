"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the floating-point bar is max|du| <= 0.05 on the 0-255 scale for
results with FP32 output (the solver's stated tolerance), and the relative
residual of the returned image, evaluated in FP64 by the oracle, must meet the
requested tol.  Single sweeps compare the FP32 kernel with the FP64 oracle
sweep taking the same steps; their bound (2e-3 absolute) is derived in the
test below from FP32 rounding of k CG steps."""
import zlib

import numpy as np
import pytest

import synth
from oracle import inpaint_ref as ref
from oracle import oras_ref as oras

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_03946_gb300 import binding as B  # noqa: E402
from paper_2110_03946_gb300.inpaint import Inpainter  # noqa: E402

DEV = torch.device("cuda:0")
TOL_U = 0.05


def _t(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


# ----------------------------------------------------------------------- steps
@pytest.mark.parametrize("H,W,C", [(37, 52, 1), (64, 64, 3), (1, 9, 2), (7, 1, 1), (301, 257, 3)])
def test_restrict_matches_oracle(H, W, C):
    rng = np.random.default_rng(H * 1000 + W)
    f = rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)
    m = (rng.uniform(size=(H, W)) < 0.1).astype(np.uint8)
    fd = np.where(m != 0, f, 0).astype(np.float32)
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    mc = torch.zeros((Hc, Wc), dtype=torch.uint8, device=DEV)
    fc = torch.zeros((C, Hc, Wc), dtype=torch.float32, device=DEV)
    md, fdd = _t(m, torch.uint8), _t(fd)
    B.check(B.dd_restrict(H, W, C, md.data_ptr(), fdd.data_ptr(), mc.data_ptr(), fc.data_ptr()), "restrict")
    torch.cuda.synchronize()
    ofc, omc = oras.restrict_level(fd.astype(np.float64), m)
    assert np.array_equal(mc.cpu().numpy(), omc)                      # integer work: bit-exact
    assert np.max(np.abs(fc.cpu().numpy() - ofc)) <= 1e-4             # mean of <= 4 FP32 values


@pytest.mark.parametrize("Hc,Wc,H,W,C", [(9, 12, 18, 24, 1), (5, 7, 9, 13, 3), (1, 1, 2, 1, 1), (135, 240, 270, 480, 2)])
def test_prolong_matches_oracle(Hc, Wc, H, W, C):
    rng = np.random.default_rng(Hc * 7 + W)
    uc = rng.uniform(0, 255, size=(C, Hc, Wc)).astype(np.float32)
    m = (rng.uniform(size=(H, W)) < 0.2).astype(np.uint8)
    f = rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)
    out = torch.zeros((C, H, W), dtype=torch.float32, device=DEV)
    ucd, md, fd = _t(uc), _t(m, torch.uint8), _t(f)
    B.check(B.dd_prolong(Hc, Wc, H, W, C, ucd.data_ptr(), 0, 0, out.data_ptr()), "prolong")
    torch.cuda.synchronize()
    exp = oras.prolong_bilinear(uc.astype(np.float64), H, W)
    assert np.max(np.abs(out.cpu().numpy() - exp)) <= 1e-3
    B.check(B.dd_prolong(Hc, Wc, H, W, C, ucd.data_ptr(), md.data_ptr(), fd.data_ptr(), out.data_ptr()), "prolong")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got[:, m != 0], f[:, m != 0])
    assert np.max(np.abs(got[:, m == 0] - exp[:, m == 0])) <= 1e-3


def test_residual_norms_match_oracle():
    f, m = synth.make_frame(130, 97, 3, 0.05, "uniform", 99)
    rng = np.random.default_rng(3)
    u = np.where(m != 0, f, rng.uniform(0, 255, size=f.shape)).astype(np.float32)
    md, fd, ud = _t(m, torch.uint8), _t(f), _t(u)      # keep the buffers alive during the call
    rc, norms, refs = B.dd_residual_norms(130, 97, 3, md.data_ptr(), fd.data_ptr(), ud.data_ptr())
    B.check(rc, "residual")
    exp = ref.residual_norms(u.astype(np.float64), f, m)
    exp0 = ref.residual_norms(ref.initial_guess(f, m), f, m)
    assert np.allclose(norms, exp, rtol=1e-5)          # FP32 sums of r^2 per block
    assert np.allclose(refs, exp0, rtol=1e-5)


SWEEP_CASES = [
    # H, W, C, block, overlap, k, p_robin, density, pattern, warps per block tile
    (64, 64, 1, 32, 4, 8, 0.3, 0.05, "uniform", 1),
    (100, 83, 2, 32, 6, 16, 0.25, 0.03, "edge", 1),       # ragged last blocks
    (100, 83, 2, 32, 6, 16, 0.25, 0.03, "edge", 2),       # two warps per block
    (100, 83, 2, 32, 3, 16, 0.15, 0.03, "edge", 4),       # four warps per block
    (45, 70, 1, 16, 3, 6, 1.0, 0.08, "uniform", 1),       # RAS, odd overlap
    (150, 140, 1, 64, 4, 12, 0.3, 0.04, "edge", 4),       # multi-warp tiles
    (150, 140, 1, 64, 5, 12, 0.3, 0.04, "edge", 8),
    (20, 24, 1, 32, 6, 5, 0.3, 0.1, "uniform", 1),        # image smaller than a block
    (20, 24, 1, 32, 6, 5, 0.3, 0.1, "uniform", 4),
]


@pytest.mark.parametrize("H,W,C,b,o,k,p,d,pat,nw", SWEEP_CASES)
def test_single_and_triple_sweep_match_oracle(H, W, C, b, o, k, p, d, pat, nw):
    """Max error bound 2e-3: k FP32 CG steps on |v| <= 255 with local
    condition numbers <= ~100 lose ~k * kappa * 2^-24 * 255 <= 1e-3."""
    f, m = synth.make_frame(H, W, C, d, pat, 17)
    u0 = ref.initial_guess(f, m)
    with Inpainter(m, f, block=b, overlap=o, local_cg_iters=k, robin_p=p, levels=1, precision="fp32",
                   tile_warps=nw) as ip:
        ip.set_iterate(u0.astype(np.float32))
        norms = ip.sweep(1)
        u1 = ip.get_iterate().cpu().numpy()
        e1, rn = oras.oras_sweep(u0, f, m, b, o, p, k)
        assert np.max(np.abs(u1 - e1)) <= 2e-3
        assert np.allclose(norms, rn, rtol=1e-5)
        assert np.array_equal(u1[:, m != 0], f[:, m != 0].astype(np.float32))
        ip.sweep(2)
        u3 = ip.get_iterate().cpu().numpy()
        e3 = e1
        for _ in range(2):
            e3, _ = oras.oras_sweep(e3, f, m, b, o, p, k)
        assert np.max(np.abs(u3 - e3)) <= 6e-3


# ----------------------------------------------------------------------- solves
SOLVE_CASES = [
    # name, H, W, C, params
    ("gray256_fp32_1level", 256, 256, 1, dict(block=32, overlap=4, levels=1, precision="fp32")),
    ("gray256_fp32ref_3level", 256, 256, 1, dict(block=32, overlap=4, levels=3, precision="fp32_ref")),
    ("rgb_fp16ref", 200, 330, 3, dict(block=32, overlap=6, levels=3, precision="fp16_ref")),
    ("rgb_bf16ref", 200, 330, 3, dict(block=32, overlap=6, levels=3, precision="bf16_ref")),
    ("rgb_b64", 190, 260, 3, dict(block=64, overlap=4, levels=2, precision="fp32_ref")),
    ("rgb_b16", 190, 260, 2, dict(block=16, overlap=2, levels=2, precision="fp32")),
    ("gray256_cg_1level", 256, 256, 1, dict(levels=1, precision="fp32", solver="cg", max_sweeps=2000)),
    ("rgb_mlcg_3level", 200, 330, 3, dict(levels=3, precision="fp32", solver="cg", max_sweeps=2000,
                                          coarse_sweeps=200, coarse_tol=1e-3)),
    ("rgb_correction_3level", 200, 330, 3, dict(levels=3, precision="fp32", ml_mode="correction")),
    # the sweep predicted to be a level's last with a looser local tolerance (device loops, and launches)
    ("rgb_final_rtol", 200, 330, 3, dict(levels=3, precision="fp32", local_rtol=0.05, final_local_rtol=0.5)),
    ("gray256_final_rtol_launches", 256, 256, 1, dict(levels=2, precision="fp32", local_rtol=0.05,
                                                      final_local_rtol=0.35, device_loop=0)),
    # the absolute local stop (blocks below their share of the tolerance take no CG step)
    ("rgb_local_atol", 200, 330, 3, dict(levels=3, precision="fp32", local_rtol=0.05, local_atol=0.5,
                                         final_local_rtol=0.35)),
    ("gray256_local_atol_launches", 256, 256, 1, dict(levels=2, precision="fp32", local_atol=0.9, device_loop=0)),
    ("rgb_local_atol_fp16ref", 200, 330, 3, dict(levels=3, precision="fp16_ref", local_rtol=0.05, local_atol=0.5)),
    ("gray256_correction_2level_launches", 256, 256, 1, dict(levels=2, precision="fp32", ml_mode="correction",
                                                             correction_sweeps=3, device_loop=0)),
    # two solved levels with a 1/8 coarse grid (two pass-through dyadic levels between them)
    ("rgb_2level_coarse8", 270, 480, 3, dict(block=64, overlap=4, levels=2, coarse_factor=8, precision="fp32")),
    ("rgb_2level_coarse4_launches", 200, 330, 3, dict(levels=2, coarse_factor=4, precision="fp32", device_loop=0)),
]


@pytest.mark.parametrize("name,H,W,C,params", SOLVE_CASES)
def test_solve_matches_oracle(name, H, W, C, params):
    if name.startswith("gray256"):
        f, m = synth.workload_frame("gray256_uniform5")
    else:
        f, m = synth.make_frame(H, W, C, 0.04, "edge", zlib.crc32(name.encode()) % 1000)
    tol = 1e-6
    with Inpainter(m, f, **params) as ip:
        u = ip.solve(tol).cpu().numpy()
        st = ip.stats()
    exact = ref.solve_direct(f, m)
    err = np.max(np.abs(u - exact))
    rel = ref.rel_residual(u.astype(np.float64), f, m)
    print(f"{name}: max|du|={err:.2e} relres={rel.max():.2e} stats={st}")
    assert st["converged"]
    assert err <= TOL_U
    assert np.all(rel <= tol)
    assert np.allclose(st["rel_residual"][:C], rel, rtol=1e-5, atol=1e-12)
    assert np.array_equal(u[:, m != 0], f[:, m != 0].astype(np.float32))
    if params.get("coarse_factor", 2) > 2:   # only the solved levels sweep
        step = {4: 2, 8: 3}[params["coarse_factor"]]
        per = st["sweeps_per_level"]
        assert all(per[l] == 0 for l in range(1, step)) and per[step] > 0


@pytest.mark.parametrize("solver", ["oras", "cg"])
@pytest.mark.parametrize("H,W", [(1, 40), (40, 1), (5, 5), (33, 17), (2, 2), (70, 131)])
def test_degenerate_shapes(H, W, solver):
    """Single rows and columns, tiny images and widths that are not a multiple
    of 4 (the CG kernels work on float4 groups of columns)."""
    rng = np.random.default_rng(H * 100 + W)
    f = rng.uniform(0, 255, size=(1, H, W)).astype(np.float32)
    m = np.zeros((H, W), dtype=np.uint8)
    m.flat[rng.choice(H * W, size=max(1, H * W // 10), replace=False)] = 1
    if solver == "cg":
        prm = dict(levels=2, precision="fp32", solver="cg", max_sweeps=4000, coarse_sweeps=2000)
    else:
        prm = dict(levels=3, precision="fp32_ref")
    with Inpainter(m, f, **prm) as ip:
        u = ip.solve(1e-6).cpu().numpy()
        st = ip.stats()
    assert st["converged"]
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U


def test_single_known_pixel_and_all_known():
    """One known pixel: the solution is that value everywhere.  It is the
    worst-conditioned case of the method (every block without the pixel is a
    Neumann problem held only by the Robin interfaces), so it gets the full
    dyadic hierarchy and a large sweep budget."""
    f = np.full((1, 50, 60), 0.0, dtype=np.float32)
    f[0, 20, 30] = 200.0
    m = np.zeros((50, 60), dtype=np.uint8)
    m[20, 30] = 1
    with Inpainter(m, f, levels=6, max_sweeps=5000, coarse_sweeps=400, coarse_tol=1e-4) as ip:
        u = ip.solve(1e-6).cpu().numpy()
    assert np.max(np.abs(u - 200.0)) <= TOL_U               # constant extension of one value
    m[:] = 1
    g = np.random.default_rng(0).uniform(0, 255, size=(2, 50, 60)).astype(np.float32)
    with Inpainter(m, g) as ip:
        u = ip.solve(1e-6).cpu().numpy()
        assert ip.stats()["sweeps_total"] == 0
    assert np.array_equal(u, g)


def test_empty_mask_is_an_error():
    m = torch.zeros((16, 16), dtype=torch.uint8, device=DEV)
    v = torch.zeros((1, 16, 16), dtype=torch.float32, device=DEV)
    with pytest.raises(B.DDError) as ei:
        Inpainter(m, v)
    assert ei.value.code == B.DD_EEMPTYMASK


def test_sweep_limit_reports_not_converged():
    f, m = synth.make_frame(128, 128, 1, 0.02, "uniform", 5)
    with Inpainter(m, f, levels=1, precision="fp32", max_sweeps=2, local_cg_iters=2) as ip:
        with pytest.raises(B.DDError) as ei:
            ip.solve(1e-9)
        assert ei.value.code == B.DD_ENOTCONVERGED
        u = ip.solve(1e-9, allow_unconverged=True)
        assert torch.isfinite(u).all()


def test_host_inputs_path():
    from paper_2110_03946_gb300 import inpaint as I
    f, m = synth.make_frame(80, 90, 2, 0.05, "uniform", 8)
    p = I.make_params(levels=2, inputs_on_device=0)
    fc = np.ascontiguousarray(f, dtype=np.float32)
    mc = np.ascontiguousarray(m, dtype=np.uint8)
    rc, h = B.dd_inpaint_create(80, 90, 2, mc.ctypes.data, fc.ctypes.data, p)
    B.check(rc, "create")
    out = torch.empty((2, 80, 90), dtype=torch.float32, device=DEV)
    B.check(B.dd_inpaint_solve(h, out.data_ptr(), 1e-6, None), "solve")
    B.dd_inpaint_destroy(h)
    assert np.max(np.abs(out.cpu().numpy() - ref.solve_direct(f, m))) <= TOL_U


def test_warm_start_same_answer():
    f, m = synth.make_frame(120, 160, 3, 0.04, "edge", 21)
    frames = synth.shifted_sequence(f, 2, 77)
    m2 = synth.uniform_mask(120, 160, 0.04, np.random.default_rng(5))
    with Inpainter(m, frames[0]) as ip:
        ip.solve(1e-6)
        cold = ip.stats()["sweeps_total"]
        ip.set_data(m2, frames[1], keep_iterate=True)
        u = ip.solve(1e-6).cpu().numpy()
    assert np.max(np.abs(u - ref.solve_direct(frames[1], m2))) <= TOL_U
    assert cold >= 0


def test_repeatable_bitwise():
    f, m = synth.make_frame(150, 170, 3, 0.04, "edge", 31)
    with Inpainter(m, f, precision="fp16_ref") as ip:
        a = ip.solve(1e-6).cpu().numpy()
        b = ip.solve(1e-6).cpu().numpy()
    assert np.array_equal(a, b)


def test_repeatable_bitwise_under_concurrency():
    """Tiles go to the persistent CTAs through an atomic counter, so which CTA
    solves which tile differs between runs, most of all when other solves share
    the GPU; the residual sums are exact fixed-point sums, so the norms, every
    stop decision and the output must not change."""
    f, m = synth.make_frame(720, 1280, 3, 0.03, "edge", 37)
    prm = dict(block=32, overlap=3, local_cg_iters=20, local_rtol=0.05, robin_p=0.15, levels=3, precision="fp32")
    with Inpainter(m, f, **prm) as ip:
        alone = ip.solve(1e-6).cpu().numpy()
        st0 = ip.stats()
    ips = [Inpainter(m, f, **prm) for _ in range(4)]
    streams = [torch.cuda.Stream(DEV) for _ in ips]
    outs = [torch.empty(f.shape, dtype=torch.float32, device=DEV) for _ in ips]
    try:
        for _ in range(2):
            for ip, s, o in zip(ips, streams, outs):
                B.check(B.dd_inpaint_solve_async(ip._h, o.data_ptr(), 1e-6, s), "solve_async")
            for ip, s in zip(ips, streams):
                B.check(B.dd_inpaint_solve_finish(ip._h, s), "finish")
            for ip, o in zip(ips, outs):
                st = ip.stats()
                assert np.array_equal(o.cpu().numpy(), alone)
                assert st["rel_residual"] == st0["rel_residual"]
                assert st["sweeps_per_level"] == st0["sweeps_per_level"]
    finally:
        for ip in ips:
            ip.close()


def test_many_channels_more_tiles_than_ctas():
    """16 channels of 300 x 290 pixels: 1760 tiles of 32 x 32 at stride 29, more
    than the persistent CTAs, so CTAs take tiles of several channels and each
    channel's exact residual sum collects partials from many CTAs."""
    f, m = synth.make_frame(290, 300, 16, 0.04, "edge", 41)
    prm = dict(block=32, overlap=3, local_cg_iters=20, local_rtol=0.05, robin_p=0.15, levels=2, precision="fp32")
    with Inpainter(m, f, **prm) as ip:
        u = ip.solve(1e-6).cpu().numpy()
        st = ip.stats()
        u2 = ip.solve(1e-6).cpu().numpy()
        assert ip.stats()["rel_residual"] == st["rel_residual"]
    assert st["converged"] and np.array_equal(u, u2)
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= TOL_U
    assert np.all(ref.rel_residual(u.astype(np.float64), f, m) <= 1e-6)


@pytest.mark.parametrize("solver", ["oras", "cg"])
def test_device_loop_matches_launches(solver):
    """The level iterations repeated in a CUDA graph loop on the device give the
    launch path's answer: the same kernels run in the same order until the
    stop test, so equal sweep counts mean bitwise-equal results."""
    f, m = synth.make_frame(180, 230, 3, 0.04, "edge", 41)
    prm = dict(levels=3, precision="fp32", solver=solver, max_sweeps=3000 if solver == "cg" else 400,
               coarse_sweeps=400 if solver == "cg" else 12)
    out = {}
    for loop in (0, 1):
        with Inpainter(m, f, device_loop=loop, **prm) as ip:
            out[loop] = (ip.solve(1e-6).cpu().numpy(), ip.stats())
    (u0, s0), (u1, s1) = out[0], out[1]
    exact = ref.solve_direct(f, m)
    for u, st in ((u0, s0), (u1, s1)):
        assert st["converged"]
        assert np.max(np.abs(u - exact)) <= TOL_U
    if s0["sweeps_per_level"] == s1["sweeps_per_level"]:
        assert np.array_equal(u0, u1)


def test_device_loop_graph_reused_across_solves():
    """A second solve with the same tolerance reuses the level loop graphs and
    gives the bitwise-same answer; a new tolerance rebuilds them."""
    f, m = synth.make_frame(140, 150, 2, 0.05, "uniform", 43)
    with Inpainter(m, f, levels=3, precision="fp32") as ip:
        a = ip.solve(1e-6).cpu().numpy()
        b = ip.solve(1e-6).cpu().numpy()
        c = ip.solve(1e-4)
        st = ip.stats()
        d = ip.solve(1e-6).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(a, d)
    assert max(st["rel_residual"][:2]) <= 1e-4 and torch.isfinite(c).all()


@pytest.mark.parametrize("levels,m", [(2, 1), (3, 2)])
def test_correction_pass_matches_oracle(levels, m):
    """One pass of DD_ML_CORRECTION (a fine sweep, then the coarse-grid
    correction) against the oracle's pass from the same iterate."""
    b, o, k, p = 16, 4, 8, 0.3
    f, msk = synth.make_frame(70, 90, 2, 0.04, "edge", 31 + levels)
    with Inpainter(msk, f, block=b, overlap=o, local_cg_iters=k, robin_p=p, levels=levels, precision="fp32",
                   ml_mode="correction", correction_sweeps=m) as ip:
        u0 = ref.initial_guess(f, msk).astype(np.float32)
        ip.set_iterate(torch.as_tensor(u0))
        ip.sweep(1)
        u1 = ip.get_iterate().cpu().numpy()
    hier = oras.build_hierarchy(f, msk, levels)
    e1, _ = oras.correction_pass(u0.astype(np.float64), f, msk, hier, b, o, p, k, m)
    assert np.max(np.abs(u1 - e1)) <= 2e-3
    assert np.array_equal(u1[:, msk != 0], f[:, msk != 0].astype(np.float32))



@pytest.mark.parametrize("levels", [2, 3])
def test_correction_pass_with_coarse_cg_matches_oracle(levels):
    """One pass of DD_ML_CORRECTION whose coarse equation is solved by the
    small-grid CG (to relative residual 1e-3) against the oracle's pass with
    an exact coarse solve, from the same iterate.  The tolerance allows the
    CG's 1e-3 on the correction's size."""
    b, o, k, p = 16, 4, 8, 0.3
    f, msk = synth.make_frame(70, 90, 2, 0.04, "edge", 41 + levels)
    with Inpainter(msk, f, block=b, overlap=o, local_cg_iters=k, robin_p=p, levels=levels, precision="fp32",
                   ml_mode="correction", correction_cg=500) as ip:
        u0 = ref.initial_guess(f, msk).astype(np.float32)
        ip.set_iterate(torch.as_tensor(u0))
        ip.sweep(1)
        u1 = ip.get_iterate().cpu().numpy()
    hier = oras.build_hierarchy(f, msk, levels)
    e1, _ = oras.correction_pass(u0.astype(np.float64), f, msk, hier, b, o, p, k, 0, coarse_exact=True)
    us, _ = oras.oras_sweep(u0.astype(np.float64), f, msk, b, o, p, k)
    corr = float(np.max(np.abs(e1 - us)))
    assert corr > 0.0
    assert np.max(np.abs(u1 - e1)) <= 2e-3 + 1e-2 * corr
    assert np.array_equal(u1[:, msk != 0], f[:, msk != 0].astype(np.float32))


@pytest.mark.parametrize("rtol", [0.1, 0.02])
def test_sweep_with_local_rtol_matches_oracle(rtol):
    """Local CG with the relative stop: the block's CG ends once its residual
    fell by rtol (decided on the kernel's FP32 (r, r), on the oracle's FP64)."""
    b, o, k, p = 32, 6, 16, 0.25
    f, m = synth.make_frame(100, 83, 2, 0.03, "edge", 17)
    u0 = ref.initial_guess(f, m)
    with Inpainter(m, f, block=b, overlap=o, local_cg_iters=k, robin_p=p, levels=1, precision="fp32",
                   local_rtol=rtol) as ip:
        ip.set_iterate(u0.astype(np.float32))
        ip.sweep(1)
        u1 = ip.get_iterate().cpu().numpy()
    e1, _ = oras.oras_sweep(u0, f, m, b, o, p, k, local_rtol=rtol)
    assert np.max(np.abs(u1 - e1)) <= 2e-3
