"""Pins of the oracle's Schwarz and multilevel steps (paper Sec. 3-4)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import inpaint_ref as ref
from oracle import oras_ref as oras

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _case(rng, H, W, d=0.08):
    f = rng.uniform(0, 255, size=(H, W))
    m = (rng.uniform(size=(H, W)) < d).astype(np.uint8)
    m[rng.integers(H), rng.integers(W)] = 1
    return f, m


def test_paper_local_problem_count():
    """Sec. 4: block 32, overlap 6 -> 36852 local problems for 4K RGB."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_layout_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for W, H, C, b, o, n in (map(int, r) for r in rows):
        assert oras.block_count(W, b, o) * oras.block_count(H, b, o) * C == n
        assert len(oras.subdomains(H, W, b, o)) * C == n


@pytest.mark.parametrize("n,b,o", [(3840, 32, 6), (2160, 32, 6), (256, 32, 4), (1920, 64, 4),
                                   (100, 32, 5), (31, 32, 6), (5, 32, 6), (33, 16, 1), (97, 96, 8)])
def test_axis_partition_of_unity(n, b, o):
    """sum_i R_i^T D_i R_i = I on one axis: cores are disjoint, cover every
    pixel once, and lie inside their block; blocks cover the axis."""
    blocks = oras.axis_blocks(n, b, o)
    own = np.zeros(n, dtype=int)
    cov = np.zeros(n, dtype=int)
    for j, (lo, hi, olo, ohi) in enumerate(blocks):
        assert 0 <= lo < hi <= n and hi - lo <= b
        assert lo <= olo < ohi <= hi
        own[olo:ohi] += 1
        cov[lo:hi] += 1
        for x in range(olo, ohi):
            assert oras.owner_of(x, n, b, o) == j
    assert np.all(own == 1) and np.all(cov >= 1)
    assert blocks[-1][1] == n


def test_partition_of_unity_2d():
    H, W, b, o = 45, 70, 16, 3
    acc = np.zeros((H, W), dtype=int)
    for (y0, y1, x0, x1, oy0, oy1, ox0, ox1) in oras.subdomains(H, W, b, o):
        acc[oy0:oy1, ox0:ox1] += 1
    assert np.all(acc == 1)


def test_ras_local_matrix_is_RART(rng):
    """With p_R = 1 the local matrix is literally R_i A R_i^T (Eq.
    eq:ras-local-problem), R_i built as a 0/1 selection matrix."""
    f, m = _case(rng, 20, 23)
    A = ref.assemble_A(m)
    for blk in oras.subdomains(20, 23, 8, 2)[::5]:
        idx, M = oras.local_matrix(A, m, blk, 1.0)
        R = sp.csr_matrix((np.ones(idx.size), (np.arange(idx.size), idx)), shape=(idx.size, 20 * 23))
        assert abs(M - R @ A @ R.T).max() == 0.0


def test_oras_interface_diagonal(rng):
    """ORAS changes only interface diagonals of unknown pixels, by (p_R - 1)
    per in-image neighbour outside the block."""
    H, W = 12, 12
    m = np.zeros((H, W), dtype=np.uint8); m[0, 0] = 1
    A = ref.assemble_A(m)
    blk = (4, 8, 4, 8, 0, 0, 0, 0)
    idx, M1 = oras.local_matrix(A, m, blk, 1.0)
    _, Mp = oras.local_matrix(A, m, blk, 0.25)
    d = (Mp - M1).diagonal().reshape(4, 4)
    exp = np.zeros((4, 4))
    exp[0, :] += 1; exp[-1, :] += 1; exp[:, 0] += 1; exp[:, -1] += 1
    assert np.allclose(d, -0.75 * exp)
    assert abs((Mp - M1) - sp.diags((Mp - M1).diagonal())).max() == 0.0


def test_local_cg_exact_after_n_steps(rng):
    """CG terminates in at most n steps in exact arithmetic: with k = n it
    matches a dense solve of the local SPD system."""
    f, m = _case(rng, 10, 10, 0.3)
    A = ref.assemble_A(m)
    blk = oras.subdomains(10, 10, 5, 1)[4]
    idx, M = oras.local_matrix(A, m, blk, 0.4)
    unk = m.ravel()[idx] == 0
    Muu = M[unk][:, unk]
    rhs = rng.normal(size=unk.sum())
    x = oras.cg_fixed(Muu, rhs, int(unk.sum()))
    assert np.max(np.abs(x - np.linalg.solve(Muu.toarray(), rhs))) <= 1e-8
    # symmetric positive definite
    D = Muu.toarray()
    assert np.allclose(D, D.T) and np.linalg.eigvalsh(D).min() > 0


def test_single_block_one_sweep_is_exact(rng):
    """One block covering the image: R = I, no interface, so one sweep with
    an exact local solve gives the solution of A u = b."""
    f, m = _case(rng, 13, 17)
    u1, rn = oras.oras_sweep(ref.initial_guess(f, m), f, m, 32, 6, 0.3, None)
    assert np.max(np.abs(u1 - ref.solve_direct(f, m))) <= 1e-9
    assert rn[0] == pytest.approx(ref.residual_norms(ref.initial_guess(f, m), f, m)[0])


@pytest.mark.parametrize("p,k", [(1.0, None), (0.3, None), (0.3, 8), (0.1, 4)])
def test_fixed_point_is_exact_solution(rng, p, k):
    f, m = _case(rng, 40, 36, 0.06)
    u, n = oras.oras_solve(f, m, 12, 3, p, k, 1e-10, 400)
    assert ref.rel_residual(u, f, m)[0] <= 1e-10
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= 1e-6


def test_sweep_keeps_known_pixels(rng):
    f, m = _case(rng, 30, 30)
    u, _ = oras.oras_sweep(ref.initial_guess(f, m), f, m, 10, 2, 0.3, 5)
    assert np.array_equal(u[m != 0], f[m != 0])


def test_oras_beats_ras():
    """Sec. 3: ORAS converges faster than RAS (soft check, exact local solves)."""
    import synth
    f, m = synth.make_frame(96, 96, 1, 0.05, "uniform", 11)
    _, n_ras = oras.oras_solve(f, m, 32, 4, 1.0, None, 1e-6, 100)
    _, n_oras = oras.oras_solve(f, m, 32, 4, 0.3, None, 1e-6, 100)
    assert n_oras < n_ras


def test_restrict_hand_example():
    """Worked 3x4 -> 2x2 example: a coarse pixel is known iff one of its
    (up to) four fine pixels is known; its value is the mean of the known
    fine values (Sec. 4)."""
    f = np.array([[10., 20., 30., 40.],
                  [50., 60., 70., 80.],
                  [90., 11., 12., 13.]])
    m = np.array([[1, 0, 0, 0],
                  [0, 1, 0, 0],
                  [1, 1, 0, 1]], dtype=np.uint8)
    fc, mc = oras.restrict_level(f, m)
    assert mc.tolist() == [[1, 0], [1, 1]]
    assert fc[0, 0] == pytest.approx((10 + 60) / 2)
    assert fc[1, 0] == pytest.approx((90 + 11) / 2)
    assert fc[1, 1] == pytest.approx(13.0)
    assert fc[0, 1] == 0.0


def test_restrict_invariants(rng):
    f, m = _case(rng, 37, 52, 0.05)
    fc, mc = oras.restrict_level(f, m)
    assert mc.shape == (19, 26)
    assert mc.mean() >= m.mean()                       # density grows (Sec. 4)
    fcc, _ = oras.restrict_level(np.full_like(f, 9.5), m)
    assert np.all(fcc[mc != 0] == 9.5)
    for Y in range(19):
        for X in range(26):
            blk_m = m[2 * Y:2 * Y + 2, 2 * X:2 * X + 2] != 0
            blk_f = f[2 * Y:2 * Y + 2, 2 * X:2 * X + 2]
            assert bool(mc[Y, X]) == bool(blk_m.any())
            if blk_m.any():
                assert blk_f[blk_m].min() - 1e-12 <= fc[Y, X] <= blk_f[blk_m].max() + 1e-12


def test_prolong_reproduces_affine():
    Hc, Wc = 9, 12
    Y, X = np.mgrid[0:Hc, 0:Wc].astype(float)
    uc = 2.0 * X - 3.0 * Y + 1.0
    u = oras.prolong_bilinear(uc, 18, 24)
    y, x = np.mgrid[0:18, 0:24].astype(float)
    exp = 2.0 * (x - 0.5) / 2 - 3.0 * (y - 0.5) / 2 + 1.0
    inner = (slice(1, 17), slice(1, 23))                # away from the clamp
    assert np.max(np.abs(u[inner] - exp[inner])) <= 1e-12
    assert np.allclose(oras.prolong_bilinear(np.full((4, 5), 3.0), 7, 9), 3.0)


def test_prolong_convex(rng):
    uc = rng.uniform(-5, 5, size=(6, 7))
    u = oras.prolong_bilinear(uc, 11, 14)
    assert u.min() >= uc.min() - 1e-12 and u.max() <= uc.max() + 1e-12


def test_cascade_converges_to_solution():
    import synth
    f, m = synth.make_frame(64, 80, 1, 0.05, "edge", 5)
    u, counts = oras.cascade_solve(f, m, 3, 16, 4, 0.3, 8, 1e-8, 200, 1e-2)
    assert len(counts) == 3
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= 1e-4


# ------------------------------------------- coarse-grid correction (two-level)
def test_restrict_sum_hand_example():
    """3x5 -> 2x3: each coarse pixel sums its 2x2 block inside the image."""
    r = np.arange(15, dtype=float).reshape(3, 5)
    exp = np.array([[0 + 1 + 5 + 6, 2 + 3 + 7 + 8, 4 + 9],
                    [10 + 11, 12 + 13, 14]], dtype=float)
    assert np.array_equal(oras.restrict_sum(r), exp)


@pytest.mark.parametrize("H,W", [(8, 8), (7, 9), (1, 5), (5, 1)])
def test_restrict_sum_conserves_total(rng, H, W):
    r = rng.normal(size=(2, H, W))
    rc = oras.restrict_sum(r)
    assert rc.shape == (2, (H + 1) // 2, (W + 1) // 2)
    assert np.allclose(rc.sum(axis=(1, 2)), r.sum(axis=(1, 2)), rtol=0, atol=1e-12)


def test_correction_pass_keeps_the_solution(rng):
    """The exact solution has r = 0, so the coarse correction adds nothing and
    the sweep leaves it unchanged: it is a fixed point of the corrected pass."""
    f, m = _case(rng, 36, 44, 0.06)
    hier = oras.build_hierarchy(f, m, 3)
    us = ref.solve_direct(f, m)
    u1, _ = oras.correction_pass(us, f, m, hier, 12, 3, 0.3, 8, 2)
    assert np.max(np.abs(u1 - us)) <= 1e-8


def test_correction_pass_converges_and_helps_in_large_holes():
    """Corrected passes converge to the direct solution; on a sparse mask with
    large unsampled regions (low-frequency error that the local solves spread
    slowly) they need fewer fine passes than plain sweeps (soft check)."""
    import synth
    f, m = synth.make_frame(64, 64, 1, 0.01, "uniform", 21)
    hier = oras.build_hierarchy(f, m, 3)
    us = ref.solve_direct(f, m)
    u_c = ref.initial_guess(f, m)
    u_p = u_c.copy()
    A = ref.assemble_A(m)
    for _ in range(6):
        u_c, _ = oras.correction_pass(u_c, f, m, hier, 16, 4, 0.3, 8, 3)
        u_p, _ = oras.oras_sweep(u_p, f, m, 16, 4, 0.3, 8, A=A)
    err_c = np.max(np.abs(u_c - us))
    err_p = np.max(np.abs(u_p - us))
    assert err_c < 0.5 * err_p
    for _ in range(30):
        u_c, _ = oras.correction_pass(u_c, f, m, hier, 16, 4, 0.3, 8, 3)
    assert np.max(np.abs(u_c - us)) <= 1e-4


def test_correction_step_never_raises_the_energy_error(rng):
    """omega = (r, d) / (d, A d) minimises ||u* - u - omega d||_A, so the
    corrected iterate is never worse in the A-norm than the swept one."""
    f, m = _case(rng, 40, 52, 0.03)
    hier = oras.build_hierarchy(f, m, 3)
    us = ref.solve_direct(f, m)

    def energy(u):
        e = (us - u) * (m == 0)
        return float((e * ref.apply_A(e, m)).sum())

    u = ref.initial_guess(f, m)
    for _ in range(4):
        swept, _ = oras.oras_sweep(u, f, m, 12, 3, 0.3, 6)
        u, _ = oras.correction_pass(u, f, m, hier, 12, 3, 0.3, 6, 1)
        assert energy(u) <= energy(swept) * (1 + 1e-12) + 1e-18


def test_cg_relative_stop(rng):
    """rtol = 0 is the fixed-step CG; rtol > 0 stops at the first iterate whose
    residual fell by the factor rtol, which the fixed-step run passes through."""
    n = 60
    Mr = rng.normal(size=(n, n))
    M = sp.csr_matrix(Mr @ Mr.T + n * np.eye(n))
    rhs = rng.normal(size=n)
    x_fixed = oras.cg_fixed(M, rhs, 12)
    assert np.array_equal(oras.cg_fixed(M, rhs, 12, 0.0), x_fixed)
    x_rel = oras.cg_fixed(M, rhs, 12, 1e-3)
    res = np.linalg.norm(rhs - M @ x_rel) / np.linalg.norm(rhs)
    assert res <= 1e-3
    steps = [oras.cg_fixed(M, rhs, j) for j in range(13)]
    hit = next(j for j, xj in enumerate(steps) if np.linalg.norm(rhs - M @ xj) <= 1e-3 * np.linalg.norm(rhs))
    assert np.allclose(x_rel, steps[hit], rtol=0, atol=1e-12)


def test_local_rtol_sweep_still_converges(rng):
    f, m = _case(rng, 40, 36, 0.06)
    A = ref.assemble_A(m)
    u = ref.initial_guess(f, m)
    for _ in range(60):
        u, _ = oras.oras_sweep(u, f, m, 12, 3, 0.3, 16, A=A, local_rtol=0.05)
    assert np.max(np.abs(u - ref.solve_direct(f, m))) <= 1e-6


def _cg_one_reduction(M, rhs, k):
    """The CUDA sweep's form of the local CG, written here in FP64: each step
    forms (p, Ap), (Ap, Ap) and the measured (r, r) together; alpha uses the
    measured (r, r), beta = alpha (Ap, Ap)/(p, Ap) - 1 (the recurrence
    |r - alpha Ap|^2 = alpha^2 (Ap, Ap) - (r, r), valid since (r, Ap) = (p, Ap))."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    for _ in range(k):
        Ap = M @ p
        pq, qq, rr = float(p @ Ap), float(Ap @ Ap), float(r @ r)
        if not (pq > 0.0 and rr > 0.0):
            break
        alpha = rr / pq
        beta = alpha * qq / pq - 1.0
        x += alpha * p
        r -= alpha * Ap
        p = r + beta * p
    return x


def test_one_reduction_cg_step_equals_textbook_cg(rng):
    """The kernel's one-reduction step gives the textbook CG iterates (Saad,
    the oracle's cg_fixed) to rounding, on ORAS local problems with Robin
    interfaces and scattered known pixels, for every step count."""
    f, m = _case(rng, 40, 40, 0.05)
    A = ref.assemble_A(m)
    for blk in oras.subdomains(40, 40, 16, 3)[:4]:
        idx, M = oras.local_matrix(A, m, blk, 0.15)
        unk = m.ravel()[idx] == 0
        Muu = M[unk][:, unk].tocsr()
        rhs = rng.normal(size=int(unk.sum()))
        for k in (1, 2, 5, 10, 20):
            a, b = oras.cg_fixed(Muu, rhs, k), _cg_one_reduction(Muu, rhs, k)
            assert np.max(np.abs(a - b)) <= 1e-9 * max(1.0, np.max(np.abs(a)))


# ------------------------------------------------ absolute local stop (reading C7)
def _block_local_residuals(u, f, m, b, o):
    """||R_i r|| over the unknown pixels of each block, r = b - A u."""
    r = ref.residual(u[None], f[None], m)[0].ravel()
    H, W = m.shape
    out = []
    for y0, y1, x0, x1, *_ in oras.subdomains(H, W, b, o):
        yy, xx = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        idx = (yy * W + xx).ravel()
        out.append(np.linalg.norm(r[idx][m.ravel()[idx] == 0]))
    return np.array(out), np.linalg.norm(r)


def test_block_residuals_bound_the_global_residual(rng):
    """The argument behind local_atol < 1: the owned cores partition the image,
    so the blocks' local residuals squared sum to at least ||r||^2."""
    f, m = _case(rng, 37, 53, 0.05)
    u = rng.uniform(0, 255, size=f.shape)
    u[m != 0] = f[m != 0]
    for b, o in [(16, 2), (12, 5), (8, 1)]:
        loc, glob = _block_local_residuals(u, f, m, b, o)
        assert np.sum(loc ** 2) >= glob ** 2 * (1 - 1e-12)


def test_absolute_local_stop_below_one_converges(rng):
    f, m = _case(rng, 40, 56, 0.05)
    us = ref.solve_direct(f, m)
    for kappa in (0.5, 0.9):
        u, n = oras.oras_solve(f, m, 16, 3, 0.3, 12, 1e-8, 300, local_rtol=0.05, local_atol=kappa)
        assert n < 300
        assert np.all(ref.rel_residual(u, f, m) <= 1e-8)
        assert np.max(np.abs(u - us)) <= 1e-4


def test_absolute_local_stop_at_or_above_one_can_stall(rng):
    """With kappa >= 1 every block can sit below its share while the stop test
    fails: then no block iterates and a sweep returns its input unchanged."""
    f, m = _case(rng, 40, 56, 0.05)
    b, o, kappa = 16, 3, 3.0
    u0 = ref.initial_guess(f, m)
    loc, glob = _block_local_residuals(u0, f, m, b, o)
    nblk = loc.size
    tol = loc.max() * np.sqrt(nblk) / (kappa * glob)   # every block exactly at its kappa-share
    assert tol < 1.0                                     # the stop test ||r|| <= tol ||r0|| fails at u0
    at = oras.absolute_local_tol(f, m, b, o, tol, kappa)
    u1, _ = oras.oras_sweep(u0, f, m, b, o, 0.3, 12, local_atol=at * (1 + 1e-9))
    assert np.array_equal(u1, u0)


def test_exact_coarse_correction_on_the_fine_grid_gives_the_solution(rng):
    """With a one-level hierarchy the coarse grid is the fine grid: the exact
    correction e = A^-1 r is the whole error, omega = (r, e) / (e, A e) = 1,
    and the corrected iterate is the solution of Eq. eq:ls."""
    f, m = _case(rng, 30, 41, 0.06)
    hier = oras.build_hierarchy(f, m, 1)
    u0 = ref.initial_guess(f, m)
    u1, _ = oras.correction_pass(u0, f, m, hier, 12, 3, 0.3, 4, 0, coarse_exact=True)
    assert np.max(np.abs(u1 - ref.solve_direct(f, m))) <= 1e-8
