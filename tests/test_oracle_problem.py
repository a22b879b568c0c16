"""Pins of the oracle's problem definition (paper Sec. 2, Eq. eq:homdiff/eq:ls)
against facts fixed by the mathematics, not by the oracle itself:
variational characterisation, closed forms, invariants, brute force."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import inpaint_ref as ref


def _random_case(rng, H, W, nknown=None):
    f = rng.uniform(0, 255, size=(H, W))
    m = np.zeros(H * W, dtype=np.uint8)
    k = nknown if nknown is not None else max(1, int(rng.integers(1, H * W + 1)))
    m[rng.choice(H * W, size=k, replace=False)] = 1
    return f, m.reshape(H, W)


def _dirichlet_energy_minimiser(f, mask):
    """Variational route (independent of A): the inpainting solution
    minimises sum over in-image neighbour pairs of (u_p - u_q)^2 subject to
    u = f on the known pixels (reflecting boundaries = no pairs across the
    border).  Solved as a dense least-squares problem on the incidence matrix."""
    H, W = mask.shape
    N = H * W
    rows = []
    for y in range(H):
        for x in range(W):
            p = y * W + x
            if x + 1 < W:
                rows.append((p, p + 1))
            if y + 1 < H:
                rows.append((p, p + W))
    D = np.zeros((len(rows), N))
    for e, (p, q) in enumerate(rows):
        D[e, p], D[e, q] = 1.0, -1.0
    known = mask.ravel() != 0
    fv = f.ravel()
    u = fv * known
    if (~known).any() and len(rows):
        sol, *_ = np.linalg.lstsq(D[:, ~known], -D[:, known] @ fv[known], rcond=None)
        u[~known] = sol
    return u.reshape(H, W)


@pytest.mark.parametrize("shape,nknown", [
    ((7, 9), None), ((12, 12), None), ((16, 16), 1), ((16, 16), 255),
    ((1, 13), 3), ((11, 1), 2), ((5, 5), 25), ((3, 8), 1)])
def test_direct_matches_variational_minimiser(rng, shape, nknown):
    f, m = _random_case(rng, *shape, nknown)
    u = ref.solve_direct(f, m)
    e = _dirichlet_energy_minimiser(f, m)
    assert np.max(np.abs(u - e)) <= 1e-9


@pytest.mark.parametrize("shape,nknown", [((16, 16), None), ((16, 16), 1), ((9, 14), 4), ((1, 16), 2)])
def test_cg_matches_direct(rng, shape, nknown):
    f, m = _random_case(rng, *shape, nknown)
    ud = ref.solve_direct(f, m)
    uc, it, rel = ocg.solve_cg(f, m, tol=1e-13)
    assert rel[0] <= 1e-13
    assert np.max(np.abs(uc - ud)) <= 1e-9


def test_cg_matches_direct_seeded_frame():
    import synth
    f, m = synth.make_frame(96, 80, 2, 0.03, "edge", 7)
    ud = ref.solve_direct(f, m)
    uc, it, rel = ocg.solve_cg(f, m, tol=1e-12)
    assert np.all(rel <= 1e-12)
    assert np.max(np.abs(uc - ud)) <= 1e-8


def test_known_pixels_reproduced(rng):
    f, m = _random_case(rng, 20, 17, 30)
    ud = ref.solve_direct(f, m)
    uc, _, _ = ocg.solve_cg(f, m)
    k = m != 0
    assert np.array_equal(uc[k], f[k])                  # imposed exactly
    assert np.max(np.abs(ud[k] - f[k])) <= 1e-12


def test_constant_image(rng):
    m = _random_case(rng, 19, 23, 7)[1]
    f = np.full((19, 23), 77.25)
    assert np.max(np.abs(ref.solve_direct(f, m) - 77.25)) <= 1e-11
    uc, _, _ = ocg.solve_cg(f, m)
    assert np.max(np.abs(uc - 77.25)) <= 1e-9


def test_min_max_principle(rng):
    for _ in range(5):
        f, m = _random_case(rng, 15, 21, int(rng.integers(1, 40)))
        u = ref.solve_direct(f, m)
        k = m != 0
        assert u.min() >= f[k].min() - 1e-9
        assert u.max() <= f[k].max() + 1e-9


def _one_row_closed_form(f, known_idx, n):
    """Piecewise-linear interpolation between consecutive known pixels,
    constant extension beyond the first and last known pixel (the
    reflecting end makes the boundary difference vanish)."""
    u = np.empty(n)
    ks = sorted(known_idx)
    for i in range(n):
        if i <= ks[0]:
            u[i] = f[ks[0]]
        elif i >= ks[-1]:
            u[i] = f[ks[-1]]
        else:
            j = max(k for k in ks if k <= i)
            l = min(k for k in ks if k >= i)
            u[i] = f[j] if j == l else f[j] + (f[l] - f[j]) * (i - j) / (l - j)
    return u


@pytest.mark.parametrize("n,known", [(13, [3, 7, 8]), (20, [0, 19]), (9, [4]), (30, [2, 11, 12, 25])])
def test_one_row_closed_form(rng, n, known):
    f = rng.uniform(0, 255, size=n)
    m = np.zeros(n, dtype=np.uint8)
    m[known] = 1
    exp = _one_row_closed_form(f, known, n)
    assert np.max(np.abs(ref.solve_direct(f[None, :], m[None, :])[0] - exp)) <= 1e-9
    assert np.max(np.abs(ref.solve_direct(f[:, None], m[:, None])[:, 0] - exp)) <= 1e-9
    uc, _, _ = ocg.solve_cg(f[None, :], m[None, :], tol=1e-14)
    assert np.max(np.abs(uc[0] - exp)) <= 1e-8


@pytest.mark.parametrize("kind", ["linear", "saddle", "xy"])
def test_harmonic_reproduction(rng, kind):
    """The 5-point stencil is exact for discrete harmonic functions: with the
    outer ring known, u = f for f linear, x^2 - y^2 or x*y."""
    H, W = 14, 17
    y, x = np.mgrid[0:H, 0:W].astype(float)
    f = {"linear": 3.0 * x - 2.0 * y + 5.0, "saddle": x * x - y * y, "xy": x * y}[kind]
    m = np.zeros((H, W), dtype=np.uint8)
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = 1
    m[rng.integers(1, H - 1, 6), rng.integers(1, W - 1, 6)] = 1
    assert np.max(np.abs(ref.solve_direct(f, m) - f)) <= 1e-9


def test_superposition_and_symmetry(rng):
    f, m = _random_case(rng, 12, 10, 9)
    g = rng.uniform(0, 255, size=f.shape)
    a, b = 0.7, -1.3
    lhs = ref.solve_direct(a * f + b * g, m)
    rhs = a * ref.solve_direct(f, m) + b * ref.solve_direct(g, m)
    assert np.max(np.abs(lhs - rhs)) <= 1e-9
    u = ref.solve_direct(f, m)
    assert np.max(np.abs(ref.solve_direct(f.T.copy(), m.T.copy()) - u.T)) <= 1e-9
    assert np.max(np.abs(ref.solve_direct(f[::-1].copy(), m[::-1].copy()) - u[::-1])) <= 1e-9
    assert np.max(np.abs(ref.solve_direct(f[:, ::-1].copy(), m[:, ::-1].copy()) - u[:, ::-1])) <= 1e-9


def test_separable_columns(rng):
    """f depends on x only and whole columns are known: each row is the 1-D
    problem, so u(x, y) is the 1-D closed form for every y."""
    H, W = 9, 25
    fx = rng.uniform(0, 255, size=W)
    cols = [4, 5, 13, 20]
    m = np.zeros((H, W), dtype=np.uint8)
    m[:, cols] = 1
    u = ref.solve_direct(np.tile(fx, (H, 1)), m)
    exp = _one_row_closed_form(fx, cols, W)
    assert np.max(np.abs(u - exp[None, :])) <= 1e-9


def test_laplacian_properties(rng):
    u = rng.normal(size=(2, 8, 11))
    v = rng.normal(size=(2, 8, 11))
    Lu = ref.laplacian(u)
    # constants are in the kernel; the total flux vanishes (reflecting boundary)
    assert np.max(np.abs(ref.laplacian(np.full((8, 11), 3.0)))) == 0.0
    assert np.max(np.abs(Lu.sum(axis=(1, 2)))) <= 1e-12
    # symmetry <Lu, v> = <u, Lv>
    assert abs((Lu * v).sum() - (u * ref.laplacian(v)).sum()) <= 1e-10
    # interior value on x^2 + 2y^2 is 2 + 4 = 6
    y, x = np.mgrid[0:8, 0:11].astype(float)
    assert np.allclose(ref.laplacian(x * x + 2 * y * y)[1:-1, 1:-1], 6.0)
    # an isolated spike: centre -deg, each in-image neighbour +1
    s = np.zeros((5, 5)); s[0, 2] = 1.0
    Ls = ref.laplacian(s)
    assert Ls[0, 2] == -3.0 and Ls[0, 1] == 1.0 and Ls[0, 3] == 1.0 and Ls[1, 2] == 1.0
    # the sparse assembly agrees with the stencil
    L = ref.assemble_L(8, 11)
    assert np.max(np.abs(L @ u[0].ravel() - Lu[0].ravel())) <= 1e-12


def test_relative_residual(rng):
    f, m = _random_case(rng, 10, 12, 6)
    assert ref.rel_residual(ref.initial_guess(f, m), f, m)[0] == pytest.approx(1.0)
    assert ref.rel_residual(ref.solve_direct(f, m), f, m)[0] <= 1e-12


def test_empty_mask_rejected():
    with pytest.raises(ValueError):
        ref.solve_direct(np.ones((4, 4)), np.zeros((4, 4), dtype=np.uint8))
    with pytest.raises(ValueError):
        ocg.solve_cg(np.ones((4, 4)), np.zeros((4, 4), dtype=np.uint8))


def test_all_known():
    f = np.arange(12.0).reshape(3, 4)
    m = np.ones((3, 4), dtype=np.uint8)
    assert np.array_equal(ref.solve_direct(f, m), f)
    uc, it, _ = ocg.solve_cg(f, m)
    assert np.array_equal(uc, f) and it[0] == 0
