"""Restricted additive Schwarz steps in the paper's order (FP64).

TEST INFRASTRUCTURE ONLY -- imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the library.

Sec. 3: the image domain is covered by overlapping subdomains Omega_i.  In
iteration n the residual r^n = b - A u^n is formed; on every subdomain the
local problem  R_i A R_i^T v_i = R_i r^n  (Eq. eq:ras-local-problem) is solved;
the corrections are added back with a partition of unity,
u^{n+1} = u^n + sum_i R_i^T D_i v_i,  sum_i R_i^T D_i R_i = I.  The local
problems keep the reflecting image boundary of A; at artificial subdomain
interfaces RAS implicitly imposes a zero Dirichlet value, ORAS replaces it by a
Robin (Dirichlet/Neumann) combination.  Sec. 4: blocks of side 32 with an
overlap of 6 pixels, local problems solved by conjugate gradients, and a
coarse-to-fine multilevel variant over three dyadic levels: a coarse pixel is
known iff one of its four fine pixels is known; its value averages the fine
values; the coarse solution initialises the next finer level.

Readings taken where the text is silent or garbled:
* R_i is the |Omega_i| x N 0/1 selection matrix (the text prints N x |Omega_i|),
  D_i a |Omega_i| x |Omega_i| diagonal.
* Blocks of side b start at multiples of the stride s = b - o; the count per
  axis is max(1, ceil((n - o) / s)) and the last block is clipped to the image.
  For 3840x2160 RGB with b = 32, o = 6 this gives 148 x 83 x 3 = 36852 local
  problems, the number the paper states in Sec. 4.
* D_i is 0/1 ownership: pixel x on an axis belongs to block
  clamp(floor((x - floor(o/2)) / s), 0, n - 1).
* ORAS interface condition: for an unknown pixel p of Omega_i and each in-image
  neighbour q outside Omega_i, the diagonal of the local matrix receives +p_R
  instead of the +1 of the implicit zero-Dirichlet (RAS) condition; p_R = 1 is
  RAS, p_R -> 0 the Neumann limit.
* Local CG: a fixed number k of iterations from v = 0 (k = None: exact local
  solve).  Known pixels have identity rows in A, so v = R_i r there.
* Coarse values average the KNOWN fine values of the 2x2 block (the decoder has
  no values at unknown pixels); odd sizes give ceil(n/2) coarse pixels.
* Prolongation (not stated in the paper): cell-centred bilinear interpolation
  with clamping at the border; fine known pixels are then reset to f.
"""
from __future__ import annotations


import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import inpaint_ref as ref

__all__ = [
    "axis_blocks", "block_count", "owner_of", "subdomains", "local_matrix",
    "cg_fixed", "oras_sweep", "oras_solve", "restrict_level", "prolong_bilinear",
    "build_hierarchy", "cascade_solve", "restrict_sum", "correction_pass",
]


# ---------------------------------------------------------------- layout (Sec. 4)
def block_count(n: int, b: int, o: int) -> int:
    """Blocks per axis: max(1, ceil((n - o) / (b - o)))."""
    s = b - o
    if s <= 0:
        raise ValueError("block must exceed overlap")
    return max(1, -(-(n - o) // s))


def axis_blocks(n: int, b: int, o: int):
    """[(start, end, own_lo, own_hi)] per block along one axis."""
    s = b - o
    nb = block_count(n, b, o)
    h = o // 2
    out = []
    for j in range(nb):
        lo, hi = j * s, min(j * s + b, n)
        own_lo = 0 if j == 0 else j * s + h
        own_hi = n if j == nb - 1 else (j + 1) * s + h
        out.append((lo, hi, own_lo, own_hi))
    return out


def owner_of(x: int, n: int, b: int, o: int) -> int:
    s = b - o
    return min(max((x - o // 2) // s, 0), block_count(n, b, o) - 1)


def subdomains(H: int, W: int, b: int, o: int):
    """List of (y0, y1, x0, x1, oy0, oy1, ox0, ox1): block and owned core."""
    out = []
    for (y0, y1, oy0, oy1) in axis_blocks(H, b, o):
        for (x0, x1, ox0, ox1) in axis_blocks(W, b, o):
            out.append((y0, y1, x0, x1, oy0, oy1, ox0, ox1))
    return out


# ------------------------------------------------------ local problem (Sec. 3)
def local_matrix(A, mask, blk, p_robin: float):
    """R_i A R_i^T for block blk with the ORAS interface modification.

    Returns (idx, M): idx the global pixel indices of Omega_i (row-major
    within the block), M the sparse |Omega_i| x |Omega_i| local matrix."""
    H, W = mask.shape
    y0, y1, x0, x1 = blk[:4]
    yy, xx = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    idx = (yy * W + xx).ravel()
    M = A[idx][:, idx].tolil()
    known = mask.ravel()[idx] != 0
    # number of in-image neighbours outside the block, per local pixel
    nout = np.zeros(idx.size)
    ly, lx = (yy - y0).ravel(), (xx - x0).ravel()
    gy, gx = yy.ravel(), xx.ravel()
    nout += ((ly == 0) & (gy > 0))
    nout += ((ly == y1 - y0 - 1) & (gy < H - 1))
    nout += ((lx == 0) & (gx > 0))
    nout += ((lx == x1 - x0 - 1) & (gx < W - 1))
    diag = M.diagonal()
    diag = diag + np.where(known, 0.0, (p_robin - 1.0) * nout)
    M.setdiag(diag)
    return idx, M.tocsr()


def cg_fixed(M, rhs, k, rtol=0.0, atol=0.0):
    """Conjugate gradients (Saad 2003, the CG algorithm of Ch. 6) from x = 0
    for k iterations; stops early if (r, r) or (p, Ap) is not positive, or,
    with rtol > 0, once ||r|| <= rtol ||r_0||, or, with atol > 0, once
    ||r|| <= atol (checked before each step).  k = None solves exactly."""
    if k is None:
        if rhs.size == 0:
            return rhs.copy()
        return spla.spsolve(M.tocsc(), rhs) if rhs.size > 1 else rhs / M.toarray()[0, 0]
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    rr_stop = max(rtol * rtol * rr, atol * atol)
    for _ in range(k):
        if not rr > 0.0 or rr <= rr_stop:
            break
        Ap = M @ p
        pAp = float(p @ Ap)
        if not pAp > 0.0:
            break
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return x


def oras_sweep(u, f, mask, b, o, p_robin, k, g=None, A=None, local_rtol=0.0, local_atol=None):
    """One ORAS iteration: returns (u_next, ||r^n|| per channel).

    u, f: (C, H, W).  g (optional, (C,H,W)): extra source term on unknown
    pixels, i.e. the sweep solves A u = C f + (I - C) g (used for correction
    equations).  r^n is the residual of the INPUT iterate u^n.  local_rtol > 0
    lets each local CG stop once its residual fell by that factor (the paper
    runs a fixed number of steps; 0 keeps that).  local_atol (optional, C
    values): each local CG of channel c also stops once its residual norm is at
    most local_atol[c] (an absolute local stop; see oras_solve)."""
    u = np.asarray(u, dtype=np.float64)
    two_d = u.ndim == 2
    u3 = u[None] if two_d else u
    f3 = np.asarray(f, dtype=np.float64)
    f3 = f3[None] if f3.ndim == 2 else f3
    mask = np.asarray(mask)
    C, H, W = u3.shape
    if A is None:
        A = ref.assemble_A(mask)
    r = ref.residual(u3, f3, mask)
    if g is not None:
        g3 = np.asarray(g, dtype=np.float64)
        g3 = g3[None] if g3.ndim == 2 else g3
        r = r + (mask == 0) * g3
    rn = np.sqrt((r * r).reshape(C, -1).sum(axis=1))
    out = u3.copy().reshape(C, -1)
    rflat = r.reshape(C, -1)
    for blk in subdomains(H, W, b, o):
        y0, y1, x0, x1, oy0, oy1, ox0, ox1 = blk
        idx, M = local_matrix(A, mask, blk, p_robin)
        known = mask.ravel()[idx] != 0
        unk = ~known
        # D_i: ownership of the block's pixels
        yy, xx = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        own = ((yy >= oy0) & (yy < oy1) & (xx >= ox0) & (xx < ox1)).ravel()
        Muu = M[unk][:, unk]
        Muk = M[unk][:, known]
        for c in range(C):
            rl = rflat[c, idx]
            v = np.zeros(idx.size)
            v[known] = rl[known]               # identity rows of A
            rhs = rl[unk] - Muk @ v[known]
            at = 0.0 if local_atol is None else float(local_atol[c])
            v[unk] = cg_fixed(Muu, rhs, k, local_rtol, at)
            out[c, idx[own]] += v[own]
    out = out.reshape(C, H, W)
    return (out[0] if two_d else out), rn


def absolute_local_tol(f, mask, b, o, tol, kappa):
    """Per channel, the absolute local stop kappa * tol * ||b - A u0|| /
    sqrt(blocks): a block's share of the stop test ||b - A u|| <= tol ||b - A u0||,
    scaled by kappa.  Since the blocks' owned cores partition the image, the
    sum over blocks of their local residuals squared is at least ||b - A u||^2:
    with kappa < 1, while the stop test fails some block is above its share."""
    f3 = np.asarray(f, dtype=np.float64)
    f3 = f3[None] if f3.ndim == 2 else f3
    mask = np.asarray(mask)
    r0 = ref.residual(ref.initial_guess(f3, mask), f3, mask)
    ref_n = np.sqrt((r0 * r0).reshape(f3.shape[0], -1).sum(axis=1))
    nblk = len(subdomains(mask.shape[0], mask.shape[1], b, o))
    return kappa * tol * ref_n / np.sqrt(nblk)


def oras_solve(f, mask, b, o, p_robin, k, tol, max_sweeps, u0=None, local_rtol=0.0, local_atol=0.0):
    """Iterate ORAS sweeps from u0 (default C f) until the relative residual
    (reference u0 = C f) of the current iterate is <= tol for every channel.
    local_atol = kappa > 0: the absolute local stop of absolute_local_tol.
    Returns (u, sweeps_applied)."""
    mask = np.asarray(mask)
    A = ref.assemble_A(mask)
    u = ref.initial_guess(f, mask) if u0 is None else np.array(u0, dtype=np.float64)
    at = absolute_local_tol(f, mask, b, o, tol, local_atol) if local_atol > 0 else None
    for n in range(max_sweeps + 1):
        if np.all(ref.rel_residual(u, f, mask) <= tol):
            return u, n
        if n == max_sweeps:
            break
        u, _ = oras_sweep(u, f, mask, b, o, p_robin, k, A=A, local_rtol=local_rtol, local_atol=at)
    return u, max_sweeps


# ------------------------------------------------------- multilevel (Sec. 4)
def restrict_level(f, mask):
    """Dyadic subsampling of mask and known values.

    Coarse pixel (Y, X) covers fine pixels {2Y, 2Y+1} x {2X, 2X+1} (those
    inside the image).  It is known iff at least one of them is known; its
    value is the average of the known fine values (0 where unknown)."""
    f3 = np.asarray(f, dtype=np.float64)
    two_d = f3.ndim == 2
    f3 = f3[None] if two_d else f3
    mask = np.asarray(mask) != 0
    C, H, W = f3.shape
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    cnt = np.zeros((Hc, Wc))
    acc = np.zeros((C, Hc, Wc))
    for dy in (0, 1):
        for dx in (0, 1):
            m = mask[dy::2, dx::2]
            hh, ww = m.shape
            cnt[:hh, :ww] += m
            acc[:, :hh, :ww] += f3[:, dy::2, dx::2] * m
    maskc = (cnt > 0).astype(np.uint8)
    fc = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
    return (fc[0] if two_d else fc), maskc


def prolong_bilinear(uc, H, W):
    """Cell-centred bilinear interpolation of a coarse grid to H x W.

    Fine pixel i lies at coarse coordinate (i - 0.5) / 2; the coarse samples
    are at integers; coordinates are clamped to [0, n_c - 1]."""
    uc = np.asarray(uc, dtype=np.float64)
    two_d = uc.ndim == 2
    uc3 = uc[None] if two_d else uc
    C, Hc, Wc = uc3.shape

    def weights(n, nc):
        t = np.clip((np.arange(n) - 0.5) / 2.0, 0.0, nc - 1)
        i0 = np.floor(t).astype(int)
        i1 = np.minimum(i0 + 1, nc - 1)
        return i0, i1, t - i0

    y0, y1, wy = weights(H, Hc)
    x0, x1, wx = weights(W, Wc)
    top = uc3[:, y0][:, :, x0] * (1 - wx) + uc3[:, y0][:, :, x1] * wx
    bot = uc3[:, y1][:, :, x0] * (1 - wx) + uc3[:, y1][:, :, x1] * wx
    out = top * (1 - wy)[:, None] + bot * wy[:, None]
    return out[0] if two_d else out


def build_hierarchy(f, mask, levels):
    """[(f_l, mask_l)] from fine (l = 0) to coarsest (l = levels - 1)."""
    hier = [(np.asarray(f, dtype=np.float64), np.asarray(mask))]
    for _ in range(levels - 1):
        hier.append(restrict_level(*hier[-1]))
    return hier


def cascade_solve(f, mask, levels, b, o, p_robin, k, tol, max_sweeps, coarse_tol):
    """Coarse-to-fine ORAS: solve the coarsest level to coarse_tol, prolong
    as the initialisation of the next finer level, ..., the finest to tol.
    Returns (u, sweeps per level, coarsest first)."""
    hier = build_hierarchy(f, mask, levels)
    u = None
    counts = []
    for lvl in range(levels - 1, -1, -1):
        fl, ml = hier[lvl]
        if u is not None:
            H, W = ml.shape
            u = prolong_bilinear(u, H, W)
            u = np.where(ml != 0, fl, u)
        t = tol if lvl == 0 else coarse_tol
        u, n = oras_solve(fl, ml, b, o, p_robin, k, t, max_sweeps, u0=u)
        counts.append(n)
    return u, counts


# ------------------------------------------ coarse-grid correction (two-level)
def restrict_sum(r):
    """Sum of a fine grid over each 2x2 block {2Y, 2Y+1} x {2X, 2X+1} (the parts
    inside the image); ceil(n/2) coarse pixels per axis.  With the h = 1
    stencil the coarse operator represents the Laplacian times 4, so the sum
    (4 x the block mean) is the restricted right-hand side."""
    r3 = np.asarray(r, dtype=np.float64)
    two_d = r3.ndim == 2
    r3 = r3[None] if two_d else r3
    C, H, W = r3.shape
    out = np.zeros((C, (H + 1) // 2, (W + 1) // 2))
    for dy in (0, 1):
        for dx in (0, 1):
            part = r3[:, dy::2, dx::2]
            out[:, :part.shape[1], :part.shape[2]] += part
    return out[0] if two_d else out


def correction_pass(u, f, mask, hier, b, o, p_robin, k, m, coarse_exact=False):
    """One fine ORAS sweep followed by a coarse-grid correction on the coarsest
    level of hier (from build_hierarchy): the fine residual r = b - A u (zero
    on known pixels) is summed down to that level, the correction equation
    A_c e = R r (e = 0 on coarse-known pixels) gets m ORAS sweeps from e = 0,
    and e, prolonged bilinearly level by level to d (zero on known fine
    pixels), is added with the step omega = (r, d) / (d, A d) per channel: the
    minimiser of the A-norm of the error along d (A is SPD on the unknowns;
    the rediscretised coarse problem is not the Galerkin one, so the plain
    step can overshoot).  coarse_exact: the correction equation is solved
    exactly (sparse LU) instead of by m ORAS sweeps.  Returns (u_next, ||r^n||
    of the input per channel)."""
    mask = np.asarray(mask)
    u1, rn = oras_sweep(u, f, mask, b, o, p_robin, k)
    two_d = np.asarray(u1).ndim == 2
    u3 = u1[None] if two_d else u1
    f3 = np.asarray(f, dtype=np.float64)
    f3 = f3[None] if f3.ndim == 2 else f3
    r = ref.residual(u3, f3, mask)
    for _ in range(len(hier) - 1):
        r = restrict_sum(r)
    _, mask_c = hier[-1]
    e = np.zeros_like(r)
    if coarse_exact:   # A_c e = r on coarse-unknown pixels, e = 0 on coarse-known ones
        lu = spla.splu(ref.assemble_A(mask_c).tocsc())
        for c in range(r.shape[0]):
            rhs = np.where(np.asarray(mask_c) != 0, 0.0, r[c]).ravel()
            e[c] = lu.solve(rhs).reshape(r.shape[1:])
    else:
        for _ in range(m):
            e, _ = oras_sweep(e, np.zeros_like(r), mask_c, b, o, p_robin, k, g=r)
    for lvl in range(len(hier) - 2, -1, -1):
        H, W = np.asarray(hier[lvl][1]).shape
        e = prolong_bilinear(e, H, W)
    r0 = ref.residual(u3, f3, mask)
    d = (mask == 0) * e
    Ad = ref.apply_A(d, mask)
    num = (r0 * d).reshape(d.shape[0], -1).sum(axis=1)
    den = (d * Ad).reshape(d.shape[0], -1).sum(axis=1)
    omega = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    out = u3 + omega[:, None, None] * d
    return (out[0] if two_d else out), rn

