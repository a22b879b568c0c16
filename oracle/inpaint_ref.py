"""The inpainting problem written out from its definition (FP64).

TEST INFRASTRUCTURE ONLY -- imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the library.

Paper Sec. 2: the continuous model c(u - f) - (1 - c) Lap(u) = 0 with
reflecting (homogeneous Neumann) image boundaries (Eq. eq:inp) is discretised
with finite differences as  C(u - f) - (I - C) L u = 0  (Eq. eq:homdiff), i.e.
A u = b with A = C - (I - C) L and b = C f (Eq. eq:ls).  C is the diagonal
0/1 mask matrix; colour images give one such system per channel with the same
A (end of Sec. 2).

Readings taken where the paper is silent:
* grid size h = 1 (the scale of L does not change u);
* L is the 5-point Laplacian with reflecting boundaries: for pixel p,
  (L u)_p = sum over the in-image 4-neighbours q of (u_q - u_p); a mirrored
  ghost equals u_p, so its term vanishes;
* "relative residual" (Sec. 4-5) = ||b - A u||_2 / ||b - A u0||_2 per channel,
  with the fixed reference u0 = C f (known values, zeros elsewhere); if that
  reference norm is 0 the absolute norm is used.
Arrays are (C, H, W) float64 (a 2-D array is one channel); masks are (H, W).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "laplacian", "apply_A", "rhs_b", "residual", "residual_norms",
    "rel_residual", "initial_guess", "assemble_L", "assemble_A", "solve_direct",
]


def _as3(a):
    a = np.asarray(a, dtype=np.float64)
    return a[None] if a.ndim == 2 else a


def laplacian(u):
    """(L u)_p = sum_{q in N(p)} (u_q - u_p); neighbours outside the image
    are dropped (reflecting boundary, Sec. 2)."""
    u = np.asarray(u, dtype=np.float64)
    Lu = np.zeros_like(u)
    dv = u[..., 1:, :] - u[..., :-1, :]      # edge (y, y+1) in each column
    Lu[..., :-1, :] += dv
    Lu[..., 1:, :] -= dv
    dh = u[..., :, 1:] - u[..., :, :-1]      # edge (x, x+1) in each row
    Lu[..., :, :-1] += dh
    Lu[..., :, 1:] -= dh
    return Lu


def apply_A(u, mask):
    """A u = C u - (I - C) L u  (Eq. eq:ls)."""
    c = (np.asarray(mask) != 0).astype(np.float64)
    u = np.asarray(u, dtype=np.float64)
    return c * u - (1.0 - c) * laplacian(u)


def rhs_b(f, mask):
    """b = C f  (Eq. eq:ls)."""
    c = (np.asarray(mask) != 0).astype(np.float64)
    return c * np.asarray(f, dtype=np.float64)


def initial_guess(f, mask):
    """u0 = C f: the known values, zero on the inpainting domain."""
    return rhs_b(f, mask)


def residual(u, f, mask):
    """r = b - A u."""
    return rhs_b(f, mask) - apply_A(u, mask)


def residual_norms(u, f, mask):
    """Per-channel ||b - A u||_2 (float64 array of length C)."""
    r = _as3(residual(u, f, mask))
    return np.sqrt((r * r).reshape(r.shape[0], -1).sum(axis=1))


def rel_residual(u, f, mask):
    """Per-channel relative residual ||b - A u|| / ||b - A u0||, u0 = C f."""
    num = residual_norms(u, f, mask)
    den = residual_norms(initial_guess(f, mask), f, mask)
    den = np.where(den > 0, den, 1.0)
    return num / den


def assemble_L(H: int, W: int):
    """Sparse N x N 5-point Laplacian with reflecting boundaries, pixel
    index p = y*W + x.  Built edge by edge: each in-image neighbour pair
    (p, q) adds +1 at (p,q),(q,p) and -1 at (p,p),(q,q)."""
    N = H * W
    idx = np.arange(N).reshape(H, W)
    pairs = [
        (idx[:, :-1].ravel(), idx[:, 1:].ravel()),   # horizontal edges
        (idx[:-1, :].ravel(), idx[1:, :].ravel()),   # vertical edges
    ]
    rows, cols, vals = [], [], []
    for p, q in pairs:
        rows += [p, q, p, q]
        cols += [q, p, p, q]
        vals += [np.ones(p.size), np.ones(p.size), -np.ones(p.size), -np.ones(p.size)]
    if rows:
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def assemble_A(mask):
    """Sparse A = C - (I - C) L  (Eq. eq:ls) for an (H, W) mask."""
    mask = np.asarray(mask)
    H, W = mask.shape
    c = (mask.ravel() != 0).astype(np.float64)
    L = assemble_L(H, W)
    return (sp.diags(c) - sp.diags(1.0 - c) @ L).tocsr()


def solve_direct(f, mask):
    """Exact solution of A u = b per channel by sparse LU (SuperLU).

    Raises ValueError for an empty mask: with no known pixel, A is singular
    under the reflecting boundary conditions."""
    f3 = _as3(f)
    mask = np.asarray(mask)
    if not np.any(mask):
        raise ValueError("empty mask: A is singular")
    C, H, W = f3.shape
    lu = spla.splu(assemble_A(mask).tocsc())
    b = rhs_b(f3, mask).reshape(C, -1)
    u = np.stack([lu.solve(b[c]) for c in range(C)]).reshape(C, H, W)
    return u if np.asarray(f).ndim == 3 else u[0]
