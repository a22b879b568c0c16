"""Seeded synthetic inputs for homogeneous diffusion inpainting.

This module only draws input data: smooth colour fields and sparse masks of
known pixels, in the shapes of the paper's 4K colour decoding workload
(Sec. 5: a 3840x2160 RGB photograph with 5 % stored pixels).  The paper's test
image and its Voronoi-densified mask are not available, so seeded stand-ins are
used.  It holds none of the solver's arithmetic: both the CPU oracle and the
CUDA path receive the arrays it returns.

Recipe (all draws from numpy's PCG64, one child stream per channel and one for
the mask, spawned from ``SeedSequence(seed)``):

* field, per channel: 20 isotropic Gaussians with centres uniform in the image,
  sigma uniform in [min(H,W)/32, min(H,W)/4] and amplitude uniform in [-1, 1],
  plus 3 step edges (a line through a uniform point at a uniform angle; one side
  is raised by a jump uniform in [-0.5, 0.5]); affinely rescaled to [0, 255] and
  stored as float32.
* uniform mask: exactly round(d*H*W) pixels drawn without replacement.
* edge-clustered mask: exactly round(d*H*W) pixels drawn without replacement
  with probability proportional to g + 0.05*mean(g), where g is the
  channel-mean central-difference gradient magnitude of the field.  The floor
  keeps holes in flat regions bounded.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "smooth_field", "uniform_mask", "edge_clustered_mask", "make_frame",
    "Workload", "WORKLOADS", "workload_frame", "shifted_sequence",
]


def _children(seed: int, n: int):
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(int(seed)).spawn(n)]


def smooth_field(H: int, W: int, rng: np.random.Generator,
                 n_gauss: int = 20, n_edges: int = 3) -> np.ndarray:
    """One channel: sum of Gaussians plus step edges, rescaled to [0, 255]."""
    y = np.arange(H, dtype=np.float64)
    x = np.arange(W, dtype=np.float64)
    m = float(min(H, W))
    field = np.zeros((H, W), dtype=np.float64)
    for _ in range(n_gauss):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        sig = rng.uniform(m / 32.0, m / 4.0)
        amp = rng.uniform(-1.0, 1.0)
        gy = np.exp(-0.5 * ((y - cy) / sig) ** 2)
        gx = np.exp(-0.5 * ((x - cx) / sig) ** 2)
        field += amp * np.outer(gy, gx)
    for _ in range(n_edges):
        py, px = rng.uniform(0, H), rng.uniform(0, W)
        th = rng.uniform(0.0, np.pi)
        jump = rng.uniform(-0.5, 0.5)
        side = ((x[None, :] - px) * np.cos(th) + (y[:, None] - py) * np.sin(th)) > 0
        field += jump * side
    lo, hi = field.min(), field.max()
    if hi > lo:
        field = (field - lo) * (255.0 / (hi - lo))
    else:
        field = np.full_like(field, 127.5)
    return field.astype(np.float32)


def _count(H: int, W: int, density: float) -> int:
    return int(min(H * W, max(0, round(density * H * W))))


def uniform_mask(H: int, W: int, density: float, rng: np.random.Generator) -> np.ndarray:
    """uint8 (H, W) mask with exactly round(density*H*W) ones."""
    k = _count(H, W, density)
    m = np.zeros(H * W, dtype=np.uint8)
    if k:
        m[rng.choice(H * W, size=k, replace=False)] = 1
    return m.reshape(H, W)


def edge_clustered_mask(f: np.ndarray, density: float, rng: np.random.Generator) -> np.ndarray:
    """uint8 (H, W) mask, probability ~ gradient magnitude + 5 % of its mean.

    Weighted sampling without replacement by exponential keys
    (Efraimidis-Spirakis): the k pixels with the smallest Exp(1)/w are taken.
    """
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    k = _count(H, W, density)
    g = np.zeros((H, W), dtype=np.float64)
    for c in range(C):
        gy = np.gradient(f[c], axis=0) if H > 1 else np.zeros((H, W))
        gx = np.gradient(f[c], axis=1) if W > 1 else np.zeros((H, W))
        g += np.sqrt(gx * gx + gy * gy)
    g /= C
    mg = g.mean()
    w = (g + 0.05 * mg).ravel() if mg > 0 else np.ones(H * W)
    keys = rng.exponential(size=H * W) / w
    m = np.zeros(H * W, dtype=np.uint8)
    if k:
        m[np.argpartition(keys, k - 1)[:k]] = 1
    return m.reshape(H, W)


def make_frame(H: int, W: int, C: int, density: float, pattern: str, seed: int):
    """Return (f float32 (C,H,W), mask uint8 (H,W)) for one seeded frame."""
    rngs = _children(seed, C + 1)
    f = np.stack([smooth_field(H, W, rngs[c]) for c in range(C)])
    if pattern == "uniform":
        mask = uniform_mask(H, W, density, rngs[C])
    elif pattern == "edge":
        mask = edge_clustered_mask(f, density, rngs[C])
    else:
        raise ValueError(f"unknown mask pattern {pattern!r}")
    return f, mask


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic decoding workload (shape, mask, solver layout)."""
    name: str
    H: int
    W: int
    C: int
    density: float
    pattern: str
    block: int
    overlap: int
    seed_base: int


# Named by what they are.  Seeds: 1000*k + frame for the k-th workload.
WORKLOADS = {
    "gray256_uniform5": Workload("gray256_uniform5", 256, 256, 1, 0.05, "uniform", 32, 4, 1000),
    "rgb1080p_edge4": Workload("rgb1080p_edge4", 1080, 1920, 3, 0.04, "edge", 64, 4, 2000),
    "rgb4k_edge3": Workload("rgb4k_edge3", 2160, 3840, 3, 0.03, "edge", 32, 6, 3000),
}


def workload_frame(name: str, frame: int = 0):
    w = WORKLOADS[name]
    return make_frame(w.H, w.W, w.C, w.density, w.pattern, w.seed_base + frame)


def shifted_sequence(f0: np.ndarray, length: int, seed: int, sigma: float = 2.0):
    """Video stand-in: frame t+1 = frame t shifted by 1..3 px (reflect-padded)
    in a random direction plus Gaussian noise (sigma), clamped to [0, 255]."""
    rng = _children(seed, 1)[0]
    frames = [np.asarray(f0, dtype=np.float32)]
    for _ in range(1, length):
        prev = frames[-1].astype(np.float64)
        mag = int(rng.integers(1, 4))
        ang = rng.uniform(0, 2 * np.pi)
        dy, dx = int(round(mag * np.sin(ang))), int(round(mag * np.cos(ang)))
        H, W = prev.shape[-2:]
        pad = 4
        P = np.pad(prev, [(0, 0)] * (prev.ndim - 2) + [(pad, pad), (pad, pad)], mode="reflect")
        nxt = P[..., pad - dy:pad - dy + H, pad - dx:pad - dx + W]
        nxt = nxt + rng.normal(0.0, sigma, size=nxt.shape)
        frames.append(np.clip(nxt, 0.0, 255.0).astype(np.float32))
    return frames
