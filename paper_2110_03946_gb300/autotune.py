"""Autotuner for the ORAS solver parameters.

Searches block side, overlap, local CG steps and their relative stop, Robin
weight, number of levels and coarse tolerance for the smallest device time to a relative residual
``tol`` on sample frames: for every block side a coordinate descent (one
parameter at a time over its candidates, repeated while something improves and
time is left), keeping the best result over block sides.  Every trial
runs through the C ABI; a trial counts only if its solve converged.  Results
are cached in a JSON file keyed by frame shape, mask density (1 % buckets),
precision and tolerance.

python -m paper_2110_03946_gb300.autotune --workload rgb4k_edge3 --out tuned.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import binding as B
from .inpaint import PRECISIONS, make_params

SPACE = {
    "block": [16, 32, 64, 96],
    "overlap": [1, 2, 3, 4, 5, 6, 8],
    "local_cg_iters": [2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 24, 28, 32],
    "local_rtol": [0.0, 0.01, 0.02, 0.03, 0.05, 0.1],   # 0.0 = always local_cg_iters steps
    "robin_p": [0.0, 0.1, 0.15, 0.2, 0.3, 0.5, 1.0],   # 0.0 = library default
    "levels": [1, 2, 3, 4, 5, 6],
    "coarse_tol": [1e-1, 1e-2, 3e-3, 1e-3, 3e-4],
    "final_local_rtol": [0.0, 0.2, 0.35, 0.5],   # 0.0 = the predicted-last sweep uses local_rtol too
    "local_atol": [0.0, 0.3, 0.5, 0.7],          # 0.0 = no absolute local stop (values >= 1 can stall)
}
START = {"block": 32, "overlap": 6, "local_cg_iters": 16, "local_rtol": 0.0, "robin_p": 0.0, "levels": 3,
         "coarse_tol": 1e-2, "final_local_rtol": 0.0, "local_atol": 0.0}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def cache_key(H: int, W: int, C: int, density: float, precision: str, tol: float) -> str:
    return f"{H}x{W}x{C}|d{int(round(density * 100))}|{precision}|tol{tol:g}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def lookup(H, W, C, density, precision, tol, path: str = DEFAULT_CACHE, nearest: bool = True):
    """Tuned parameters for this shape/density/precision, or None.  Without an
    entry for the density's 1 % bucket, the entry of the same shape, precision
    and tolerance with the nearest density (nearest=True)."""
    cache = load_cache(path)
    ent = cache.get(cache_key(H, W, C, density, precision, tol))
    if ent is None and nearest:
        prefix = f"{H}x{W}x{C}|d"
        suffix = f"|{precision}|tol{tol:g}"
        want = int(round(density * 100))
        cands = []
        for k, v in cache.items():
            if k.startswith(prefix) and k.endswith(suffix):
                try:
                    d = int(k[len(prefix):-len(suffix)])
                except ValueError:
                    continue
                cands.append((abs(d - want), d, v))
        if cands:
            ent = min(cands, key=lambda t: (t[0], t[1]))[2]
    return dict(ent["params"]) if ent else None


class _Trial:
    """Solves the sample frames with one parameter set; device ms per frame."""

    def __init__(self, frames, precision, tol, reps=1):
        self.frames = frames
        self.precision = precision
        self.tol = tol
        self.reps = reps
        C, H, W = frames[0][1].shape
        self.out = torch.empty((C, H, W), dtype=torch.float32, device=frames[0][1].device)

    def __call__(self, prm: dict) -> float:
        m0, v0 = self.frames[0]
        C, H, W = v0.shape
        p = make_params(precision=self.precision, **prm)
        rc, h = B.dd_inpaint_create(H, W, C, m0.data_ptr(), v0.data_ptr(), p)
        if rc != B.DD_OK:
            return float("inf")
        try:
            stream = torch.cuda.current_stream(v0.device)
            total, n = 0.0, 0
            for rep in range(self.reps + 1):           # the first pass warms up
                for m, v in self.frames:
                    if B.dd_inpaint_set_data(h, m.data_ptr(), v.data_ptr(), 0) != B.DD_OK:
                        return float("inf")
                    if B.dd_inpaint_solve(h, self.out.data_ptr(), self.tol, stream) != B.DD_OK:
                        return float("inf")
                    rc, st = B.dd_inpaint_stats(h)
                    if rep > 0:
                        total += st.ms_total
                        n += 1
            return total / max(n, 1)
        finally:
            B.dd_inpaint_destroy(h)


def autotune(frames, precision: str = "fp32", tol: float = 1e-6, budget_s: float = 60.0,
             space: dict | None = None, start: dict | None = None, log=None):
    """Block-major coordinate descent: for every block side, descend over the
    other parameters from the start point; keep the best overall.
    frames: list of (mask uint8 (H,W), values f32 (C,H,W)) CUDA tensors.
    Returns (best_params, best_ms, trials)."""
    space = dict(space or SPACE)
    blocks = space.pop("block", [32])
    trial = _Trial(frames, precision, tol)
    seen = {}
    t0 = time.time()
    best, best_ms = None, float("inf")
    for b in blocks:
        per = max(1.0, (budget_s - (time.time() - t0)) / max(1, len(blocks) - blocks.index(b)))
        cand, ms = _descend(trial, seen, dict(start or START, block=b), space, per, log)
        if ms < best_ms:
            best, best_ms = cand, ms
    return best, best_ms, seen


def _descend(trial, seen, best, space, budget_s, log):

    def score(prm):
        key = json.dumps(prm, sort_keys=True)
        if key not in seen:
            if prm["overlap"] >= prm["block"]:
                seen[key] = float("inf")
            else:
                seen[key] = trial(prm)
                if log:
                    log(f"{seen[key]:9.3f} ms  {prm}")
        return seen[key]

    best_ms = score(best)
    t0 = time.time()
    improved = True
    while improved and time.time() - t0 < budget_s:
        improved = False
        for name, values in space.items():
            for v in values:
                if time.time() - t0 >= budget_s:
                    break
                cand = dict(best, **{name: v})
                ms = score(cand)
                if ms < best_ms * 0.99:
                    best, best_ms, improved = cand, ms, True
    return best, best_ms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="rgb4k_edge3")
    ap.add_argument("--shape", default=None, help="HxWxC instead of the workload's shape")
    ap.add_argument("--density", type=float, default=None, help="mask density instead of the workload's")
    ap.add_argument("--pattern", default=None, choices=["uniform", "edge"])
    ap.add_argument("--mix", default=None,
                    help="sample frames of mixed masks, e.g. 0.02:edge,0.04:uniform,0.08:edge (density:pattern per "
                         "frame; the cache key takes --density)")
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--holdout", type=int, default=0,
                    help="held-out frames per sample mask (new seeds): the tuned winner is kept only if it also "
                         "beats the previous entry and the given fallbacks on them")
    ap.add_argument("--fallback", action="append", default=[],
                    help="JSON parameter set that the held-out check compares against (repeatable)")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--budget", type=float, default=120.0, help="seconds")
    ap.add_argument("--blocks", default="16,32,64,96", help="block sides to search")
    ap.add_argument("--start", default=None, help="JSON start point (default: the cached entry, else START)")
    ap.add_argument("--out", default=DEFAULT_CACHE)
    a = ap.parse_args()
    import dataclasses

    import synth
    w = synth.WORKLOADS[a.workload]
    if a.shape:
        H, W, C = (int(v) for v in a.shape.lower().split("x"))
        w = dataclasses.replace(w, name=f"{H}x{W}x{C}", H=H, W=W, C=C)
    if a.density is not None:
        w = dataclasses.replace(w, density=a.density)
    if a.pattern:
        w = dataclasses.replace(w, pattern=a.pattern)
    dev = torch.device("cuda", 0)
    masks = [(w.density, w.pattern)] * a.frames
    if a.mix:
        masks = [(float(d), pat) for d, pat in (item.split(":") for item in a.mix.split(","))]
    frames = []
    for j, (dens, pat) in enumerate(masks):
        f, m = synth.make_frame(w.H, w.W, w.C, dens, pat, w.seed_base + 50 + j)
        frames.append((torch.as_tensor(m).to(dev), torch.as_tensor(f).to(dev)))
    space = dict(SPACE, block=[int(b) for b in a.blocks.split(",")])
    if a.precision != "fp32":   # the outer correction's inner tolerance (ignored by FP32 solves)
        space["inner_tol"] = [1e-2, 3e-3, 1e-3]
    start = json.loads(a.start) if a.start else lookup(w.H, w.W, w.C, w.density, a.precision, a.tol, a.out,
                                                       nearest=False)
    if start:
        start = dict(START, **start)
    best, ms, seen = autotune(frames, a.precision, a.tol, a.budget, space=space, start=start,
                              log=lambda s: print(s, flush=True))
    entry = {"params": best, "ms_per_frame": ms, "trials": len(seen), "workload": w.name,
             "pattern": w.pattern,
             "sample_seeds": [w.seed_base + 50 + j for j in range(len(masks))],
             "sample_masks": [f"{d:g}:{pat}" for d, pat in masks]}
    if a.holdout > 0:
        # the winner against the start point and the fallbacks on frames it was not tuned on
        held = []
        for r in range(a.holdout):
            for j, (dens, pat) in enumerate(masks):
                f, m = synth.make_frame(w.H, w.W, w.C, dens, pat, w.seed_base + 150 + 16 * r + j)
                held.append((torch.as_tensor(m).to(dev), torch.as_tensor(f).to(dev)))
        trial = _Trial(held, a.precision, a.tol)
        cands = [("tuned", best)] + ([("start", start)] if start else [])
        cands += [(f"fallback{i}", dict(START, **json.loads(fb))) for i, fb in enumerate(a.fallback)]
        scored = []
        for name, prm in cands:
            hms = trial(prm)
            print(f"held-out {hms:9.3f} ms  {name} {prm}", flush=True)
            scored.append((hms, name, prm))
        hms, name, prm = min(scored, key=lambda t: t[0])
        entry.update(params=prm, holdout_ms_per_frame=hms, holdout_winner=name,
                     holdout_seeds=[w.seed_base + 150 + 16 * r + j for r in range(a.holdout)
                                    for j in range(len(masks))])
        best, ms = prm, hms
    cache = load_cache(a.out)
    cache[cache_key(w.H, w.W, w.C, w.density, a.precision, a.tol)] = entry
    with open(a.out, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    print(json.dumps({"best": best, "ms_per_frame": ms, "trials": len(seen)}))


if __name__ == "__main__":
    main()
