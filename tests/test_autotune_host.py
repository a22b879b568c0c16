"""Host logic of the autotuner, without a GPU: the coordinate descent over the
parameter space (with a synthetic cost in place of timed solves) and the
cache keyed by frame shape, mask density, precision and tolerance."""
import json

import pytest

pytest.importorskip("torch")

from paper_2110_03946_gb300 import autotune  # noqa: E402

SPACE = {
    "overlap": [1, 2, 3, 4, 6],
    "local_cg_iters": [8, 12, 16, 20, 24],
    "robin_p": [0.0, 0.1, 0.15, 0.3],
}
START = {"block": 32, "overlap": 6, "local_cg_iters": 16, "robin_p": 0.0}


def _cost(prm):
    # separable, minimum at overlap 3, k 20, robin 0.15
    return (1.0 + abs(prm["overlap"] - 3) + 0.1 * abs(prm["local_cg_iters"] - 20)
            + 10.0 * abs(prm["robin_p"] - 0.15))


def test_descent_reaches_the_minimum_of_a_separable_cost():
    calls = []

    def trial(prm):
        calls.append(dict(prm))
        return _cost(prm)

    seen = {}
    best, ms = autotune._descend(trial, seen, dict(START), SPACE, budget_s=60.0, log=None)
    assert best == {"block": 32, "overlap": 3, "local_cg_iters": 20, "robin_p": 0.15}
    assert ms == pytest.approx(1.0)
    # every parameter set is timed once
    assert len(calls) == len({json.dumps(c, sort_keys=True) for c in calls}) == len(seen)


def test_overlap_not_below_block_is_never_timed():
    timed = []

    def trial(prm):
        timed.append(prm)
        return 1.0

    seen = {}
    autotune._descend(trial, seen, {"block": 4, "overlap": 1}, {"overlap": [1, 3, 4, 6]}, budget_s=10.0, log=None)
    assert all(p["overlap"] < p["block"] for p in timed)
    assert seen[json.dumps({"block": 4, "overlap": 4}, sort_keys=True)] == float("inf")
    assert seen[json.dumps({"block": 4, "overlap": 6}, sort_keys=True)] == float("inf")


def test_gains_under_one_percent_do_not_move_the_point():
    def trial(prm):
        return 100.0 - 0.5 * (prm["overlap"] == 3)    # 0.5 % better: ignored

    best, ms = autotune._descend(trial, {}, {"block": 32, "overlap": 6}, {"overlap": [3, 6]}, budget_s=10.0, log=None)
    assert best["overlap"] == 6 and ms == 100.0


def test_cache_key_and_lookup(tmp_path):
    key = autotune.cache_key(2160, 3840, 3, 0.031, "fp32", 1e-6)
    assert key == "2160x3840x3|d3|fp32|tol1e-06"
    path = tmp_path / "tuned.json"
    path.write_text(json.dumps({key: {"params": {"block": 32, "overlap": 3}, "ms_per_frame": 3.0}}))
    assert autotune.lookup(2160, 3840, 3, 0.029, "fp32", 1e-6, path=str(path)) == {"block": 32, "overlap": 3}
    assert autotune.lookup(2160, 3840, 3, 0.03, "fp16_ref", 1e-6, path=str(path)) is None
    assert autotune.lookup(2160, 3840, 3, 0.03, "fp32", 1e-6, path=str(tmp_path / "missing.json")) is None


def test_committed_cache_has_the_bench_entries():
    for precision in ("fp32", "fp16_ref"):
        prm = autotune.lookup(2160, 3840, 3, 0.03, precision, 1e-6)
        assert prm is not None and prm["overlap"] < prm["block"]
        assert set(prm) <= set(autotune.SPACE)


def test_lookup_falls_back_to_the_nearest_density(tmp_path):
    path = tmp_path / "tuned.json"
    cache = {autotune.cache_key(720, 1280, 3, 0.02, "fp32", 1e-6): {"params": {"overlap": 2}},
             autotune.cache_key(720, 1280, 3, 0.08, "fp32", 1e-6): {"params": {"overlap": 8}},
             autotune.cache_key(720, 1280, 3, 0.05, "fp16_ref", 1e-6): {"params": {"overlap": 5}}}
    path.write_text(json.dumps(cache))
    look = lambda d, **kw: autotune.lookup(720, 1280, 3, d, "fp32", 1e-6, str(path), **kw)
    assert look(0.02) == {"overlap": 2}                 # exact bucket
    assert look(0.03) == {"overlap": 2}                 # nearest density
    assert look(0.07) == {"overlap": 8}
    assert look(0.05) == {"overlap": 2}                 # a tie goes to the lower density
    assert look(0.03, nearest=False) is None
    assert autotune.lookup(1080, 1920, 3, 0.03, "fp32", 1e-6, str(path)) is None   # other shape
