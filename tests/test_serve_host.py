"""Host logic of the serving loop and of the multi-GPU replicas, without a GPU:
a simulated backend with a virtual clock, and two gloo ranks on CPU."""
import os

import numpy as np
import pytest

from paper_2110_03946_gb300 import replicas
from paper_2110_03946_gb300.serve import Request, Server


class FakeBackend:
    """Virtual clock; a solve takes cold_s (or warm_s when warm-started)."""

    def __init__(self, cold_s=0.010, warm_s=0.004, bytes_per_px=16):
        self.t = 0.0
        self.cold_s, self.warm_s = cold_s, warm_s
        self.bpp = bytes_per_px
        self.jobs = {}
        self.created = 0
        self.live = set()
        self.log = []

    def now(self):
        return self.t

    def sleep(self, s):
        self.t += s

    def idle(self):
        self.t = min(j["done"] for j in self.jobs.values() if j["done"] is not None)

    def bytes_for(self, shape):
        H, W, C = shape
        return H * W * C * self.bpp

    def create(self, req):
        h = self.created
        self.created += 1
        self.live.add(h)
        self.jobs[h] = {"done": None, "req": None}
        return h, self.bytes_for(req.shape)

    def destroy(self, h):
        self.live.discard(h)
        self.jobs.pop(h, None)

    def submit(self, h, req, warm, fresh):
        assert not (fresh and warm)
        self.jobs[h] = {"done": self.t + (self.warm_s if warm else self.cold_s), "req": req, "warm": warm}
        self.log.append(("start", req.rid, h, self.t, warm))

    def ready(self, h):
        j = self.jobs[h]
        return j["done"] is not None and self.t >= j["done"] - 1e-12

    def finish(self, h):
        j = self.jobs[h]
        j["done"] = None
        return 0, ("image", j["req"].rid)


def _req(rid, t, H=8, W=8, C=1, seq=None, ft=0):
    return Request(rid, t, np.ones((H, W), np.uint8), np.zeros((C, H, W), np.float32), seq, ft)


def test_all_served_with_metrics():
    b = FakeBackend()
    srv = Server(b, hbm_budget=10 * 8 * 8 * 16)
    reqs = [_req(i, 0.001 * i) for i in range(20)]
    res, m = srv.run(reqs, realtime=True)
    assert [r.rid for r in res] == list(range(20))
    assert m["requests"] == 20 and m["failures"] == 0
    assert m["p99_ms"] >= m["p50_ms"] >= 10.0 - 1e-9
    assert m["peak_hbm_bytes"] <= 10 * 8 * 8 * 16


class GreedyBackend(FakeBackend):
    """A backend whose slots turn out larger than its estimate."""

    def __init__(self, actual_factor=1.5, **kw):
        super().__init__(**kw)
        self.factor = actual_factor

    def create(self, req):
        h, n = super().create(req)
        return h, int(n * self.factor)


def test_budget_holds_when_slots_exceed_their_estimate():
    # estimate 1024 B per slot, actual 1536 B: the budget of 4096 B fits 2 actual
    # slots, though 4 estimated ones would seem to fit; admission must hold it
    b = GreedyBackend(actual_factor=1.5)
    budget = 4 * 8 * 8 * 16
    srv = Server(b, hbm_budget=budget)
    reqs = [_req(i, 0.0) for i in range(12)]
    res, m = srv.run(reqs, realtime=True)
    assert m["failures"] == 0 and len(res) == 12
    assert m["peak_hbm_bytes"] <= budget
    assert len(b.live) <= 2


def test_slot_larger_than_the_budget_waits_instead_of_overrunning():
    # a slot that is actually larger than the whole budget is given up at once
    b = GreedyBackend(actual_factor=3.0)
    budget = 2 * 8 * 8 * 16
    srv = Server(b, hbm_budget=budget)
    with pytest.raises(RuntimeError, match="cannot be admitted"):
        srv.run([_req(0, 0.0)], realtime=True)
    assert not b.live and srv.peak_bytes <= budget


def test_concurrent_slots_overlap():
    b = FakeBackend()
    srv = Server(b, hbm_budget=3 * 8 * 8 * 16)
    res, m = srv.run([_req(i, 0.0) for i in range(6)], realtime=True)
    starts = sorted(r.start for r in res)
    assert starts[:3] == [0.0, 0.0, 0.0]          # three slots fit the budget and start together
    assert m["slots_created"] == 3
    assert m["max_ms"] == pytest.approx(20.0)      # two rounds of 10 ms


def test_video_frames_in_order_and_warm():
    b = FakeBackend()
    srv = Server(b, hbm_budget=4 * 8 * 8 * 16)
    reqs = [_req(i, 0.0005 * i, seq=7, ft=i) for i in range(6)]
    res, m = srv.run(reqs, realtime=True)
    starts = {rid: t for (ev, rid, h, t, w) in b.log}
    for i in range(1, 6):
        assert starts[i] >= res[i - 1].done - 1e-12  # frame i starts after frame i-1 is done
    assert m["warm_starts"] == 5                     # every frame after the first reuses the iterate
    assert all(r.warm for r in res[1:]) and not res[0].warm


def test_budget_evicts_idle_slots_of_other_shapes():
    b = FakeBackend()
    budget = 16 * 16 * 16 + 8 * 8 * 16              # one large and one small slot
    srv = Server(b, hbm_budget=budget)
    reqs = [_req(0, 0.0, 16, 16), _req(1, 0.0, 8, 8), _req(2, 0.05, 12, 12), _req(3, 0.1, 16, 16)]
    res, m = srv.run(reqs, realtime=True)
    assert m["failures"] == 0 and m["evictions"] >= 1
    assert m["peak_hbm_bytes"] <= budget
    assert len(b.live) <= 2


def test_slot_over_budget_is_an_error():
    srv = Server(FakeBackend(), hbm_budget=100)
    with pytest.raises(ValueError):
        srv.run([_req(0, 0.0)], realtime=True)


def test_offline_mode_skips_idle_time():
    b = FakeBackend()
    srv = Server(b, hbm_budget=8 * 8 * 16)
    res, m = srv.run([_req(0, 0.0), _req(1, 5.0)], realtime=False)
    assert res[1].latency == pytest.approx(0.010)


def test_prewarm_creates_idle_slots_within_budget():
    b = FakeBackend()
    one = 8 * 8 * 16
    srv = Server(b, hbm_budget=3 * one + 16 * 16 * 16)
    reqs = [_req(0, 0.0), _req(1, 0.0, 16, 16), _req(2, 0.0), _req(3, 0.05)]
    made = srv.prewarm(reqs, per_shape=2)
    assert made == 3 and b.created == 3              # 2 small + 1 large fill the budget; no eviction
    assert srv.bytes_in_use <= srv.budget and srv.evictions == 0
    res, m = srv.run(reqs, realtime=True)
    assert m["failures"] == 0 and b.created == 3     # the stream found its slots already created
    assert [r.rid for r in res] == [0, 1, 2, 3]


def test_shard_covers_all_frames_once():
    items = list(range(11))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert replicas.seed_offset(0) != replicas.seed_offset(1)


def _worker(rank, world_size, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world_size))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    mine = replicas.shard(range(10), rank, world_size)
    elapsed = 1.0 + rank                        # rank 1 is the slower replica
    t = replicas.max_over_ranks(elapsed)
    total = replicas.sum_over_ranks(len(mine))
    out.put((rank, t, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_total_frames():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, total in got:
        assert t == 2.0 and total == 10.0
    assert replicas.max_over_ranks(3.5) == 3.5     # without a process group: the value itself
