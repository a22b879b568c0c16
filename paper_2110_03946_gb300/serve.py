"""Continuous-batching server for inpainting decode requests.

Requests (one frame each: mask + known values, optionally part of a video
sequence) arrive over time.  The server keeps a pool of solver slots (one
dd_inpaint handle and one CUDA stream each, keyed by frame shape) inside an
HBM budget and, whenever a slot is free, starts the next admissible request on
it with the asynchronous C ABI, so the solves of several requests overlap on
the device.  A frame of a video sequence is routed to the slot that holds the
previous frame's iterate and warm-started from it (the slot's solver keeps the
iterate); frames of one sequence are served in order.  When the budget is
exhausted, idle slots of other shapes are evicted, least recently used first.

The scheduling logic talks to a backend interface; ``CudaBackend`` runs the
real solver, and tests can drive the server with a simulated backend.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds on the server clock
    mask: object                   # (H, W) uint8, host (pinned torch tensor or numpy) or device
    values: object                 # (C, H, W) float32
    seq: int | None = None         # video sequence id (None: independent frame)
    t: int = 0                     # frame index inside the sequence

    @property
    def shape(self):
        C, H, W = self.values.shape
        return (H, W, C)


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    start: float
    done: float
    status: int
    warm: bool
    slot: int
    output: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class _Slot:
    sid: int
    shape: tuple
    handle: object
    nbytes: int
    busy: bool = False
    req: Request | None = None
    start: float = 0.0
    warm: bool = False
    seq: int | None = None         # sequence whose last frame's iterate the slot holds
    t: int = -1
    last_used: float = 0.0


class Server:
    """Admission, slot management and completion tracking over a backend."""

    def __init__(self, backend, hbm_budget: int, max_slots: int = 64):
        self.b = backend
        self.budget = int(hbm_budget)
        self.max_slots = max_slots
        self.slots: list[_Slot] = []
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.max_queue = 0
        self._next_sid = 0
        self.evictions = 0

    # -- slot pool -----------------------------------------------------------------
    def _free_slot(self, req: Request):
        """A free slot for req: the one holding the previous frame of its
        sequence (warm), else any free slot of its shape (cold)."""
        if req.seq is not None:
            for s in self.slots:
                if not s.busy and s.seq == req.seq and s.t == req.t - 1 and s.shape == req.shape:
                    return s, True
        cands = [s for s in self.slots if not s.busy and s.shape == req.shape]
        if not cands:
            return None, False
        # prefer a slot that holds no sequence another waiting frame will want
        cands.sort(key=lambda s: (s.seq is not None, s.last_used))
        return cands[0], False

    def _make_room(self, need: int, keep_shape) -> bool:
        while self.bytes_in_use + need > self.budget or len(self.slots) >= self.max_slots:
            idle = [s for s in self.slots if not s.busy and s.shape != keep_shape]
            if not idle:
                idle = [s for s in self.slots if not s.busy]
                if not idle:
                    return False
            victim = min(idle, key=lambda s: s.last_used)
            self.b.destroy(victim.handle)
            self.slots.remove(victim)
            self.bytes_in_use -= victim.nbytes
            self.evictions += 1
        return True

    def _new_slot(self, req: Request):
        need = self.b.bytes_for(req.shape)
        if need > self.budget:
            raise ValueError(f"a single {req.shape} slot needs {need} bytes, over the budget {self.budget}")
        # evicting only idle slots of other shapes keeps capacity where it is used
        if not self._make_room(need, req.shape):
            return None
        handle, nbytes = self.b.create(req)
        if nbytes > need:
            # the slot holds more than estimated (the backend's estimate is
            # raised for the next time): make room for the actual size, else
            # give the slot up and let the request wait
            if nbytes > self.budget or not self._make_room(nbytes, req.shape):
                self.b.destroy(handle)
                return None
        s = _Slot(self._next_sid, req.shape, handle, nbytes)
        self._next_sid += 1
        self.slots.append(s)
        self.bytes_in_use += nbytes
        self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
        return s

    def prewarm(self, requests, per_shape: int = 1) -> int:
        """Create idle slots before traffic arrives: per_shape slots for each
        distinct shape among requests (loaded with the first request of that
        shape), as far as the HBM budget and the slot limit allow without
        evicting.  The first requests of a shape then find a slot whose
        allocations and device-loop graphs already exist.  Returns the number
        of slots created."""
        first = {}
        for r in requests:
            first.setdefault(r.shape, r)
        made = 0
        for shape, r in first.items():
            for _ in range(per_shape):
                need = self.b.bytes_for(shape)
                if self.bytes_in_use + need > self.budget or len(self.slots) >= self.max_slots:
                    break
                if self._new_slot(r) is None:
                    break
                made += 1
        return made

    # -- main loop -----------------------------------------------------------------
    def run(self, requests, realtime: bool = True, on_result=None):
        """Serve all requests; returns (results sorted by rid, metrics).
        on_result(result) is called at each completion, while result.output
        (the slot's buffer) still holds that request's image."""
        for s in self.slots:   # sequence ids are local to one run
            s.seq, s.t = None, -1
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: list[Request] = []
        results: list[Result] = []
        seq_next = {}                         # sequence -> next frame index allowed to start
        for r in pending:
            if r.seq is not None:
                seq_next.setdefault(r.seq, r.t)
                seq_next[r.seq] = min(seq_next[r.seq], r.t)
        t0 = self.b.now()
        clock = (lambda: self.b.now() - t0)
        n = len(pending)
        while len(results) < n:
            now = clock()
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            self.max_queue = max(self.max_queue, len(waiting))
            # admit every waiting request that can start now (arrival order)
            progressed = False
            for req in list(waiting):
                if req.seq is not None and seq_next.get(req.seq) != req.t:
                    continue                  # its previous frame is not finished yet
                slot, warm = self._free_slot(req)
                if slot is None:
                    slot = self._new_slot(req)
                    warm = False
                    if slot is None:
                        continue
                    fresh = True
                else:
                    fresh = False
                slot.busy, slot.req, slot.start, slot.warm = True, req, clock(), warm
                self.b.submit(slot.handle, req, warm=warm, fresh=fresh)
                waiting.remove(req)
                progressed = True
            # complete finished solves
            for s in self.slots:
                if s.busy and self.b.ready(s.handle):
                    status, out = self.b.finish(s.handle)
                    req = s.req
                    done = clock()
                    res = Result(req.rid, req.arrival, s.start, done, status, s.warm, s.sid, out)
                    if on_result is not None:
                        on_result(res)
                    res.output = None
                    results.append(res)
                    s.busy, s.req, s.last_used = False, None, done
                    s.seq, s.t = (req.seq, req.t) if req.seq is not None else (None, -1)
                    if req.seq is not None:
                        seq_next[req.seq] = req.t + 1
                    progressed = True
            if not progressed:
                busy = any(s.busy for s in self.slots)
                if not busy and not waiting and pending:
                    wait = pending[0].arrival - clock()
                    if realtime and wait > 0:
                        self.b.sleep(wait)
                    elif not realtime:
                        # offline: jump the clock forward to the next arrival
                        t0 -= max(wait, 0.0)
                elif busy:
                    self.b.idle()
                elif waiting and not busy:
                    raise RuntimeError("requests cannot be admitted: budget or slot limit too small")
        results.sort(key=lambda r: r.rid)
        lat = np.array([r.latency for r in results]) * 1e3
        span = max(r.done for r in results) - min(r.arrival for r in results)
        metrics = {
            "requests": n,
            "frames_per_s": n / span if span > 0 else float("inf"),
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()),
            "warm_starts": int(sum(r.warm for r in results)),
            "slots_created": self._next_sid,
            "evictions": self.evictions,
            "peak_hbm_bytes": self.peak_bytes,
            "max_queue": self.max_queue,
            "failures": int(sum(r.status != 0 for r in results)),
        }
        return results, metrics

    def close(self):
        for s in self.slots:
            self.b.destroy(s.handle)
        self.slots.clear()
        self.bytes_in_use = 0


class CudaBackend:
    """The real solver: one dd_inpaint handle and stream per slot, inputs from
    pinned host memory (copied inside the timed request), results left on the
    device (or copied back when host_output is set).  per_shape: optional
    {(H, W, C): params} overriding params for frames of that shape (e.g. the
    autotuner's entries)."""

    def __init__(self, params: dict, tol: float = 1e-6, device="cuda", host_output: bool = True,
                 per_shape: dict | None = None):
        import torch

        from . import binding as B
        from .inpaint import make_params
        self.torch, self.B = torch, B
        self.dev = torch.device(device)
        self.tol = tol
        self._make_params = make_params
        self.params = dict(params)
        self.per_shape = dict(per_shape or {})
        self.host_output = host_output
        self._state = {}
        self._bytes_cache = {}

    def params_for(self, shape) -> dict:
        return dict(self.per_shape.get(tuple(shape), self.params))

    def now(self) -> float:
        return time.perf_counter()

    def sleep(self, s: float):
        time.sleep(min(s, 0.05))

    def idle(self):
        time.sleep(0)

    def bytes_for(self, shape) -> int:
        """Device bytes of one slot: the handle (an estimate until a slot of
        this shape has been created, then the handle's own count) and the
        slot's output buffer."""
        if shape not in self._bytes_cache:
            H, W, C = shape
            # pitched FP32 planes: f and two iterates per level, levels shrink by 4
            P = (W + 31) // 32 * 32
            lv = 4.0 / 3.0
            est = int(C * H * P * 4 * 3 * lv + H * W * 2 + (1 << 22))
            self._bytes_cache[shape] = est
        H, W, C = shape
        return self._bytes_cache[shape] + C * H * W * 4

    def create(self, req: Request):
        torch, B = self.torch, self.B
        C, H, W = req.values.shape
        m = _host_u8(torch, req.mask)
        v = _host_f32(torch, req.values)
        prm = self._make_params(inputs_on_device=0, precision="fp32", **self.params_for((H, W, C)))
        rc, h = B.dd_inpaint_create(H, W, C, m.data_ptr(), v.data_ptr(), prm)
        B.check(rc, "dd_inpaint_create")
        rc, st = B.dd_inpaint_stats(h)
        stream = torch.cuda.Stream(self.dev)
        out = torch.empty((C, H, W), dtype=torch.float32, device=self.dev)
        host = torch.empty((C, H, W), dtype=torch.float32).pin_memory() if self.host_output else None
        self._state[h.value] = {"stream": stream, "out": out, "host": host, "inputs": None}
        self._bytes_cache[(H, W, C)] = max(self._bytes_cache.get((H, W, C), 0), int(st.device_bytes))
        return h, int(st.device_bytes) + out.numel() * out.element_size()

    def destroy(self, h):
        self.torch.cuda.synchronize(self.dev)
        self.B.dd_inpaint_destroy(h)
        self._state.pop(h.value, None)

    def submit(self, h, req: Request, warm: bool, fresh: bool):
        torch, B = self.torch, self.B
        s = self._state[h.value]
        m = _host_u8(torch, req.mask)
        v = _host_f32(torch, req.values)
        s["inputs"] = (m, v)                  # keep the pinned inputs alive until finish
        if not fresh:
            B.check(B.dd_inpaint_set_data_async(h, m.data_ptr(), v.data_ptr(), int(warm), s["stream"]),
                    "set_data_async")
        elif warm:
            raise ValueError("a fresh slot cannot warm-start")
        B.check(B.dd_inpaint_solve_async(h, s["out"].data_ptr(), self.tol, s["stream"]), "solve_async")
        if s["host"] is not None:
            with torch.cuda.stream(s["stream"]):
                s["host"].copy_(s["out"], non_blocking=True)
        s["event"] = torch.cuda.Event()
        s["event"].record(s["stream"])

    def ready(self, h) -> bool:
        return self._state[h.value]["event"].query()

    def finish(self, h):
        torch, B = self.torch, self.B
        s = self._state[h.value]
        rc = B.dd_inpaint_solve_finish(h, s["stream"])
        rcs, st = B.dd_inpaint_stats(h)
        if s["host"] is not None and st.host_continued:
            s["host"].copy_(s["out"])         # the finish rewrote the output: copy the final result
        s["inputs"] = None
        return rc, (s["host"] if s["host"] is not None else s["out"])


def _host_u8(torch, m):
    t = torch.as_tensor(m)
    if t.dtype != torch.uint8:
        t = (t != 0).to(torch.uint8)
    if t.is_cuda:
        t = t.cpu()
    return t.contiguous() if t.is_pinned() else t.contiguous().pin_memory()


def _host_f32(torch, v):
    t = torch.as_tensor(v)
    if t.dtype != torch.float32:
        t = t.to(torch.float32)
    if t.is_cuda:
        t = t.cpu()
    return t.contiguous() if t.is_pinned() else t.contiguous().pin_memory()


# ---------------------------------------------------------------- workload
def make_pool(shapes, n_frames: int, n_masks: int, density_range, seed: int, pinned: bool = True):
    """Per shape (H, W, C): one seeded video sequence of n_frames (frame t+1 is
    frame t shifted by 1..3 px, reflect-padded, plus Gaussian noise sigma 2,
    see synth.shifted_sequence) and n_masks uniform masks with densities in
    density_range.  Returned as torch tensors (pinned host memory)."""
    import torch

    import synth
    pool = {}
    rng = np.random.default_rng(seed)
    for k, (H, W, C) in enumerate(shapes):
        f0, _ = synth.make_frame(H, W, C, 0.05, "uniform", seed + 17 * k)
        frames = synth.shifted_sequence(f0, n_frames, seed + 17 * k + 1)
        masks = [synth.uniform_mask(H, W, rng.uniform(*density_range), rng) for _ in range(n_masks)]
        conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()) if pinned else \
            (lambda a: torch.from_numpy(np.ascontiguousarray(a)))
        pool[(H, W, C)] = ([conv(f) for f in frames], [conv(m) for m in masks])
    return pool


def poisson_stream(rate: float, duration: float, shapes, shape_probs, seq_len: int, seed: int, pool):
    """Requests of the serving benchmark: Poisson arrivals at `rate` per second
    over `duration` seconds.  Each arrival continues an open video sequence
    (probability 0.85, when one is open) or opens a new one with a shape drawn
    from shape_probs; a sequence has seq_len frames taken in order from the
    shape's pooled sequence (wrapping), each with a pooled mask."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    active = []                               # [seq id, shape, start offset, next t]
    seq_id = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if active and rng.uniform() < 0.85:
            a = active[rng.integers(len(active))]
        else:
            shape = shapes[rng.choice(len(shapes), p=shape_probs)]
            a = [seq_id, shape, int(rng.integers(1 << 16)), 0]
            seq_id += 1
            active.append(a)
        seq, shape, off, ft = a
        frames, masks = pool[shape]
        f = frames[(off + ft) % len(frames)]
        m = masks[int(rng.integers(len(masks)))]
        reqs.append(Request(len(reqs), t, m, f, seq, ft))
        a[3] = ft + 1
        if a[3] >= seq_len:
            active.remove(a)
    return reqs
