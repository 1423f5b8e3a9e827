"""Request loop for concealment as a service: damaged frames arrive over time, are admitted
while device memory allows, and run in batches that overlap on the GPU.

  - Memory: everything a request needs on the device lives in preallocated arenas, one per
    stream: a pinned host arena and a device arena of the same size, bump-allocated per
    batch and reset when the batch completes.  Nothing is allocated or page-locked per
    request.  The device-memory budget counts the arenas and the contexts' scratch.
  - Admission: FIFO; a request joins the batch being formed for a free stream while its
    frame and mask fit that stream's arena (no reordering, so no starvation).
  - Continuous batching: whenever a stream is free and requests are waiting, the admitted
    waiting requests go out as one skmmse_conceal_batch launch on that stream (its own
    context, so concurrent launches never share scratch).  Requests that arrive while other
    batches run start on the next free stream.  Each stream's context runs its persistent
    launch with the SM's CTA slots divided among the streams (1 CTA per SM each for 2
    streams), so the launches of different streams are resident on the device together
    instead of queueing behind each other.
  - Device concurrency is measured on the device: each launch's first-CTA start and last-CTA
    end (global timer) give its resident interval; the loop reports the mean number of
    launches resident while the device is busy.
  - State on the GPU: a batch's frames and masks go to the device in one copy, are concealed
    in place, and return in one copy, all in the stream's order.

Latency of a request = the host's observation of its batch's completion - its arrival time.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds from the start of the run
    frame: np.ndarray         # uint8 [H, W]
    mb_lost: np.ndarray       # uint8 [ceil(H/16), ceil(W/16)]
    t_done: float | None = None
    result: np.ndarray | None = None

    @property
    def nbytes(self) -> int:
        return 2 * self.frame.nbytes + self.mb_lost.nbytes

    @property
    def n_lost(self) -> int:
        return int((self.mb_lost != 0).sum())


class Admission:
    """Device-memory admission: FIFO, admit while the in-flight bytes fit the budget."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.in_flight = 0
        self.waiting: collections.deque = collections.deque()

    def arrive(self, req):
        self.waiting.append(req)

    def admit(self, limit: int | None = None) -> list:
        out = []
        while self.waiting and (limit is None or len(out) < limit):
            r = self.waiting[0]
            if r.nbytes > self.budget:
                raise ValueError(f"request {r.rid} needs {r.nbytes} bytes, above the budget")
            if self.in_flight + r.nbytes > self.budget:
                break
            self.waiting.popleft()
            self.in_flight += r.nbytes
            out.append(r)
        return out

    def release(self, reqs):
        for r in reqs:
            self.in_flight -= r.nbytes
        assert self.in_flight >= 0


def _align(v: int, a: int = 256) -> int:
    return (v + a - 1) // a * a


class Arena:
    """A pinned host buffer and a device buffer of the same size; a batch's frames and masks
    take consecutive 256-byte-aligned pieces (the same offsets on both sides), so one copy
    each way moves the whole batch."""

    def __init__(self, nbytes: int):
        import torch
        self.nbytes = int(nbytes)
        self.host = torch.empty(self.nbytes, dtype=torch.uint8).pin_memory()
        self.dev = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.used = 0

    def reset(self):
        self.used = 0

    def fits(self, reqs_bytes: int) -> bool:
        return self.used + reqs_bytes <= self.nbytes

    def take(self, nbytes: int) -> int:
        off = _align(self.used)
        assert off + nbytes <= self.nbytes
        self.used = off + nbytes
        return off

    @staticmethod
    def request_bytes(r: Request) -> int:
        return _align(r.frame.nbytes) + _align(r.mb_lost.nbytes)


def resident_concurrency(intervals) -> dict:
    """Mean and largest number of launches resident on the device while it is busy, from
    launch intervals [(t0, t1)] in ns (sweep over the start and end events)."""
    ev = sorted([(t0, 1) for t0, t1 in intervals if t1 > t0] + [(t1, -1) for t0, t1 in intervals if t1 > t0])
    busy = total = 0.0
    cur = peak = 0
    last = None
    for t, d in ev:
        if last is not None and cur > 0:
            busy += t - last
            total += (t - last) * cur
        cur += d
        peak = max(peak, cur)
        last = t
    return {"mean_resident_launches": total / busy if busy > 0 else 0.0, "max_resident_launches": peak,
            "device_busy_s": busy * 1e-9}


@dataclass
class _Batch:
    reqs: list
    stream: object
    event: object
    views: list = field(default_factory=list)   # (offset, shape) of each result in the arena


class ServeLoop:
    """Runs a request stream through the library on cuda:0 with `n_streams` overlapping
    batches, each stream with its own context and arena of `arena_bytes`."""

    def __init__(self, params=None, n_streams: int = 2, arena_bytes: int = 128 << 20, max_batch: int = 64):
        import torch
        from . import skmmse
        self.torch = torch
        self.sk = skmmse
        self.p = params if params is not None else skmmse.params("efficient")
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.ctxs = [skmmse.Context() for _ in range(n_streams)]
        # divide the SMs' CTA slots among the streams' persistent launches (occupancy: 2)
        per = max(1, 2 // n_streams)
        for c in self.ctxs:
            c.set_config(per, 64, 64)
        self.arenas = [Arena(arena_bytes) for _ in range(n_streams)]
        self.busy = [None] * n_streams
        self.waiting: collections.deque = collections.deque()
        self.max_batch = max_batch
        self.max_overlap = 0
        self.n_batches = 0
        self.intervals = []
        props = torch.cuda.get_device_properties(0)
        # preallocated device memory: the arenas and each context's whitened-vector buffer
        # (1849 x 32 floats per persistent CTA of the largest grid); a context's work-queue
        # scratch grows on demand to the largest batch and is then reused
        self.prealloc_device_bytes = n_streams * (arena_bytes + props.multi_processor_count * 2 * 1849 * 32 * 4)

    def _launch(self, si: int, reqs: list):
        torch = self.torch
        s, ar = self.streams[si], self.arenas[si]
        ar.reset()
        b = _Batch(reqs, s, torch.cuda.Event())
        frames, masks = [], []
        for r in reqs:  # pack the batch into the pinned arena
            fo = ar.take(r.frame.nbytes)
            mo = ar.take(r.mb_lost.nbytes)
            ar.host[fo:fo + r.frame.nbytes].numpy()[:] = r.frame.reshape(-1)
            ar.host[mo:mo + r.mb_lost.nbytes].numpy()[:] = r.mb_lost.reshape(-1)
            frames.append(ar.dev[fo:fo + r.frame.nbytes].view(r.frame.shape))
            masks.append(ar.dev[mo:mo + r.mb_lost.nbytes].view(r.mb_lost.shape))
            b.views.append((fo, r.frame.shape))
        n = ar.used
        with torch.cuda.stream(s):
            ar.dev[:n].copy_(ar.host[:n], non_blocking=True)
            # conceal in place: the frame buffers become the results
            self.ctxs[si].conceal_batch(frames, masks, self.p, outs=frames, stream=s)
            ar.host[:n].copy_(ar.dev[:n], non_blocking=True)
            b.event.record(s)
        self.busy[si] = b
        self.n_batches += 1
        self.max_overlap = max(self.max_overlap, sum(x is not None for x in self.busy))

    def _poll(self, t0: float) -> int:
        done = 0
        for si, b in enumerate(self.busy):
            if b is not None and b.event.query():
                now = time.perf_counter() - t0
                ar = self.arenas[si]
                for r, (off, shape) in zip(b.reqs, b.views):
                    r.result = ar.host[off:off + int(np.prod(shape))].numpy().reshape(shape).copy()
                    r.t_done = now
                st = self.ctxs[si].read_stats(b.stream)
                self.intervals.append((st["t_first_ns"], st["t_last_ns"]))
                self.busy[si] = None
                done += len(b.reqs)
        return done

    def _form_batch(self, si: int) -> list:
        ar = self.arenas[si]
        ar.reset()
        out, need = [], 0
        while self.waiting and len(out) < self.max_batch:
            r = self.waiting[0]
            nb = Arena.request_bytes(r)
            if nb > ar.nbytes:
                raise ValueError(f"request {r.rid} needs {nb} bytes, above the arena")
            if need + nb > ar.nbytes:
                break
            need += nb
            out.append(self.waiting.popleft())
        return out

    def run(self, requests: list, realtime: bool = True) -> dict:
        """Serve `requests` (sorted by arrival).  With realtime, arrivals follow the wall
        clock; otherwise all requests are present at t = 0."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        n = len(reqs)
        i = 0
        finished = 0
        self.intervals = []
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            while i < n and (not realtime or reqs[i].t_arrival <= now):
                self.waiting.append(reqs[i])
                i += 1
            finished += self._poll(t0)
            free = [si for si, b in enumerate(self.busy) if b is None]
            if free and self.waiting:
                batch = self._form_batch(free[0])
                if batch:
                    self._launch(free[0], batch)
                    continue
            if i < n and realtime and not any(self.busy) and not self.waiting:
                time.sleep(max(0.0, min(reqs[i].t_arrival - now, 0.002)))
            else:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        lat = np.array([r.t_done - (r.t_arrival if realtime else 0.0) for r in reqs])
        mbs = sum(r.n_lost for r in reqs)
        return {"requests": n, "wall_s": wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
                "mbs_per_s": mbs / wall, "lost_mbs": mbs, "batches": self.n_batches,
                "max_overlap": self.max_overlap, "prealloc_device_bytes": self.prealloc_device_bytes,
                **resident_concurrency(self.intervals)}

    def close(self):
        for c in self.ctxs:
            c.close()


def make_requests(n: int, seed: int = 0, rate_hz: float = 600.0, pool_per_size: int = 8,
                  loss_lo: float = 0.02, loss_hi: float = 0.30):
    """Serving stream: Poisson arrivals at rate_hz, sizes 1/3 each 352x288 / 1280x720 /
    1920x1080, loss U[loss_lo, loss_hi] (half isolated blocks, half runs).  Frame contents
    cycle through a pool of `pool_per_size` seeded frames per size (generating 20,000
    distinct 1080p frames on the host would dominate the run); every request has its own
    seeded loss map."""
    from . import synth
    pool = {}
    out = []
    for rid, (t, w, h, fseed, mseed) in enumerate(synth.stream_requests(seed, n, rate_hz)):
        key = (w, h, fseed % pool_per_size)
        if key not in pool:
            pool[key] = synth.make_frame(w, h, seed * 1000 + key[2] + 17 * w)
        m = synth.loss_mixed(w, h, mseed, loss_lo, loss_hi)
        out.append(Request(rid, t, pool[key], m))
    return out
