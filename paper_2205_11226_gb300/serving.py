"""Request loop for concealment as a service: damaged frames arrive over time, are admitted
while device memory allows, and run in batches that overlap on the GPU.

  - Admission: every request needs device memory for its frame, its output and its block
    map; a request is admitted when the bytes of the requests in flight plus its own stay
    within the budget, oldest first (no reordering, so no starvation).
  - Continuous batching: whenever a stream is free and requests are waiting, all admitted
    waiting requests go out as one skmmse_conceal_batch launch on that stream (its own
    context, so concurrent launches never share scratch).  Requests that arrive while other
    batches run are admitted as memory frees up and start on the next free stream, so their
    work overlaps with the batches already on the device.
  - State on the GPU: a request's frame is copied in once, concealed on the device, and its
    result is copied back to pinned host memory in the same stream order.

Latency of a request = completion of its device->host copy - its arrival time.
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


@dataclass
class _Batch:
    reqs: list
    stream: object
    event: object
    dev: list = field(default_factory=list)
    host_out: list = field(default_factory=list)


class ServeLoop:
    """Runs a request stream through the library on cuda:0 with `n_streams` overlapping
    batches and a device-memory budget."""

    def __init__(self, params=None, n_streams: int = 3, budget_bytes: int = 2 << 30,
                 max_batch: int = 64):
        import torch
        from . import skmmse
        self.torch = torch
        self.sk = skmmse
        self.p = params if params is not None else skmmse.params("efficient")
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.ctxs = [skmmse.Context() for _ in range(n_streams)]
        self.busy = [None] * n_streams
        self.adm = Admission(budget_bytes)
        self.max_batch = max_batch
        self.max_overlap = 0
        self.n_batches = 0

    def _launch(self, si: int, reqs: list, t0: float):
        torch = self.torch
        s = self.streams[si]
        b = _Batch(reqs, s, torch.cuda.Event())
        with torch.cuda.stream(s):
            frames, masks = [], []
            for r in reqs:
                hf = torch.from_numpy(r.frame).pin_memory()
                hm = torch.from_numpy(r.mb_lost).pin_memory()
                df = torch.empty(hf.shape, dtype=torch.uint8, device="cuda")
                dm = torch.empty(hm.shape, dtype=torch.uint8, device="cuda")
                df.copy_(hf, non_blocking=True)
                dm.copy_(hm, non_blocking=True)
                frames.append(df)
                masks.append(dm)
            # conceal in place: the frame buffer becomes the result
            self.ctxs[si].conceal_batch(frames, masks, self.p, outs=frames, stream=s)
            for df in frames:
                ho = torch.empty(df.shape, dtype=torch.uint8).pin_memory()
                ho.copy_(df, non_blocking=True)
                b.host_out.append(ho)
            b.dev = frames + masks
            b.event.record(s)
        self.busy[si] = b
        self.n_batches += 1
        self.max_overlap = max(self.max_overlap, sum(x is not None for x in self.busy))

    def _poll(self, t0: float) -> int:
        done = 0
        for si, b in enumerate(self.busy):
            if b is not None and b.event.query():
                now = time.perf_counter() - t0
                for r, ho in zip(b.reqs, b.host_out):
                    r.result = ho.numpy()
                    r.t_done = now
                self.adm.release(b.reqs)
                self.busy[si] = None
                done += len(b.reqs)
        return done

    def run(self, requests: list, realtime: bool = True) -> dict:
        """Serve `requests` (sorted by arrival).  With realtime, arrivals follow the wall
        clock; otherwise all requests are present at t = 0."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        n = len(reqs)
        i = 0
        finished = 0
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            while i < n and (not realtime or reqs[i].t_arrival <= now):
                self.adm.arrive(reqs[i])
                i += 1
            finished += self._poll(t0)
            free = [si for si, b in enumerate(self.busy) if b is None]
            if free and self.adm.waiting:
                batch = self.adm.admit(self.max_batch)
                if batch:
                    self._launch(free[0], batch, t0)
                    continue
            if i < n and realtime and not any(self.busy) and not self.adm.waiting:
                time.sleep(max(0.0, min(reqs[i].t_arrival - now, 0.002)))
            else:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        lat = np.array([r.t_done - (r.t_arrival if realtime else 0.0) for r in reqs])
        mbs = sum(r.n_lost for r in reqs)
        return {"requests": n, "wall_s": wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
                "mbs_per_s": mbs / wall, "lost_mbs": mbs, "batches": self.n_batches,
                "max_overlap": self.max_overlap}

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
