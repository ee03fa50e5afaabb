"""Continuous-batching render server over resident PlenOctrees.

Requests (tree, camera of any resolution, arrival time) enter a wait queue.
A request is admitted when its output buffer fits the HBM budget left after
the resident trees and the outputs already in flight; admitted requests are
packed, as they come, into ``pot_render_batch`` launches (one work list per
launch, mixed trees and resolutions) on a small ring of CUDA streams, so work
that arrives while earlier launches run overlaps with them on the device.
Requests of at most ``priority_pixels`` pixels go, in their own work lists,
to a stream of higher priority: the batch kernel's blocks each render one
tile and end, so the GPU starts their blocks between those of large
requests already running.
Completion is read from CUDA events; a finished request releases its budget.
Outputs of finished requests are handed to the caller (``on_done``); when
the caller consumes them there, device memory held by outputs stays within
the admission budget; without ``on_done`` the finished images stay on the
requests, outside the budget, for the caller to keep or drop.
Mode ``alone`` renders one request per launch on one stream, in arrival order
(the baseline the batching is compared with).

All GPU work runs in libpot kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import render_batch


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    tree_id: int
    cam: object             # camera record (80 bytes, synth.CAMERA_DTYPE)
    out_bytes: int = 0
    rgb: object = None
    t_admit: float = -1.0
    t_launch: float = -1.0
    t_done: float = -1.0
    rejected: bool = False

    @property
    def rays(self) -> int:
        return int(self.cam["width"]) * int(self.cam["height"])


class Admission:
    """HBM accounting: resident tree bytes + bytes of outputs held by admitted requests."""

    def __init__(self, budget_bytes: int, resident_bytes: int):
        if resident_bytes > budget_bytes:
            raise ValueError("resident trees exceed the HBM budget")
        self.budget = int(budget_bytes)
        self.resident = int(resident_bytes)
        self.used = 0

    def fits(self, nbytes: int) -> bool:
        return self.resident + self.used + nbytes <= self.budget

    def take(self, nbytes: int) -> bool:
        if not self.fits(nbytes):
            return False
        self.used += nbytes
        return True

    def release(self, nbytes: int) -> None:
        self.used -= nbytes
        assert self.used >= 0


class RenderServer:
    def __init__(self, trees, hbm_budget_bytes: int, streams: int = 3, max_rays_per_launch: int = 8 << 20,
                 bg=(0.0, 0.0, 0.0), gamma: float = 1e-4, device="cuda", launcher=None, clock=None,
                 allocator=None, stream_factory=None, priority_pixels: int = 0):
        self.trees = trees
        resident = sum(int(t.info()["bytes"]) for t in trees) if launcher is None else 0
        self.adm = Admission(hbm_budget_bytes, resident)
        self.n_streams = streams
        # batch mode: requests of at most this many pixels are launched on a
        # stream of higher priority (0: no such stream), so that they start
        # between the blocks of large requests already on the GPU
        self.priority_pixels = int(priority_pixels)
        self.max_rays = max_rays_per_launch
        self.bg, self.gamma, self.device = tuple(bg), float(gamma), device
        self.clock = clock or time.perf_counter
        # injectable for host-only tests
        self.launcher = launcher or self._launch_gpu
        self.allocator = allocator or self._alloc_gpu
        self.stream_factory = stream_factory or self._streams_gpu

    # -- GPU plumbing -------------------------------------------------------
    def _alloc_gpu(self, req: Request):
        import torch
        return torch.empty((int(req.cam["height"]), int(req.cam["width"]), 3), dtype=torch.float32,
                           device=self.device)

    def _streams_gpu(self, n, high=False):
        import torch
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        return [torch.cuda.Stream(device=self.device, priority=(hi if high else 0)) for _ in range(n)]

    def _launch_gpu(self, reqs, stream):
        import torch
        items = [(self.trees[r.tree_id], r.cam, r.rgb, self.bg, self.gamma, None) for r in reqs]
        with torch.cuda.stream(stream):
            render_batch(items, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev

    # -- the loop -------------------------------------------------------------
    def run(self, requests, mode: str = "batch", on_done=None):
        """Serves ``requests`` (sorted by arrival) in real time; returns the requests with timestamps.

        ``on_done(request)`` is called as each request completes (its image in
        ``request.rgb``); the server then drops its reference to the image, so
        the bytes it returns to the budget are really free.  Without it,
        completed images stay on the requests: they leave the budget at
        completion and are the caller's to free."""
        assert mode in ("batch", "alone")
        n_streams = self.n_streams if mode == "batch" else 1
        per_launch = None if mode == "batch" else 1
        streams = self.stream_factory(n_streams)
        free = collections.deque(range(n_streams))
        hp = mode == "batch" and self.priority_pixels > 0
        if hp:   # one more stream slot, of high priority, for small requests
            streams = list(streams) + list(self.stream_factory(1, high=True))
        hp_free = hp
        arrivals = collections.deque(requests)
        waiting = collections.deque()
        ready = collections.deque()
        inflight = []               # (stream index, event, [requests])
        t0 = self.clock()
        now = 0.0
        while arrivals or waiting or ready or inflight:
            now = self.clock() - t0
            while arrivals and arrivals[0].arrival <= now:
                waiting.append(arrivals.popleft())
            # admission in arrival order, by HBM footprint of the output; a
            # request that cannot fit even into an idle server is rejected
            while waiting:
                r = waiting[0]
                r.out_bytes = 12 * r.rays
                if self.adm.resident + r.out_bytes > self.adm.budget:
                    waiting.popleft()
                    r.rejected = True
                    r.t_done = now
                    continue
                if not self.adm.take(r.out_bytes):
                    break
                waiting.popleft()
                r.rgb = self.allocator(r)
                r.t_admit = now
                ready.append(r)
            # completions
            still = []
            for si, ev, reqs in inflight:
                if ev.query():
                    t = self.clock() - t0
                    for r in reqs:
                        r.t_done = t
                        if on_done is not None:
                            on_done(r)
                            r.rgb = None
                        self.adm.release(r.out_bytes)
                    if si == n_streams:
                        hp_free = True
                    else:
                        free.append(si)
                else:
                    still.append((si, ev, reqs))
            inflight = still
            # small requests first, on the high-priority stream
            if hp and hp_free and any(r.rays <= self.priority_pixels for r in ready):
                batch, rest, rays = [], collections.deque(), 0
                for r in ready:
                    if r.rays <= self.priority_pixels and rays + r.rays <= self.max_rays:
                        batch.append(r)
                        rays += r.rays
                    else:
                        rest.append(r)
                ready = rest
                t = self.clock() - t0
                for r in batch:
                    r.t_launch = t
                hp_free = False
                inflight.append((n_streams, self.launcher(batch, streams[n_streams]), batch))
            # launches: everything admitted so far (up to the ray cap) in one work list
            while ready and free:
                batch, rays = [], 0
                while ready and (not batch or rays + ready[0].rays <= self.max_rays):
                    if per_launch is not None and len(batch) >= per_launch:
                        break
                    r = ready.popleft()
                    batch.append(r)
                    rays += r.rays
                si = free.popleft()
                t = self.clock() - t0
                for r in batch:
                    r.t_launch = t
                inflight.append((si, self.launcher(batch, streams[si]), batch))
            # while launches are in flight, poll their events without sleeping (a
            # sleep lasts tens of microseconds, which would add to every latency);
            # sleep only when waiting for the next arrival
            if not inflight and not (ready and (free or hp_free)) and \
                    not (arrivals and arrivals[0].arrival <= self.clock() - t0):
                time.sleep(2e-5)
        return requests


def summarize(requests, wall: float | None = None) -> dict:
    rejected = sum(1 for r in requests if r.rejected)
    requests = [r for r in requests if not r.rejected]
    lat = np.array([r.t_done - r.arrival for r in requests]) * 1e3
    rays = sum(r.rays for r in requests)
    t_end = max(r.t_done for r in requests)
    t_start = min(r.arrival for r in requests)
    span = wall if wall is not None else (t_end - t_start)
    by_res = {}
    for r, l in zip(requests, lat):
        by_res.setdefault(f"{int(r.cam['width'])}x{int(r.cam['height'])}", []).append(l)
    return {"requests": len(requests), "rejected": rejected, "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "max_ms": round(float(lat.max()), 3), "rays": int(rays),
            "mrays_s": round(rays / span / 1e6, 2), "span_s": round(span, 4),
            "by_resolution": {k: {"n": len(v), "p50_ms": round(float(np.percentile(v, 50)), 3),
                                  "p99_ms": round(float(np.percentile(v, 99)), 3)}
                              for k, v in sorted(by_res.items())},
            # arrival -> launch (queueing + admission + host work) and launch -> completion seen
            "p50_wait_ms": round(float(np.percentile([(r.t_launch - r.arrival) * 1e3 for r in requests], 50)), 3),
            "p50_run_ms": round(float(np.percentile([(r.t_done - r.t_launch) * 1e3 for r in requests], 50)), 3)}
