"""Continuous-batching render server over a resident Gaussian scene.

Requests (a camera each, any resolution) arrive over time.  Whenever one of
`streams` slots is free, the server takes the requests that have arrived, in
arrival order, as long as they fit the memory budget for sort and tile
buffers and the batch has at most `max_views` views, and hands them to that
slot's worker thread, which renders them as one batch on the slot's CUDA
stream: one gs_preprocess over all the batch's views, one shared gs_bin_sort
(the view is part of the global tile id) and one gs_render_fwd launch over
every tile of every view.  The admission loop never waits for a launch: the
preprocess's read-back of the entry count and the wait for completion block
only the slot's worker (the library calls release the interpreter lock), so
requests arriving meanwhile are admitted to the other slots at once.  Batches
on different slots overlap on the device.  Completion is stamped with a CUDA
event on the batch's stream, so latencies are device-accurate:
latency = completion - arrival, queueing included.

With streams=1 and max_views=1 the same loop serves one request at a time
in arrival order (the baseline).

Admission is two-phase because a batch's sort memory is only known after
preprocessing: a request is admitted on an estimate (its tiles times a
running entries-per-tile estimate), and the reservation is corrected to the
exact workspace sizes once the batch's entry count is known.

Each slot keeps its device buffers (workspaces and outputs) and grows them
when a batch needs more, so requests do not go through the allocator (before
the clock starts, every slot renders the trace's largest requests once so
that its buffers begin at their working size); and
each slot has a second, high-priority stream for batches above big_pixels
pixels, the slowest requests, whose blocks are then scheduled first when
they overlap smaller work.
"""
from __future__ import annotations

import gc
import math
import queue
import sys
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import raster


@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the trace start
    cam: object
    done: float | None = None   # seconds after the trace start (device time)
    # seconds after the trace start (host clock) at which the slot's worker
    # began launching the request's batch: latency splits into the wait
    # before it (queue and admission) and the service after it
    started: float | None = None
    batch: int = -1
    image: torch.Tensor | None = None
    # set by the caller at any time before the request is admitted: the
    # server then drops it (done stays None, batch -1)
    cancelled: bool = False

    @property
    def pixels(self) -> int:
        return int(self.cam.width) * int(self.cam.height)


@dataclass
class _Batch:
    bid: int
    reqs: list
    stream: torch.cuda.Stream
    reserved: int
    event: torch.cuda.Event
    keep: list = field(default_factory=list)    # tensors alive until completion


class RenderServer:
    def __init__(self, g: raster.GaussianTensors, budget_bytes: int = 24 << 30, streams: int = 3,
                 max_views: int = 16, keep_images: bool = False, cfg=None, entries_per_tile: float = 3000.0,
                 big_pixels: int | None = 4_000_000):
        self.g = g
        self.budget = int(budget_bytes)
        self.n_slots = int(streams)
        self.max_views = int(max_views)
        self.keep_images = keep_images
        self.cfg = cfg or raster.make_config()
        self.ept = float(entries_per_tile)          # running estimate of entries per tile
        # each slot has a normal and a high-priority stream; batches of more
        # than big_pixels pixels (the slowest requests, which set the latency
        # tail) run on the high-priority one, so that their blocks are
        # scheduled first when they overlap smaller work
        self.big_pixels = big_pixels
        lo, hi = torch.cuda.Stream.priority_range()
        self.streams = [torch.cuda.Stream(priority=lo) for _ in range(self.n_slots)]
        self.hi_streams = [torch.cuda.Stream(priority=hi) for _ in range(self.n_slots)]
        # per-slot device buffers, grown on demand and reused by the slot's
        # batches (a slot runs one batch at a time), so serving does not go
        # through the allocator per request
        self.slot_bufs = [dict() for _ in range(self.n_slots)]
        self.reserved = 0
        self.peak_reserved = 0
        self.batches_run = 0
        self.views_run = 0
        self._lock = threading.Lock()

    # -------------------------------------------------------------- memory
    @staticmethod
    def _tiles(cam) -> int:
        return math.ceil(cam.width / 16) * math.ceil(cam.height / 16)

    def _estimate(self, cam) -> int:
        """Bytes a request is admitted on: its share of the preprocess
        workspace, its estimated sort workspace and its outputs."""
        pre = self.g.n * 176
        sort = int(self._tiles(cam) * self.ept * 16 * 1.25) + (2 << 20)
        out = cam.width * cam.height * 24
        return pre + sort + out

    # -------------------------------------------------------------- buffers
    def _buf(self, slot: int, name: str, nbytes: int) -> torch.Tensor:
        """The first nbytes of the slot's buffer `name` (uint8), grown by 25 %
        headroom when too small."""
        b = self.slot_bufs[slot].get(name)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(int(nbytes * 1.25), 256), dtype=torch.uint8, device="cuda")
            self.slot_bufs[slot][name] = b
        return b[:max(nbytes, 1)]

    def _outputs(self, slot: int, plan) -> dict:
        """Forward outputs of the plan carved from the slot's output buffer."""
        P = int(plan.total_pixels)
        layout = (("image", 3 * P, torch.float32), ("final_T", P, torch.float32), ("n_contrib", P, torch.int32),
                  ("depth", P, torch.float32), ("imax", P, torch.int32))
        offs, o = [], 0
        for _, cnt, _ in layout:
            offs.append(o)
            o += (4 * cnt + 255) // 256 * 256
        buf = self._buf(slot, "out", o)
        return {name: buf[off: off + 4 * cnt].view(dt) for (name, cnt, dt), off in zip(layout, offs)}

    # -------------------------------------------------------------- one batch
    def _launch(self, reqs: list, slot: int, bid: int, est: int) -> _Batch:
        big = self.big_pixels is not None and sum(r.pixels for r in reqs) > self.big_pixels
        s = self.hi_streams[slot] if big else self.streams[slot]
        with torch.cuda.stream(s):
            cams = [r.cam for r in reqs]
            plan = raster.make_plan(self.g.n, cams)
            pre_ws = self._buf(slot, "pre", raster.preprocess_workspace_size(plan))
            raster.preprocess(plan, self.g.struct(), self.cfg, pre_ws, stream=s)
            sort_ws = self._buf(slot, "sort", raster.bin_sort_workspace_size(plan))
            raster.bin_sort(plan, pre_ws, sort_ws, stream=s)
            outs = self._outputs(slot, plan)
            raster.render_fwd(plan, self.cfg, pre_ws, sort_ws, outs, stream=s)
            if self.keep_images:
                for v, r in enumerate(reqs):
                    r.image = raster.view_image(outs["image"], plan, v).clone()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        actual = pre_ws.numel() + sort_ws.numel() + sum(t.numel() * t.element_size() for t in outs.values())
        tiles = sum(self._tiles(c) for c in cams)
        with self._lock:
            if tiles:
                self.ept = 0.8 * self.ept + 0.2 * (plan.n_entries / tiles)
            self.reserved += actual - est           # correct the admission estimate
            self.peak_reserved = max(self.peak_reserved, self.reserved)
        return _Batch(bid, reqs, s, actual, ev, [])

    # -------------------------------------------------------------- the loop
    def serve(self, trace: list) -> list:
        """Serves `trace` (Requests sorted by arrival) in real time; returns it
        with `done` filled in.  Python's cyclic garbage collector is paused
        for the duration (its sweeps stall the launch loop), and the
        interpreter's thread switch interval is shortened so that the slot
        workers and the admission loop hand over quickly."""
        was = gc.isenabled()
        interval = sys.getswitchinterval()
        gc.disable()
        sys.setswitchinterval(2e-5)
        try:
            self._prewarm(trace)
            return self._serve(trace)
        finally:
            sys.setswitchinterval(interval)
            if was:
                gc.enable()

    def _prewarm(self, trace: list, k: int = 3) -> None:
        """Before the clock starts: every slot renders the trace's k largest
        requests once, alone and then together, and its buffers are then
        grown by half again, so that they have reached their working size and
        no request waits on the allocator.  The admission accounting is reset
        afterwards."""
        big = sorted(trace, key=lambda r: -r.pixels)[:k]
        if not big:
            return
        for slot in range(self.n_slots):
            groups = [[r] for r in big] + ([big] if len(big) > 1 and len(big) <= self.max_views else [])
            for grp in groups:
                reqs = [Request(-1, 0.0, r.cam) for r in grp]
                self._launch(reqs, slot, -1, 0).event.synchronize()
            # headroom for requests with more entries than the warm ones
            for name, b in list(self.slot_bufs[slot].items()):
                self._buf(slot, name, int(b.numel() * 1.5))
        torch.cuda.synchronize()
        self.reserved = 0
        self.peak_reserved = 0

    def _worker(self, slot: int, jobs: "queue.Queue", st: dict) -> None:
        """One slot: launches each batch it is given (the preprocess's read-back
        of the entry count blocks this thread only; the calls release the
        interpreter lock), waits for the batch on the device, stamps its
        requests and frees the slot."""
        while True:
            job = jobs.get()
            if job is None:
                return
            reqs, bid, est = job
            try:
                started = time.perf_counter() - st["t0"]
                for r in reqs:
                    r.started = started
                b = self._launch(reqs, slot, bid, est)
                b.event.synchronize()
                done = st["t0_ev"].elapsed_time(b.event) / 1e3
                for r in reqs:
                    r.done = done
                    r.batch = bid
                with st["cv"]:
                    self.reserved -= b.reserved
                    st["free"].append(slot)
                    st["inflight"] -= 1
                    st["cv"].notify()
            except BaseException as exc:         # handed to the admission loop
                with st["cv"]:
                    st["error"] = exc
                    st["inflight"] -= 1
                    st["free"].append(slot)
                    st["cv"].notify()

    def _serve(self, trace: list) -> list:
        pending = list(trace)
        queue_: list = []
        cv = threading.Condition(self._lock)      # guards reserved, the free slots and the error
        st = {"cv": cv, "free": list(range(self.n_slots)), "inflight": 0, "error": None}
        jobs = [queue.Queue() for _ in range(self.n_slots)]
        workers = [threading.Thread(target=self._worker, args=(k, jobs[k], st), daemon=True)
                   for k in range(self.n_slots)]
        for w in workers:
            w.start()
        torch.cuda.synchronize()
        st["t0_ev"] = torch.cuda.Event(enable_timing=True)
        st["t0_ev"].record(torch.cuda.current_stream())
        t0 = time.perf_counter()
        st["t0"] = t0
        bid = 0
        try:
            while True:
                with cv:
                    if st["error"] is not None:
                        raise st["error"]
                    now = time.perf_counter() - t0
                    while pending and pending[0].arrival <= now:
                        queue_.append(pending.pop(0))
                    # admit and hand batches to free slots
                    while queue_ and st["free"]:
                        take, need = [], 0
                        while queue_ and len(take) < self.max_views:
                            if queue_[0].cancelled:
                                queue_.pop(0)
                                continue
                            est = self._estimate(queue_[0].cam)
                            if take and self.reserved + need + est > self.budget:
                                break
                            if not take and self.reserved + est > self.budget and st["inflight"]:
                                break
                            take.append(queue_.pop(0))
                            need += est
                        if not take:
                            break
                        slot = st["free"].pop(0)
                        self.reserved += need
                        self.peak_reserved = max(self.peak_reserved, self.reserved)
                        st["inflight"] += 1
                        jobs[slot].put((take, bid, need))
                        bid += 1
                        self.batches_run += 1
                        self.views_run += len(take)
                    if not pending and not queue_ and st["inflight"] == 0:
                        break
                    # sleep until just before the next arrival or until a slot
                    # reports back; the last 0.2 ms are spun (a timed wait wakes
                    # up too late for sub-millisecond latencies)
                    wait = (pending[0].arrival - (time.perf_counter() - t0)) if pending else 0.05
                    if queue_ and not st["free"]:
                        wait = 0.05
                    if wait > 3e-4:
                        cv.wait(timeout=min(wait - 2e-4, 0.05))
                time.sleep(0)                        # let the slot workers take the interpreter
        finally:
            for q in jobs:
                q.put(None)
            for w in workers:
                w.join()
        torch.cuda.synchronize()
        return trace


def poisson_trace(n: int, rate: float, seed: int = 3, sizes=None) -> list:
    """n requests with exponential inter-arrival times (mean 1/rate), poses on
    a sphere of radius U[3, 6] looking at the origin and resolutions drawn
    uniformly from `sizes` (fovx 60 degrees)."""
    from . import scenes
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return [Request(i, float(t[i]), scenes.sphere_camera(rng, sizes)) for i in range(n)]


def latency_stats(reqs: list, skip: int = 0) -> dict:
    """Latency percentiles and throughput of the served requests after the
    first `skip` (cancelled requests, which have no completion, are left out),
    with the split of the slowest request's latency into its wait before its
    batch began launching and its service after that."""
    reqs = [r for r in reqs[skip:] if r.done is not None]
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    pix = sum(r.pixels for r in reqs)
    out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "requests": len(lat),
           "mpix_per_s": pix / span / 1e6}
    if all(r.started is not None for r in reqs):
        wait = np.array([r.started - r.arrival for r in reqs]) * 1e3
        service = lat - wait
        worst = int(lat.argmax())
        out.update({"wait_p99_ms": float(np.percentile(wait, 99)), "service_p99_ms": float(np.percentile(service, 99)),
                    "slowest_wait_ms": float(wait[worst]), "slowest_service_ms": float(service[worst])})
    return out
