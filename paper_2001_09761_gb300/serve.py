"""Continuous-batching server for CLUE events.

Requests (one event each: host x, y, layer, energy) arrive at any time.  The
server thread:

* admits a waiting request into the region being filled when the region has
  room (hits and events) and the device-memory budget covers the event's
  estimated footprint; otherwise the request waits (back-pressure);
* copies an admitted event's inputs into a resident device region on a copy
  stream as soon as it is admitted, so copies overlap the batch computing on
  the device;
* launches the filled region as one batch (``clue_run_batch``, all sizes
  mixed) as soon as the device has room for it (at most ``max_inflight``
  batches queued), then starts filling the next free region;
* when a batch is done (results on the device, or on the host if asked),
  resolves each request's future and releases its budget.

Each event's result is identical whether it runs alone or in any batch
(bit-exact; the library's per-event ids and canonical arithmetic guarantee
it).  Latency is measured from ``submit`` to the future's resolution.

The device work goes through a backend object (``GpuBackend`` over libclue);
the scheduling above is independent of it, so it can be exercised with a fake
backend on a machine without a GPU.
"""
from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

#: Device bytes per admitted hit held against the budget: inputs (16) and
#: outputs (5) in the region plus the pipeline's scratch per hit.
BYTES_PER_HIT = 16 + 5 + 120


@dataclass
class _Request:
    x: object
    y: object
    layer: object
    energy: object
    n: int
    t_submit: float
    future: Future
    rid: int
    keep: list = field(default_factory=list)   # host copies alive until staged


@dataclass
class _Region:
    idx: int
    state: str = "free"        # free -> filling -> running -> free
    reqs: list = field(default_factory=list)
    offsets: list = field(default_factory=lambda: [0])
    hits: int = 0
    handle: object = None


class GpuBackend:
    """Resident device regions on one GPU, clustered through libclue.

    Results are returned as device tensors (an int32 cluster-id and a uint8
    seed view per event of one copy of the batch's outputs, made on the
    compute stream right after the batch), so a request is complete when its
    results are on the device.  With ``host_results`` they are copied to host numpy arrays
    instead.
    """

    def __init__(self, device=0, extent=(-250.0, 250.0, -250.0, 250.0), max_layers=100,
                 params=(2.0, 2.0, 2.0, 4.0), region_hits=8_000_000, n_regions=3, tuning=None,
                 host_results=False):
        import torch

        from . import clue
        self.torch, self.clue = torch, clue
        self.dev = torch.device("cuda", device)
        self.params = tuple(float(v) for v in params)
        self.cl = clue.Clusterer(device=device, extent=extent, max_layers=max_layers,
                                 use_graphs=False)
        if tuning:
            self.cl.tuning = tuning
        self.copy_stream = torch.cuda.Stream(device=self.dev)
        self.capacity = int(region_hits)
        self.n_regions = n_regions
        self.host_results = host_results
        mk = lambda dt: torch.empty(self.capacity, dtype=dt, device=self.dev)
        self.bufs = [dict(x=mk(torch.float32), y=mk(torch.float32), l=mk(torch.int32),
                          e=mk(torch.float32), cid=mk(torch.int32), seed=mk(torch.uint8))
                     for _ in range(n_regions)]
        if host_results:
            pin = lambda dt: torch.empty(self.capacity, dtype=dt).pin_memory()
            for bf in self.bufs:
                bf["hcid"], bf["hseed"] = pin(torch.int32), pin(torch.uint8)

    def stage(self, region: int, offset: int, req: _Request):
        """Queue the copy of one event's inputs into a region (one library
        call for the four arrays; host tensors or numpy arrays of the right
        dtypes, pinned for asynchronous copies)."""
        if req.n == 0:
            return
        t = self.torch
        b = self.bufs[region]
        srcs = []
        for arr, dt, tdt in ((req.x, np.float32, t.float32), (req.y, np.float32, t.float32),
                             (req.layer, np.int32, t.int32),
                             (req.energy, np.float32, t.float32)):
            if isinstance(arr, t.Tensor):
                a = arr.to(tdt).contiguous()
                ptr = a.data_ptr()
            else:
                a = np.ascontiguousarray(arr, dtype=dt)
                ptr = a.ctypes.data
            req.keep.append(a)
            srcs.append(ptr)
        rc = self.clue.clue_stage_event(*srcs, req.n, b["x"].data_ptr(), b["y"].data_ptr(),
                                        b["l"].data_ptr(), b["e"].data_ptr(), offset,
                                        self.copy_stream.cuda_stream)
        if rc:
            raise self.clue.ClueError(rc, "clue_stage_event")

    def launch(self, region: int, offsets):
        """Cluster the region's events as one batch; returns a handle whose
        completion event covers the per-event result copies."""
        t, clue = self.torch, self.clue
        b = self.bufs[region]
        ready = self.copy_stream.record_event()
        cs = self.cl.stream
        cs.wait_event(ready)
        offs = np.asarray(offsets, np.int64)
        n = int(offs[-1])
        rc = clue.clue_run_batch(self.cl.ctx, b["x"].data_ptr(), b["y"].data_ptr(),
                                 b["l"].data_ptr(), b["e"].data_ptr(), offs, len(offs) - 1,
                                 *self.params, b["cid"].data_ptr(), b["seed"].data_ptr())
        if rc:
            raise clue.ClueError(rc, "clue_run_batch", clue.clue_last_message(self.cl.ctx))
        outs = None
        with t.cuda.stream(cs):
            if self.host_results:
                b["hcid"][:n].copy_(b["cid"][:n], non_blocking=True)
                b["hseed"][:n].copy_(b["seed"][:n], non_blocking=True)
            else:  # one copy per batch; each request gets a view of it
                cid_all, seed_all = b["cid"][:n].clone(), b["seed"][:n].clone()
                outs = [(cid_all[a:z], seed_all[a:z])
                        for a, z in zip(offs[:-1].tolist(), offs[1:].tolist())]
        return {"done": cs.record_event(), "outs": outs}

    def ready(self, handle) -> bool:
        return handle["done"].query()

    def fetch(self, region: int, handle, k: int, a: int, b: int):
        if not self.host_results:
            return handle["outs"][k]
        buf = self.bufs[region]
        return buf["hcid"][a:b].numpy().copy(), buf["hseed"][a:b].numpy().copy()

    def check(self) -> int:
        """Deferred device errors (waits for the device); 0 if none."""
        return self.clue.clue_sync(self.cl.ctx)

    def close(self):
        self.cl.close()


class Server:
    """Continuous batching over a backend; see the module docstring."""

    def __init__(self, backend, max_events_per_batch=512, max_inflight=2,
                 mem_budget_bytes=None, min_launch_hits=0, poll_s=50e-6):
        self.be = backend
        self.max_events = max_events_per_batch
        self.max_inflight = min(max_inflight, backend.n_regions - 1)
        self.budget = mem_budget_bytes if mem_budget_bytes is not None else float("inf")
        self.min_launch_hits = min_launch_hits
        self.poll_s = poll_s
        self.regions = [_Region(i) for i in range(backend.n_regions)]
        self.inbox: queue.Queue = queue.Queue()
        self.waiting: list = []
        self.used = 0
        self.lat = []
        self.done_hits = 0
        self.t_first = None
        self.t_last = None
        self.batches = 0
        self.batch_sizes = []
        self.errors = 0
        self._rid = 0
        self._stop = threading.Event()
        self._lock = threading.Lock()
        self.thread = threading.Thread(target=self._loop, name="clue-serve", daemon=True)
        self.thread.start()

    # -- client side ---------------------------------------------------------
    def submit(self, x, y, layer, energy) -> Future:
        fut: Future = Future()
        n = int(len(x))
        with self._lock:
            rid = self._rid
            self._rid += 1
        if n > self.be.capacity or n * BYTES_PER_HIT > self.budget:
            fut.set_exception(ValueError(f"event of {n} hits exceeds the server's capacity"))
            return fut
        self.inbox.put(_Request(x, y, layer, energy, n, time.perf_counter(), fut, rid))
        return fut

    def close(self, check=True):
        self._stop.set()
        self.thread.join()
        rc = self.be.check() if check else 0
        self.be.close()
        if rc:
            raise RuntimeError(f"device reported error {rc} for a served batch")

    def stats(self) -> dict:
        lat = np.array(self.lat) * 1e3
        span = (self.t_last - self.t_first) if self.t_first is not None and self.t_last else 0.0
        return {
            "events": len(self.lat),
            "hits": self.done_hits,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
            "mhits_per_s": self.done_hits / span / 1e6 if span > 0 else None,
            "batches": self.batches,
            "mean_events_per_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
        }

    # -- server thread -------------------------------------------------------
    def _filling(self):
        for r in self.regions:
            if r.state == "filling":
                return r
        for r in self.regions:
            if r.state == "free":
                r.state = "filling"
                r.reqs, r.offsets, r.hits = [], [0], 0
                return r
        return None

    def _admit(self):
        while True:
            try:
                self.waiting.append(self.inbox.get_nowait())
            except queue.Empty:
                break
        admitted = False
        while self.waiting:
            req = self.waiting[0]
            reg = self._filling()
            if reg is None:
                break
            if reg.hits + req.n > self.be.capacity or len(reg.reqs) >= self.max_events:
                break  # region full: launch it first
            cost = req.n * BYTES_PER_HIT
            if self.used + cost > self.budget:
                break  # device budget exhausted: wait for completions
            self.waiting.pop(0)
            if self.t_first is None:
                self.t_first = req.t_submit
            self.be.stage(reg.idx, reg.hits, req)
            reg.reqs.append(req)
            reg.hits += req.n
            reg.offsets.append(reg.hits)
            self.used += cost
            admitted = True
        return admitted

    def _running(self):
        return [r for r in self.regions if r.state == "running"]

    def _launch(self, force=False):
        reg = next((r for r in self.regions if r.state == "filling" and r.reqs), None)
        if reg is None:
            return False
        running = self._running()
        if len(running) >= self.max_inflight:
            return False
        full = (reg.hits >= self.min_launch_hits or not running or force or
                (self.waiting and (reg.hits + self.waiting[0].n > self.be.capacity)))
        if not full:
            return False
        reg.handle = self.be.launch(reg.idx, reg.offsets)
        reg.state = "running"
        reg.seq = self.batches
        self.batches += 1
        self.batch_sizes.append(len(reg.reqs))
        return True

    def _complete(self):
        progressed = False
        for reg in sorted(self._running(), key=lambda r: r.seq):
            if not self.be.ready(reg.handle):
                break  # batches finish in launch order on one stream
            now = time.perf_counter()
            for k, req in enumerate(reg.reqs):
                cid, seed = self.be.fetch(reg.idx, reg.handle, k, reg.offsets[k],
                                          reg.offsets[k + 1])
                self.lat.append(now - req.t_submit)
                self.done_hits += req.n
                self.used -= req.n * BYTES_PER_HIT
                req.future.set_result((cid, seed))
            self.t_last = now
            reg.state = "free"
            reg.reqs = []
            progressed = True
        return progressed

    def _loop(self):
        try:
            while True:
                busy = self._complete()
                busy |= self._admit()
                busy |= self._launch()
                if self._stop.is_set() and self.inbox.empty() and not self.waiting and \
                        not any(r.reqs for r in self.regions):
                    break
                if self._stop.is_set():
                    busy |= self._launch(force=True)
                if not busy:
                    time.sleep(self.poll_s)
        except BaseException as exc:  # fail every request still held
            self.errors += 1
            for r in self.regions:
                for req in r.reqs:
                    if not req.future.done():
                        req.future.set_exception(exc)
            for req in self.waiting:
                if not req.future.done():
                    req.future.set_exception(exc)
            while True:
                try:
                    req = self.inbox.get_nowait()
                except queue.Empty:
                    break
                req.future.set_exception(exc)


def offered_load(server: Server, pool, rate_events_per_s: float, n_requests: int, seed=0):
    """Submit n_requests events drawn cyclically from `pool` (list of
    (x, y, layer, energy) tuples) at Poisson arrival times; wait for all."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_events_per_s, n_requests)
    order = rng.integers(0, len(pool), n_requests)
    t0 = time.perf_counter()
    t_next = t0
    futs = []
    for k in range(n_requests):
        t_next += gaps[k]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)  # releases the interpreter lock for the server thread
        futs.append(server.submit(*pool[order[k]]))
    for f in futs:
        f.result()
    return futs
