"""Continuous-batching server for CLUE events: a thin binding of the
library's native server (``clue_server_*`` in include/clue.h).

Requests (one event each: host x, y, layer, energy) arrive at any time, from
any thread.  The library's worker thread admits each into the device region
being filled while the region has room and the memory budget covers it (else
the request waits), copies its inputs there at once on a copy stream, and
launches a filled region as one ``clue_run_batch`` as soon as fewer than
``max_inflight`` batches are queued on the device; results are copied back
into each request's own output arrays (host or device) and a stream callback
marks it done (no polling).  Each event's result is the same whether it runs
alone or in any batch.  Latency runs from ``submit`` to the results in the
request's output arrays.

This module only marshals arguments: scheduling, copies and clustering all
run in libclue.  The scheduler itself (serve_core.cpp) is tested on a CPU
with a fake device (tests/serve_fake.cpp).
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import clue

#: Device bytes an admitted hit holds against a server's memory budget:
#: inputs (16) and outputs (5) in the region plus the run's scratch.
BYTES_PER_HIT = 16 + 5 + 120


class ClueServerOpts(ctypes.Structure):
    _fields_ = [("region_hits", ctypes.c_int64), ("n_regions", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("max_events_per_batch", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64)]


def _lib():
    lib = clue.load()
    if not getattr(lib, "_server_sigs", False):
        P, F, I64 = ctypes.c_void_p, ctypes.c_float, ctypes.c_int64
        lib.clue_server_default_opts.argtypes = [ctypes.POINTER(ClueServerOpts)]
        lib.clue_server_default_opts.restype = None
        lib.clue_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(clue.ClueOpts),
                                           ctypes.POINTER(ClueServerOpts), F, F, F, F,
                                           ctypes.c_char_p]
        lib.clue_server_create.restype = ctypes.c_int
        lib.clue_server_submit.argtypes = [P, P, P, P, P, I64, P, P, ctypes.POINTER(I64)]
        lib.clue_server_submit.restype = ctypes.c_int
        lib.clue_server_wait.argtypes = [P, I64, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]
        lib.clue_server_wait.restype = ctypes.c_int
        lib.clue_server_stats.argtypes = [P, P, P, I64]
        lib.clue_server_stats.restype = I64
        lib.clue_server_reset_stats.argtypes = [P]
        lib.clue_server_reset_stats.restype = ctypes.c_int
        lib.clue_server_destroy.argtypes = [P]
        lib.clue_server_destroy.restype = None
        lib._server_sigs = True
    return lib


class Ticket:
    """One submitted event.  ``result()`` waits for it and returns its
    (cluster_id int32, is_seed uint8) output arrays."""

    def __init__(self, server, ticket, keep, cid, seed):
        self._srv, self._t, self._keep = server, ticket, keep
        self._cid, self._seed = cid, seed
        self._done, self.latency_ms, self._rc = False, None, 0

    def result(self, timeout=None):
        if not self._done:
            rc, st, lat = self._srv.wait_raw(self._t, timeout)
            if rc == clue.CLUE_ERR_TIMEOUT:
                raise TimeoutError(f"event not done within {timeout} s")
            if rc:
                raise clue.ClueError(rc, "clue_server_wait")
            self._done, self._keep, self.latency_ms, self._rc = True, None, lat, st
        if self._rc:
            raise clue.ClueError(self._rc, "served event")
        return self._cid, self._seed


class Server:
    """A CLUE server on one GPU (see the module docstring).  ``params`` is
    (d_c, rho_c, delta_c, delta_o) for every event."""

    def __init__(self, device=0, extent=(-250.0, 250.0, -250.0, 250.0), max_layers=100,
                 params=(2.0, 2.0, 2.0, 4.0), region_hits=16_000_000, n_regions=3,
                 max_inflight=2, max_events_per_batch=512, mem_budget_bytes=0, tuning=None):
        import torch
        self.torch = torch
        lib = _lib()
        o = clue.clue_default_opts()
        o.device = device
        o.x_min, o.x_max, o.y_min, o.y_max = (float(v) for v in extent)
        o.max_layers = int(max_layers)
        so = ClueServerOpts()
        lib.clue_server_default_opts(ctypes.byref(so))
        so.region_hits, so.n_regions = int(region_hits), int(n_regions)
        so.max_inflight, so.max_events_per_batch = int(max_inflight), int(max_events_per_batch)
        so.mem_budget_bytes = int(mem_budget_bytes)
        h = ctypes.c_void_p()
        rc = lib.clue_server_create(ctypes.byref(h), ctypes.byref(o), ctypes.byref(so),
                                    *[float(v) for v in params],
                                    tuning.encode() if tuning else None)
        if rc:
            raise clue.ClueError(rc, "clue_server_create")
        self._h = h.value
        self.capacity = int(region_hits)
        self.device = torch.device("cuda", device)

    def submit(self, x, y, layer, energy, out=None) -> Ticket:
        """Queue one event: host arrays (numpy, or torch CPU tensors; pinned
        ones give asynchronous copies).  The results go to `out` = (cluster_id,
        is_seed) arrays or tensors, host or device, else to new CUDA tensors
        on the server's device.  Raises ValueError for an event the server
        cannot take (larger than a region or the memory budget)."""
        t = self.torch
        keep, ptrs = [], []
        for a, dt, tdt in ((x, np.float32, t.float32), (y, np.float32, t.float32),
                           (layer, np.int32, t.int32), (energy, np.float32, t.float32)):
            if isinstance(a, t.Tensor):
                a = a.to(tdt).contiguous()
                ptrs.append(a.data_ptr())
            else:
                a = np.ascontiguousarray(a, dtype=dt)
                ptrs.append(a.ctypes.data)
            keep.append(a)
        n = int(len(keep[0]))
        if out is None:
            out = (t.empty(n, dtype=t.int32, device=self.device),
                   t.empty(n, dtype=t.uint8, device=self.device))
        cid, seed = out
        keep += [cid, seed]
        ptr = lambda a: a.data_ptr() if isinstance(a, t.Tensor) else a.ctypes.data
        tk = self.submit_raw(*ptrs, n, ptr(cid), ptr(seed))
        return Ticket(self, tk, keep, cid, seed)

    def submit_raw(self, x, y, layer, energy, n, cluster_id, is_seed) -> int:
        """clue_server_submit on raw pointers (ints); returns the ticket.  The
        caller keeps all six arrays alive until wait_raw reports the event."""
        tk = ctypes.c_int64(0)
        rc = _lib().clue_server_submit(self._h, x, y, layer, energy, int(n), cluster_id,
                                       is_seed, ctypes.byref(tk))
        if rc == clue.CLUE_ERR_ARG:
            raise ValueError(f"event of {n} hits exceeds the server's capacity")
        if rc:
            raise clue.ClueError(rc, "clue_server_submit")
        return tk.value

    def wait_raw(self, ticket, timeout=None):
        """clue_server_wait: (return code, the event's status, latency ms)."""
        lat, st = ctypes.c_double(0.0), ctypes.c_int32(0)
        rc = _lib().clue_server_wait(self._h, int(ticket),
                                     -1.0 if timeout is None else float(timeout),
                                     ctypes.byref(st), ctypes.byref(lat))
        return rc, st.value, lat.value

    def stats(self) -> dict:
        lib = _lib()
        out = (ctypes.c_double * 6)()
        n = lib.clue_server_stats(self._h, out, None, 0)
        lat = (ctypes.c_double * max(1, n))()
        n = lib.clue_server_stats(self._h, out, lat, n)
        lat = np.frombuffer(lat, np.float64)[:n]
        span = out[4]
        return {
            "events": int(out[0]), "hits": int(out[1]), "batches": int(out[2]),
            "rejected": int(out[3]),
            "p50_ms": float(np.percentile(lat, 50)) if n else None,
            "p99_ms": float(np.percentile(lat, 99)) if n else None,
            "mean_ms": float(lat.mean()) if n else None,
            "mhits_per_s": out[1] / span / 1e6 if span > 0 else None,
            "mean_events_per_batch": out[5],
            "latency": "submit to results in the request's output arrays",
        }

    def reset_stats(self):
        """Start the counters and latencies again (e.g. after a warm-up)."""
        _lib().clue_server_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib().clue_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def offered_load(server, pool, rate_events_per_s: float, n_requests: int, seed=0):
    """Submit n_requests events drawn from `pool` (list of (x, y, layer,
    energy) host tensors, pinned for asynchronous copies) at Poisson arrival
    times, then wait for all; returns the latencies (ms).  The results go to
    a ring of device buffers (four regions' worth of hits), so the driver
    allocates nothing per request and submits fast enough for tens of
    thousands of events per second; before a slice of the ring is reused, the
    events still writing into it are waited for."""
    from collections import deque
    t = server.torch
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_events_per_s, n_requests)
    order = rng.integers(0, len(pool), n_requests)
    src = [(x.data_ptr(), y.data_ptr(), l.data_ptr(), e.data_ptr(), int(x.numel()))
           for x, y, l, e in pool]
    ring_n = 4 * server.capacity
    cid = t.empty(ring_n, dtype=t.int32, device=server.device)
    sd = t.empty(ring_n, dtype=t.uint8, device=server.device)
    c0, s0 = cid.data_ptr(), sd.data_ptr()
    at, lat, pending = 0, [], deque()  # pending: (ticket, first slot, hits), ring order

    def finish():
        tk, _, _ = pending.popleft()
        rc, st, ms = server.wait_raw(tk)
        if rc or st:
            raise clue.ClueError(rc or st, "served event")
        lat.append(ms)

    t_next = time.perf_counter()
    for k in range(n_requests):
        t_next += gaps[k]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        xp, yp, lp, ep, n = src[order[k]]
        if at + n > ring_n:
            at = 0
        while pending and pending[0][1] < at + n and at < pending[0][1] + pending[0][2]:
            finish()  # the oldest event still writes where this one will
        pending.append((server.submit_raw(xp, yp, lp, ep, n, c0 + 4 * at, s0 + at), at, n))
        at += n
    while pending:
        finish()
    return lat
