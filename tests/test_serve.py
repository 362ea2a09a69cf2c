"""Continuous-batching server: scheduling on CPU with a fake backend, and on
the GPU each served result against the oracle's clustering of the event
alone."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

from paper_2001_09761_gb300 import gen
from paper_2001_09761_gb300.serve import BYTES_PER_HIT, Server, offered_load


class FakeBackend:
    """Stands in for the GPU: 'clusters' an event as cid = int(x) and records
    what the scheduler did.  Each batch takes `delay` seconds."""

    def __init__(self, capacity=1000, n_regions=3, delay=0.002):
        self.capacity, self.n_regions, self.delay = capacity, n_regions, delay
        self.staged = {}
        self.launched = []
        self.lock = threading.Lock()

    def stage(self, region, offset, req):
        self.staged[(region, offset)] = np.asarray(req.x)

    def launch(self, region, offsets):
        out = np.concatenate([self.staged[(region, a)] for a in offsets[:-1]]) \
            if len(offsets) > 1 else np.zeros(0)
        self.launched.append(list(offsets))
        return {"t": time.perf_counter() + self.delay, "region": region,
                "cid": out.astype(np.int32), "seed": (out > 0).astype(np.uint8)}

    def ready(self, h):
        return time.perf_counter() >= h["t"]

    def fetch(self, region, h, k, a, b):
        return h["cid"][a:b].copy(), h["seed"][a:b].copy()

    def check(self):
        return 0

    def close(self):
        pass


def _ev(rng, n, tag):
    return (np.full(n, tag, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32),
            np.ones(n, np.float32))


def test_every_request_gets_its_own_result():
    be = FakeBackend()
    srv = Server(be)
    rng = np.random.default_rng(0)
    sizes = rng.integers(1, 400, 200)
    futs = [srv.submit(*_ev(rng, int(n), k)) for k, n in enumerate(sizes)]
    for k, (f, n) in enumerate(zip(futs, sizes)):
        cid, seed = f.result(timeout=30)
        assert cid.shape == (n,) and (cid == k).all()
    srv.close()
    st = srv.stats()
    assert st["events"] == 200 and st["hits"] == int(sizes.sum())
    assert st["mean_events_per_batch"] > 1  # requests were batched together
    for offs in be.launched:
        assert offs[-1] <= be.capacity


def test_memory_budget_gates_admission():
    be = FakeBackend(capacity=10_000, delay=0.003)
    budget = 600 * BYTES_PER_HIT
    srv = Server(be, mem_budget_bytes=budget)
    peak = []
    orig = srv._admit

    def spy():
        r = orig()
        peak.append(srv.used)
        return r
    srv._admit = spy
    rng = np.random.default_rng(1)
    futs = [srv.submit(*_ev(rng, 250, k)) for k in range(40)]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    assert max(peak) <= budget
    assert all(offs[-1] <= 500 for offs in be.launched)  # at most 2 events fit the budget


def test_oversized_request_is_rejected():
    srv = Server(FakeBackend(capacity=100))
    f = srv.submit(*_ev(None, 101, 0))
    with pytest.raises(ValueError):
        f.result(timeout=5)
    ok = srv.submit(*_ev(None, 100, 3))
    assert (ok.result(timeout=5)[0] == 3).all()
    srv.close()


def test_requests_arriving_during_a_batch_join_the_next_one():
    be = FakeBackend(delay=0.05)
    srv = Server(be, max_inflight=1)
    first = srv.submit(*_ev(None, 10, 1))
    time.sleep(0.01)  # first batch is now on the "device"
    later = [srv.submit(*_ev(None, 10, k)) for k in range(2, 8)]
    for f in [first, *later]:
        f.result(timeout=10)
    srv.close()
    assert be.launched[0] == [0, 10]
    assert len(be.launched[1]) - 1 == 6  # all six late arrivals in one batch


def test_offered_load_driver_poisson():
    srv = Server(FakeBackend(delay=0.001))
    pool = [_ev(None, n, n) for n in (5, 50, 200)]
    futs = offered_load(srv, pool, rate_events_per_s=2000.0, n_requests=100, seed=3)
    srv.close()
    assert all(f.done() for f in futs)
    st = srv.stats()
    assert st["events"] == 100 and st["p99_ms"] >= st["p50_ms"] > 0


@pytest.mark.gpu
def test_served_results_equal_events_alone():
    """Served events (batched with others of every size) against the oracle,
    element by element: each result is the one the event has alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2001_09761_gb300.serve import GpuBackend
    rng = np.random.default_rng(5)
    sizes = [int(v) for v in np.exp(rng.uniform(np.log(1e3), np.log(4e5), 30))] + [1, 0, 7]
    events = [gen.make_event(n, 100, 3000 + k, "blobs") for k, n in enumerate(sizes)]
    be = GpuBackend(device=0, extent=gen.EXTENT, max_layers=100, params=gen.PARAMS_BLOBS,
                    region_hits=1_500_000, n_regions=3)
    srv = Server(be, max_events_per_batch=16)
    futs = [srv.submit(ev.x, ev.y, ev.layer, ev.energy) for ev in events]
    results = [f.result(timeout=120) for f in futs]
    srv.close()
    assert srv.stats()["batches"] < len(events)  # events really were batched
    for ev, (cid, seed) in zip(events, results):
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
        assert np.array_equal(cid.cpu().numpy(), ref["cluster_id"])
        assert np.array_equal(seed.cpu().numpy(), ref["is_seed"])


@pytest.mark.gpu
def test_served_stream_up_to_2M_hit_events():
    """The served stream's size range (log-uniform 10k-2M hits, 100 layers,
    one event of exactly 2M) through the benchmark's server configuration
    (16M-hit regions, three of them, results on the host), with Poisson
    arrivals; every result against the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2001_09761_gb300.serve import GpuBackend
    sizes = [int(v) for v in gen.batch_sizes(11, 1e4, 2e6, seed=7)] + [2_000_000]
    events = [gen.make_event(n, 100, 6000 + k, "blobs") for k, n in enumerate(sizes)]
    pool = [(ev.x, ev.y, ev.layer, ev.energy) for ev in events]
    be = GpuBackend(device=0, extent=gen.EXTENT, max_layers=100, params=gen.PARAMS_BLOBS,
                    region_hits=16_000_000, n_regions=3, host_results=True)
    srv = Server(be)
    rng = np.random.default_rng(11)
    futs = []
    for k in rng.permutation(len(pool)).tolist() + [len(pool) - 1]:
        futs.append((k, srv.submit(*pool[k])))
        time.sleep(float(rng.exponential(0.002)))
    results = [(k, f.result(timeout=300)) for k, f in futs]
    srv.close()
    refs = {}
    for k, (cid, seed) in results:
        if k not in refs:
            refs[k] = oracle.run_event(events[k], gen.PARAMS_BLOBS, 100)
        assert np.array_equal(np.asarray(cid), refs[k]["cluster_id"]), f"event {k}"
        assert np.array_equal(np.asarray(seed), refs[k]["is_seed"]), f"event {k}"
    assert max(sizes) == 2_000_000
