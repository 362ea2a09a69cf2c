"""Continuous-batching server.

On the CPU: the library's scheduler (paper_2001_09761_gb300/csrc/
serve_core.cpp, the same code the GPU server runs) over a fake device
(tests/serve_fake.cpp, built here with g++): every request gets its own
result, requests are batched, the memory budget gates admission, oversized
requests are rejected, late arrivals join the next batch, nothing is lost at
shutdown.  On the GPU: every served result (to host or device arrays) against
the oracle's clustering of the event alone.
"""
from __future__ import annotations

import ctypes
import subprocess
import threading
import time
from pathlib import Path

import numpy as np
import pytest

from paper_2001_09761_gb300 import gen

ROOT = Path(__file__).resolve().parents[1]
BPH = 141  # bytes per admitted hit against a budget (as the library's server)


@pytest.fixture(scope="module")
def fake(tmp_path_factory):
    out = tmp_path_factory.mktemp("servefake") / "libservefake.so"
    csrc = ROOT / "paper_2001_09761_gb300" / "csrc"
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                    str(ROOT / "tests" / "serve_fake.cpp"), str(csrc / "serve_core.cpp"),
                    f"-I{ROOT / 'include'}", f"-I{csrc}", "-o", str(out)], check=True)
    lib = ctypes.CDLL(str(out))
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.fake_server_create.argtypes = [I64, I32, D, I32, I32, I64, I64]
    lib.fake_server_create.restype = P
    lib.fake_server_submit.argtypes = [P, P, I64, P, P, ctypes.POINTER(I64)]
    lib.fake_server_wait.argtypes = [P, I64, D, ctypes.POINTER(I32), ctypes.POINTER(D)]
    lib.fake_server_launched.argtypes = [P, P, I64]
    lib.fake_server_launched.restype = I64
    lib.fake_server_max_staged.argtypes = [P]
    lib.fake_server_max_staged.restype = I64
    lib.fake_server_stats.argtypes = [P, P]
    lib.fake_server_stop.argtypes = [P]
    lib.fake_server_destroy.argtypes = [P]
    return lib


class FakeServer:
    def __init__(self, lib, capacity=1000, n_regions=3, delay=0.002, max_events=512,
                 max_inflight=2, budget=0):
        self.lib = lib
        self.h = lib.fake_server_create(capacity, n_regions, delay, max_events, max_inflight,
                                        budget, BPH)
        self.keep = {}

    def submit(self, n, tag):
        x = np.full(n, tag, np.float32)
        cid, seed = np.full(n, -9, np.int32), np.zeros(n, np.uint8)
        t = ctypes.c_int64(0)
        rc = self.lib.fake_server_submit(self.h, x.ctypes.data, n, cid.ctypes.data,
                                         seed.ctypes.data, ctypes.byref(t))
        if rc == 0:
            self.keep[t.value] = (x, cid, seed)
        return rc, t.value

    def wait(self, t, timeout=30.0):
        st, lat = ctypes.c_int32(0), ctypes.c_double(0.0)
        rc = self.lib.fake_server_wait(self.h, t, timeout, ctypes.byref(st), ctypes.byref(lat))
        return rc, st.value, self.keep[t][1], lat.value

    def batches(self):
        buf = np.zeros(1 << 16, np.int64)
        n = self.lib.fake_server_launched(self.h, buf.ctypes.data, buf.size)
        out, cur = [], []
        for v in buf[:n].tolist():
            if v < 0:
                out.append(cur)
                cur = []
            else:
                cur.append(v)
        return out

    def stats(self):
        out = np.zeros(6)
        self.lib.fake_server_stats(self.h, out.ctypes.data)
        return dict(events=int(out[0]), hits=int(out[1]), batches=int(out[2]),
                    rejected=int(out[3]), span=out[4], mean_events=out[5])

    def close(self):
        self.lib.fake_server_destroy(self.h)


def test_every_request_gets_its_own_result(fake):
    srv = FakeServer(fake)
    sizes = np.random.default_rng(0).integers(1, 400, 200)
    tickets = [srv.submit(int(n), k)[1] for k, n in enumerate(sizes)]
    for k, (t, n) in enumerate(zip(tickets, sizes)):
        rc, st, cid, lat = srv.wait(t)
        assert rc == 0 and st == 0 and lat > 0
        assert cid.shape == (n,) and (cid == k).all()
    st, batches = srv.stats(), srv.batches()
    srv.close()
    assert st["events"] == 200 and st["hits"] == int(sizes.sum())
    assert st["mean_events"] > 1  # requests were batched together
    for offs in batches:
        assert offs[-1] <= 1000


def test_memory_budget_gates_admission(fake):
    budget = 600 * BPH
    srv = FakeServer(fake, capacity=10_000, delay=0.003, budget=budget)
    tickets = [srv.submit(250, k)[1] for k in range(40)]
    for k, t in enumerate(tickets):
        assert (srv.wait(t)[2] == k).all()
    peak = fake.fake_server_max_staged(srv.h)
    batches = srv.batches()
    srv.close()
    assert peak <= 600  # hits held at once never passed the budget
    assert all(offs[-1] <= 500 for offs in batches)  # at most 2 events fit the budget


def test_oversized_request_is_rejected(fake):
    srv = FakeServer(fake, capacity=100)
    rc, _ = srv.submit(101, 0)
    assert rc == 1  # CLUE_ERR_ARG, nothing queued
    rc, t = srv.submit(100, 3)
    assert rc == 0 and (srv.wait(t)[2] == 3).all()
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_requests_arriving_during_a_batch_join_the_next_one(fake):
    srv = FakeServer(fake, delay=0.05, max_inflight=1)
    first = srv.submit(10, 1)[1]
    time.sleep(0.01)  # the first batch is now on the "device"
    later = [srv.submit(10, k)[1] for k in range(2, 8)]
    for t in [first, *later]:
        srv.wait(t)
    b = srv.batches()
    srv.close()
    assert b[0] == [0, 10]
    assert len(b[1]) - 1 == 6  # all six late arrivals in one batch


def test_wait_times_out_then_completes(fake):
    srv = FakeServer(fake, delay=0.2)
    t = srv.submit(5, 4)[1]
    rc, *_ = srv.wait(t, timeout=0.01)
    assert rc == 5  # CLUE_ERR_TIMEOUT: not done yet, the ticket stays
    rc, st, cid, _ = srv.wait(t, timeout=10.0)
    assert rc == 0 and (cid == 4).all()
    srv.close()


def test_shutdown_completes_everything_queued(fake):
    srv = FakeServer(fake, delay=0.005, capacity=50)
    tickets = [srv.submit(40, k)[1] for k in range(30)]  # one event per batch
    fake.fake_server_stop(srv.h)  # returns once all 30 are done
    assert srv.stats()["events"] == 30
    for k, t in enumerate(tickets):
        assert (srv.wait(t, timeout=0.0)[2] == k).all()
    rc, _ = srv.submit(1, 0)
    assert rc == 6  # CLUE_ERR_STATE after stop
    srv.close()


def test_many_submitting_threads(fake):
    srv = FakeServer(fake, delay=0.001, capacity=5000)
    results, lock = {}, threading.Lock()

    def client(c):
        for k in range(50):
            tag = c * 1000 + k
            t = srv.submit(1 + (k * 7) % 90, tag)[1]
            with lock:
                results[tag] = t
    th = [threading.Thread(target=client, args=(c,)) for c in range(6)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for tag, t in results.items():
        assert (srv.wait(t)[2] == tag).all()
    st = srv.stats()
    srv.close()
    assert st["events"] == 300


@pytest.mark.gpu
def test_served_results_equal_events_alone():
    """Served events (batched with others of every size) against the oracle,
    element by element: each result is the one the event has alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2001_09761_gb300 import build
    from paper_2001_09761_gb300.serve import Server
    build.build()
    rng = np.random.default_rng(5)
    sizes = [int(v) for v in np.exp(rng.uniform(np.log(1e3), np.log(4e5), 30))] + [1, 0, 7]
    events = [gen.make_event(n, 100, 3000 + k, "blobs") for k, n in enumerate(sizes)]
    srv = Server(device=0, extent=gen.EXTENT, max_layers=100, params=gen.PARAMS_BLOBS,
                 region_hits=1_500_000, n_regions=3, max_events_per_batch=16)
    # results to pinned host arrays for half the events, to device tensors
    # (the default) for the other half
    outs = [(torch.empty(ev.n, dtype=torch.int32, pin_memory=True),
             torch.empty(ev.n, dtype=torch.uint8, pin_memory=True)) if k % 2 else None
            for k, ev in enumerate(events)]
    tickets = [srv.submit(ev.x, ev.y, ev.layer, ev.energy, out=o)
               for ev, o in zip(events, outs)]
    results = [t.result(timeout=120) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["batches"] < len(events)  # events really were batched
    for k, (ev, (cid, seed)) in enumerate(zip(events, results)):
        assert cid.is_cuda == (k % 2 == 0)
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
        assert np.array_equal(cid.cpu().numpy(), ref["cluster_id"])
        assert np.array_equal(seed.cpu().numpy(), ref["is_seed"])


@pytest.mark.gpu
def test_served_stream_up_to_2M_hit_events():
    """The served stream's size range (log-uniform 10k-2M hits, 100 layers,
    one event of exactly 2M) through the benchmark's server configuration
    (16M-hit regions, three of them) with Poisson arrivals from pinned host
    memory; every result against the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2001_09761_gb300 import build
    from paper_2001_09761_gb300.serve import Server
    build.build()
    sizes = [int(v) for v in gen.batch_sizes(11, 1e4, 2e6, seed=7)] + [2_000_000]
    events = [gen.make_event(n, 100, 6000 + k, "blobs") for k, n in enumerate(sizes)]
    pin = lambda a: torch.from_numpy(a).pin_memory()
    pool = [(pin(ev.x), pin(ev.y), pin(ev.layer), pin(ev.energy)) for ev in events]
    srv = Server(device=0, extent=gen.EXTENT, max_layers=100, params=gen.PARAMS_BLOBS,
                 region_hits=16_000_000, n_regions=3)
    rng = np.random.default_rng(11)
    tickets = []
    for k in rng.permutation(len(pool)).tolist() + [len(pool) - 1]:
        tickets.append((k, srv.submit(*pool[k])))
        time.sleep(float(rng.exponential(0.002)))
    results = [(k, t.result(timeout=300)) for k, t in tickets]
    srv.close()
    refs = {}
    for k, (cid, seed) in results:
        if k not in refs:
            refs[k] = oracle.run_event(events[k], gen.PARAMS_BLOBS, 100)
        assert np.array_equal(cid.cpu().numpy(), refs[k]["cluster_id"]), f"event {k}"
        assert np.array_equal(seed.cpu().numpy(), refs[k]["is_seed"]), f"event {k}"
    assert max(sizes) == 2_000_000


@pytest.mark.gpu
def test_served_event_with_bad_input_fails_alone_later_events_succeed():
    """A served event whose layer is out of range fails with CLUE_ERR_INPUT
    (raised on the device, read back per batch); a later event is fine."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import build, clue
    from paper_2001_09761_gb300.serve import Server
    build.build()
    srv = Server(device=0, extent=gen.EXTENT, max_layers=10, params=gen.PARAMS_BLOBS,
                 region_hits=100_000, n_regions=2, max_inflight=1)
    bad = gen.make_event(2000, 10, 1, "blobs")
    layer = bad.layer.copy()
    layer[5] = 99
    t = srv.submit(bad.x, bad.y, layer, bad.energy)
    with pytest.raises(clue.ClueError) as ei:
        t.result(timeout=60)
    assert ei.value.code == clue.CLUE_ERR_INPUT
    good = gen.make_event(3000, 10, 2, "blobs")
    cid, _ = srv.submit(good.x, good.y, good.layer, good.energy).result(timeout=60)
    srv.close()
    cid = cid.cpu().numpy()
    assert (cid >= -1).all() and (cid >= 0).any()


@pytest.mark.gpu
def test_offered_load_driver_on_gpu():
    """The benchmark's load driver: Poisson submissions of pinned pool events
    whose results go to a reused ring of device buffers (small regions, so the
    ring wraps many times); every request completes and the counters agree."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import build
    from paper_2001_09761_gb300.serve import Server, offered_load
    build.build()
    pin = lambda a: torch.from_numpy(a).pin_memory()
    pool = []
    for k, n in enumerate([3000, 20000, 70000, 150000]):
        ev = gen.make_event(n, 100, 40 + k, "blobs")
        pool.append((pin(ev.x), pin(ev.y), pin(ev.layer), pin(ev.energy)))
    srv = Server(device=0, extent=gen.EXTENT, max_layers=100, params=gen.PARAMS_BLOBS,
                 region_hits=400_000, n_regions=3)
    lat = offered_load(srv, pool, rate_events_per_s=20_000.0, n_requests=400, seed=2)
    st = srv.stats()
    srv.close()
    assert len(lat) == 400 and min(lat) > 0
    assert st["events"] == 400 and st["batches"] < 400
    assert st["p99_ms"] >= st["p50_ms"] > 0
