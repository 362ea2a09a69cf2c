"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerance: 0.  Cluster ids, seed flags and nearest-higher indices are integer
outputs and must match exactly; rho (the exact sum rounded once) and delta
(a fixed fp32 operation order, no fused multiply-add) are compared bit for
bit.
"""
from __future__ import annotations

import json
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2001_09761_gb300 import gen

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def clue_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import build, clue
    build.build()
    clue.load()
    return clue


def _cl(clue_mod, extent=(-250.0, 250.0, -250.0, 250.0), layers=128, **kw):
    return clue_mod.Clusterer(device=0, extent=extent, max_layers=layers, **kw)


def _gpu_all(cl, ev, params):
    cid, seed = cl.run(ev.x, ev.y, ev.layer, ev.energy, params)
    rho, delta, nh = cl.intermediates()
    cl.sync()
    return dict(cluster_id=cid.cpu().numpy(), is_seed=seed.cpu().numpy(),
                rho=rho.cpu().numpy(), delta=delta.cpu().numpy(), nh=nh.cpu().numpy())


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def assert_parity(g, ref, keys=("cluster_id", "is_seed", "rho", "delta", "nh")):
    for k in keys:
        a, b = g[k], ref[k]
        if a.dtype.kind == "f":
            bad = np.nonzero(_bits(a) != _bits(b))[0]
        else:
            bad = np.nonzero(a != b.astype(a.dtype))[0]
        assert bad.size == 0, f"{k}: {bad.size} mismatches, first {bad[:8]}: {a[bad[:8]]} vs {b[bad[:8]]}"


class Ev:
    def __init__(self, x, y, layer, energy):
        self.x = np.asarray(x, np.float32)
        self.y = np.asarray(y, np.float32)
        self.layer = np.asarray(layer, np.int32)
        self.energy = np.asarray(energy, np.float32)
        self.n = self.x.shape[0]


@pytest.mark.parametrize("name", sorted(p.stem for p in GOLDEN.glob("*.json")))
def test_golden_fixtures(clue_mod, name):
    d = json.loads((GOLDEN / f"{name}.json").read_text())
    cl = _cl(clue_mod, d["extent"], d["n_layers"])
    g = _gpu_all(cl, Ev(d["x"], d["y"], d["layer"], d["w"]), d["params"])
    exp = d["expected"]
    assert g["cluster_id"].tolist() == exp["cluster_id"]
    assert g["is_seed"].tolist() == exp["is_seed"]
    assert g["nh"].tolist() == exp["nh"]
    assert _bits(g["rho"]).tolist() == _bits(np.array(exp["rho"], np.float32)).tolist()
    d2 = np.array([np.inf if v == "inf" else v for v in exp["delta2"]], np.float32)
    assert _bits(g["delta"]).tolist() == _bits(np.sqrt(d2)).tolist()


CASES = [
    ("blobs", 2400, 3, gen.PARAMS_BLOBS, 0, (-40.0, 40.0, -40.0, 40.0)),
    ("blobs", 1500, 1, (2.0, 1.0, 1.0, 3.0), 1, (-40.0, 40.0, -40.0, 40.0)),
    ("irregular", 20000, 2, gen.PARAMS_IRREGULAR, 2, (-60.0, 60.0, -60.0, 60.0)),
    ("paper", 20000, 4, gen.PARAMS_PAPER, 3, (-100.0, 100.0, -100.0, 100.0)),
    ("uniform", 5000, 1, (6.0, 3.0, 4.0, 8.0), 4, (-40.0, 40.0, -40.0, 40.0)),
    ("blobs", 3000, 2, (2.0, 2.0, 6.0, 1.0), 5, (-40.0, 40.0, -40.0, 40.0)),
    ("blobs", 10_000, 10, gen.PARAMS_BLOBS, 0, gen.EXTENT),
    ("irregular", 50_000, 5, gen.PARAMS_IRREGULAR, 7, gen.EXTENT),
]


@pytest.mark.parametrize("expand", [0, 1], ids=["frontier", "chase"])
@pytest.mark.parametrize("kind,n,L,params,seed,ext", CASES)
def test_parity_vs_oracle(clue_mod, kind, n, L, params, seed, ext, expand):
    ev = gen.make_event(n, L, seed, kind, extent=ext)
    cl = _cl(clue_mod, ext, L, expand=expand)
    g = _gpu_all(cl, ev, params)
    ref = oracle.run_event(ev, params, L, extent=ext)
    assert_parity(g, ref)


@pytest.mark.parametrize("density", ["FUSED", "SEPARATE"])
@pytest.mark.parametrize("kind,n,L,params,seed,ext", CASES)
def test_parity_forced_density_kernels(clue_mod, kind, n, L, params, seed, ext, density):
    """Both density forms, forced on every case (the default picks one per
    run): the fused kernel, whose dense or wide tiles go to the list-driven
    nh kernel, and the separate rho and nh kernels give the oracle's bytes."""
    ev = gen.make_event(n, L, seed, kind, extent=ext)
    cl = _cl(clue_mod, ext, L, density=getattr(clue_mod, f"CLUE_DENSITY_{density}"))
    assert_parity(_gpu_all(cl, ev, params), oracle.run_event(ev, params, L, extent=ext))


@pytest.mark.parametrize("kind,n,L,seed,ext", [
    ("irregular", 50_000, 5, 7, gen.EXTENT),
    ("blobs", 20_000, 2, 8, (-40.0, 40.0, -40.0, 40.0)),
    ("uniform", 30_000, 1, 9, (-60.0, 60.0, -60.0, 60.0)),
])
def test_fused_kernel_at_the_smallest_staging(clue_mod, kind, n, L, seed, ext):
    """The fused kernel forced at the smallest staging capacity (1792 records),
    so that tiles take every path it has: the halo's densities from the
    widened staging where their windows fit it, by walks in global memory
    where they do not, and the list-driven nh kernel for bands past it."""
    ev = gen.make_event(n, L, seed, kind, extent=ext)
    params = gen.PARAMS_IRREGULAR if kind == "irregular" else gen.PARAMS_BLOBS
    cl = _cl(clue_mod, ext, L, density=clue_mod.CLUE_DENSITY_FUSED)
    cl.tuning = cl.tuning.replace("band 0", "band 1792")
    assert "band 1792" in cl.tuning
    assert_parity(_gpu_all(cl, ev, params), oracle.run_event(ev, params, L, extent=ext))


@pytest.mark.parametrize("per_layer,block", [(8000, 128), (12600, 128), (12600, 64),
                                             (22000, 256)])
def test_fused_kernel_halo_windows_kept_and_looked_up(clue_mod, per_layer, block):
    """The fused kernel's halo densities with every number of halo hits per
    thread.  Bins of 8 cm on the 500 cm extent give 63 bins per row, so a
    layer of h hits has about h / 63 per grid row, and a 1024-hit tile's band
    holds about two rows' worth of halo hits (its first and last rows'
    neighbours): about 250, 400 and 700 for 8000, 12600 and 22000 hits per
    layer.  So tiles have their halo within the three windows per thread that
    the kernel keeps from its sizing pass (8000 hits at 128 threads, most
    tiles at 22000 hits and 256 threads), past them (a fourth window looked up
    again: over half the tiles at 12600 hits and 128 threads, some at 22000),
    past the four halo hits a thread takes (12600 hits at 64 threads: the
    halo's densities by walks in global memory), and a widened band past the
    staging (some tiles at 22000).  The staging capacity is raised to 2560
    records so most widened bands fit."""
    L = 3
    ev = gen.make_event(per_layer * L, L, 21, "blobs")
    cl = _cl(clue_mod, gen.EXTENT, L, bin_size=8.0, block_size=block,
             density=clue_mod.CLUE_DENSITY_FUSED)
    cl.tuning = cl.tuning.replace("band 0", "band 2560")
    assert "band 2560" in cl.tuning
    assert_parity(_gpu_all(cl, ev, gen.PARAMS_BLOBS),
                  oracle.run_event(ev, gen.PARAMS_BLOBS, L))


def test_parity_scaling_event_full_size(clue_mod):
    """100 layers x 10k hits (1M hits), the largest single event of the
    scaling sweep, compared in full."""
    ev = gen.scaling_event(10_000, 0)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    g = _gpu_all(cl, ev, gen.PARAMS_BLOBS)
    ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
    assert_parity(g, ref)


def test_full_batch_in_the_bench_configuration(clue_mod):
    """The benchmark's workload at full size (256 events, 65.2M hits) in its
    launch configuration: autotuned bins, then a replayed CUDA graph.  Six
    events spread over the size range are checked in full against the oracle
    (every output, intermediates included); every event of the batch is
    checked for the numbering of Algorithm 3 (seed ids 0..k-1 in ascending
    seed index, every other id in [-1, k))."""
    import torch
    evs = gen.uneven_batch()
    x, y, l, e, offs = gen.concat(evs)
    n = int(offs[-1])
    d = lambda a: torch.from_numpy(a).cuda()
    tx, ty, tl, te = d(x), d(y), d(l), d(e)
    cid = torch.empty(n, dtype=torch.int32, device="cuda")
    seed = torch.empty(n, dtype=torch.uint8, device="cuda")
    cl = _cl(clue_mod, gen.EXTENT, 100)
    cl.autotune(tx, ty, tl, te, offs, gen.PARAMS_BLOBS, reps=1)
    for _ in range(3):  # direct, captured, replayed
        cl.run_batch(tx, ty, tl, te, offs, gen.PARAMS_BLOBS, out=(cid, seed))
    rho, delta, nh = cl.intermediates()
    cl.sync()
    c, sd = cid.cpu().numpy(), seed.cpu().numpy()
    order = np.argsort([ev.n for ev in evs])
    for i in order[[0, 51, 102, 153, 204, 255]]:
        a, z = int(offs[i]), int(offs[i + 1])
        g = dict(cluster_id=c[a:z], is_seed=sd[a:z], rho=rho[a:z].cpu().numpy(),
                 delta=delta[a:z].cpu().numpy(), nh=nh[a:z].cpu().numpy())
        assert_parity(g, oracle.run_event(evs[i], gen.PARAMS_BLOBS, 100))
    for i in range(len(evs)):
        a, z = int(offs[i]), int(offs[i + 1])
        ci, si = c[a:z], sd[a:z].astype(bool)
        k = int(si.sum())
        assert np.array_equal(ci[si], np.arange(k))
        assert np.all((ci[~si] >= -1) & (ci[~si] < k))


@pytest.mark.parametrize("bin_size,block", [(2.0, 128), (3.0, 256), (4.5, 64), (9.0, 256),
                                             (25.0, 128)])
def test_bin_size_and_block_do_not_change_results(clue_mod, bin_size, block):
    ext = (-80.0, 80.0, -80.0, 80.0)
    ev = gen.make_event(30_000, 3, 31, "irregular", extent=ext)
    ref = oracle.run_event(ev, gen.PARAMS_IRREGULAR, 3, extent=ext)
    cl = _cl(clue_mod, ext, 3, bin_size=bin_size, block_size=block)
    assert_parity(_gpu_all(cl, ev, gen.PARAMS_IRREGULAR), ref)


@pytest.mark.parametrize("sizes", [[0, 1, 5000, 20000, 0, 1234, 40000, 7], [3000, 0, 0, 12000, 0]],
                         ids=["mixed", "empty_last"])
def test_batch_equals_events_alone(clue_mod, sizes):
    """Every event of a batch (empty ones included, also as the last event,
    where the grid fill's run table ends) clusters as it does alone."""
    evs = [gen.make_event(n, 100, 500 + i, "blobs") for i, n in enumerate(sizes)]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    rho, delta, nh = cl.intermediates()
    cl.sync()
    cid, seed, rho, nh = (t.cpu().numpy() for t in (cid, seed, rho, nh))
    for i, ev in enumerate(evs):
        a, b = offs[i], offs[i + 1]
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
        assert np.array_equal(cid[a:b], ref["cluster_id"]), i
        assert np.array_equal(seed[a:b], ref["is_seed"]), i
        assert np.array_equal(_bits(rho[a:b]), _bits(ref["rho"])), i
        assert np.array_equal(nh[a:b], ref["nh"]), i


def test_repeated_runs_are_identical_and_graph_replay(clue_mod):
    ev = gen.make_event(60_000, 20, 9, "blobs")
    cl = _cl(clue_mod, gen.EXTENT, 20, use_graphs=True)
    outs = []
    for _ in range(6):  # first direct, second captured, the rest replayed
        cid, seed = cl.run(ev.x, ev.y, ev.layer, ev.energy, gen.PARAMS_BLOBS)
        cl.sync()
        outs.append((cid.cpu().numpy().copy(), seed.cpu().numpy().copy()))
    ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 20)
    for c, s in outs:
        assert np.array_equal(c, ref["cluster_id"]) and np.array_equal(s, ref["is_seed"])


def test_profiled_graph_replay_keeps_each_runs_times(clue_mod):
    """With profiling on, captured graphs stamp a ring of event sets, so the
    times of the last 4 runs stay readable while later runs are queued, and
    profiling changes no result."""
    import torch
    evs = [gen.make_event(n, 100, 60 + i, "blobs") for i, n in enumerate((30_000, 70_000))]
    x, y, l, e, offs = gen.concat(evs)
    d = lambda a: torch.from_numpy(a).cuda()
    tx, ty, tl, te = d(x), d(y), d(l), d(e)
    n = int(offs[-1])
    cid = torch.empty(n, dtype=torch.int32, device="cuda")
    seed = torch.empty(n, dtype=torch.uint8, device="cuda")
    cl = _cl(clue_mod, gen.EXTENT, 100, use_graphs=True)
    cl.set_profiling(True)
    for r in range(7):  # direct, captured, then replays through all four sets
        cl.run_batch(tx, ty, tl, te, offs, gen.PARAMS_BLOBS, out=(cid, seed))
        if r >= 1:
            prev = cl.kernel_times(back=1)  # read while run r is queued
            assert {"fill_cells", "density", "nh_rest", "assign"} <= set(prev)
    times = [cl.kernel_times(back=k) for k in range(4)]
    for t in times:
        assert set(t) == set(times[0]) and all(v >= 0 for v in t.values())
    with pytest.raises(clue_mod.ClueError):
        cl.kernel_times(back=4)
    cl.sync()
    c = cid.cpu().numpy()
    for i, ev in enumerate(evs):
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
        assert np.array_equal(c[offs[i]:offs[i + 1]], ref["cluster_id"])


@pytest.mark.parametrize("chi,s", [(0, 0.0), (1, 1.0), (2, 0.8)])
def test_exact_rho_with_adversarial_weights(clue_mod, chi, s):
    """Reading R4 on the GPU: weights over 1e-38..1e30, both signs,
    subnormals and zeros, so many windows fail the fast path's exactness
    proof and take the integer accumulator; every output is bit-exact, for
    the flat, Gaussian and exponential kernels."""
    from exactsum import adversarial_weights
    ev = gen.make_event(30_000, 5, 77, "blobs")
    w = adversarial_weights(np.random.default_rng(5), ev.n)
    cl = _cl(clue_mod, gen.EXTENT, 5, chi=chi, chi_param=s)
    ev2 = gen.Event(ev.x, ev.y, ev.layer, w)
    assert_parity(_gpu_all(cl, ev2, gen.PARAMS_BLOBS),
                  oracle.run(ev.x, ev.y, ev.layer, w, gen.PARAMS_BLOBS, 5, chi=chi,
                             chi_param=s))


@pytest.mark.parametrize("span", [15, 36, 37, 38, 39])
def test_fixed_point_rho_at_its_bounds(clue_mod, span):
    """The flat kernel sums an event's weights in 64-bit fixed point when
    24 + (exponent span) + bitlen(window candidates) <= 63.  Weights of both
    signs span `span` binary orders (both ends present), in dense blobs so
    windows hold dozens of candidates: span 15 takes the fixed point
    everywhere, 36-38 leave it only a few candidate bits (most windows fall
    back to the integer accumulator), 39 leaves the event on TwoSum.  Every
    output is bit-exact against the oracle."""
    ev = gen.make_event(20_000, 4, 78, "blobs")
    rng = np.random.default_rng(span)
    e = rng.integers(0, span + 1, ev.n)
    e[:2] = (0, span)
    w = np.ldexp(1.0 + rng.integers(0, 1 << 23, ev.n) / float(1 << 23), e - 20)
    w = (w * np.where(rng.random(ev.n) < 0.2, -1.0, 1.0)).astype(np.float32)
    cl = _cl(clue_mod, gen.EXTENT, 4)
    ev2 = gen.Event(ev.x, ev.y, ev.layer, w)
    assert_parity(_gpu_all(cl, ev2, gen.PARAMS_BLOBS),
                  oracle.run(ev.x, ev.y, ev.layer, w, gen.PARAMS_BLOBS, 4))


def test_weight_ranges_per_event_in_one_batch(clue_mod):
    """The rho arithmetic is chosen per event from its weights: a normal
    event (fixed point), one whose weights are all zero (no range: TwoSum),
    one with a single nonzero weight, and one spanning 60 binary orders
    (TwoSum), in one batch; every event matches the oracle bit for bit."""
    evs = [gen.make_event(n, 10, 880 + i, "blobs") for i, n in enumerate([6000, 5000, 4000, 7000])]
    rng = np.random.default_rng(88)
    ws = [evs[0].energy,
          np.zeros(evs[1].n, np.float32),
          np.where(np.arange(evs[2].n) == 17, 3.5, 0.0).astype(np.float32),
          np.ldexp(1.0, rng.integers(-30, 31, evs[3].n)).astype(np.float32)]
    evs = [gen.Event(ev.x, ev.y, ev.layer, w) for ev, w in zip(evs, ws)]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 10)
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    rho, delta, nh = cl.intermediates()
    cl.sync()
    cid, seed, rho, nh = (t.cpu().numpy() for t in (cid, seed, rho, nh))
    for i, ev in enumerate(evs):
        a, b = offs[i], offs[i + 1]
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 10)
        assert np.array_equal(_bits(rho[a:b]), _bits(ref["rho"])), i
        assert np.array_equal(cid[a:b], ref["cluster_id"]), i
        assert np.array_equal(seed[a:b], ref["is_seed"]), i
        assert np.array_equal(nh[a:b], ref["nh"]), i


def test_exact_rho_of_coincident_sets(clue_mod):
    """Hits at one point are mutual neighbours, so rho is the rounded exact
    sum of the whole set: rounding up, to even, to a subnormal, to zero by
    cancellation, to infinity and across a power of two, against the oracle."""
    from exactsum import adversarial_weights
    rng = np.random.default_rng(11)
    sets = [adversarial_weights(rng, int(rng.integers(1, 60))) for _ in range(40)]
    sets += [np.array(v, np.float32) for v in (
        [1.0, 2.0 ** -24, 2.0 ** -25], [1.0, 2.0 ** -24], [1.0 + 2.0 ** -23, 2.0 ** -24],
        [2.0 ** -149] * 5, [3.0e38, 3.0e38, -1.0], [1e30, -1e30, 2.0 ** -140], [5.0, -5.0],
        [1.0, 1.0 - 2.0 ** -24, 2.0 ** -25])]
    cl = _cl(clue_mod, (-1.0, 1.0, -1.0, 1.0), 1)
    for w in sets:
        z = np.zeros(w.size, np.float32)
        ev = gen.Event(z, z, np.zeros(w.size, np.int32), w)
        g = _gpu_all(cl, ev, (1.0, 0.0, 1.0, 1.0))
        ref = oracle.run(z, z, ev.layer, w, (1.0, 0.0, 1.0, 1.0), 1, (-1.0, 1.0, -1.0, 1.0))
        assert_parity(g, ref)


def test_calls_under_a_callers_capture_are_refused(clue_mod):
    """While the caller captures the context's stream into a graph of its own,
    a run is refused (CLUE_ERR_STATE) without touching the capture; outside it
    the context works as before."""
    import torch
    ev = gen.make_event(20_000, 10, 91, "blobs")
    d = lambda a: torch.from_numpy(a).cuda()
    tx, ty, tl, te = d(ev.x), d(ev.y), d(ev.layer), d(ev.energy)
    cid = torch.empty(ev.n, dtype=torch.int32, device="cuda")
    seed = torch.empty(ev.n, dtype=torch.uint8, device="cuda")
    cl = _cl(clue_mod, gen.EXTENT, 10)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cl.stream):
        rc = clue_mod.clue_run(cl.ctx, tx.data_ptr(), ty.data_ptr(), tl.data_ptr(),
                               te.data_ptr(), ev.n, *gen.PARAMS_BLOBS, cid.data_ptr(),
                               seed.data_ptr())
        cid.fill_(0)  # the caller's own captured work
    assert rc == clue_mod.CLUE_ERR_STATE
    assert "captured" in clue_mod.clue_last_message(cl.ctx)
    g.replay()
    torch.cuda.synchronize()
    assert_parity(_gpu_all(cl, ev, gen.PARAMS_BLOBS), oracle.run_event(ev, gen.PARAMS_BLOBS, 10))


def test_distinct_events_back_to_back_through_graph_templates(clue_mod):
    """Events new to the context, queued back to back with no sync between
    them, all go through the same executable graph updated per call while
    earlier launches may still run; every event's result is the oracle's."""
    import torch
    evs = [gen.make_event(n, 20, 300 + i, "blobs")
           for i, n in enumerate([3000 + 997 * i for i in range(24)])]
    x, y, l, e, offs = gen.concat(evs)
    d = lambda a: torch.from_numpy(a).cuda()
    tx, ty, tl, te = d(x), d(y), d(l), d(e)
    n = int(offs[-1])
    cid = torch.empty(n, dtype=torch.int32, device="cuda")
    seed = torch.empty(n, dtype=torch.uint8, device="cuda")
    cl = _cl(clue_mod, gen.EXTENT, 20, use_graphs=True)
    for i in range(len(evs)):
        a, z = int(offs[i]), int(offs[i + 1])
        cl.run(tx[a:z], ty[a:z], tl[a:z], te[a:z], gen.PARAMS_BLOBS, out=(cid[a:z], seed[a:z]))
    cl.sync()
    c, sd = cid.cpu().numpy(), seed.cpu().numpy()
    for i, ev in enumerate(evs):
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 20)
        a, z = int(offs[i]), int(offs[i + 1])
        assert np.array_equal(c[a:z], ref["cluster_id"]), i
        assert np.array_equal(sd[a:z], ref["is_seed"]), i


def test_host_pointer_path(clue_mod):
    evs = [gen.make_event(n, 100, 700 + i, "blobs") for i, n in enumerate([3000, 25000, 9000])]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    for _ in range(3):
        cid, seed = cl.run_batch_host(x, y, l, e, offs, gen.PARAMS_BLOBS)
        for i, ev in enumerate(evs):
            ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
            assert np.array_equal(cid[offs[i]:offs[i + 1]], ref["cluster_id"])
            assert np.array_equal(seed[offs[i]:offs[i + 1]], ref["is_seed"])


def test_host_pointer_path_pipelined_chunks(clue_mod):
    """A 10M-hit batch is split into several chunks whose copies overlap the
    clustering; the results equal the device-pointer path's."""
    evs = [gen.make_event(n, 100, 1700 + i, "blobs")
           for i, n in enumerate([900_000, 1_500_000, 2_000_000, 700_000, 2_500_000, 30_000,
                                  1_200_000, 1_300_000])]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    dcid, dseed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    cl.sync()
    dcid, dseed = dcid.cpu().numpy(), dseed.cpu().numpy()
    for _ in range(3):  # the second call replays captured graphs
        hcid, hseed = cl.run_batch_host(x, y, l, e, offs, gen.PARAMS_BLOBS)
        assert np.array_equal(hcid, dcid) and np.array_equal(hseed, dseed)
    ref = oracle.run_event(evs[5], gen.PARAMS_BLOBS, 100)
    assert np.array_equal(hcid[offs[5]:offs[6]], ref["cluster_id"])


def test_host_pointer_path_tapered_chunks(clue_mod):
    """A batch above 32M hits is cut into chunks of about an eighth of it and a
    small last one; the results equal the device-pointer path's."""
    base = [gen.make_event(n, 100, 2700 + i, "blobs")
            for i, n in enumerate([1_300_000, 700_000, 2_100_000, 40_000, 900_000])]
    evs = [base[i % len(base)] for i in range(34)]  # 34 events, about 34M hits
    x, y, l, e, offs = gen.concat(evs)
    assert offs[-1] >= 32 << 20
    cl = _cl(clue_mod, gen.EXTENT, 100)
    dcid, dseed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    cl.sync()
    dcid, dseed = dcid.cpu().numpy(), dseed.cpu().numpy()
    hcid, hseed = cl.run_batch_host(x, y, l, e, offs, gen.PARAMS_BLOBS)
    assert np.array_equal(hcid, dcid) and np.array_equal(hseed, dseed)
    ref = oracle.run_event(base[3], gen.PARAMS_BLOBS, 100)
    for i in (3, 28):  # the same small event in an early chunk and in a late one
        assert np.array_equal(hcid[offs[i]:offs[i + 1]], ref["cluster_id"])


def test_host_pointer_path_error_in_a_later_chunk(clue_mod):
    """A NaN coordinate in the second chunk of a pipelined call (the first
    event alone fills the first chunk) is reported by the call, and the
    context works afterwards."""
    sizes = [1_200_000, 500_000, 2_000_000, 2_000_000, 2_000_000, 1_000_000]
    evs = [gen.make_event(n, 100, 3700 + i, "blobs") for i, n in enumerate(sizes)]
    x, y, l, e, offs = gen.concat(evs)
    assert offs[-1] >= 8 << 20
    cl = _cl(clue_mod, gen.EXTENT, 100)
    bad = x.copy()
    bad[offs[1] + 5] = np.nan
    with pytest.raises(clue_mod.ClueError) as ei:
        cl.run_batch_host(bad, y, l, e, offs, gen.PARAMS_BLOBS)
    assert ei.value.code == clue_mod.CLUE_ERR_INPUT
    hcid, hseed = cl.run_batch_host(x, y, l, e, offs, gen.PARAMS_BLOBS)
    dcid, dseed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    cl.sync()
    assert np.array_equal(hcid, dcid.cpu().numpy()) and np.array_equal(hseed, dseed.cpu().numpy())


def test_edge_cases(clue_mod):
    cl = _cl(clue_mod, (-10.0, 10.0, -10.0, 10.0), 4)
    p = (1.0, 0.5, 1.0, 2.0)
    # empty event: no-op
    z = np.zeros(0, np.float32)
    cid, seed = cl.run(z, z, np.zeros(0, np.int32), z, p)
    cl.sync()
    assert cid.numel() == 0
    # one hit
    g = _gpu_all(cl, Ev([0.3], [0.1], [2], [1.0]), p)
    assert g["cluster_id"].tolist() == [0] and g["is_seed"].tolist() == [1]
    # hits far outside the extent fall into edge bins and still cluster right
    rng = np.random.default_rng(0)
    ev = Ev(rng.normal(0, 30, 3000), rng.normal(0, 30, 3000), rng.integers(0, 4, 3000),
            rng.exponential(1.0, 3000))
    assert_parity(_gpu_all(cl, ev, p), oracle.run_event(ev, p, 4, extent=(-10.0, 10.0, -10.0, 10.0)))


@pytest.mark.parametrize("params", [
    (2.0, 2.0, 0.0, 0.0),      # d_m = 0: no nearest-higher search
    (400.0, 2.0, 2.0, 4.0),    # d_c spans the layer: every hit neighbours every other
    (2.0, -1.0, 2.0, 4.0),     # rho_c below every density: no outlier
    (2.0, 1e30, 2.0, 4.0),     # rho_c above every density: no seed, all outliers or noise
], ids=["dm0", "dc_huge", "rhoc_negative", "rhoc_huge"])
def test_degenerate_parameters(clue_mod, params):
    """The method's degenerate parameter choices, bit-exact against the oracle."""
    ext = (-100.0, 100.0, -100.0, 100.0)
    ev = gen.make_event(4000, 4, 61, "blobs", extent=ext)
    cl = _cl(clue_mod, ext, 4)
    assert_parity(_gpu_all(cl, ev, params), oracle.run_event(ev, params, 4, extent=ext))


def test_dense_cells_and_exact_ties(clue_mod):
    """Thousands of hits in one bin (windows of thousands of candidates);
    identical coordinates give exact distance ties."""
    rng = np.random.default_rng(1)
    n = 6000
    x = np.concatenate([rng.normal(0, 0.3, n // 2), np.full(n // 4, 1.5), rng.uniform(-3, 3, n // 4)])
    y = np.concatenate([rng.normal(0, 0.3, n // 2), np.full(n // 4, -1.0), rng.uniform(-3, 3, n // 4)])
    w = rng.exponential(1.0, n)
    ev = Ev(x, y, np.zeros(n, np.int32), w)
    ext = (-5.0, 5.0, -5.0, 5.0)
    cl = _cl(clue_mod, ext, 1, bin_size=2.5)
    p = (0.5, 3.0, 0.7, 1.0)
    assert_parity(_gpu_all(cl, ev, p), oracle.run_event(ev, p, 1, extent=ext))


@pytest.mark.parametrize("form", ["two_level", "fine_grid", "many_layers", "long_segment"])
def test_grid_fill_forms(clue_mod, form):
    """Both forms of the grid fill, bit-exact against the oracle: the two-level
    sort, the direct sort that a layer of more than 16384 cells or more than
    1024 layers falls back to, and a 30000-hit layer segment (longer than the
    two-level sort permutes in shared memory).  The profiled kernel names show which ran."""
    ext = (-100.0, 100.0, -100.0, 100.0)
    rng = np.random.default_rng(71)
    kw, L = {}, 8
    if form == "long_segment":
        L = 1
        ev = gen.make_event(30_000, 1, 72, "blobs", extent=ext)
    elif form == "many_layers":
        L = 5000
        n = 20_000
        ev = Ev(rng.uniform(-100, 100, n), rng.uniform(-100, 100, n),
                rng.integers(0, L, n), rng.exponential(1.0, n))
    elif form == "fine_grid":  # bins of d_c over 500 x 500: ~40000 cells per layer
        ext = (-250.0, 250.0, -250.0, 250.0)
        ev = gen.make_event(20_000, L, 73, "blobs", extent=ext)
        kw = dict(bin_size=2.0)
    else:
        ev = gen.make_event(20_000, L, 73, "blobs", extent=ext)
    cl = _cl(clue_mod, ext, L, **kw)
    cl.set_profiling(True)
    assert_parity(_gpu_all(cl, ev, gen.PARAMS_BLOBS),
                  oracle.run_event(ev, gen.PARAMS_BLOBS, L, extent=ext))
    direct = form in ("fine_grid", "many_layers")
    names = set(cl.kernel_times())
    assert ("fill_count" in names) == direct and ("fill_cells" in names) == (not direct)


def test_cell_sort_builds_and_their_long_segments(clue_mod):
    """The cell sort's two builds in one batch, each meeting a segment longer
    than it permutes in shared memory: an event of few hits per layer on
    average (the 128-thread build) whose hits all sit in one layer (a
    30000-hit segment, past that build's 4096), beside events of many hits
    per layer (the 512-thread build), one with a 20000-hit layer."""
    ext = (-60.0, 60.0, -60.0, 60.0)
    L = 40
    crowded = gen.make_event(30_000, 1, 81, "blobs", extent=ext)  # layer 0 only
    sparse = gen.make_event(8_000, L, 82, "blobs", extent=ext)
    dense = gen.make_event(60_000, 3, 83, "blobs", extent=ext)     # ~20000 hits per layer
    evs = [crowded, sparse, dense]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, ext, L, bin_size=4.0)  # 30 x 30 cells per layer: the small build's limit
    cl.set_profiling(True)
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    cl.sync()
    cid, seed = cid.cpu().numpy(), seed.cpu().numpy()
    assert "fill_cells" in cl.kernel_times()
    for i, ev in enumerate(evs):
        ref = oracle.run_event(ev, gen.PARAMS_BLOBS, L, extent=ext)
        assert np.array_equal(cid[offs[i]:offs[i + 1]], ref["cluster_id"]), i
        assert np.array_equal(seed[offs[i]:offs[i + 1]], ref["is_seed"]), i


@pytest.mark.parametrize("expand", [0, 1], ids=["frontier", "chase"])
def test_wide_tree_one_node_with_many_followers(clue_mod, expand):
    """2000 hits on a circle of radius 3 around one heavy hit.  They are
    farther apart than d_c, so each has rho = its own weight 1 (equal, so none
    is higher than another), and the centre (rho 1000) is every one's
    nearest-higher within d_m = 4: one frontier node hands its id to 2000
    followers spread over many threads."""
    k = 2000
    ang = np.arange(k) * (2 * np.pi / k)
    x = np.concatenate([[0.0], 3 * np.cos(ang), [50.0]])
    y = np.concatenate([[0.0], 3 * np.sin(ang), [50.0]])
    w = np.concatenate([[1000.0], np.ones(k), [5.0]])
    ev = Ev(x, y, np.zeros(k + 2, np.int32), w)
    p = (0.005, 0.5, 4.0, 4.0)
    ext = (-100.0, 100.0, -100.0, 100.0)
    cl = _cl(clue_mod, ext, 1, expand=expand)
    ref = oracle.run_event(ev, p, 1, extent=ext)
    assert (ref["nh"][1:k + 1] == 0).all() and (ref["cluster_id"][1:k + 1] == 0).all()
    assert_parity(_gpu_all(cl, ev, p), ref)


@pytest.mark.parametrize("expand", [0, 1], ids=["frontier", "chase"])
def test_batch_expand_modes_agree(clue_mod, expand):
    evs = [gen.make_event(n, 100, 800 + i, k) for i, (n, k) in
           enumerate([(30000, "blobs"), (50000, "irregular"), (3, "blobs"), (0, "blobs")])]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100, expand=expand)
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_IRREGULAR)
    cl.sync()
    cid = cid.cpu().numpy()
    for i, ev in enumerate(evs):
        ref = oracle.run_event(ev, gen.PARAMS_IRREGULAR, 100)
        assert np.array_equal(cid[offs[i]:offs[i + 1]], ref["cluster_id"])


def test_long_chain(clue_mod):
    """A line of hits with rising weights: nh chains of length ~1000."""
    n = 1000
    x = np.arange(n, dtype=np.float64)
    w = 1.0 + np.arange(n) * 1e-3
    ev = Ev(x - 500.0, np.zeros(n), np.zeros(n, np.int32), w)
    p = (1.5, 1.0, 2.0, 3.0)
    ext = (-600.0, 600.0, -10.0, 10.0)
    for expand in (0, 1):
        cl = _cl(clue_mod, ext, 1, expand=expand)
        assert_parity(_gpu_all(cl, ev, p), oracle.run_event(ev, p, 1, extent=ext))
    cl = _cl(clue_mod, ext, 1)
    ref = oracle.run_event(ev, p, 1, extent=ext)
    assert_parity(_gpu_all(cl, ev, p), ref)


def _chain_1000():
    n = 1000
    x = np.arange(n, dtype=np.float64)
    w = 1.0 + np.arange(n) * 1e-3
    ev = Ev(x - 500.0, np.zeros(n), np.zeros(n, np.int32), w)
    return ev, (1.5, 1.0, 2.0, 3.0), (-600.0, 600.0, -10.0, 10.0)


@pytest.mark.parametrize("expand", [0, 1], ids=["frontier", "chase"])
def test_walk_limit_runs_out_and_reports_timeout(clue_mod, expand):
    """The 1000-hit chain (one cluster, depth 999) under walk limits too short
    for it: 10 steps (the bounded walk alone) and 66 (the 64-step walk and two
    pointer-jumping rounds).  The device gives up on the hits it cannot reach
    (-1), the next clue_sync returns CLUE_ERR_TIMEOUT, and the context stays
    usable.  With 74 (ten rounds) the chain resolves exactly."""
    ev, p, ext = _chain_1000()
    ref = oracle.run_event(ev, p, 1, extent=ext)
    assert ref["n_seeds"] == 1 and (ref["cluster_id"] == 0).all()
    for limit in (10, 66):
        cl = _cl(clue_mod, ext, 1, expand=expand, walk_limit=limit)
        cid, seed = cl.run(ev.x, ev.y, ev.layer, ev.energy, p)
        with pytest.raises(clue_mod.ClueError) as ei:
            cl.sync()
        assert ei.value.code == clue_mod.CLUE_ERR_TIMEOUT
        c = cid.cpu().numpy()
        assert set(np.unique(c).tolist()) == {-1, 0}
        assert c[-1] == 0 and c[0] == -1  # the seed is resolved, the chain's far end is not
        assert np.array_equal(seed.cpu().numpy(), ref["is_seed"])
        small = gen.make_event(3000, 1, 5, "blobs", extent=ext)
        g = _gpu_all(cl, small, gen.PARAMS_BLOBS)  # syncs: no error left behind
        assert_parity(g, oracle.run_event(small, gen.PARAMS_BLOBS, 1, extent=ext))
        cl.close()
    cl = _cl(clue_mod, ext, 1, expand=expand, walk_limit=74)
    assert_parity(_gpu_all(cl, ev, p), ref)


def _serpentine_chain(n, row_len=1300):
    """n hits on a serpentine path, 1.5 cm apart along rows 3 cm apart, with
    weights rising along the path (exact in fp32): every hit's nearest-higher
    is the next hit or, at a row's end, one of the next row's first two, so
    the event is one cluster whose tree is a single chain of depth ~n."""
    i = np.arange(n)
    r, c = i // row_len, i % row_len
    c = np.where(r % 2 == 0, c, row_len - 1 - c)
    x = c * 1.5 - row_len * 0.75
    y = r * 3.0 - 240.0
    w = 1.0 + i * 2.0 ** -20
    return Ev(x, y, np.zeros(n, np.int32), w)


@pytest.mark.parametrize("expand", [0, 1], ids=["frontier", "chase"])
def test_chain_of_200k_hits(clue_mod, expand):
    """A 200k-hit chain, resolved by the bounded walk plus pointer jumping in
    about log2(200k / 64) rounds, against the oracle in full."""
    ev = _serpentine_chain(200_000)
    p = (2.0, 1.0, 3.5, 4.0)
    ext = (-1000.0, 1000.0, -250.0, 250.0)
    ref = oracle.run_event(ev, p, 1, extent=ext)
    assert ref["n_seeds"] == 1 and (ref["cluster_id"] == 0).all()
    depth, j = 0, 0  # the chain really is deep: follow nh from the first hit
    while j >= 0 and depth <= ev.n:
        j, depth = int(ref["nh"][j]), depth + 1
    assert depth > 190_000
    cl = _cl(clue_mod, ext, 1, expand=expand)
    assert_parity(_gpu_all(cl, ev, p), ref)


def test_invalid_inputs_reported_at_sync(clue_mod):
    cl = _cl(clue_mod, gen.EXTENT, 4)
    x = np.zeros(100, np.float32)
    x[7] = np.nan
    cl.run(x, np.zeros(100), np.zeros(100, np.int32), np.ones(100), gen.PARAMS_BLOBS)
    with pytest.raises(clue_mod.ClueError) as ei:
        cl.sync()
    assert ei.value.code == clue_mod.CLUE_ERR_INPUT
    cl.sync()  # error cleared
    bad_layer = np.full(50, 4, np.int32)
    cl.run(np.zeros(50), np.zeros(50), bad_layer, np.ones(50), gen.PARAMS_BLOBS)
    with pytest.raises(clue_mod.ClueError):
        cl.sync()
    with pytest.raises(clue_mod.ClueError) as ei:
        cl.run(np.zeros(5), np.zeros(5), np.zeros(5, np.int32), np.ones(5), (0.0, 1.0, 1.0, 1.0))
    assert ei.value.code == clue_mod.CLUE_ERR_ARG


@pytest.mark.parametrize("tile", [64, 256, 512, 1024])
@pytest.mark.parametrize("block", [0, 128, 512])
def test_tile_length_and_block_do_not_change_results(clue_mod, tile, block):
    """Every tuning choice of the table (hits per tile, so hits per thread, per
    size class; the density kernels' block) gives the same bytes: a batch with
    an event in each size class, against the oracle."""
    evs = [gen.make_event(n, 100, 700 + i, "blobs") for i, n in
           enumerate([12000, 50000, 150000, 400000, 1_100_000])]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    lines = [ln for ln in cl.tuning.splitlines() if ln.startswith("class")]
    cl.tuning = "\n".join(" ".join(ln.split()[:4] + [str(tile)]) for ln in lines) + \
        f"\nblock {block}\n"
    assert all(ln.split()[4] == str(tile) for ln in cl.tuning.splitlines()
               if ln.startswith("class"))
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    rho, delta, nh = cl.intermediates()
    cl.sync()
    c, sd = cid.cpu().numpy(), seed.cpu().numpy()
    r, d, h = rho.cpu().numpy(), delta.cpu().numpy(), nh.cpu().numpy()
    for i, ev in enumerate(evs):
        a, z = offs[i], offs[i + 1]
        g = dict(cluster_id=c[a:z], is_seed=sd[a:z], rho=r[a:z], delta=d[a:z], nh=h[a:z])
        assert_parity(g, oracle.run_event(ev, gen.PARAMS_BLOBS, 100))


def test_autotune_keeps_results(clue_mod):
    evs = [gen.make_event(n, 100, 900 + i, "blobs") for i, n in enumerate([15000, 60000, 200000])]
    x, y, l, e, offs = gen.concat(evs)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    table = cl.autotune(x, y, l, e, offs, gen.PARAMS_BLOBS, reps=1)
    assert "block" in table
    cid, seed = cl.run_batch(x, y, l, e, offs, gen.PARAMS_BLOBS)
    cl.sync()
    cid = cid.cpu().numpy()
    for i, ev in enumerate(evs):
        assert np.array_equal(cid[offs[i]:offs[i + 1]],
                              oracle.run_event(ev, gen.PARAMS_BLOBS, 100)["cluster_id"])
    cl.tuning = table  # round-trips through the text format
    assert cl.tuning == table
    assert len([ln for ln in table.splitlines() if ln.startswith("class")]) == 6
    for ln in table.splitlines():
        if ln.startswith("class"):
            assert int(ln.split()[4]) in (256, 512, 1024)


def test_stage_times_and_launch_count(clue_mod):
    ev = gen.make_event(100_000, 100, 3, "blobs")
    for expand, last in ((0, {"expand_level", "complete", "jump"}), (1, {"assign", "jump"})):
        cl = _cl(clue_mod, gen.EXTENT, 100, expand=expand)
        cl.set_profiling(True)
        cl.run(ev.x, ev.y, ev.layer, ev.energy, gen.PARAMS_BLOBS)
        st = cl.stage_times()
        assert list(st) == ["grid_fill", "density", "decide_followers", "expand"]
        assert all(v >= 0 for v in st.values())
        kt = cl.kernel_times()
        assert {"fill_cells", "density", "nh_rest"} | last <= set(kt)
        # two-level grid fill with a one-CTA segment scan (4); chase: one-CTA
        # seed-rank scan that also writes the seed codes; both end with the
        # pointer-jumping kernel
        assert cl.launch_count() == (4 + 20 if expand == 0 else 9)


def test_paper_parameter_workload(clue_mod):
    """Sec. 4.2's workload shape (unit weights, sigma 3 cm blobs, 5% noise,
    d_c = 3, rho_c = 8, delta_c = delta_o = 5, bin 5 cm), 100 layers x 2k hits."""
    ev = gen.make_event(200_000, 100, 11, "paper")
    cl = _cl(clue_mod, gen.EXTENT, 100, bin_size=5.0)
    assert_parity(_gpu_all(cl, ev, gen.PARAMS_PAPER), oracle.run_event(ev, gen.PARAMS_PAPER, 100))


def test_noise_shrinks_as_delta_o_grows_on_gpu(clue_mod):
    """Fig. 4: with delta_c fixed and at least every delta_o, a larger delta_o
    demotes fewer outliers, so the noise can only shrink; each run is also
    bit-exact with the oracle."""
    ext = (-80.0, 80.0, -80.0, 80.0)
    ev = gen.make_event(8000, 1, 21, "blobs", extent=ext)
    cl = _cl(clue_mod, ext, 1)
    prev = None
    for do in (0.5, 1.0, 2.0, 4.0):
        p = (2.0, 2.0, 4.0, do)
        g = _gpu_all(cl, ev, p)
        assert_parity(g, oracle.run_event(ev, p, 1, extent=ext))
        noise = int((g["cluster_id"] < 0).sum())
        if prev is not None:
            assert noise <= prev
        prev = noise


@pytest.mark.parametrize("chi,s", [(1, 1.5), (2, 0.8)], ids=["gaussian", "exponential"])
def test_chi_kernels_parity(clue_mod, chi, s):
    """Eq. 3's Gaussian and exponential kernels: rho (and everything after it)
    bit-exact with the oracle, both computing chi with the same fp32 exp."""
    for kind, n, L, params, seed, ext in [("blobs", 30000, 10, gen.PARAMS_BLOBS, 2, gen.EXTENT),
                                          ("irregular", 20000, 2, gen.PARAMS_IRREGULAR, 3,
                                           (-60.0, 60.0, -60.0, 60.0))]:
        ev = gen.make_event(n, L, seed, kind, extent=ext)
        cl = _cl(clue_mod, ext, L, chi=chi, chi_param=s)
        ref = oracle.run_event(ev, params, L, extent=ext, chi=chi, chi_param=s)
        assert_parity(_gpu_all(cl, ev, params), ref)


def test_scratch_limit_fails_cleanly_then_recovers(clue_mod):
    """An injected scratch limit makes a run fail with CLUE_ERR_OOM before any
    allocation; the context stays usable for runs that fit."""
    small = gen.make_event(2000, 4, 1, "blobs")
    big = gen.make_event(400_000, 100, 2, "blobs")
    cl = _cl(clue_mod, gen.EXTENT, 100, max_scratch_bytes=20_000_000)
    cid, _ = cl.run(small.x, small.y, small.layer, small.energy, gen.PARAMS_BLOBS)
    cl.sync()
    with pytest.raises(clue_mod.ClueError) as ei:
        cl.run(big.x, big.y, big.layer, big.energy, gen.PARAMS_BLOBS)
    assert ei.value.code == clue_mod.CLUE_ERR_OOM
    cid2, _ = cl.run(small.x, small.y, small.layer, small.energy, gen.PARAMS_BLOBS)
    cl.sync()
    assert np.array_equal(cid.cpu().numpy(), cid2.cpu().numpy())


def test_unit_weight_partition_invariant_under_permutation(clue_mod):
    """With unit weights rho is an exact integer, so relabelling the hits only
    relabels the clusters, on the GPU path."""
    ev = gen.make_event(300_000, 100, 5, "paper")
    perm = np.random.default_rng(2).permutation(ev.n)
    cl = _cl(clue_mod, gen.EXTENT, 100)
    a, _ = cl.run(ev.x, ev.y, ev.layer, ev.energy, gen.PARAMS_PAPER)
    b, _ = cl.run(ev.x[perm], ev.y[perm], ev.layer[perm], ev.energy[perm], gen.PARAMS_PAPER)
    cl.sync()
    a, b = a.cpu().numpy(), b.cpu().numpy()[np.argsort(perm)]
    # same partition: a bijection between the id sets
    pairs = set(zip(a.tolist(), b.tolist()))
    assert len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))
    assert ((a < 0) == (b < 0)).all()
