"""GPU parity at the full sizes of the benchmarked workloads, against the oracle.

Every output of the CUDA path (cluster ids, seed flags, and the
intermediates rho, delta, nh) is compared element by element with the CPU
oracle, tolerance 0, on the events the benchmark reports:

* the 5M-hit irregular event (50 layers x 100k hits: ellipses, rings, 30 %
  noise and four dense hotspot discs per layer, whose windows hold thousands
  of candidates), clustered in full;
* the 0.1M-1M scaling sweep (100 layers x {1k..10k} hits): all ten sizes at
  seed 0 and all ten seeds at 1M hits;
* each event run as the benchmark runs it: the same call three times (direct
  launches, then captured into a CUDA graph, then the graph replayed) and the
  replay's outputs compared.

Served events are compared with the oracle in tests/test_serve.py.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2001_09761_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clue_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import build, clue
    build.build()
    clue.load()
    return clue


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _check(g, ref, what):
    for k in ("cluster_id", "is_seed", "rho", "delta", "nh"):
        a, b = g[k], ref[k]
        if a.dtype.kind == "f":
            bad = np.nonzero(_bits(a) != _bits(b))[0]
        else:
            bad = np.nonzero(a != b.astype(a.dtype))[0]
        assert bad.size == 0, (f"{what} {k}: {bad.size} of {a.size} differ, first "
                               f"{bad[:6]}: {a[bad[:6]]} vs {b[bad[:6]]}")


def _gpu_replayed(clue_mod, ev, layers, params):
    """The event run three times through one context (direct launches,
    capture, graph replay), outputs of the replay."""
    import torch
    cl = clue_mod.Clusterer(device=0, extent=gen.EXTENT, max_layers=layers)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, l, e = d(ev.x), d(ev.y), d(ev.layer), d(ev.energy)
    cid = torch.full((ev.n,), -9, dtype=torch.int32, device="cuda")
    seed = torch.full((ev.n,), 9, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        cl.run(x, y, l, e, params, out=(cid, seed))
    rho, delta, nh = cl.intermediates()
    cl.sync()
    out = dict(cluster_id=cid.cpu().numpy(), is_seed=seed.cpu().numpy(),
               rho=rho.cpu().numpy(), delta=delta.cpu().numpy(), nh=nh.cpu().numpy())
    cl.close()
    return out


def test_irregular_5M_event_in_full(clue_mod):
    ev = gen.irregular_event(0)
    assert ev.n == 5_000_000
    g = _gpu_replayed(clue_mod, ev, 50, gen.PARAMS_IRREGULAR)
    ref = oracle.run_event(ev, gen.PARAMS_IRREGULAR, 50)
    _check(g, ref, "irregular 5M")
    assert ref["n_seeds"] > 1000 and (ref["cluster_id"] < 0).any()


SWEEP = [(h, 0) for h in range(1000, 10001, 1000)] + [(10_000, s) for s in range(1, 10)]


@pytest.mark.parametrize("h,seed", SWEEP, ids=[f"{100 * h}_s{s}" for h, s in SWEEP])
def test_scaling_sweep_event(clue_mod, h, seed):
    ev = gen.scaling_event(h, seed)
    g = _gpu_replayed(clue_mod, ev, 100, gen.PARAMS_BLOBS)
    ref = oracle.run_event(ev, gen.PARAMS_BLOBS, 100)
    _check(g, ref, f"sweep {100 * h} hits seed {seed}")
