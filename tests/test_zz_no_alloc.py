"""clue_run_static: single-event clustering that allocates nothing.

Callers that cannot allocate device memory (inside another framework's memory
pool, in a real-time loop where an allocation could block or fail, or in a
plugin whose host owns all device memory) use clue_run_static, whose scratch
is a fixed array in the library's device memory.  This test calls it through
the C ABI with device pointers and checks its outputs against clue_run's, with
the tolerance of every other parity test here (0: identical bytes), on two
calls in a row, so the second call runs on scratch the first one left behind.
It lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2001_09761_gb300 import gen

pytestmark = pytest.mark.gpu


def _static(clue, torch, ev, params, extent, layers, stream):
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    x, y = t(ev.x, torch.float32), t(ev.y, torch.float32)
    l, e = t(ev.layer, torch.int32), t(ev.energy, torch.float32)
    cid = torch.full((ev.n,), -7, dtype=torch.int32, device=dev)
    seed = torch.full((ev.n,), 7, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    rc = clue.clue_run_static(x.data_ptr(), y.data_ptr(), l.data_ptr(), e.data_ptr(), ev.n,
                              *[float(v) for v in params], *[float(v) for v in extent], layers,
                              cid.data_ptr(), seed.data_ptr(), stream)
    return rc, cid.cpu().numpy(), seed.cpu().numpy()


def test_static_scratch_entry_point_matches_clue_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import build, clue
    build.build()
    clue.load()
    stream = torch.cuda.Stream()
    cases = [  # two calls in a row; the second is smaller, on stale scratch
        (gen.make_event(60000, 20, 41, "irregular"), gen.PARAMS_IRREGULAR, gen.EXTENT, 20),
        (gen.make_event(9000, 6, 42, "blobs", extent=(-50.0, 50.0, -50.0, 50.0)),
         gen.PARAMS_BLOBS, (-50.0, 50.0, -50.0, 50.0), 6),
    ]
    for ev, params, extent, layers in cases:
        cl = clue.Clusterer(device=0, extent=extent, max_layers=layers)
        ref_cid, ref_seed = cl.run(ev.x, ev.y, ev.layer, ev.energy, params)
        cl.sync()
        ref_cid, ref_seed = ref_cid.cpu().numpy(), ref_seed.cpu().numpy()
        cl.close()
        rc, cid, seed = _static(clue, torch, ev, params, extent, layers, stream.cuda_stream)
        assert rc == clue.CLUE_OK, clue.clue_strerror(rc)
        assert np.array_equal(cid, ref_cid)
        assert np.array_equal(seed, ref_seed)
        assert (ref_cid >= 0).any() and (ref_cid < 0).any()


def _ref(clue, ev, params, extent, layers):
    cl = clue.Clusterer(device=0, extent=extent, max_layers=layers)
    cid, seed = cl.run(ev.x, ev.y, ev.layer, ev.energy, params)
    cl.sync()
    out = cid.cpu().numpy(), seed.cpu().numpy()
    cl.close()
    return out


def test_static_entry_point_at_its_limits():
    """The largest event the array holds (CLUE_STATIC_MAX_HITS hits, 64 full
    tiles) on a grid of 1000 layers, whose first bin size gives more cells
    than the array holds, so the bins are widened several times; then a tiny
    d_c, whose first grid would overflow any integer, widened to fit as well.
    Both give clue_run's results (the bin size never changes them)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import clue
    clue.load()
    stream = torch.cuda.Stream()
    n = clue.CLUE_STATIC_MAX_HITS
    ev = gen.make_event(n, 1000, 43, "blobs")
    assert ev.n == n and int(ev.layer.max()) == 999
    tiny = (1e-15, 0.5, 2.0, 4.0)  # only coincident hits are within d_c
    for params in (gen.PARAMS_BLOBS, tiny):
        ref_cid, ref_seed = _ref(clue, ev, params, gen.EXTENT, 1000)
        rc, cid, seed = _static(clue, torch, ev, params, gen.EXTENT, 1000, stream.cuda_stream)
        assert rc == clue.CLUE_OK, clue.clue_strerror(rc)
        assert np.array_equal(cid, ref_cid)
        assert np.array_equal(seed, ref_seed)


def test_static_entry_point_rejects_oversized_events():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import clue
    clue.load()
    n = clue.CLUE_STATIC_MAX_HITS + 1
    rc = clue.clue_run_static(1, 1, 1, 1, n, 2.0, 2.0, 2.0, 4.0, -250.0, 250.0, -250.0, 250.0,
                              100, 1, 1, None)
    assert rc == clue.CLUE_ERR_ARG


def test_static_entry_point_rejects_too_many_layers():
    """More layers than the array has cells: no bin size can fit, so the call
    is refused before anything runs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_09761_gb300 import clue
    clue.load()
    rc = clue.clue_run_static(1, 1, 1, 1, 100, 2.0, 2.0, 2.0, 4.0, -250.0, 250.0, -250.0, 250.0,
                              clue.CLUE_STATIC_MAX_CELLS + 1, 1, 1, None)
    assert rc == clue.CLUE_ERR_ARG
