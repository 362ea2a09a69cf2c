"""Pins for the CPU oracle: it is checked against things other than itself.

* hand-derived golden fixtures (tests/golden/*.json, each citing the passage
  it follows);
* an O(n^2) brute force written from the definitions (no grid, recursive
  expansion instead of Algorithm 3's stack);
* library routines: scipy's KD-tree for neighbour sets and nearest-higher
  search, networkx for the follower forest, exact rational sums (Python
  fractions) for rho;
* the paper's invariants (Sec. 2.2) and symmetries of the definitions.
"""
from __future__ import annotations

import json
import math
from pathlib import Path

import numpy as np
import pytest

from brute import brute_clue
from exactsum import adversarial_weights, exact_rho
from paper_2001_09761_gb300 import gen

GOLDEN = Path(__file__).resolve().parent / "golden"
KEYS = ["rho", "delta2", "nh", "is_seed", "is_outlier", "cluster_id"]


def _fixture(name):
    d = json.loads((GOLDEN / f"{name}.json").read_text())
    exp = {k: np.array([np.inf if v == "inf" else v for v in d["expected"][k]])
           for k in d["expected"]}
    return d, exp


@pytest.mark.parametrize("name", sorted(p.stem for p in GOLDEN.glob("*.json")))
def test_golden_fixture(oracle_mod, name):
    d, exp = _fixture(name)
    out = oracle_mod.run(d["x"], d["y"], d["layer"], d["w"], d["params"], d["n_layers"],
                         d["extent"])
    for k in KEYS:
        want = exp[k].astype(out[k].dtype)
        assert np.array_equal(out[k], want), (k, out[k], want)
    # the brute force agrees with the same hand-derived values
    b = brute_clue(d["x"], d["y"], d["layer"], d["w"], d["params"])
    for k in KEYS:
        assert np.array_equal(b[k], exp[k].astype(b[k].dtype)), k


def _assert_same(a, b, keys=KEYS):
    for k in keys:
        assert a[k].dtype == b[k].dtype or k in ("nh",), k
        if a[k].dtype.kind == "f":
            assert np.array_equal(a[k].view(np.uint32), b[k].astype(np.float32).view(np.uint32)), k
        else:
            assert np.array_equal(a[k], b[k]), (k, np.nonzero(a[k] != b[k])[0][:10])


SMALL_EVENTS = [
    ("blobs", 2400, 3, gen.PARAMS_BLOBS, 0),
    ("blobs", 1500, 1, (2.0, 1.0, 1.0, 3.0), 1),
    ("irregular", 2000, 2, gen.PARAMS_IRREGULAR, 2),
    ("paper", 2000, 2, gen.PARAMS_PAPER, 3),
    ("uniform", 1800, 1, (6.0, 3.0, 4.0, 8.0), 4),
    ("blobs", 1000, 2, (2.0, 2.0, 6.0, 1.0), 5),   # delta_c > delta_o
]


@pytest.mark.parametrize("kind,n,L,params,seed", SMALL_EVENTS)
def test_oracle_matches_brute_force(oracle_mod, kind, n, L, params, seed):
    # Shrink the extent so that small events are dense enough to form chains.
    ext = (-40.0, 40.0, -40.0, 40.0)
    ev = gen.make_event(n, L, seed, kind, extent=ext)
    o = oracle_mod.run_event(ev, params, L, extent=ext)
    b = brute_clue(ev.x, ev.y, ev.layer, ev.energy, params)
    _assert_same(o, b)
    assert o["n_seeds"] == int(b["is_seed"].sum())


def test_oracle_independent_of_extent_and_clamping(oracle_mod):
    """Hits far outside the grid extent land in edge bins (reading R10); the
    result equals the brute force, which has no grid at all."""
    ev = gen.make_event(1500, 2, 7, "blobs", extent=(-30.0, 30.0, -30.0, 30.0))
    for ext in [(-5.0, 5.0, -5.0, 5.0), (-1000.0, 1000.0, -3.0, 200.0), (0.0, 1.0, 0.0, 1.0)]:
        o = oracle_mod.run_event(ev, gen.PARAMS_BLOBS, 2, extent=ext)
        b = brute_clue(ev.x, ev.y, ev.layer, ev.energy, gen.PARAMS_BLOBS)
        _assert_same(o, b)


def test_isolated_hits_closed_form(oracle_mod):
    """All hits farther apart than d_c and d_m: rho_i = w_i (Eq. 3 with only
    j = i), delta = +inf, seed iff w > rho_c, outlier iff w < rho_c."""
    g = np.arange(40, dtype=np.float32)
    x = (g % 8) * 10.0
    y = (g // 8) * 10.0
    w = np.linspace(0.5, 3.5, 40).astype(np.float32)
    w[7] = 2.0  # exactly rho_c: neither seed nor outlier, no nh -> noise
    out = oracle_mod.run(x, y, np.zeros(40, np.int32), w, (1.0, 2.0, 1.0, 2.0), 1)
    assert np.array_equal(out["rho"], w)
    assert np.all(np.isinf(out["delta2"])) and np.all(out["nh"] == -1)
    assert np.array_equal(out["is_seed"], (w > 2.0).astype(np.uint8))
    assert np.array_equal(out["is_outlier"], (w < 2.0).astype(np.uint8))
    seeds = np.nonzero(w > 2.0)[0]
    exp = np.full(40, -1)
    exp[seeds] = np.arange(seeds.size)
    assert np.array_equal(out["cluster_id"], exp)


def test_invariants_on_generated_events(oracle_mod):
    """Sec. 2.2: seeds have rho > rho_c and delta > delta_c, outliers rho < rho_c
    and delta > delta_o; every clustered hit reaches its seed through nh links
    without crossing another seed or an outlier; noise reaches an outlier or a
    hit with no nearest-higher; ids are 0..k-1 in ascending seed index."""
    for kind, params in [("blobs", gen.PARAMS_BLOBS), ("irregular", gen.PARAMS_IRREGULAR)]:
        ev = gen.make_event(20000, 4, 11, kind, extent=(-100.0, 100.0, -100.0, 100.0))
        o = oracle_mod.run_event(ev, params, 4, extent=(-100.0, 100.0, -100.0, 100.0))
        dc, rhoc, delta_c, delta_o = (np.float32(v) for v in params)
        rho, d2, nh = o["rho"], o["delta2"], o["nh"]
        seed, outl, cid = o["is_seed"].astype(bool), o["is_outlier"].astype(bool), o["cluster_id"]
        assert np.all(rho[seed] > rhoc) and np.all(d2[seed] > delta_c * delta_c)
        assert np.all(rho[outl] < rhoc) and np.all(d2[outl] > delta_o * delta_o)
        assert not np.any(seed & outl)
        seeds = np.nonzero(seed)[0]
        assert np.array_equal(cid[seeds], np.arange(seeds.size))
        has = nh >= 0
        assert np.all(rho[nh[has]] > rho[has])
        assert np.all(ev.layer[nh[has]] == ev.layer[has])
        dm = max(delta_c, delta_o)
        assert np.all(d2[has] < dm * dm) and np.all(np.isinf(d2[~has]))
        for i in range(ev.n):
            j = i
            while not seed[j] and not outl[j] and nh[j] >= 0:
                j = nh[j]
            assert cid[i] == (cid[j] if seed[j] else -1)


@pytest.mark.parametrize("params", [(2.0, 2.0, 0.0, 0.0), (400.0, 2.0, 2.0, 4.0),
                                    (2.0, -1.0, 2.0, 4.0), (2.0, 1e30, 2.0, 4.0)],
                         ids=["dm0", "dc_huge", "rhoc_negative", "rhoc_huge"])
def test_degenerate_parameters_match_brute_force(oracle_mod, params):
    """No nearest-higher search (d_m = 0); d_c spanning the layer (every rho
    of a layer equal, so every hit is a seed, Eq. 4 with R6); rho_c below or
    above every density: oracle and brute force agree bit for bit."""
    ext = (-100.0, 100.0, -100.0, 100.0)
    ev = gen.make_event(600, 2, 61, "blobs", extent=ext)
    o = oracle_mod.run_event(ev, params, 2, extent=ext)
    _assert_same(o, brute_clue(ev.x, ev.y, ev.layer, ev.energy, params))
    if params[0] == 400.0:
        assert o["is_seed"].all() and (o["nh"] == -1).all()
    if params[1] == 1e30:
        assert not o["is_seed"].any() and (o["cluster_id"] == -1).all()


def test_rho_is_exact_sum_rounded_once(oracle_mod):
    """Reading R4: rho_i is the exact rational sum of w_j over N_dc(i) rounded
    once to fp32 (ties to even), checked hit by hit with Python's exact
    fractions on weights chosen so that any fp32 running sum would differ."""
    ev = gen.make_event(600, 1, 3, "irregular", extent=(-15.0, 15.0, -15.0, 15.0))
    w = adversarial_weights(np.random.default_rng(7), ev.n)
    dc = np.float32(2.0)
    o = oracle_mod.run(ev.x, ev.y, ev.layer, w, gen.PARAMS_IRREGULAR, 1,
                       (-15.0, 15.0, -15.0, 15.0))
    x, y = ev.x, ev.y
    dx = x[None, :] - x[:, None]
    dy = y[None, :] - y[:, None]
    near = (dx * dx + dy * dy) < dc * dc
    for i in range(ev.n):
        want = exact_rho(w[near[i]])
        assert o["rho"][i].view(np.uint32) == want.view(np.uint32), (i, o["rho"][i], want)


def test_rho_exact_sum_of_coincident_hits(oracle_mod):
    """All hits of a layer at one point are mutual neighbours, so every rho
    is the rounded exact sum of the whole layer: the summation alone, on
    sets built to round up, down, to even, to a subnormal, to zero by
    cancellation, to infinity and up across a power of two."""
    rng = np.random.default_rng(11)
    sets = [adversarial_weights(rng, int(rng.integers(1, 60))) for _ in range(120)]
    sets += [np.array([1.0, 2.0 ** -24, 2.0 ** -25], np.float32),             # up (not a tie)
             np.array([1.0, 2.0 ** -24], np.float32),                          # tie, to even
             np.array([1.0 + 2.0 ** -23, 2.0 ** -24], np.float32),             # tie, to even (up)
             np.array([2.0 ** -149] * 5, np.float32),                          # subnormal
             np.array([3.0e38, 3.0e38, -1.0], np.float32),                     # overflow
             np.array([1e30, -1e30, 2.0 ** -140], np.float32),                 # cancellation
             np.array([5.0, -5.0], np.float32),                                # exact zero
             np.array([1.0, 1.0 - 2.0 ** -24, 2.0 ** -25], np.float32)]        # up into 2.0
    for w in sets:
        n = w.size
        z = np.zeros(n, np.float32)
        o = oracle_mod.run(z, z, np.zeros(n, np.int32), w, (1.0, 0.0, 1.0, 1.0), 1,
                           (-1.0, 1.0, -1.0, 1.0))
        want = exact_rho(w)
        assert np.all(o["rho"].view(np.uint32) == want.view(np.uint32)), (w, o["rho"][0], want)


def test_neighbour_sets_match_kdtree(oracle_mod):
    """Unit weights make rho an exact integer count of N_dc(i); scipy's KD-tree
    counts the same points (hits within 1e-4 of the d_c circle are skipped,
    since the KD-tree works in fp64 with <=)."""
    spatial = pytest.importorskip("scipy.spatial")
    ev = gen.make_event(5000, 2, 5, "paper", extent=(-60.0, 60.0, -60.0, 60.0))
    dc = 3.0
    o = oracle_mod.run_event(ev, gen.PARAMS_PAPER, 2, extent=(-60.0, 60.0, -60.0, 60.0))
    for l in range(2):
        idx = np.nonzero(ev.layer == l)[0]
        pts = np.stack([ev.x[idx], ev.y[idx]], 1).astype(np.float64)
        tree = spatial.cKDTree(pts)
        cnt = np.array([len(v) for v in tree.query_ball_point(pts, dc)])
        edge = np.array([len(v) for v in tree.query_ball_point(pts, dc + 1e-4)]) != \
            np.array([len(v) for v in tree.query_ball_point(pts, dc - 1e-4)])
        assert np.array_equal(o["rho"][idx][~edge], cnt[~edge].astype(np.float32))
        assert (~edge).sum() > 0.9 * idx.size


def test_nearest_higher_matches_kdtree(oracle_mod):
    """nh_i from Eq. 4 against a KD-tree ball query of radius d_m filtered by
    rho_j > rho_i, nearest first, smaller index on a tie (fp64 distances;
    hits whose best two candidates are within 1e-4 are skipped)."""
    spatial = pytest.importorskip("scipy.spatial")
    params = gen.PARAMS_BLOBS
    ext = (-50.0, 50.0, -50.0, 50.0)
    ev = gen.make_event(4000, 1, 9, "blobs", extent=ext)
    o = oracle_mod.run_event(ev, params, 1, extent=ext)
    pts = np.stack([ev.x, ev.y], 1).astype(np.float64)
    tree = spatial.cKDTree(pts)
    dm = max(params[2], params[3])
    checked = 0
    for i, nb in enumerate(tree.query_ball_point(pts, dm + 1e-4)):
        nb = np.array([j for j in nb if o["rho"][j] > o["rho"][i]], dtype=np.int64)
        d = np.hypot(pts[nb, 0] - pts[i, 0], pts[nb, 1] - pts[i, 1]) if nb.size else np.zeros(0)
        if nb.size and np.any(np.abs(d - dm) < 1e-4):
            continue
        keep = d < dm
        nb, d = nb[keep], d[keep]
        if nb.size == 0:
            assert o["nh"][i] == -1
            checked += 1
            continue
        order = np.lexsort((nb, d))
        if nb.size > 1 and d[order[1]] - d[order[0]] < 1e-4:
            continue
        assert o["nh"][i] == nb[order[0]]
        assert abs(math.sqrt(o["delta2"][i]) - d[order[0]]) < 1e-4
        checked += 1
    assert checked > 0.95 * ev.n


def test_expansion_matches_networkx_forest(oracle_mod):
    """Algorithm 3's expansion equals, per seed, the set of descendants of the
    seed in the follower forest (edges nh_j -> j for every hit that is neither
    seed nor outlier), computed by networkx."""
    nx = pytest.importorskip("networkx")
    ext = (-60.0, 60.0, -60.0, 60.0)
    ev = gen.make_event(6000, 3, 13, "irregular", extent=ext)
    o = oracle_mod.run_event(ev, gen.PARAMS_IRREGULAR, 3, extent=ext)
    G = nx.DiGraph()
    G.add_nodes_from(range(ev.n))
    follower = (o["is_seed"] == 0) & (o["is_outlier"] == 0) & (o["nh"] >= 0)
    G.add_edges_from((int(o["nh"][j]), int(j)) for j in np.nonzero(follower)[0])
    exp = np.full(ev.n, -1)
    for k, s in enumerate(np.nonzero(o["is_seed"])[0]):
        exp[s] = k
        for d in nx.descendants(G, int(s)):
            assert exp[d] == -1
            exp[d] = k
    assert np.array_equal(o["cluster_id"], exp)


def _partition(cid):
    """Canonical form of a clustering: the sorted tuple of member sets."""
    groups = {}
    for i, c in enumerate(cid):
        if c >= 0:
            groups.setdefault(int(c), []).append(i)
    return sorted(tuple(v) for v in groups.values())


@pytest.mark.parametrize("kind", ["paper", "blobs"])
def test_permutation_invariance(oracle_mod, kind):
    """rho is a function of the neighbour set alone (R4), so relabelling the
    hits permutes rho bit for bit and can only change cluster ids, not the
    partition, barring distance ties (unit weights for "paper", real-valued
    energies for "blobs")."""
    ext = (-40.0, 40.0, -40.0, 40.0)
    ev = gen.make_event(3000, 2, 17, kind, extent=ext)
    params = gen.PARAMS_PAPER if kind == "paper" else gen.PARAMS_BLOBS
    a = oracle_mod.run_event(ev, params, 2, extent=ext)
    perm = np.random.default_rng(1).permutation(ev.n)
    b = oracle_mod.run(ev.x[perm], ev.y[perm], ev.layer[perm], ev.energy[perm],
                       params, 2, extent=ext)
    inv = np.argsort(perm)
    assert np.array_equal(b["rho"][inv], a["rho"])
    back = b["cluster_id"][inv]
    assert _partition(back) == _partition(a["cluster_id"])
    assert np.array_equal(b["is_seed"][inv], a["is_seed"])


def test_translation_invariance_on_lattice(oracle_mod):
    """Integer coordinates translate exactly in fp32; distances, and so every
    output, are unchanged by an integer shift of one layer."""
    rng = np.random.default_rng(3)
    n = 1500
    x = rng.integers(-30, 30, n).astype(np.float32)
    y = rng.integers(-30, 30, n).astype(np.float32)
    w = rng.integers(1, 4, n).astype(np.float32)
    L = np.zeros(n, np.int32)
    p = (2.5, 5.0, 2.0, 3.0)
    a = oracle_mod.run(x, y, L, w, p, 1)
    b = oracle_mod.run(x + 7, y - 13, L, w, p, 1)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


def test_noise_shrinks_as_delta_o_grows(oracle_mod):
    """Fig. 4: a larger delta_o demotes fewer outliers.  With delta_c fixed at
    least as large as every delta_o, d_m = delta_c does not move, nh and delta
    are fixed, and the outlier set can only shrink."""
    ext = (-80.0, 80.0, -80.0, 80.0)
    ev = gen.make_event(8000, 1, 21, "blobs", extent=ext)
    prev_out, prev_noise = None, None
    for do in (0.5, 1.0, 2.0, 4.0):
        o = oracle_mod.run_event(ev, (2.0, 2.0, 4.0, do), 1, extent=ext)
        out = set(np.nonzero(o["is_outlier"])[0])
        noise = int((o["cluster_id"] < 0).sum())
        if prev_out is not None:
            assert out <= prev_out and noise <= prev_noise
        prev_out, prev_noise = out, noise
    assert len(prev_out) > 0


def test_layers_do_not_interact(oracle_mod):
    """Eq. 2 only relates hits on the same layer: an event equals the union of
    its layers clustered one by one (ids renumbered in index order)."""
    ext = (-30.0, 30.0, -30.0, 30.0)
    ev = gen.make_event(2000, 3, 23, "blobs", extent=ext)
    full = oracle_mod.run_event(ev, gen.PARAMS_BLOBS, 3, extent=ext)
    for l in range(3):
        idx = np.nonzero(ev.layer == l)[0]
        one = oracle_mod.run(ev.x[idx], ev.y[idx], np.zeros(idx.size, np.int32),
                             ev.energy[idx], gen.PARAMS_BLOBS, 1, extent=ext)
        assert np.array_equal(one["rho"], full["rho"][idx])
        assert np.array_equal(one["is_seed"], full["is_seed"][idx])
        nh = full["nh"][idx]
        assert np.array_equal(np.where(nh >= 0, np.searchsorted(idx, nh), -1), one["nh"])
        assert _partition(one["cluster_id"]) == [tuple(np.searchsorted(idx, g)) for g in
                                                 _partition(np.where(np.isin(np.arange(ev.n), idx), full["cluster_id"], -1))]


def test_input_errors(oracle_mod):
    x = np.zeros(3, np.float32)
    ok = dict(y=np.zeros(3, np.float32), layer=np.zeros(3, np.int32), energy=np.ones(3, np.float32))
    with pytest.raises(ValueError):
        oracle_mod.run(np.array([0, np.nan, 1], np.float32), ok["y"], ok["layer"], ok["energy"],
                       gen.PARAMS_BLOBS, 1)
    with pytest.raises(ValueError):
        oracle_mod.run(x, ok["y"], np.array([0, 1, 0], np.int32), ok["energy"], gen.PARAMS_BLOBS, 1)
    with pytest.raises(ValueError):
        oracle_mod.run(x, ok["y"], ok["layer"], ok["energy"], (0.0, 1.0, 1.0, 1.0), 1)
    empty = oracle_mod.run(np.zeros(0, np.float32), np.zeros(0, np.float32),
                           np.zeros(0, np.int32), np.zeros(0, np.float32), gen.PARAMS_BLOBS, 1)
    assert empty["n_seeds"] == 0 and empty["cluster_id"].size == 0


def test_generators_are_seeded_and_shaped():
    a = gen.single_event_10k(0)
    b = gen.single_event_10k(0)
    assert a.n == 10_000 and np.array_equal(a.x, b.x) and np.array_equal(a.energy, b.energy)
    assert a.x.dtype == np.float32 and a.layer.dtype == np.int32
    assert np.bincount(a.layer).tolist() == [1000] * 10
    assert not np.array_equal(gen.single_event_10k(1).x, a.x)
    sizes = gen.batch_sizes()
    assert sizes.size == 256 and sizes.min() >= 10_000 and sizes.max() <= 1_000_000
    irr = gen.make_event(10_000, 2, 0, "irregular")
    assert irr.n == 10_000


def test_chi_exp_within_two_ulp_of_exp(oracle_mod):
    """The oracle's fp32 exp used by the Gaussian and exponential kernels of
    Eq. 3, against float64 exp: at most 2 ULP of the fp32 result on a dense
    grid of [-86.9, 0], exactly 1 at 0, and 0 below -87."""
    a = np.concatenate([np.linspace(-86.9, 0.0, 40001), -np.logspace(-12, 0, 2001)]).astype(np.float32)
    mine = np.array([oracle_mod.chi_exp(v) for v in a], np.float64)
    ref = np.exp(a.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(mine - ref) / ulp) <= 2.0
    assert oracle_mod.chi_exp(0.0) == 1.0 and oracle_mod.chi_exp(-0.0) == 1.0
    assert oracle_mod.chi_exp(-87.5) == 0.0 and oracle_mod.chi_exp(-1e30) == 0.0


@pytest.mark.parametrize("chi,s", [(1, 1.0), (1, 2.5), (2, 0.7), (2, 3.0)])
def test_chi_rho_within_bound_of_exact(oracle_mod, chi, s):
    """rho with the Gaussian (1) or exponential (2) kernel of Eq. 3: against
    the exact float64 sum of chi(d_ij) w_j over the same neighbours, within the
    recursive-summation bound plus the per-term error of chi (2 ULP of exp,
    the fp32 argument and the product rounding): |err| <= 24 u sum|t| +
    (m-1) u sum|t|."""
    ext = (-15.0, 15.0, -15.0, 15.0)
    ev = gen.make_event(700, 1, 4, "irregular", extent=ext)
    dc = 2.0
    o = oracle_mod.run_event(ev, (dc, 3.0, 2.0, 4.0), 1, extent=ext, chi=chi, chi_param=s)
    x, y, w = ev.x, ev.y, ev.energy
    dx = x[None, :] - x[:, None]
    dy = y[None, :] - y[:, None]
    d2 = dx * dx + dy * dy
    near = d2 < np.float32(dc) * np.float32(dc)
    dd = np.hypot(x[None, :].astype(np.float64) - x[:, None], y[None, :].astype(np.float64) - y[:, None])
    chi_true = np.exp(-dd * dd / (2 * s * s)) if chi == 1 else np.exp(-dd / s)
    t = np.where(near, chi_true * w[None, :].astype(np.float64), 0.0)
    m = near.sum(1)
    exact = t.sum(1)
    u = 2.0 ** -24
    bound = (24 * u + (m - 1) * u) * np.abs(t).sum(1) + 1e-37
    assert np.all(np.abs(o["rho"].astype(np.float64) - exact) <= bound)
    # R4: the exact sum of the fp32 terms fl(chi * w), chi from the oracle's
    # own exp (pinned above), rounded once
    inv = np.float32(1.0) / (np.float32(2.0) * np.float32(s) * np.float32(s)) if chi == 1 \
        else np.float32(1.0) / np.float32(s)
    for i in range(0, ev.n, 7):
        js = np.nonzero(near[i])[0]
        arg = (d2[i, js] * inv) if chi == 1 else (np.sqrt(d2[i, js]) * inv)
        terms = np.array([np.float32(oracle_mod.chi_exp(-float(a))) for a in arg.astype(np.float32)],
                         np.float32) * w[js]
        assert o["rho"][i].view(np.uint32) == exact_rho(terms).view(np.uint32)
    # and the flat kernel is the special case chi = 1
    flat = oracle_mod.run_event(ev, (dc, 3.0, 2.0, 4.0), 1, extent=ext)
    big = oracle_mod.run_event(ev, (dc, 3.0, 2.0, 4.0), 1, extent=ext, chi=0, chi_param=0.0)
    assert np.array_equal(flat["rho"], big["rho"])
