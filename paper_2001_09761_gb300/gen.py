"""Seeded synthetic calorimeter events for the CLUE hot path.

This module only draws random numbers: it holds none of the clustering
arithmetic, so both the CPU oracle tests and the GPU path can take their inputs
from it without sharing any of the method.

An event is a structure of arrays over its hits (the layout of Sec. 3 of the
paper): ``x``, ``y`` float32 (cm), ``layer`` int32, ``energy`` float32 (the
weight w of Eq. 3).  The paper's own timing workload (Sec. 4.2) is "100 layers,
Gaussian energy blobs plus uniform noise"; the recipes below reproduce that
shape with the sizes of the benchmark configurations:

* ``blobs``: per layer, ``round(0.09 * h)`` Gaussian blobs of 10 hits each
  (uniform centres in the extent, sigma 1 cm, energy ~ Exp(mean 1)), the rest
  uniform noise hits with energy ~ U(0, 0.1).
* ``irregular``: per layer, 30% uniform noise and 70% cluster hits: half of them
  in elongated ellipses (sigma 0.5 x 2.5 cm, random orientation, 20 hits each),
  half in rings (radius U(3.75, 4.25) cm, 40 hits each); 10% of the cluster hits
  are moved into 4 dense discs of radius 5 cm (hotspots).  Energy ~ lognormal(0, 1).
* ``paper``: Sec. 4.2's parameters: unit weights, Gaussian blobs with sigma 3 cm,
  5% uniform noise.

After generation the hits of an event are shuffled by a seeded permutation, so
no consumer can rely on any input order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

EXTENT = (-250.0, 250.0, -250.0, 250.0)


@dataclass
class Event:
    x: np.ndarray
    y: np.ndarray
    layer: np.ndarray
    energy: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _split_per_layer(n: int, n_layers: int) -> np.ndarray:
    """Hits per layer: n spread as evenly as possible over n_layers."""
    base = n // n_layers
    h = np.full(n_layers, base, dtype=np.int64)
    h[: n - base * n_layers] += 1
    return h


def _uniform(rng, k, extent):
    x0, x1, y0, y1 = extent
    return rng.uniform(x0, x1, k), rng.uniform(y0, y1, k)


def _blob_layer(rng, h, extent, hits_per_blob=10, blob_frac=0.9, sigma=1.0,
                unit_weight=False):
    nb = int(round(blob_frac * h / hits_per_blob))
    nb = min(nb, h // hits_per_blob)
    nblob_hits = nb * hits_per_blob
    cx, cy = _uniform(rng, nb, extent)
    bx = np.repeat(cx, hits_per_blob) + sigma * rng.standard_normal(nblob_hits)
    by = np.repeat(cy, hits_per_blob) + sigma * rng.standard_normal(nblob_hits)
    nn = h - nblob_hits
    nx, ny = _uniform(rng, nn, extent)
    if unit_weight:
        e = np.ones(h)
    else:
        e = np.concatenate([rng.exponential(1.0, nblob_hits), rng.uniform(0.0, 0.1, nn)])
    return np.concatenate([bx, nx]), np.concatenate([by, ny]), e


def _irregular_layer(rng, h, extent):
    n_noise = int(round(0.3 * h))
    n_clu = h - n_noise
    n_hot = int(round(0.1 * n_clu))
    n_shape = n_clu - n_hot
    n_ell_hits = n_shape // 2
    n_ring_hits = n_shape - n_ell_hits
    xs, ys = [], []
    # ellipses: sigma_minor 0.5, sigma_major 2.5 (axis ratio 1:5), 20 hits each
    ne = (n_ell_hits + 19) // 20
    cx, cy = _uniform(rng, ne, extent)
    th = rng.uniform(0.0, math.pi, ne)
    a = 2.5 * rng.standard_normal(ne * 20)
    b = 0.5 * rng.standard_normal(ne * 20)
    c, s = np.repeat(np.cos(th), 20), np.repeat(np.sin(th), 20)
    xs.append((np.repeat(cx, 20) + c * a - s * b)[:n_ell_hits])
    ys.append((np.repeat(cy, 20) + s * a + c * b)[:n_ell_hits])
    # rings: radius U(3.75, 4.25) around 4 cm, 40 hits each
    nr = (n_ring_hits + 39) // 40
    cx, cy = _uniform(rng, nr, extent)
    r = rng.uniform(3.75, 4.25, nr * 40)
    phi = rng.uniform(0.0, 2 * math.pi, nr * 40)
    xs.append((np.repeat(cx, 40) + r * np.cos(phi))[:n_ring_hits])
    ys.append((np.repeat(cy, 40) + r * np.sin(phi))[:n_ring_hits])
    # hotspots: 4 discs of radius 5 cm, uniform in the disc
    hx, hy = _uniform(rng, 4, extent)
    which = rng.integers(0, 4, n_hot)
    rr = 5.0 * np.sqrt(rng.uniform(0.0, 1.0, n_hot))
    pp = rng.uniform(0.0, 2 * math.pi, n_hot)
    xs.append(hx[which] + rr * np.cos(pp))
    ys.append(hy[which] + rr * np.sin(pp))
    nx, ny = _uniform(rng, n_noise, extent)
    xs.append(nx)
    ys.append(ny)
    e = rng.lognormal(0.0, 1.0, h)
    return np.concatenate(xs), np.concatenate(ys), e


def make_event(n: int, n_layers: int, seed: int, kind: str = "blobs",
               extent=EXTENT) -> Event:
    """One event of n hits over n_layers layers, drawn from recipe ``kind``."""
    rng = np.random.default_rng(seed)
    hs = _split_per_layer(n, n_layers)
    X, Y, L, E = [], [], [], []
    for l, h in enumerate(hs):
        h = int(h)
        if h == 0:
            continue
        if kind == "blobs":
            x, y, e = _blob_layer(rng, h, extent)
        elif kind == "irregular":
            x, y, e = _irregular_layer(rng, h, extent)
        elif kind == "paper":
            x, y, e = _blob_layer(rng, h, extent, hits_per_blob=10, blob_frac=0.95,
                                  sigma=3.0, unit_weight=True)
        elif kind == "uniform":
            x, y = _uniform(rng, h, extent)
            e = rng.exponential(1.0, h)
        else:
            raise ValueError(f"unknown event kind {kind!r}")
        X.append(x)
        Y.append(y)
        L.append(np.full(h, l, dtype=np.int32))
        E.append(e)
    if not X:
        z = np.zeros(0, np.float32)
        return Event(z, z.copy(), np.zeros(0, np.int32), z.copy())
    perm = rng.permutation(n)
    return Event(np.concatenate(X).astype(np.float32)[perm],
                 np.concatenate(Y).astype(np.float32)[perm],
                 np.concatenate(L).astype(np.int32)[perm],
                 np.concatenate(E).astype(np.float32)[perm])


# --- the benchmark workloads -------------------------------------------------

#: CLUE parameters (d_c, rho_c, delta_c, delta_o) of each workload.
PARAMS_BLOBS = (2.0, 2.0, 2.0, 4.0)
PARAMS_IRREGULAR = (2.0, 3.0, 2.0, 4.0)
#: Sec. 4.2 of the paper: d_c = 3, rho_c = 8, delta_c = delta_o = 5.
PARAMS_PAPER = (3.0, 8.0, 5.0, 5.0)


def single_event_10k(seed: int = 0) -> Event:
    """10 layers x 1,000 hits, blob/noise recipe (the small workload)."""
    return make_event(10_000, 10, seed, "blobs")


def scaling_event(hits_per_layer: int, seed: int) -> Event:
    """100 layers x hits_per_layer hits (0.1M-1M hits), blob/noise recipe."""
    return make_event(100 * hits_per_layer, 100, seed, "blobs")


def batch_sizes(n_events: int = 256, lo: float = 1e4, hi: float = 1e6,
                seed: int = 0) -> np.ndarray:
    """Event sizes log-uniform in [lo, hi], drawn with ``seed``."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n_events)).astype(np.int64)


def uneven_batch(n_events: int = 256, lo: float = 1e4, hi: float = 1e6,
                 size_seed: int = 0, first_event_seed: int = 1000):
    """Events of log-uniform size over 100 layers; event e uses seed 1000+e."""
    sizes = batch_sizes(n_events, lo, hi, size_seed)
    return [make_event(int(n), 100, first_event_seed + e, "blobs")
            for e, n in enumerate(sizes)]


def irregular_event(seed: int = 0, hits_per_layer: int = 100_000,
                    n_layers: int = 50) -> Event:
    """50 layers x 100k hits of ellipses, rings, hotspots and 30% noise."""
    return make_event(hits_per_layer * n_layers, n_layers, seed, "irregular")


def concat(events):
    """Concatenate events into one batch: SoA arrays plus int64 offsets[E+1]."""
    offs = np.zeros(len(events) + 1, np.int64)
    offs[1:] = np.cumsum([ev.n for ev in events])
    cat = lambda f, dt: (np.concatenate([getattr(ev, f) for ev in events]).astype(dt)
                         if events else np.zeros(0, dt))
    return (cat("x", np.float32), cat("y", np.float32), cat("layer", np.int32),
            cat("energy", np.float32), offs)


def poisson_arrivals(rate_per_s: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
