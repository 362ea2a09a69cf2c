"""O(n^2) brute-force CLUE in numpy: the definitions with no spatial index.

A test-only pin for the oracle.  It follows the paper's definitions directly:
N_d(i) is every hit of i's layer with d_ij < d (Eq. 2 with Omega = the whole
layer, allowed since Omega only has to contain N), rho by Eq. 3 with the flat
kernel as the exact rational sum rounded once to fp32 (reading R4),
nh/delta by Eq. 4 with the smaller index winning
a distance tie, the seed/outlier rule of Sec. 2.2, and cluster ids through the
recursion "a follower inherits the id of its nearest-higher" (the closed form
of passing ids down the follower chains) rather than a stack.

Distances are the oracle's fp32 reading: dx, dy, their squares and the sum
each rounded to float32 on its own (numpy float32 ufuncs do exactly that).
"""
from __future__ import annotations

import sys

import numpy as np

from exactsum import exact_rho


def brute_clue(x, y, layer, w, params):
    dc, rhoc, delta_c, delta_o = (np.float32(v) for v in params)
    dm = max(delta_o, delta_c)
    dc2, dm2 = dc * dc, dm * dm
    dcs2, dos2 = delta_c * delta_c, delta_o * delta_o
    x = np.asarray(x, np.float32)
    y = np.asarray(y, np.float32)
    w = np.asarray(w, np.float32)
    layer = np.asarray(layer)
    n = x.shape[0]
    rho = np.zeros(n, np.float32)
    d2best = np.full(n, np.inf, np.float32)
    nh = np.full(n, -1, np.int64)
    for l in np.unique(layer):
        idx = np.nonzero(layer == l)[0]          # ascending global indices
        xl, yl, wl = x[idx], y[idx], w[idx]
        dx = xl[None, :] - xl[:, None]             # [i, j] = x_j - x_i, fp32
        dy = yl[None, :] - yl[:, None]
        d2 = (dx * dx) + (dy * dy)                 # fp32, separately rounded
        near = d2 < dc2
        r = np.array([exact_rho(wl[near[i]]) for i in range(idx.shape[0])], np.float32)
        rho[idx] = r
        cand = (d2 < dm2) & (r[None, :] > r[:, None])
        masked = np.where(cand, d2, np.float32(np.inf))
        j = np.argmin(masked, axis=1)              # first (smallest j) minimum
        has = cand.any(axis=1)
        d2best[idx[has]] = masked[has, j[has]]
        nh[idx[has]] = idx[j[has]]
    seed = (rho > rhoc) & (d2best > dcs2)
    outl = (rho < rhoc) & (d2best > dos2)
    sid = np.full(n, -1, np.int64)
    sid[seed] = np.arange(int(seed.sum()))
    cid = np.full(n, -2, np.int64)

    sys.setrecursionlimit(max(10000, 4 * n))

    def resolve(i):
        if cid[i] != -2:
            return cid[i]
        if seed[i]:
            v = sid[i]
        elif outl[i] or nh[i] < 0:
            v = -1
        else:
            v = resolve(nh[i])
        cid[i] = v
        return v

    for i in range(n):
        resolve(i)
    return dict(rho=rho, delta2=d2best, nh=nh.astype(np.int32), is_seed=seed.astype(np.uint8),
                is_outlier=outl.astype(np.uint8), cluster_id=cid.astype(np.int32))
