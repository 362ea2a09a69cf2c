"""Exact sums of fp32 values and their correct rounding to fp32, written from
the IEEE 754 definition (test infrastructure, independent of the oracle).

``round_to_f32(v)`` returns the fp32 value nearest to the rational ``v``,
ties to the one with an even significand, by comparing ``v`` with its two
fp32 neighbours; ``exact_rho(w)`` is reading R4 of the density: the exact sum
of fp32 terms rounded once.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

_MAX = Fraction(float(np.finfo(np.float32).max))
_TOP = _MAX + Fraction(2) ** (127 - 24)  # halfway to 2^128: rounds to inf


def round_to_f32(v: Fraction) -> np.float32:
    if v == 0:
        return np.float32(0.0)
    if v < 0:
        return np.float32(-round_to_f32(-v))
    if v >= _TOP:
        return np.float32(np.inf)
    if v > _MAX:  # between the largest finite value and the halfway point
        return np.float32(_MAX)
    f = np.float32(float(v))  # within an ulp or two; adjust below
    while Fraction(float(f)) > v:
        f = np.nextafter(f, np.float32(-np.inf))
    while Fraction(float(np.nextafter(f, np.float32(np.inf)))) <= v:
        f = np.nextafter(f, np.float32(np.inf))
    lo, hi = f, np.nextafter(f, np.float32(np.inf))  # lo <= v < hi
    dlo, dhi = v - Fraction(float(lo)), Fraction(float(hi)) - v
    if dlo < dhi:
        return lo
    if dhi < dlo:
        return hi
    return lo if int(lo.view(np.uint32)) % 2 == 0 else hi


def exact_rho(terms) -> np.float32:
    """The exact sum of the fp32 terms, rounded once (R4)."""
    return round_to_f32(sum((Fraction(float(t)) for t in np.asarray(terms, np.float32)),
                            Fraction(0)))


def adversarial_weights(rng, n):
    """fp32 weights that make fp32 running sums order-dependent: magnitudes
    from 1e-38 to 1e30, both signs, subnormals, zeros and exact cancellations."""
    kind = rng.integers(0, 6, n)
    w = np.where(kind == 0, rng.exponential(1.0, n),
        np.where(kind == 1, 10.0 ** rng.uniform(-38, 30, n),
        np.where(kind == 2, -rng.exponential(1.0, n),
        np.where(kind == 3, rng.integers(1, 2 ** 20, n) * 2.0 ** -149,
        np.where(kind == 4, 0.0, 1.0 + rng.integers(0, 8, n) * 2.0 ** -24)))))
    return w.astype(np.float32)
