"""Python loader for the CPU oracle (``clue_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the CUDA library.  The
library itself never imports this package.

``build()`` compiles the oracle with gcc (``-O2 -ffp-contract=off``, no fast
math, so every fp32 operation rounds on its own, as the oracle's readings
require).  ``run()`` clusters one event and returns its per-hit arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = _DIR / "clue_oracle.c"
_LIB = _DIR / "liboracle.so"
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]


def build(force: bool = False) -> Path:
    """Compile the oracle into oracle/liboracle.so (skipped when up to date)."""
    if not force and _LIB.exists() and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB.with_suffix(f".so.{os.getpid()}")
    subprocess.run(["gcc", *CFLAGS, str(_SRC), "-o", str(tmp), "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        f = lib.oracle_clue_chi
        P = ctypes.c_void_p
        F = ctypes.c_float
        f.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int32, F, F, F, F, F, F, F, F,
                      ctypes.c_int32, F, P, P, P, P, P, P, P, P]
        f.restype = ctypes.c_int
        lib.oracle_chi_exp.argtypes = [F]
        lib.oracle_chi_exp.restype = F
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def chi_exp(a: float) -> float:
    """The oracle's fp32 exp(a) for a <= 0 (used by the Gaussian and
    exponential kernels)."""
    return float(_load().oracle_chi_exp(float(a)))


def run(x, y, layer, energy, params, n_layers, extent=(-250.0, 250.0, -250.0, 250.0),
        chi=0, chi_param=0.0):
    """Cluster one event; returns a dict of numpy arrays (see clue_oracle.c).

    params = (d_c, rho_c, delta_c, delta_o); chi = 0 flat, 1 Gaussian, 2
    exponential kernel with width chi_param.  Raises ValueError on the
    oracle's error codes.
    """
    lib = _load()
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    layer = np.ascontiguousarray(layer, np.int32)
    energy = np.ascontiguousarray(energy, np.float32)
    n = x.shape[0]
    out = dict(rho=np.empty(n, np.float32), delta=np.empty(n, np.float32),
               delta2=np.empty(n, np.float32), nh=np.empty(n, np.int32),
               is_seed=np.empty(n, np.uint8), is_outlier=np.empty(n, np.uint8),
               cluster_id=np.empty(n, np.int32))
    k = ctypes.c_int64(0)
    dc, rhoc, delta_c, delta_o = params
    rc = lib.oracle_clue_chi(n, _ptr(x), _ptr(y), _ptr(layer), _ptr(energy), int(n_layers),
                         *[float(v) for v in extent], float(dc), float(rhoc),
                         float(delta_c), float(delta_o), int(chi), float(chi_param),
                         _ptr(out["rho"]), _ptr(out["delta"]), _ptr(out["delta2"]),
                         _ptr(out["nh"]), _ptr(out["is_seed"]), _ptr(out["is_outlier"]),
                         _ptr(out["cluster_id"]), ctypes.byref(k))
    if rc != 0:
        raise ValueError(f"oracle_clue returned {rc}")
    out["n_seeds"] = int(k.value)
    return out


def run_event(ev, params, n_layers, extent=(-250.0, 250.0, -250.0, 250.0), chi=0,
              chi_param=0.0):
    return run(ev.x, ev.y, ev.layer, ev.energy, params, n_layers, extent, chi, chi_param)


def run_batch(x, y, layer, energy, offsets, params, n_layers,
              extent=(-250.0, 250.0, -250.0, 250.0)):
    """Cluster each event of a concatenated batch on its own; per-event ids."""
    outs = [run(x[a:b], y[a:b], layer[a:b], energy[a:b], params, n_layers, extent)
            for a, b in zip(offsets[:-1], offsets[1:])]
    keys = ["rho", "delta", "delta2", "nh", "is_seed", "is_outlier", "cluster_id"]
    res = {k: (np.concatenate([o[k] for o in outs]) if outs else np.zeros(0))
           for k in keys}
    res["n_seeds"] = [o["n_seeds"] for o in outs]
    return res
