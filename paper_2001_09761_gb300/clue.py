"""Thin ctypes binding of libclue.so (include/clue.h).

Argument marshalling only: every step of the clustering runs in the library's
CUDA kernels.  The functions ``clue_*`` mirror the C ABI one to one (pointers
are passed as ints, e.g. ``tensor.data_ptr()``); ``Clusterer`` wraps a context
with torch CUDA tensors for device memory and a torch stream.

Importing this module never falls back to anything: if libclue.so is missing
or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libclue.so"

CLUE_OK, CLUE_ERR_ARG, CLUE_ERR_INPUT, CLUE_ERR_OOM, CLUE_ERR_CUDA, CLUE_ERR_TIMEOUT, \
    CLUE_ERR_STATE = range(7)

#: Every symbol include/clue.h declares.
ABI_SYMBOLS = [
    "clue_default_opts", "clue_create", "clue_destroy", "clue_set_stream", "clue_run",
    "clue_run_batch", "clue_run_batch_host", "clue_sync", "clue_get_intermediates",
    "clue_autotune", "clue_get_tuning", "clue_set_tuning", "clue_set_profiling",
    "clue_stage_times", "clue_stage_times_back", "clue_last_launch_count", "clue_scratch_bytes", "clue_strerror",
    "clue_last_message", "clue_version", "clue_run_static", "clue_stage_event",
    "clue_server_default_opts", "clue_server_create", "clue_server_submit", "clue_server_wait",
    "clue_server_stats", "clue_server_reset_stats", "clue_server_destroy",
]


class ClueOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("x_min", ctypes.c_float), ("x_max", ctypes.c_float),
                ("y_min", ctypes.c_float), ("y_max", ctypes.c_float),
                ("max_layers", ctypes.c_int32), ("bin_size", ctypes.c_float),
                ("block_size", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("expand", ctypes.c_int32),
                ("chi", ctypes.c_int32), ("chi_param", ctypes.c_float),
                ("max_scratch_bytes", ctypes.c_int64), ("walk_limit", ctypes.c_int32),
                ("density", ctypes.c_int32)]


CLUE_EXPAND_FRONTIER, CLUE_EXPAND_CHASE = 0, 1
CLUE_DENSITY_AUTO, CLUE_DENSITY_FUSED, CLUE_DENSITY_SEPARATE = 0, 1, 2
CLUE_CHI_FLAT, CLUE_CHI_GAUSSIAN, CLUE_CHI_EXPONENTIAL = 0, 1, 2


class ClueError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        msg = f"{where}: {_strerror(code)} ({code})"
        super().__init__(msg + (f": {detail}" if detail else ""))


_lib = None
P = ctypes.c_void_p
F = ctypes.c_float
I32 = ctypes.c_int32
I64 = ctypes.c_int64


def load(path: os.PathLike | None = None):
    """Load libclue.so (raises OSError / RuntimeError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                           "(there is no fallback implementation)")
    lib = ctypes.CDLL(str(p))
    sig = {
        "clue_default_opts": (None, [ctypes.POINTER(ClueOpts)]),
        "clue_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(ClueOpts)]),
        "clue_destroy": (None, [P]),
        "clue_set_stream": (ctypes.c_int, [P, P]),
        "clue_run": (ctypes.c_int, [P, P, P, P, P, I64, F, F, F, F, P, P]),
        "clue_run_batch": (ctypes.c_int, [P, P, P, P, P, P, I32, F, F, F, F, P, P]),
        "clue_run_batch_host": (ctypes.c_int, [P, P, P, P, P, P, I32, F, F, F, F, P, P]),
        "clue_sync": (ctypes.c_int, [P]),
        "clue_get_intermediates": (ctypes.c_int, [P, P, P, P]),
        "clue_autotune": (ctypes.c_int, [P, P, P, P, P, P, I32, F, F, F, F, P, P, I32]),
        "clue_get_tuning": (I64, [P, ctypes.c_char_p, I64]),
        "clue_set_tuning": (ctypes.c_int, [P, ctypes.c_char_p]),
        "clue_set_profiling": (ctypes.c_int, [P, I32]),
        "clue_stage_times": (ctypes.c_int, [P, P, I32, ctypes.c_char_p, I64]),
        "clue_stage_times_back": (ctypes.c_int, [P, I32, P, I32, ctypes.c_char_p, I64]),
        "clue_last_launch_count": (I32, [P]),
        "clue_scratch_bytes": (I64, [P]),
        "clue_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "clue_last_message": (ctypes.c_char_p, [P]),
        "clue_version": (ctypes.c_char_p, []),
        "clue_run_static": (ctypes.c_int, [P, P, P, P, I64, F, F, F, F, F, F, F, F, I32, P, P,
                                           P]),
        "clue_stage_event": (ctypes.c_int, [P, P, P, P, I64, P, P, P, P, I64, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _strerror(code):
    try:
        return load().clue_strerror(int(code)).decode()
    except Exception:
        return "error"


# ---- one-to-one mirrors of the C ABI ---------------------------------------

def clue_default_opts() -> ClueOpts:
    o = ClueOpts()
    load().clue_default_opts(ctypes.byref(o))
    return o


def clue_create(opts: ClueOpts) -> int:
    h = P()
    rc = load().clue_create(ctypes.byref(h), ctypes.byref(opts))
    if rc:
        raise ClueError(rc, "clue_create")
    return h.value


def clue_destroy(ctx: int) -> None:
    load().clue_destroy(ctx)


def clue_set_stream(ctx, stream) -> int:
    return load().clue_set_stream(ctx, stream)


def clue_run(ctx, x, y, layer, energy, n, dc, rhoc, delta_c, delta_o, cluster_id, is_seed) -> int:
    return load().clue_run(ctx, x, y, layer, energy, n, dc, rhoc, delta_c, delta_o,
                           cluster_id, is_seed)


def _offs(offsets):
    a = np.ascontiguousarray(offsets, dtype=np.int64)
    return a, a.ctypes.data_as(P)


def clue_run_batch(ctx, x, y, layer, energy, offsets, n_events, dc, rhoc, delta_c, delta_o,
                   cluster_id, is_seed) -> int:
    a, p = _offs(offsets)
    return load().clue_run_batch(ctx, x, y, layer, energy, p, n_events, dc, rhoc, delta_c,
                                 delta_o, cluster_id, is_seed)


def clue_run_batch_host(ctx, x, y, layer, energy, offsets, n_events, dc, rhoc, delta_c,
                        delta_o, cluster_id, is_seed) -> int:
    a, p = _offs(offsets)
    return load().clue_run_batch_host(ctx, x, y, layer, energy, p, n_events, dc, rhoc,
                                      delta_c, delta_o, cluster_id, is_seed)


def clue_stage_event(x, y, layer, energy, n, dx, dy, dlayer, denergy, offset, stream) -> int:
    return load().clue_stage_event(x, y, layer, energy, n, dx, dy, dlayer, denergy, offset,
                                   stream)


def clue_sync(ctx) -> int:
    return load().clue_sync(ctx)


def clue_get_intermediates(ctx, rho, delta, nh) -> int:
    return load().clue_get_intermediates(ctx, rho, delta, nh)


def clue_autotune(ctx, x, y, layer, energy, offsets, n_events, dc, rhoc, delta_c, delta_o,
                  cluster_id, is_seed, reps) -> int:
    a, p = _offs(offsets)
    return load().clue_autotune(ctx, x, y, layer, energy, p, n_events, dc, rhoc, delta_c,
                                delta_o, cluster_id, is_seed, reps)


def clue_get_tuning(ctx) -> str:
    n = load().clue_get_tuning(ctx, None, 0)
    buf = ctypes.create_string_buffer(int(n))
    load().clue_get_tuning(ctx, buf, n)
    return buf.value.decode()


def clue_set_tuning(ctx, text: str) -> int:
    return load().clue_set_tuning(ctx, text.encode())


def clue_set_profiling(ctx, on: bool) -> int:
    return load().clue_set_profiling(ctx, 1 if on else 0)


def clue_stage_times(ctx, back=0):
    """[(kernel name, ms), ...] of the profiled run `back` runs before the
    last one (0 = the last), in launch order."""
    ms = (ctypes.c_float * 64)()
    names = ctypes.create_string_buffer(2048)
    n = load().clue_stage_times_back(ctx, int(back), ms, 64, names, 2048)
    if n < 0:
        raise ClueError(-n, "clue_stage_times_back")
    return list(zip(names.value.decode().split(","), list(ms)[:n]))


#: Pipeline step of each profiled kernel (S1 grid fill .. S5 expansion).
STAGE_OF = {"fill_layers": "grid_fill", "scan_segs": "grid_fill", "fill_place": "grid_fill",
            "fill_cells": "grid_fill",
            "fill_count": "grid_fill", "scan_cells": "grid_fill", "fill_scatter": "grid_fill",
            "fill_canon": "grid_fill", "rho": "density", "nh_delta": "density",
            "density": "density", "nh_rest": "density",
            "scan_hits": "decide_followers", "link": "decide_followers",
            "seed_codes": "decide_followers", "assign": "expand",
            "expand_level": "expand", "complete": "expand", "jump": "expand"}


def clue_last_launch_count(ctx) -> int:
    return int(load().clue_last_launch_count(ctx))


def clue_scratch_bytes(ctx) -> int:
    return int(load().clue_scratch_bytes(ctx))


def clue_strerror(code) -> str:
    return load().clue_strerror(int(code)).decode()


def clue_last_message(ctx) -> str:
    return load().clue_last_message(ctx).decode()


def clue_version() -> str:
    return load().clue_version().decode()


#: Largest event clue_run_static accepts (CLUE_STATIC_MAX_HITS).
CLUE_STATIC_MAX_HITS = 65536
#: Most grid cells (layers x bins per layer) clue_run_static's array holds.
CLUE_STATIC_MAX_CELLS = 1048576


def clue_run_static(x, y, layer, energy, n, dc, rhoc, delta_c, delta_o, x_min, x_max, y_min,
                    y_max, max_layers, cluster_id, is_seed, stream) -> int:
    """Single event with all scratch in the library's fixed device array
    (no allocation); synchronous on ``stream``."""
    return load().clue_run_static(x, y, layer, energy, n, dc, rhoc, delta_c, delta_o, x_min,
                                  x_max, y_min, y_max, max_layers, cluster_id, is_seed, stream)


# ---- torch-facing wrapper ---------------------------------------------------

def _check(rc, where, ctx=None):
    if rc:
        raise ClueError(rc, where, clue_last_message(ctx) if ctx else "")


class Clusterer:
    """A CLUE context on one GPU, with torch tensors for device memory.

    ``params`` everywhere is (d_c, rho_c, delta_c, delta_o).  Work is queued on
    the clusterer's own torch stream, ordered after the caller's current
    stream; results are ordered before later work on the current stream.
    """

    def __init__(self, device: int = 0, extent=(-250.0, 250.0, -250.0, 250.0),
                 max_layers: int = 128, bin_size: float = 0.0, block_size: int = 0,
                 use_graphs: bool = True, expand: int = CLUE_EXPAND_CHASE,
                 chi: int = CLUE_CHI_FLAT, chi_param: float = 0.0,
                 max_scratch_bytes: int = 0, walk_limit: int = 0,
                 density: int = CLUE_DENSITY_AUTO):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.device)
        o = clue_default_opts()
        o.device = device
        o.x_min, o.x_max, o.y_min, o.y_max = (float(v) for v in extent)
        o.max_layers = int(max_layers)
        o.bin_size = float(bin_size)
        o.block_size = int(block_size)
        o.use_graphs = 1 if use_graphs else 0
        o.stream = self.stream.cuda_stream
        o.expand = int(expand)
        o.chi = int(chi)
        o.chi_param = float(chi_param)
        o.max_scratch_bytes = int(max_scratch_bytes)
        o.walk_limit = int(walk_limit)
        o.density = int(density)
        self.max_layers = max_layers
        self.ctx = clue_create(o)
        self._last_n = 0
        # reused events that order the clusterer's stream after the caller's
        # current stream and back (one record and one wait each way per call)
        self._ev_in = torch.cuda.Event()
        self._ev_out = torch.cuda.Event()

    def close(self):
        if getattr(self, "ctx", None):
            clue_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _begin(self, tensors):
        cur = self.torch.cuda.current_stream(self.device)
        self._ev_in.record(cur)
        self.stream.wait_event(self._ev_in)
        for x in tensors:
            x.record_stream(self.stream)
        self._cur = cur

    def _end(self):
        self._ev_out.record(self.stream)
        self._cur.wait_event(self._ev_out)

    def _as(self, a, dtype):
        t = self.torch
        if isinstance(a, t.Tensor) and a.dtype == dtype and a.device == self.device and \
                a.is_contiguous():
            return a
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        a = a.to(device=self.device, dtype=dtype)
        return a.contiguous()

    def run(self, x, y, layer, energy, params, out=None):
        """Cluster one event; returns (cluster_id int32, is_seed uint8) tensors."""
        t = self.torch
        x, y = self._as(x, t.float32), self._as(y, t.float32)
        layer, energy = self._as(layer, t.int32), self._as(energy, t.float32)
        n = x.numel()
        cid, seed = out if out is not None else (
            t.empty(n, dtype=t.int32, device=self.device),
            t.empty(n, dtype=t.uint8, device=self.device))
        self._begin([x, y, layer, energy, cid, seed])
        rc = clue_run(self.ctx, x.data_ptr(), y.data_ptr(), layer.data_ptr(),
                      energy.data_ptr(), n, *[float(v) for v in params], cid.data_ptr(),
                      seed.data_ptr())
        _check(rc, "clue_run", self.ctx)
        self._end()
        self._last_n = n
        return cid, seed

    def run_batch(self, x, y, layer, energy, offsets, params, out=None):
        """Cluster a batch of events (concatenated arrays, host int64 offsets)."""
        t = self.torch
        x, y = self._as(x, t.float32), self._as(y, t.float32)
        layer, energy = self._as(layer, t.int32), self._as(energy, t.float32)
        offsets = np.ascontiguousarray(offsets, np.int64)
        n = x.numel()
        cid, seed = out if out is not None else (
            t.empty(n, dtype=t.int32, device=self.device),
            t.empty(n, dtype=t.uint8, device=self.device))
        self._begin([x, y, layer, energy, cid, seed])
        rc = clue_run_batch(self.ctx, x.data_ptr(), y.data_ptr(), layer.data_ptr(),
                            energy.data_ptr(), offsets, len(offsets) - 1,
                            *[float(v) for v in params], cid.data_ptr(), seed.data_ptr())
        _check(rc, "clue_run_batch", self.ctx)
        self._end()
        self._last_n = n
        return cid, seed

    def run_batch_host(self, x, y, layer, energy, offsets, params, out=None):
        """Host (numpy) arrays in and out; copies happen inside the call."""
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        layer = np.ascontiguousarray(layer, np.int32)
        energy = np.ascontiguousarray(energy, np.float32)
        offsets = np.ascontiguousarray(offsets, np.int64)
        n = x.shape[0]
        cid, seed = out if out is not None else (np.empty(n, np.int32), np.empty(n, np.uint8))
        self._ev_in.record(self.torch.cuda.current_stream(self.device))
        self.stream.wait_event(self._ev_in)
        ptr = lambda a: a.ctypes.data
        rc = clue_run_batch_host(self.ctx, ptr(x), ptr(y), ptr(layer), ptr(energy), offsets,
                                 len(offsets) - 1, *[float(v) for v in params], ptr(cid),
                                 ptr(seed))
        _check(rc, "clue_run_batch_host", self.ctx)
        self._last_n = n
        return cid, seed

    def sync(self):
        _check(clue_sync(self.ctx), "clue_sync", self.ctx)

    def intermediates(self):
        """(rho, delta, nh) of the last run as device tensors (nh per event)."""
        t = self.torch
        n = self._last_n
        rho = t.empty(n, dtype=t.float32, device=self.device)
        delta = t.empty(n, dtype=t.float32, device=self.device)
        nh = t.empty(n, dtype=t.int32, device=self.device)
        self._begin([rho, delta, nh])
        _check(clue_get_intermediates(self.ctx, rho.data_ptr(), delta.data_ptr(), nh.data_ptr()),
               "clue_get_intermediates", self.ctx)
        self._end()
        return rho, delta, nh

    def autotune(self, x, y, layer, energy, offsets, params, reps=3):
        t = self.torch
        x, y = self._as(x, t.float32), self._as(y, t.float32)
        layer, energy = self._as(layer, t.int32), self._as(energy, t.float32)
        n = x.numel()
        cid = t.empty(n, dtype=t.int32, device=self.device)
        seed = t.empty(n, dtype=t.uint8, device=self.device)
        self._begin([x, y, layer, energy, cid, seed])
        offsets = np.ascontiguousarray(offsets, np.int64)
        _check(clue_autotune(self.ctx, x.data_ptr(), y.data_ptr(), layer.data_ptr(),
                             energy.data_ptr(), offsets, len(offsets) - 1,
                             *[float(v) for v in params], cid.data_ptr(), seed.data_ptr(), reps),
               "clue_autotune", self.ctx)
        self._end()
        return clue_get_tuning(self.ctx)

    def set_profiling(self, on=True):
        _check(clue_set_profiling(self.ctx, on), "clue_set_profiling", self.ctx)

    def kernel_times(self, back=0):
        """{kernel: ms} of the last profiled run, or of the one `back` runs
        before it (repeated launches summed)."""
        out = {}
        for k, v in clue_stage_times(self.ctx, back):
            out[k] = out.get(k, 0.0) + v
        return out

    def stage_times(self):
        """{pipeline step: ms} of the last profiled run."""
        out = {}
        for k, v in clue_stage_times(self.ctx):
            st = STAGE_OF.get(k, k)
            out[st] = out.get(st, 0.0) + v
        return out

    def launch_count(self):
        return clue_last_launch_count(self.ctx)

    @property
    def tuning(self):
        return clue_get_tuning(self.ctx)

    @tuning.setter
    def tuning(self, text):
        _check(clue_set_tuning(self.ctx, text), "clue_set_tuning", self.ctx)
