#!/usr/bin/env python3
"""CLUE throughput on GB300: batched vs per-event Mhits/s, event latency.

A step is one pass of the whole pipeline (grid fill, rho, nh/delta, decision
and follower lists, expansion) over one batch of synthetic events: by default
256 events of log-uniform size 10k-1M hits over 100 layers (blob/noise recipe,
d_c = 2, rho_c = 2, delta_c = 2, delta_o = 4).  The batch (~1 GB of input) is
larger than the 129 MB L2, so no cache flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2001_09761_gb300 import gen  # noqa: E402

PARAMS = gen.PARAMS_BLOBS
METRIC = "CLUE Mhits/s on 1 GB300, batched vs per-event; p50/p99 event latency"
WORKLOAD = ("256 uneven events in one batch: hits log-uniform 10k-1M, 100 layers, "
            "blob/noise generator, d_c=2 rho_c=2 delta_c=2 delta_o=4")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_workload(rank: int, n_events: int, lo: float, hi: float):
    from paper_2001_09761_gb300 import replicas
    return gen.uneven_batch(n_events, lo, hi, *replicas.weak_seeds(rank))


def cpu_oracle_sample(events, budget_s: float):
    """Time the oracle on events of the workload until ~budget_s of CPU."""
    import oracle
    oracle.build()
    done_hits, t_total, used = 0, 0.0, 0
    order = np.argsort([ev.n for ev in events])  # small and mid events first
    for i in order[:: max(1, len(order) // 16)]:
        ev = events[i]
        t0 = time.perf_counter()
        oracle.run_event(ev, PARAMS, 100)
        t_total += time.perf_counter() - t0
        done_hits += ev.n
        used += 1
        if t_total > budget_s:
            break
    return done_hits / t_total / 1e6, f"{used} events, {done_hits} hits, {t_total:.1f} s"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    events = make_workload(0, args.events, args.lo, args.hi)
    import oracle
    oracle.build()
    # each step: a fixed bounded sample of the workload, events spread over the
    # size range, about 90 s of oracle time over all steps (~1 Mhit/s per core)
    order = np.argsort([ev.n for ev in events])
    budget_hits = max(200_000, int(1e6 * 90.0 / max(1, args.steps)))
    sample, hits = [], 0
    for i in order[:: 8]:
        if hits + events[i].n > budget_hits and sample:
            continue
        sample.append(events[i])
        hits += events[i].n
    for _ in range(args.warmup):
        oracle.run_event(sample[0], PARAMS, 100)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for ev in sample:
            oracle.run_event(ev, PARAMS, 100)
    dt = time.perf_counter() - t0
    value = hits * args.steps / dt / 1e6
    desc = (f"{len(sample)} of {len(events)} events (from every 8th by size, within "
            f"{budget_hits} hits), {hits} hits per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mhits/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle on a bounded sample)", "global_batch": len(sample),
                   "parallelism": "single-thread CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "Mhits/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "Mhits/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# Algorithmic bytes per hit of each kernel: every array the step needs is
# read once and every result written once (no re-reads, no scratch beyond
# the stage's own outputs).
ALG_BYTES = {
    "fill_layers": 4,                  # layer in (out: one int per tile and layer)
    "fill_place": 16 + 16 + 2,         # x, y, w, layer in; layered record, 16-bit cell out
    "fill_cells": 16 + 2 + 16 + 4 + 4,  # layered record, cell in; sorted record, layer, id out
    "fill_count": 16 + 4 + 4 + 4,      # x, y, w, layer in; cell, rank, cell count out
    "fill_scatter": 4 + 4 + 4 + 4,     # cell, rank, cell start in; hit id out
    "fill_canon": 4 + 16 + 16 + 4,     # id, packed record in; sorted hit, layer out
    "rho": 16 + 4 + 4,                 # x, y, w, id, layer in; rho out
    "nh_delta": 16 + 4 + 4 + 8,        # x, y, rho, id, layer in; code, (delta^2, nh) out
    "density": 16 + 4 + 4 + 4 + 4 + 8,  # x, y, w, layer, id in; rho, code, (delta^2, nh) out
    "nh_rest": 0,                      # nothing unless a tile is dense or its band too long
    "link": 4 + 4 + 4 + 1,             # code, seed rank in; id, seed flag out
    "seed_codes": 0,                   # seed bits and word ranks in (N/8 B), seeds' codes out
    "assign": 4 + 4 + 1,               # code, the nh's code in; id, seed flag out
    "expand_level": 8 + 4 + 4 + 4,     # list range, parent id, follower in; id out
    "complete": 4 + 4,                 # id in, id out
    "jump": 0,                         # nothing unless a chain outruns the bounded walk
}


# The staged floor per pipeline step, in bytes per hit (each step reads what
# it needs once and writes its result once, at minimal width): S1 grid fill
# 12 B read + 4 B index written; S2 rho 12 B gathered + 4 B written; S3
# nh/delta 12 B + 4 B rho read, 8 B (nh, delta^2) written; S4 decision 8 B
# read + 5 B written + 8 B follower lists; S5 expansion 8 B.  85 B/hit in all;
# the compulsory input and output alone are 16 + 5 = 21 B/hit.
STAGED_BYTES = {"S1": 16, "S2": 16, "S3": 24, "S4": 21, "S5": 8}
STEP_OF_KERNEL = {"fill_layers": "S1", "fill_place": "S1", "fill_cells": "S1",
                  "fill_count": "S1", "fill_scatter": "S1", "fill_canon": "S1",
                  "rho": "S2", "nh_delta": "S3", "density": "S2+S3", "nh_rest": "S3",
                  "scan_hits": "S4", "link": "S4", "seed_codes": "S4", "assign": "S4+S5",
                  "expand_level": "S5", "complete": "S5", "jump": "S5"}
COMPULSORY_BYTES = 21
STAGED_TOTAL = sum(STAGED_BYTES.values())


def staged_bytes(kernel):
    """The staged-floor bytes per hit of the step(s) a kernel carries out."""
    return sum(STAGED_BYTES[s] for s in STEP_OF_KERNEL[kernel].split("+"))


def parse_traffic():
    """Per-kernel (DRAM bytes per hit, source hash, issue-active share) from the
    committed ncu summary, keyed by kernel."""
    p = ROOT / "profiles" / "traffic.md"
    out = {}
    if not p.exists():
        return out
    for line in p.read_text().splitlines():
        f = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(f) >= 4 and f[0] in ALG_BYTES:
            try:
                issue = float(f[4]) / 100 if len(f) >= 5 else None
                out[f[0]] = (float(f[1]), f[3], issue)
            except ValueError:
                pass
    return out


# Host-side sources: a change there leaves the kernels' traffic unchanged.
HOST_SOURCES = {"clue_api.cu", "clue_static.cu", "clue_serve.cu", "serve_core.cpp",
                "serve_core.h"}


def source_hash():
    """Hash of the kernel sources' code (every file of csrc but the host-side
    ones), comments and whitespace removed, so that only a change to kernel
    code invalidates a traffic capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2001_09761_gb300" / "csrc").glob("*")):
        if f.name in HOST_SOURCES:
            continue
        code = re.sub(r"/\*.*?\*/", " ", f.read_text(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(f.name.encode() + b"\0" + " ".join(code.split()).encode())
    return h.hexdigest()[:12]


def timed_runs(cl, fn, reps):
    """Latency of `reps` synchronous calls (ms list)."""
    lat = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        cl.sync()
        lat.append((time.perf_counter() - t0) * 1e3)
    return lat


def extra_configs(torch, clue, tuning, dev, args):
    """The other workloads: each reported as Mhits/s (and latency)."""
    res = {}
    def single(ev, layers, params, reps, key):
        cl = clue.Clusterer(device=dev.index, extent=gen.EXTENT, max_layers=layers)
        cl.tuning = tuning
        x, y = torch.from_numpy(ev.x).to(dev), torch.from_numpy(ev.y).to(dev)
        l, e = torch.from_numpy(ev.layer).to(dev), torch.from_numpy(ev.energy).to(dev)
        cid = torch.empty(ev.n, dtype=torch.int32, device=dev)
        seed = torch.empty(ev.n, dtype=torch.uint8, device=dev)
        run = lambda: cl.run(x, y, l, e, params, out=(cid, seed))
        for _ in range(3):
            run()
        cl.sync()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(cl.stream)
        for _ in range(reps):
            run()
        s1.record(cl.stream)
        s1.synchronize()
        ms = s0.elapsed_time(s1) / reps
        lat = np.array(timed_runs(cl, run, reps))
        cl.close()
        return {"mhits_per_s": ev.n / (ms * 1e-3) / 1e6, "device_ms": ms,
                "latency_p50_ms": float(np.percentile(lat, 50)),
                "latency_p99_ms": float(np.percentile(lat, 99)), "hits": ev.n}

    res["single_10k"] = single(gen.single_event_10k(0), 10, PARAMS, 200, "c1")
    sweep = {}
    for h in range(1000, 10001, 3000 if args.quick else 1000):
        vals = [single(gen.scaling_event(h, s), 100, PARAMS, 10, "c2")["mhits_per_s"]
                for s in range(args.sweep_seeds)]
        sweep[str(100 * h)] = float(np.median(vals))
    res["scaling_sweep_median_mhits_per_s"] = sweep
    irr = gen.irregular_event(0)
    res["irregular_5M"] = single(irr, 50, gen.PARAMS_IRREGULAR, 5, "c4")
    # Sec. 4.2's own workload shape and parameters (bin 5 cm), 100 x 10k hits;
    # the paper's V100 numbers for it are context only (other hardware)
    pap = single(gen.make_event(1_000_000, 100, 0, "paper"), 100, gen.PARAMS_PAPER, 10, "f3")
    pap["paper_v100_context"] = {"kernels_ms": 2.37, "total_with_memcpy_ms": 6.63,
                                 "cpu_1thread_ms": 705.49, "source": "Table 2"}
    res["paper_parameters_1M"] = pap
    return res


def served(torch, clue, tuning, dev, peak_mhits, args):
    """The served stream: Poisson arrivals of events from a pool (log-uniform
    10k-2M hits, pinned host memory) through the library's server at offered
    loads of `args.loads` x the batched rate; latency from submission to the
    results on the device (the inputs' copy from the host included)."""
    from paper_2001_09761_gb300 import serve
    rng_sizes = gen.batch_sizes(args.pool, 1e4, 2e6, seed=7)
    pool = []
    for k, n in enumerate(rng_sizes):
        ev = gen.make_event(int(n), 100, 5000 + k, "blobs")
        pin = lambda a: torch.from_numpy(a).pin_memory()
        pool.append((pin(ev.x), pin(ev.y), pin(ev.layer), pin(ev.energy)))
    mean_hits = float(np.mean(rng_sizes))
    out = {"pool_events": len(pool), "mean_hits": mean_hits, "requests": args.requests,
           "latency": "submit to results on the device (host input copy included)",
           "loads": {}}
    for load in args.loads:
        free, _ = torch.cuda.mem_get_info(dev)
        srv = serve.Server(device=dev.index, extent=gen.EXTENT, max_layers=100, params=PARAMS,
                           region_hits=16_000_000, n_regions=3, tuning=tuning,
                           mem_budget_bytes=int(0.5 * free))
        serve.offered_load(srv, pool[:4], rate_events_per_s=1e3, n_requests=8, seed=1)  # warm
        srv.reset_stats()
        rate = load * peak_mhits * 1e6 / mean_hits
        serve.offered_load(srv, pool, rate_events_per_s=rate, n_requests=args.requests,
                           seed=int(load * 100))
        st = srv.stats()
        srv.close()
        st["offered_events_per_s"] = rate
        st["offered_mhits_per_s"] = rate * mean_hits / 1e6
        out["loads"][str(load)] = st
    return out


def profile_case():
    """The small case the ncu captures use: the first 40 events of the
    256-event batch (same size draw, 9.94M hits, inputs 159 MB > L2; the
    batch's mix of event sizes and so of bin sizes), clustered twice as one
    batch with the default tuning and no graph; prints nothing else."""
    from paper_2001_09761_gb300 import clue
    x, y, l, e, offs = gen.concat(make_workload(0, 40, 1e4, 1e6))
    cl = clue.Clusterer(extent=gen.EXTENT, max_layers=100, use_graphs=False)
    for _ in range(2):
        cl.run_batch(x, y, l, e, offs, PARAMS)
    cl.sync()
    print("profile case ok", int(offs[-1]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=256)
    ap.add_argument("--lo", type=float, default=1e4)
    ap.add_argument("--hi", type=float, default=1e6)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--per-event-sample", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--quick", action="store_true",
                    help="4 sweep sizes x 2 seeds, 300 requests at loads 0.1, 0.5, 0.9")
    ap.add_argument("--sweep-seeds", type=int, default=10)
    ap.add_argument("--pool", type=int, default=32)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--loads", type=float, nargs="*", default=[0.1, 0.25, 0.5, 0.75, 0.9, 1.0])
    ap.add_argument("--profile-case", action="store_true",
                    help="run the ncu case only: the batch's first 40 events, twice")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case()
    if args.warmup < 3:
        args.warmup = 3
    if args.quick:
        args.sweep_seeds, args.requests = 2, 300
        args.loads = [0.1, 0.5, 0.9]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2001_09761_gb300 import clue, replicas
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        dist = tdist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    size_seed, ev_seed = replicas.weak_seeds(rank)
    events = gen.uneven_batch(args.events, args.lo, args.hi, size_seed, ev_seed)
    x, y, l, e, offs = gen.concat(events)
    N = int(offs[-1])
    tx, ty = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    tl, te = torch.from_numpy(l).to(dev), torch.from_numpy(e).to(dev)
    cid = torch.empty(N, dtype=torch.int32, device=dev)
    seed = torch.empty(N, dtype=torch.uint8, device=dev)
    cl = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100)
    if not args.no_autotune:
        cl.autotune(tx, ty, tl, te, offs, PARAMS, reps=3)
    tuning = cl.tuning
    cl.set_profiling(True)
    for _ in range(args.warmup):
        cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
    cl.sync()
    try:
        cl.kernel_times()
    except clue.ClueError as exc:  # events not timeable in a replayed graph
        print(f"kernel timing in graph mode failed ({exc}: {clue.clue_last_message(cl.ctx)}); "
              "timing with direct launches", file=sys.stderr)
        cl = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100, use_graphs=False)
        cl.tuning = tuning
        cl.set_profiling(True)
        for _ in range(args.warmup):
            cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
        cl.sync()
    torch.cuda.synchronize()

    # ---- timed region: batched steps (graph replay) -----------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    kern = {}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(cl.stream)
    launches = 0
    for i in range(args.steps):
        cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
        launches += cl.launch_count()
        if i:  # the previous step's kernel times, while this step runs
            for k, v in cl.kernel_times(back=1).items():
                kern[k] = kern.get(k, 0.0) + v
    stop.record(cl.stream)
    if args.steps:
        for k, v in cl.kernel_times().items():
            kern[k] = kern.get(k, 0.0) + v
    stop.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms, hits_all = replicas.reduce_timing(start.elapsed_time(stop), N, dist)
    cl.sync()
    ms_per_step = ms / args.steps
    value = hits_all / (ms_per_step * 1e-3) / 1e6
    kern = {k: v / args.steps for k, v in kern.items()}
    stages = {}
    for k, v in kern.items():
        stages[clue.STAGE_OF.get(k, k)] = stages.get(clue.STAGE_OF.get(k, k), 0.0) + v

    # ---- the same batch with the level-by-level frontier expansion ---------
    cl_f = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100,
                          expand=clue.CLUE_EXPAND_FRONTIER)
    cl_f.tuning = tuning
    for _ in range(3):
        cl_f.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
    cl_f.sync()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(cl_f.stream)
    for _ in range(10):
        cl_f.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
    f1.record(cl_f.stream)
    f1.synchronize()
    frontier_value = N / (f0.elapsed_time(f1) / 10 * 1e-3) / 1e6
    cl_f.close()

    # ---- the same batch with the separate rho and nh kernels ---------------
    cl_s = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100,
                          density=clue.CLUE_DENSITY_SEPARATE)
    cl_s.tuning = tuning
    cl_s.set_profiling(True)
    for _ in range(3):
        cl_s.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
    cl_s.sync()
    sep_kern = {}
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(cl_s.stream)
    for i in range(10):
        cl_s.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
        if i:
            for k, v in cl_s.kernel_times(back=1).items():
                sep_kern[k] = sep_kern.get(k, 0.0) + v / 9
    g1.record(cl_s.stream)
    g1.synchronize()
    separate_value = N / (g0.elapsed_time(g1) / 10 * 1e-3) / 1e6
    cl_s.close()

    # ---- per-event launches (same events, one clue_run each) -------------
    # default options: each timed event is new to the context (warm-up uses
    # other events of the batch), as in a stream of incoming events
    idx = np.linspace(0, len(events) - 1, min(args.per_event_sample, len(events))).astype(int)
    pe_hits = int(sum(events[i].n for i in idx))
    views = [(int(offs[i]), int(offs[i + 1])) for i in idx]
    rest = [i for i in range(len(events)) if i not in set(idx.tolist())]
    warm = [rest[k] for k in np.linspace(0, len(rest) - 1, min(8, len(rest))).astype(int)]

    def fresh_context():
        c = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100)
        c.tuning = tuning
        for i in warm:  # events of every size class, none of them timed
            a, b = int(offs[i]), int(offs[i + 1])
            c.run(tx[a:b], ty[a:b], tl[a:b], te[a:b], PARAMS, out=(cid[a:b], seed[a:b]))
        c.sync()
        return c

    cl_pe = fresh_context()
    # each event's input and output views, made before the timed loop
    pe_args = [(tx[a:b], ty[a:b], tl[a:b], te[a:b], (cid[a:b], seed[a:b])) for a, b in views]
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(cl_pe.stream)
    for ex, ey, el, ee, eo in pe_args:
        cl_pe.run(ex, ey, el, ee, PARAMS, out=eo)
    s1.record(cl_pe.stream)
    s1.synchronize()
    per_event_value = pe_hits / (s0.elapsed_time(s1) * 1e-3) / 1e6
    cl_pe.close()
    cl_lat = fresh_context()  # each event again new to its context
    lat = []
    for a, b in views:  # one event alone, device-resident input, launch to sync
        t0 = time.perf_counter()
        cl_lat.run(tx[a:b], ty[a:b], tl[a:b], te[a:b], PARAMS, out=(cid[a:b], seed[a:b]))
        cl_lat.sync()
        lat.append((time.perf_counter() - t0) * 1e3)
    lat = np.array(lat)
    cl_lat.close()

    # ---- end to end through the host-pointer entry point -------------------
    hx = torch.from_numpy(x).pin_memory().numpy()
    hy = torch.from_numpy(y).pin_memory().numpy()
    hl = torch.from_numpy(l).pin_memory().numpy()
    he = torch.from_numpy(e).pin_memory().numpy()
    hcid = torch.empty(N, dtype=torch.int32).pin_memory().numpy()
    hseed = torch.empty(N, dtype=torch.uint8).pin_memory().numpy()
    cl_h = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100)
    cl_h.tuning = tuning
    for _ in range(2):
        cl_h.run_batch_host(hx, hy, hl, he, offs, PARAMS, out=(hcid, hseed))
    # host-timed, so the median of three trials of e2e_steps calls each
    e2e_steps = max(3, args.steps // 4)
    trials = []
    for _ in range(3):
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            cl_h.run_batch_host(hx, hy, hl, he, offs, PARAMS, out=(hcid, hseed))
        trials.append((time.perf_counter() - t0) * 1e3 / e2e_steps)
    e2e_ms, _ = replicas.reduce_timing(float(np.median(trials)), N, dist)
    e2e_value = hits_all / (e2e_ms * 1e-3) / 1e6
    ok = bool(np.array_equal(hcid, cid.cpu().numpy()))
    cl_h.close()

    # ---- roofline of the dominant kernel ------------------------------------
    # achieved = the staged-floor bytes of the kernel's step(s) per hit x the
    # hits of one launch / the kernel's CUDA-event time per launch
    dom = max((k for k in kern if k in ALG_BYTES), key=kern.get)
    peak, peak_kind = load_peaks()
    sec = kern[dom] * 1e-3
    achieved = staged_bytes(dom) * N / sec / 1e9
    traffic, issue = None, None
    tr = parse_traffic()
    if dom in tr and tr[dom][1] == source_hash():
        traffic = tr[dom][0] * N
        issue = tr[dom][2]
    step_s = ms_per_step * 1e-3
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})",
                "bytes_model": f"staged floor of step {STEP_OF_KERNEL[dom]}: "
                               f"{staged_bytes(dom)} B/hit",
                "alg_bytes_per_hit": staged_bytes(dom),
                # the same kernel against every array it really moves once
                # (packed id and decision code included)
                "kernel_bytes_per_hit": ALG_BYTES[dom],
                "kernel_bytes_frac": ALG_BYTES[dom] * N / sec / 1e9 / peak,
                # the whole step against the compulsory I/O and the staged floor
                "step_frac_compulsory_21B": COMPULSORY_BYTES * hits_all / ws / step_s / 1e9 / peak,
                "step_frac_staged_85B": STAGED_TOTAL * hits_all / ws / step_s / 1e9 / peak,
                # ncu's share of cycles issuing an instruction (same capture as
                # traffic): the density kernels are bound by issue, not bytes
                "ncu_issue_active": issue,
                "kernel_ms_per_step": kern, "stage_ms_per_step": stages}

    extra, srv = None, None
    if rank == 0 and not args.no_extra:
        extra = extra_configs(torch, clue, tuning, dev, args)
        srv = served(torch, clue, tuning, dev, value / ws, args)
    cpu = None
    if rank == 0:
        v, desc = cpu_oracle_sample(events, args.cpu_budget)
        cpu = {"value": v, "unit": "Mhits/s", "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        per_event = {"value": per_event_value, "unit": "Mhits/s", "events": len(idx),
                     "hits": pe_hits,
                     "kind": "one clue_run per event, back to back, each event new to the "
                             "context"}
        latency = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                   "kind": "one event alone (new to the context), device-resident input, "
                           "launch to sync"}
        frontier = {"value": frontier_value, "unit": "Mhits/s",
                    "kind": "same batch, CLUE_EXPAND_FRONTIER"}
        separate = {"value": separate_value, "unit": "Mhits/s",
                    "kind": "same batch, CLUE_DENSITY_SEPARATE (rho kernel, then nh kernel)",
                    "rho_ms": sep_kern.get("rho"), "nh_ms": sep_kern.get("nh_delta")}
        e2e = {"value": e2e_value, "unit": "Mhits/s", "h2d_bytes_per_step": 16 * N,
               "d2h_bytes_per_step": 5 * N, "matches_device_path": ok,
               "trials_ms_per_step": trials, "kind": "median of 3 trials of "
               f"{e2e_steps} clue_run_batch_host calls, host-timed"}
        # the compact view of every figure, last on the line so a kept tail of
        # the output still shows it
        summary = {"batched_mhits_per_s": value, "e2e_mhits_per_s": e2e_value,
                   "per_event_mhits_per_s": per_event_value,
                   "frontier_mhits_per_s": frontier_value,
                   "separate_density_mhits_per_s": separate_value,
                   "event_latency_ms_p50_p99": [latency["p50"], latency["p99"]],
                   "dominant_kernel": dom, "dominant_frac_of_hbm": roofline["frac"],
                   "step_frac_compulsory_21B": roofline["step_frac_compulsory_21B"]}
        if extra:
            summary["single_10k_mhits_per_s"] = extra["single_10k"]["mhits_per_s"]
            summary["irregular_5M_mhits_per_s"] = extra["irregular_5M"]["mhits_per_s"]
            summary["sweep_median_mhits_per_s"] = extra["scaling_sweep_median_mhits_per_s"]
        if srv:
            summary["served"] = {k: [v["mhits_per_s"], v["p50_ms"], v["p99_ms"]]
                                 for k, v in srv["loads"].items()}
            summary["served_fields"] = "load: [Mhits/s, p50 ms, p99 ms]"
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "Mhits/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": len(events) * ws,
                       "hits_per_step": hits_all, "parallelism": f"replicas x{ws}",
                       "l2": "inputs (1 GB per rank) larger than L2, no flush"},
            "gpu_launches": launches,
            "clocks": clk,
            "tuning": tuning,
            "configs": extra,
            "served": srv,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched_frontier_expansion": frontier,
            "batched_separate_density": separate,
            "per_event": per_event,
            "latency_ms": latency,
            "summary": summary,
        }))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
