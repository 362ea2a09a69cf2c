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
# algorithmic bytes per hit of the density kernels (own hit read once, outputs
# written once): rho reads x, y, w, layer and writes rho; nh/delta reads x, y,
# rho, layer and writes rho, delta^2, nh.
ALG_BYTES = {"rho": 20, "nh_delta": 28, "grid_fill": 16 + 4 + 4 + 16 + 4,
             "decide_followers": 12 + 5 + 8 + 4, "expand": 8}


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
    # weak scaling: each rank clusters its own batch of the same size
    events = gen.uneven_batch(n_events, lo, hi, size_seed=rank, first_event_seed=1000 + 100000 * rank)
    return events


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
    # each step: a fixed bounded sample of the workload (every 32nd event by size)
    order = np.argsort([ev.n for ev in events])
    sample = [events[i] for i in order[:: 32]]
    hits = sum(ev.n for ev in sample)
    for _ in range(args.warmup):
        oracle.run_event(sample[0], PARAMS, 100)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for ev in sample:
            oracle.run_event(ev, PARAMS, 100)
    dt = time.perf_counter() - t0
    value = hits * args.steps / dt / 1e6
    desc = f"{len(sample)} of {len(events)} events (every 32nd by size), {hits} hits per step"
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=256)
    ap.add_argument("--lo", type=float, default=1e4)
    ap.add_argument("--hi", type=float, default=1e6)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--per-event-sample", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local)
    from paper_2001_09761_gb300 import clue

    events = make_workload(rank, args.events, args.lo, args.hi)
    x, y, l, e, offs = gen.concat(events)
    N = int(offs[-1])
    dev = torch.device("cuda", local)
    tx, ty = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    tl, te = torch.from_numpy(l).to(dev), torch.from_numpy(e).to(dev)
    cid = torch.empty(N, dtype=torch.int32, device=dev)
    seed = torch.empty(N, dtype=torch.uint8, device=dev)
    cl = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100)
    if not args.no_autotune:
        cl.autotune(tx, ty, tl, te, offs, PARAMS, reps=1)
    cl.set_profiling(True)
    for _ in range(args.warmup):
        cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
    cl.sync()
    try:
        cl.stage_times()
    except clue.ClueError as exc:  # stage events not timeable in a replayed graph
        print(f"stage timing in graph mode failed ({exc}: {clue.clue_last_message(cl.ctx)}); "
              "timing with direct launches", file=sys.stderr)
        table = cl.tuning
        cl = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100, use_graphs=False)
        cl.tuning = table
        cl.set_profiling(True)
        for _ in range(args.warmup):
            cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
        cl.sync()
    torch.cuda.synchronize()

    # ---- timed region: batched steps -------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    stage_sum = {}
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(cl.stream)
    launches = 0
    for _ in range(args.steps):
        cl.run_batch(tx, ty, tl, te, offs, PARAMS, out=(cid, seed))
        launches += cl.launch_count()
        for k, v in cl.stage_times().items():  # waits for this step's stage events
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    stop.record(cl.stream)
    stop.synchronize()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    if pg:
        t = torch.tensor([ms], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    clk = clocks.stop()
    cl.sync()
    ms_per_step = ms / args.steps
    value = N * ws / (ms_per_step * 1e-3) / 1e6
    stages = {k: v / args.steps for k, v in stage_sum.items()}

    # ---- per-event launches (same events, one clue_run each) -------------
    cl_pe = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100, use_graphs=False)
    cl_pe.tuning = cl.tuning
    idx = np.linspace(0, len(events) - 1, min(args.per_event_sample, len(events))).astype(int)
    pe_hits = int(sum(events[i].n for i in idx))
    views = [(int(offs[i]), int(offs[i + 1])) for i in idx]
    for a, b in views[:3]:
        cl_pe.run(tx[a:b], ty[a:b], tl[a:b], te[a:b], PARAMS, out=(cid[a:b], seed[a:b]))
    cl_pe.sync()
    lat = []
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(cl_pe.stream)
    for a, b in views:
        cl_pe.run(tx[a:b], ty[a:b], tl[a:b], te[a:b], PARAMS, out=(cid[a:b], seed[a:b]))
    s1.record(cl_pe.stream)
    s1.synchronize()
    per_event_value = pe_hits / (s0.elapsed_time(s1) * 1e-3) / 1e6
    for a, b in views:  # latency of one event alone, device-resident input
        t0 = time.perf_counter()
        cl_pe.run(tx[a:b], ty[a:b], tl[a:b], te[a:b], PARAMS, out=(cid[a:b], seed[a:b]))
        cl_pe.sync()
        lat.append((time.perf_counter() - t0) * 1e3)
    lat = np.array(lat)

    # ---- end to end through the host-pointer entry point -------------------
    hx = torch.from_numpy(x).pin_memory().numpy()
    hy = torch.from_numpy(y).pin_memory().numpy()
    hl = torch.from_numpy(l).pin_memory().numpy()
    he = torch.from_numpy(e).pin_memory().numpy()
    hcid = torch.empty(N, dtype=torch.int32).pin_memory().numpy()
    hseed = torch.empty(N, dtype=torch.uint8).pin_memory().numpy()
    cl_h = clue.Clusterer(device=local, extent=gen.EXTENT, max_layers=100)
    cl_h.tuning = cl.tuning
    for _ in range(2):
        cl_h.run_batch_host(hx, hy, hl, he, offs, PARAMS, out=(hcid, hseed))
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cl_h.run_batch_host(hx, hy, hl, he, offs, PARAMS, out=(hcid, hseed))
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = N * ws / e2e_s / 1e6
    ok = bool(np.array_equal(hcid, cid.cpu().numpy()))

    # ---- roofline of the dominant kernel ------------------------------------
    dom = max(stages, key=stages.get)
    peak, peak_kind = load_peaks()
    achieved = ALG_BYTES[dom] * N / (stages[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_hit": ALG_BYTES[dom],
                "stage_ms": stages}

    cpu = None
    if rank == 0:
        v, desc = cpu_oracle_sample(events, args.cpu_budget)
        cpu = {"value": v, "unit": "Mhits/s", "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "Mhits/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": len(events) * ws,
                       "hits_per_step": N * ws, "parallelism": f"replicas x{ws}",
                       "l2": "inputs (1 GB) larger than L2, no flush"},
            "per_event": {"value": per_event_value, "unit": "Mhits/s", "events": len(idx),
                          "hits": pe_hits},
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "kind": "one event alone, device-resident input, launch to sync"},
            "e2e": {"value": e2e_value, "unit": "Mhits/s", "h2d_bytes_per_step": 16 * N,
                    "d2h_bytes_per_step": 5 * N, "matches_device_path": ok},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
            "tuning": cl.tuning,
        }))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
