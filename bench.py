#!/usr/bin/env python3
"""Benchmark of bulk transaction execution on one GB300.

Workload (debit-credit at scale): 1,000 branches, 10,000 tellers, 10,000,000
accounts with int64 balances; bulks of 2^22 transactions (account uniform or
Zipf(theta) then scrambled, delta uniform in [-99999, 99999]).  One step = one
bulk through the whole path: bulk hand-over, basic-operation extraction,
grouping sort, ranks and depths, (level, type) regrouping, execution, results
left on the device.  The headline is the plain per-bulk K-SET path with the
paper's read/write conflict model; a bounded sweep reports every strategy,
conflict model, skew and bulk size beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gputx|reference]

The reference arm times the CPU oracle (plain serial execution in timestamp
order) on the host cores on the same workload.  Under torchrun each rank runs
an independent replica (the path does not shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

BRANCHES, TELLERS, ACCOUNTS = 1000, 10_000, 10_000_000
METRIC = "txns/sec on 1 GB300 per strategy & bulk size vs plain path; p50/p99 latency"
# algorithmic bytes of one debit-credit transaction in the executor, at the
# granularity of random HBM access (one 32 B sector per random cell):
#   execution-order record (params 16 B, ts 8 B, type 4 B, index 4 B)  32 B, sequential
#   account balance: one sector read + one sector written            64 B, random
#   teller and branch balances (80 KB + 8 KB: resident in L2)           0 B
#   history row (ts, account, teller, branch, delta)                   40 B, sequential
#   output value 8 B + status 4 B                                      12 B
EXEC_BYTES_PER_TXN = 32 + 64 + 0 + 40 + 12
L2_FLUSH_BYTES = 256 << 20
# the executor kernel that dominates each headline configuration
DOMINANT_KERNEL = {("kset", "paper"): "kset_narrow_dc_kernel", ("kset", "add"): "kset_level_kernel",
                   ("part_relaxed", "paper"): "part_dc_kernel", ("tpl_relaxed", "paper"): "tpl_relaxed_kernel",
                   ("tpl_relaxed", "add"): "tpl_relaxed_kernel",
                   ("part", "paper"): "part_dc_kernel", ("part", "add"): "part_dc_kernel",
                   ("tpl", "paper"): "tpl_dc_kernel", ("tpl", "add"): "tpl_dc_kernel",
                   ("scan", "paper"): "seg64_scan_kernel", ("scan", "add"): "seg64_scan_kernel"}
# DRAM bytes (read + write) of the dominant kernel's launches for one bulk
# (the narrow runner's segments: the main run and the narrow tail) from one
# ncu capture at this configuration, keyed by (strategy, mode, bulk log2);
# each entry holds the digest of the kernel and launch-planner sources it was
# taken on, and is reported as null once those sources change
TRAFFIC = {("kset", "paper", 22): {"bytes": 341127168 + 361984 + 290942208, "digest": "3472c3d645ba694a"}}
KERNEL_SOURCES = ("common.cuh", "fastdiv.h", "engine.h", "dc.cuh", "levels.cuh", "exec_dc.cu", "exec.cu")


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1103_3105_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(strategy, mode, lg):
    t = TRAFFIC.get((strategy, mode, lg))
    if t is None or t["digest"] != kernel_digest():
        return None
    return t["bytes"]


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region.

    Sampling starts before the timed region (the first sample is awaited) and
    every sample carries its timestamp; the summary keeps those that fall in
    the marked window, widened by one sampling period on each side."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        """the timed region, as time.time() values"""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _stamp(text, fallback):
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return fallback

    def summary(self, windowed=True):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        pad = 1.5 * self.PERIOD_MS / 1e3
        for seen, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            if self.window and windowed:
                ts = self._stamp(f[0], seen)
                if ts < self.window[0] - pad or ts > self.window[1] + pad:
                    continue
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for nm, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm and windowed and self.window:
            # no sample landed inside a short window: the whole sampled span
            out = self.summary(windowed=False)
            out["window"] = "sampled span (no sample inside the timed region)"
            return out
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_throughput(units_local: float, seconds_local: float, dist=None, device=None) -> float:
    """Whole-job throughput of independent replicas (the path does not shard:
    every rank runs its own database and bulks, no data-path collective).
    Units add up over ranks; time is the slowest rank's (max over ranks)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units_local / seconds_local
    import torch
    t = torch.tensor([seconds_local, units_local], dtype=torch.float64, device=device)
    secs = t[:1].clone()
    units = t[1:].clone()
    dist.all_reduce(secs, op=dist.ReduceOp.MAX)
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return float(units.item()) / float(secs.item())


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    return 6800.0, "fallback"


def make_bulks(n, theta, count, seed0):
    return [W.dc_bulk(n, ACCOUNTS, theta, seed=W.seed_for(2, seed0 + i)) for i in range(count)]


# ---------------------------------------------------------------------------
# engine arm
# ---------------------------------------------------------------------------
def run_engine(args, rank, world, local_rank):
    import torch
    import paper_1103_3105_gb300 as G
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = 1 << args.bulk_log2
    K, Wm = args.steps, args.warmup
    # the engine and every event/flush share one explicit stream
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    cap = (3 * K + 2 * Wm + 8) * n   # history rows: device steps, serial and pipelined e2e
    db = G.Database(dc=(BRANCHES, TELLERS, ACCOUNTS), history_capacity=cap, max_bulk=n,
                    stream=stream.cuda_stream)
    db.register(G.DC_TYPES)
    bulks = make_bulks(n, args.theta, 3, 100 * rank)
    dbulks = [{k: torch.from_numpy(b[k]).to(dev) for k in ("ts", "type", "params")} for b in bulks]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    mode = G.CONFLICT_ADD if args.mode == "add" else G.CONFLICT_PAPER

    def step(i, timing=False):
        d = dbulks[i % len(dbulks)]
        b = db.submit(d["ts"], d["type"], d["params"])
        b.execute(args.strategy, conflict_mode=mode, timing=timing)
        return b

    for i in range(Wm):
        step(i).free()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = G.gputx_launch_count()
    times, exec_ms, sort_ms, stats = [], [], [], None
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        epoch0 = time.time()
        for i in range(K):
            flush.fill_(i & 0xFF)          # L2 flush between steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b = step(i, timing=True)
            e1.record(stream)
            stats = b.sync()
            times.append(e0.elapsed_time(e1))
            exec_ms.append(stats["ms_execute"])
            sort_ms.append(stats["ms_sort"])
            b.free()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark(epoch0, time.time())
    launches = G.gputx_launch_count() - launches0
    # count only the engine's kernels: the L2 flushes are torch's
    total_ms = sum(times)
    value = replica_throughput(n * K, total_ms / 1e3, dist, dev)
    total_ms = n * K * world / value * 1e3   # the slowest rank's time

    # end to end through the public API with host buffers: H2D + D2H inside
    pinned = []
    for b in bulks:
        pinned.append({k: torch.from_numpy(b[k]).pin_memory() for k in ("ts", "type", "params")})
    st_h = torch.empty(n, dtype=torch.int32).pin_memory()
    out_h = torch.empty((n, db.width), dtype=torch.int64).pin_memory()
    for i in range(max(1, Wm)):
        p = pinned[i % len(pinned)]
        b = db.submit(p["ts"].numpy(), p["type"].numpy(), p["params"].numpy())
        b.execute(args.strategy, conflict_mode=mode)
        b.results(st_h.numpy(), out_h.numpy())
        b.free()
    # one bulk at a time, L2 flushed before each (outside the timing)
    e2e_times = []
    for i in range(K):
        flush.fill_(i & 0xFF)
        p = pinned[i % len(pinned)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = db.submit(p["ts"].numpy(), p["type"].numpy(), p["params"].numpy())
        b.execute(args.strategy, conflict_mode=mode)
        b.results(st_h.numpy(), out_h.numpy())
        e2e_times.append(time.perf_counter() - t0)
        b.free()
    e2e_serial = replica_throughput(n * K, sum(e2e_times), dist, dev)
    # two bulks in flight, as a client streaming bulks uses the API: bulk i
    # is submitted (its H2D copy queued) and executed before the results of
    # bulk i-1 are read, so copies overlap the previous bulk's execution.
    # Every step's inputs and results still cross inside the timed region;
    # each step moves 117 MB of new inputs and 160 MB of history, more than L2.
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    prev = None
    for i in range(K):
        p = pinned[i % len(pinned)]
        b = db.submit(p["ts"].numpy(), p["type"].numpy(), p["params"].numpy())
        b.execute(args.strategy, conflict_mode=mode)
        if prev is not None:
            prev.results(st_h.numpy(), out_h.numpy())
            prev.free()
        prev = b
    prev.results(st_h.numpy(), out_h.numpy())
    prev.free()
    e2e_value = replica_throughput(n * K, time.perf_counter() - t0, dist, dev)

    sweep = serving = batched = subscriber = None
    if rank == 0:
        db.close()
        if args.sweep:
            sweep = run_sweep(args, G, torch, dev, stream, flush)
        if args.serve:
            serving = run_serving(args, G, torch, stream)
        if args.batched:
            batched = run_batched(args, G, torch, stream)
        if args.subscriber:
            subscriber = run_subscriber(args, G, torch, stream)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peak_hbm()
    ex = statistics.median(exec_ms)
    # the latency roofline of the level chain: the bare skeleton of a level
    # (updates of cells another SM updated at the previous level, stores,
    # cluster barrier) in the narrow runner's launch shape, with the
    # executor's traffic and with the minimum
    latency = None
    if args.strategy == "kset" and stats and stats["depth"] > 0:
        levels = stats["depth"] + 1
        def probe(*shape, **kw):   # a floor: the best of three launches
            return min(G.gputx_probe_level_chain(levels, 16, 64, *shape, **kw) for _ in range(3))
        # the runner's own shape: the account's fetch-and-add before the
        # barrier's release; after it, 9 fire-and-forget writes (teller and
        # branch additions, history row, outputs), stores in the probe
        floor_dc = probe(0, 1, 9, rmw=1)
        floor_min = probe(0, 1, 0, rmw=1)
        # the same with the fetch-and-add on random cells of a table the size
        # of the 10M accounts, prefetched two levels ahead like the runner's
        floor_rand = probe(0, 1, 9, rmw=2)
        # the same level applying its updates as loads then stores
        floor_ld_st = probe(3, 3, 7)
        measured = ex * 1e6 / levels
        latency = {"levels": levels, "measured_ns_per_level": measured,
                   "floor_ns_per_level": floor_dc, "floor_ns_per_level_min": floor_min,
                   "floor_ns_per_level_load_store": floor_ld_st, "frac": floor_dc / measured,
                   "floor_ns_per_level_random_cells": floor_rand, "frac_random_cells": floor_rand / measured,
                   "probe": "cluster 16 x 64 threads; per thread and level 1 fetch-and-add on a cell another "
                            "CTA updated at the previous level, barrier arrive (release), 9 stores, "
                            "barrier wait (acquire); best of 3 launches"}
    # L2 atomic throughput (random cells of a 10M-cell table, the 10,000
    # tellers, the 1,000 branches), beside the atomics the executor issues
    atomics = None
    if args.strategy in ("kset", "tpl") and stats:
        atomics = {f"{kind}_{name}_gops": G.gputx_probe_atomics(cells, fetch)
                   for name, cells in (("accounts", ACCOUNTS), ("tellers", TELLERS), ("branches", BRANCHES))
                   for kind, fetch in (("red", 0), ("fetch_add", 1))}
        # K-SET R/W: fetch-and-add + 2 reductions (narrow runner); K-SET ADD:
        # teller and branch reductions; TPL: one counter release per lock
        # (the branch, or the account under ADD) + the 2 reductions under ADD
        per_txn = {("kset", "paper"): 3, ("kset", "add"): 2, ("tpl", "paper"): 1,
                   ("tpl", "add"): 3}[(args.strategy, args.mode)]
        atomics["executor_gops"] = n * per_txn / (ex / 1e3) / 1e9
        atomics["executor_atomics_per_txn"] = per_txn
    achieved = n * EXEC_BYTES_PER_TXN / (ex / 1e3) / 1e9
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0))
    clocks = clk.summary()
    traffic = traffic_for(args.strategy, args.mode, args.bulk_log2)
    levels = stats["depth"] + 1 if stats else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "txn/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": total_ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic (seeded debit-credit bulks, balances start at 0)",
        "config": {"workload": f"debit-credit at scale: {BRANCHES} branches, {TELLERS} tellers, "
                               f"{ACCOUNTS} accounts, bulk 2^{args.bulk_log2}, theta {args.theta}",
                   "strategy": args.strategy, "conflict_mode": args.mode, "bulk": n,
                   "l2": "flushed between steps (256 MiB write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "txn/s", "h2d_bytes_per_step": n * (8 + 4 + 16),
                "d2h_bytes_per_step": n * (4 + 8 * db.width), "pipeline": "2 bulks in flight",
                "serial_value": e2e_serial},
        "gpu_launches": int(launches),
        "roofline": {"kernel": DOMINANT_KERNEL.get((args.strategy, args.mode), "executor"),
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind, "bytes_per_txn": EXEC_BYTES_PER_TXN,
                     "txn_per_launch_set": n, "kernel_ms": ex,
                     # the level chain, not bandwidth, bounds K-SET on a deep graph
                     "levels": levels, "ns_per_level": ex * 1e6 / levels if levels else None},
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")},
    }
    if latency is not None:
        line["latency_roofline"] = {k: latency[k] for k in ("levels", "measured_ns_per_level",
                                                             "floor_ns_per_level", "frac",
                                                             "floor_ns_per_level_random_cells",
                                                             "frac_random_cells")}
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, bulks)
    # everything else goes to the detail file; stdout ends with the compact headline
    detail = {"headline": line, "latency_roofline": latency, "atomics": atomics,
              "phases_ms": {"execute": ex, "op_sort": statistics.median(sort_ms),
                            "analysis": stats["ms_analysis"] if stats else None},
              "graph": {"depth": stats["depth"], "w0": stats["w0"], "cross": stats["cross"]} if stats else None,
              "clocks": clocks, "wall_s_timed": wall, "kernel_source_digest": kernel_digest(),
              "l2": {"l2_bytes": l2_bytes, "account_bytes": ACCOUNTS * 8,
                     "teller_branch_bytes": (TELLERS + BRANCHES) * 8},
              "sweep": sweep, "serving": serving, "batched": batched, "subscriber": subscriber}
    if args.detail_out:
        try:
            d = os.path.dirname(os.path.abspath(args.detail_out))
            os.makedirs(d, exist_ok=True)
            with open(args.detail_out, "w") as fh:
                json.dump(detail, fh, indent=1)
            line["detail"] = args.detail_out
        except OSError as e:
            line["detail"] = f"not written: {e}"
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_sweep(args, G, torch, dev, stream, flush):
    """Every strategy x conflict model x skew x bulk size, a few steps each,
    within a time budget (points past the budget are reported as skipped)."""
    t_start = time.perf_counter()
    out = []
    sizes = [14, 16, 18, 20, 22]
    # history rows for every bulk the sweep can run
    rows = 3 * 10 * 3 * sum(1 << lg for lg in sizes)
    db = G.Database(dc=(BRANCHES, TELLERS, ACCOUNTS), history_capacity=rows, max_bulk=1 << 22,
                    stream=stream.cuda_stream)
    db.register(G.DC_TYPES)
    for theta in (0.0, 0.5, 0.99):
        big = W.dc_bulk(1 << 22, ACCOUNTS, theta, seed=W.seed_for(2, 900 + int(theta * 100)))
        dbig = {k: torch.from_numpy(big[k]).to(dev) for k in ("ts", "type", "params")}
        for lg in sizes:
            n = 1 << lg
            for strategy in ("kset", "part", "tpl", "auto", "scan", "part_relaxed", "tpl_relaxed"):
                for mode_name, mode in (("paper", G.CONFLICT_PAPER), ("add", G.CONFLICT_ADD)):
                    if strategy in ("part", "scan", "part_relaxed", "auto") and mode_name == "add":
                        continue   # PART runs partitions serially, SCAN always sums: the model changes neither
                    rec = {"theta": theta, "bulk": n, "strategy": strategy, "mode": mode_name}
                    if time.perf_counter() - t_start > args.sweep_budget_s:
                        rec["skipped"] = "time budget"
                        out.append(rec)
                        continue
                    ts = []
                    st = None
                    try:
                        for i in range(3):
                            flush.fill_(i)
                            e0 = torch.cuda.Event(enable_timing=True)
                            e1 = torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            b = db.submit(dbig["ts"][:n], dbig["type"][:n], dbig["params"][:n])
                            b.execute(strategy, conflict_mode=mode, timing=True)
                            e1.record(stream)
                            try:
                                st = b.sync()
                            finally:
                                b.free()
                            if i:
                                ts.append(e0.elapsed_time(e1))
                    except G.GputxError as err:
                        # e.g. a spin lock held longer than the wait limit under
                        # extreme contention: reported, not timed
                        rec["error"] = str(err)
                        out.append(rec)
                        continue
                    ms = statistics.median(ts)
                    rec.update({"ms": ms, "txn_per_s": n / (ms / 1e3), "depth": st["depth"],
                                "w0": st["w0"], "exec_ms": st["ms_execute"], "sort_ms": st["ms_sort"],
                                "exec_hbm_frac": (n * EXEC_BYTES_PER_TXN / (st["ms_execute"] / 1e3) / 1e9
                                                  / measured_peak_hbm()[0]) if st["ms_execute"] > 0 else None})
                    out.append(rec)
    db.close()
    return out


def run_serving(args, G, torch, stream):
    """The served mix: debit-credit and subscriber schemas loaded together in a
    device-resident database of about 20 GB of live rows (20M subscribers
    with their child tables and indexes, 10M accounts, the history the
    served transactions append), open-loop Poisson arrivals of a
    50/50 mix of the two schemas' transactions.  Three serving modes:
    continuous batching (several bulks in flight), the plain per-bulk path
    (one bulk at a time, closed every deadline) and incremental 0-set
    execution.  Latency = result on the host - arrival."""
    out = []
    rates = [float(r) for r in args.serve_rates.split(",")]
    deadlines = [int(d) for d in args.serve_deadlines_us.split(",")]
    n_sub = args.serve_subscribers
    skewed_rates = [r for r in rates if r >= 20e6]
    # history rows: one per served debit-credit transaction (half the mix)
    total = int(0.52 * (sum(rates) * len(deadlines) * 3 + sum(skewed_rates) * 2) * args.serve_seconds) + (1 << 20)
    free0 = torch.cuda.mem_get_info()[0]
    # the database's size comes from its live rows (subscribers with their
    # child tables and indexes, 10M accounts); history holds what the served
    # transactions append, nothing more
    hist_rows = total
    db = G.Database(dc=(BRANCHES, TELLERS, ACCOUNTS), sub=n_sub, history_capacity=hist_rows,
                    sub_child_capacity=6 * n_sub, max_bulk=1 << 20, stream=stream.cuda_stream)
    db.register(G.DC_TYPES + G.SUB_TYPES)
    sub_t = W.sub_tables(n_sub, seed=W.seed_for(5, 1))
    for t, r in W.sub_rows(sub_t).items():
        db.load(t, r)
    torch.cuda.synchronize()
    db_bytes = free0 - torch.cuda.mem_get_info()[0]
    mode = G.CONFLICT_ADD if args.mode == "add" else G.CONFLICT_PAPER
    # every rate and deadline at the benchmark's skew, then the high rates
    # with Zipf 0.8 keys at the shorter deadline: hot subscribers and
    # accounts make each bulk's k-set chain long, so its GPU time matters
    plan = [(rate, args.theta, deadlines, ri) for ri, rate in enumerate(rates)]
    plan += [(rate, 0.8, deadlines[:1], 100 + ri) for ri, rate in enumerate(skewed_rates)]
    for rate, theta, dls, variant in plan:
        n = int(rate * args.serve_seconds)
        bulk = W.served_mix(n, ACCOUNTS, n_sub, theta, rate, seed_variant=variant)
        offs = bulk["arrival_offset_ns"]
        for deadline in dls:
            modes = (("continuous", 3, False), ("plain", 1, False), ("zero_set", 1, True))
            if theta != args.theta:
                modes = modes[:2]
            for label, inflight, zero in modes:
                if zero and rate > args.serve_zero_set_max_rate:
                    out.append({"offered_txn_per_s": rate, "deadline_us": deadline, "mode": label,
                                "skipped": "rate above --serve-zero-set-max-rate"})
                    continue
                srv = G.Server(db, deadline_us=deadline, max_bulk=1 << 20, max_inflight=inflight,
                               strategy=args.serve_strategy, conflict_mode=mode, params_per_txn=bulk["P"],
                               zero_set=zero)
                t0 = G.gputx_clock_ns() + 2_000_000
                arrivals = t0 + offs
                i = 0
                while i < n:
                    now = G.gputx_clock_ns()
                    j = int(np.searchsorted(arrivals, now, side="right"))
                    if j > i:
                        srv.submit(bulk["type"][i:j], bulk["params"][i:j], arrivals[i:j])
                        i = j
                    else:
                        time.sleep(20e-6)
                srv.drain()
                st = srv.stats()
                srv.close()
                out.append({"offered_txn_per_s": rate, "deadline_us": deadline, "mode": label, "theta": theta,
                            "max_inflight": inflight, "txn": n, "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                            "mean_us": st["mean_us"], "txn_per_s": st["txn_per_s"], "bulks": st["bulks"],
                            "max_bulk": st["max_bulk_seen"]})
    db.close()
    res = {"db_bytes": int(db_bytes), "subscribers": n_sub, "accounts": ACCOUNTS, "history_rows": hist_rows,
           "mix": "50% debit-credit, 50% subscriber (30/25/25/8/8/2/2)", "runs": out}
    if args.cpu_baseline:
        # the oracle on a bounded sample of the served stream (1M transactions)
        import oracle
        oracle.build()
        m = 1_000_000
        o = oracle.OracleDB(dc=W.dc_tables(BRANCHES, TELLERS, ACCOUNTS), sub=sub_t, hist_cap=m)
        bulk = W.served_mix(m, ACCOUNTS, n_sub, args.theta, 5e6)
        t1 = time.perf_counter()
        o.execute(bulk, R=8)
        dt = time.perf_counter() - t1
        res["cpu_baseline"] = {"value": m / dt, "unit": "txn/s", "cores": 1, "nproc": os.cpu_count(),
                               "kind": "oracle", "sample": f"{m} transactions of the served mix, serial "
                                                           f"execution in id order, {dt:.2f} s"}
    return res


def run_subscriber(args, G, torch, stream):
    """The subscriber-location schema (read-heavy, four tables): 10M
    subscribers with their access_info, special_facility and call_forwarding
    rows, bulks of 2^20 mixed transactions (30/25/25/8/8/2/2 %), subscriber
    ids uniform or Zipf 0.8.  Every strategy, the paper's R/W model."""
    t0 = time.perf_counter()
    n_sub = args.sub_subscribers
    tabs = W.sub_tables(n_sub, seed=W.seed_for(3, 1))
    db = G.Database(sub=n_sub, sub_child_capacity=6 * n_sub, max_bulk=1 << 20, stream=stream.cuda_stream)
    db.register(G.SUB_TYPES)
    for t, r in W.sub_rows(tabs).items():
        db.load(t, r)
    setup_s = time.perf_counter() - t0
    out = []
    ts0 = 0
    n = 1 << 20
    dev = torch.device("cuda", torch.cuda.current_device())
    for theta in (0.0, 0.8):
        bulk = W.sub_bulk(n, n_sub, theta, seed=W.seed_for(3, 10 + int(theta * 10)))
        # inputs resident on the device, as in the headline
        d_type = torch.from_numpy(bulk["type"]).to(dev)
        d_params = torch.from_numpy(bulk["params"]).to(dev)
        for strategy in ("kset", "part", "tpl", "auto", "part_relaxed", "tpl_relaxed"):
            rec = {"theta": theta, "bulk": n, "strategy": strategy}
            ms = []
            st = None
            try:
                for rep in range(3):
                    d_ts = torch.arange(ts0, ts0 + n, dtype=torch.int64, device=dev)
                    ts0 += n
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    b = db.submit(d_ts, d_type, d_params)
                    b.execute(strategy, timing=True)
                    e1.record(stream)
                    try:
                        st = b.sync()
                    finally:
                        b.free()
                    if rep:
                        ms.append(e0.elapsed_time(e1))
            except G.GputxError as err:
                rec["error"] = str(err)
                out.append(rec)
                continue
            m = statistics.median(ms)
            rec.update({"ms": m, "txn_per_s": n / (m / 1e3), "depth": st["depth"], "w0": st["w0"],
                        "exec_ms": st["ms_execute"], "analysis_ms": st["ms_analysis"], "ran": st["strategy"]})
            out.append(rec)
    db.close()
    res = {"subscribers": n_sub, "setup_s": setup_s, "runs": out}
    if args.cpu_baseline:
        # the oracle on one bulk of the same workload (Zipf 0.8)
        import oracle
        oracle.build()
        o = oracle.OracleDB(sub=tabs)
        bulk = W.sub_bulk(n, n_sub, 0.8, seed=W.seed_for(3, 18))
        t1 = time.perf_counter()
        o.execute(bulk, R=8)
        dt = time.perf_counter() - t1
        res["cpu_baseline"] = {"value": n / dt, "unit": "txn/s", "cores": 1, "nproc": os.cpu_count(),
                               "kind": "oracle", "sample": f"one bulk of {n} transactions (Zipf 0.8), serial "
                                                           f"execution in timestamp order, {dt:.2f} s"}
    return res


# algorithmic bytes of one order-entry transaction at the mix (45 % new-order
# with 10 lines on average, 43 % payment, 12 % order-status), one 32 B sector
# per random cell, read + write for an updated one; the 64 warehouses' and
# 640 districts' rates and year-to-date cells and the 800 KB item prices sit
# in L2 (0 B):
#   new-order     record 168 (19 params, ts, type, index), district counter
#                 64, customer discount 32, per line stock quantity/ytd/count
#                 3 x 64 + order-line row 20 (x 10), order row 33, index
#                 insert 96, customer last order 32, outputs 28   -> 2,573 B
#   payment       record 168, customer balance/ytd/count 3 x 64, output 12 -> 372 B
#   order-status  record 168, customer 2 x 32, index probe 64, order row 64,
#                 10 line amounts 96, outputs 36                  -> 492 B
OE_EXEC_BYTES_PER_TXN = round(0.45 * 2573 + 0.43 * 372 + 0.12 * 492)


def run_batched(args, G, torch, stream):
    """Order-entry streams of uneven bulks (64 warehouses x 10 districts x
    3,000 customers, 100,000 items): the graph batcher with its autotuner
    (several bulks per graph replay, each keeping its own k-sets under K-SET,
    two segments in flight once tuned) against the plain per-bulk K-SET path.
    Two streams run back to back on one database: the first tunes the
    batcher (and warms the plain path), the second is the steady state.
    Host arrays in and out (H2D and D2H inside the timing) for both.  Latency
    of a transaction = time from the stream's start until its results are on
    the host (each stream is handed over at once)."""
    n_wh, n_items = 64, 100_000
    init = W.oe_tables(n_wh, n_items=n_items, seed=W.seed_for(4))
    sizes_a, stream_a = W.oe_stream(args.batch_txns, n_wh, n_items)
    total_a = sum(sizes_a)
    sizes_b, stream_b = W.oe_stream(args.batch_txns, n_wh, n_items, variant=1, ts0=total_a)
    total_b = sum(sizes_b)
    out = {"workload": f"order-entry {n_wh} warehouses, {n_items} items, two streams of {len(sizes_a)} and "
                       f"{len(sizes_b)} bulks of 2^10..2^21 transactions ({total_a} and {total_b})",
           "txn": total_b, "bytes_per_txn": OE_EXEC_BYTES_PER_TXN}
    peak = measured_peak_hbm()[0]
    mode = G.CONFLICT_ADD if args.mode == "add" else G.CONFLICT_PAPER

    def pct(done, total):
        done.sort()
        acc, p50, p99 = 0, None, None
        for ms, k in done:
            acc += k
            if p50 is None and acc > 0.5 * total:
                p50 = ms
            if p99 is None and acc > 0.99 * total:
                p99 = ms
        return p50 * 1e3, p99 * 1e3

    for label in ("plain_kset", "batched_tuned"):
        cap = 2 * (total_a + total_b) + (1 << 22)
        db = G.Database(oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15,
                        max_bulk=1 << 21, stream=stream.cuda_stream)
        db.register(G.OE_TYPES)
        for t, rows in W.oe_rows(init).items():
            db.load(t, rows)
        bt = None
        if label == "batched_tuned":
            bt = G.Batcher(db, tune=True, params_per_txn=W.OE_PARAMS, bulk_size_max=1 << 21, conflict_mode=mode)
        rec = {}
        for phase, sizes, sb, total in (("first", sizes_a, stream_a, total_a), ("steady", sizes_b, stream_b, total_b)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if bt is None:
                i = 0
                done = []          # (ms from start, transactions) per bulk
                for k in sizes:
                    b = db.submit(sb["ts"][i:i + k], sb["type"][i:i + k], sb["params"][i:i + k])
                    b.execute("kset", conflict_mode=mode)
                    b.results()
                    b.free()
                    done.append(((time.perf_counter() - t0) * 1e3, k))
                    i += k
                p50, p99 = pct(done, total)
            else:
                bt.run_bulks(sb["ts"], sb["type"], sb["params"], sizes)
                ch = bt.choice()
                p50, p99 = ch["p50_us"], ch["p99_us"]
            dt = time.perf_counter() - t0
            rec[phase] = {"txn_per_s": total / dt, "seconds": dt, "p50_us": p50, "p99_us": p99,
                          "hbm_frac_wall": total * OE_EXEC_BYTES_PER_TXN / dt / 1e9 / peak}
        if bt is not None:
            ch = bt.choice()
            names = {G.KSET: "kset", G.TPL: "tpl", G.PART: "part"}
            rec["segments"] = ch["bulks_run"]
            rec["choice"] = {"strategy": names.get(ch["strategy"]), "segment_capacity": ch["bulk_size"],
                             "block": ch["block_threads"], "tuned": ch["tuned"],
                             "measured": [{"strategy": names.get(m["strategy"]), "capacity": m["bulk"],
                                           "block": m["block"], "ns_per_txn": m["ns_per_txn"]}
                                          for m in ch["measured"]]}
            bt.close()
        out[label] = rec
        db.close()
    if args.cpu_baseline:
        out["cpu_baseline"] = oracle_oe_rate(init, stream_a, sizes_a, args.cpu_budget_s)
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(bulks, budget_s, max_bulks=None):
    import oracle
    oracle.build()
    o = oracle.OracleDB(dc=W.dc_tables(BRANCHES, TELLERS, ACCOUNTS),
                        hist_cap=len(bulks[0]["ts"]) * (max_bulks or 64))
    done, t_exec = 0, 0.0
    k = 0
    while k == 0 or (t_exec < budget_s and (max_bulks is None or k < max_bulks)):
        b = bulks[k % len(bulks)]
        if o.hist_n + len(b["ts"]) > o.s.hist_cap:
            o.s.hist_n = 0   # reuse the history area; balances keep accumulating
        t0 = time.perf_counter()
        o.execute(b, R=1)
        t_exec += time.perf_counter() - t0
        done += len(b["ts"])
        k += 1
    return done, t_exec, k


def oracle_oe_rate(init, stream_bulk, sizes, budget_s):
    """The oracle on the order-entry stream's bulks, one after another, until
    about budget_s of CPU time (a bounded sample of the same stream)."""
    import oracle
    oracle.build()
    total = sum(sizes)
    o = oracle.OracleDB(oe=init, ord_cap=total, ol_cap=total * 15, oid_cap=1 << 16)
    i, done, t_exec = 0, 0, 0.0
    for k in sizes:
        b = {key: stream_bulk[key][i:i + k] for key in ("ts", "type", "params")}
        b["P"] = stream_bulk["P"]
        t0 = time.perf_counter()
        o.execute(b, R=4)
        t_exec += time.perf_counter() - t0
        done += k
        i += k
        if t_exec > budget_s:
            break
    return {"value": done / t_exec, "unit": "txn/s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"the first {done} transactions of the stream, serial execution in timestamp order, "
                      f"{t_exec:.1f} s on one host core"}


def cpu_baseline(args, bulks):
    done, t, k = oracle_rate(bulks, args.cpu_budget_s)
    return {"value": done / t, "unit": "txn/s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"{k} bulks of {len(bulks[0]['ts'])} transactions, serial execution in "
                      f"timestamp order (Definition 1), {t:.1f} s on one host core"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = 1 << args.bulk_log2
    bulks = make_bulks(n, args.theta, 2, 0)
    # warm-up then timed steps, each a bounded sample: one bulk of n
    for i in range(args.warmup):
        oracle_rate(bulks[i % 2:], 0.0, max_bulks=1)
    times = []
    for i in range(args.steps):
        done, t, _ = oracle_rate(bulks[i % 2:], 0.0, max_bulks=1)
        times.append(t)
    value = n * args.steps / sum(times)
    line = {
        "metric": METRIC, "value": value, "unit": "txn/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"debit-credit at scale: {BRANCHES} branches, {TELLERS} tellers, "
                               f"{ACCOUNTS} accounts, bulk 2^{args.bulk_log2}, theta {args.theta}",
                   "strategy": "serial", "bulk": n, "theta": args.theta},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "txn/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step one bulk of {n} transactions executed serially"},
        "e2e": {"value": value, "unit": "txn/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# small cases for kernel profiles (ncu): one bulk, run twice, no JSON line
# ---------------------------------------------------------------------------
PROFILE_CASES = {
    # name: (schema, bulk log2, theta, strategy, conflict mode)
    "dc_kset_paper_20": ("dc", 20, 0.0, "kset", "paper"),
    "dc_tpl_paper_20": ("dc", 20, 0.0, "tpl", "paper"),
    "dc_part_20": ("dc", 20, 0.0, "part", "paper"),
    "dc_part_zipf99_20": ("dc", 20, 0.99, "part", "paper"),
    "dc_tpl_zipf99_20": ("dc", 20, 0.99, "tpl", "paper"),
    "dc_tpl_relaxed_zipf99_20": ("dc", 20, 0.99, "tpl_relaxed", "paper"),
    "dc_scan_22": ("dc", 22, 0.0, "scan", "paper"),
    "oe_kset_paper_16": ("oe", 16, 0.0, "kset", "paper"),
    "oe_tpl_paper_16": ("oe", 16, 0.0, "tpl", "paper"),
}


def run_profile_case(name):
    import torch
    import paper_1103_3105_gb300 as G
    import __graft_entry__
    __graft_entry__.build()
    schema, lg, theta, strategy, mode_name = PROFILE_CASES[name]
    mode = G.CONFLICT_ADD if mode_name == "add" else G.CONFLICT_PAPER
    n = 1 << lg
    dev = torch.device("cuda", 0)
    if schema == "dc":
        db = G.Database(dc=(BRANCHES, TELLERS, ACCOUNTS), history_capacity=3 * n, max_bulk=n)
        db.register(G.DC_TYPES)
        bulk = W.dc_bulk(n, ACCOUNTS, theta, seed=W.seed_for(2, 22))
    else:
        n_wh, n_items = 64, 100_000
        db = G.Database(oe=(n_wh, n_items), order_capacity=4 * n, orderline_capacity=60 * n, max_bulk=n)
        db.register(G.OE_TYPES)
        for t, rows in W.oe_rows(W.oe_tables(n_wh, n_items=n_items, seed=W.seed_for(4))).items():
            db.load(t, rows)
        bulk = W.oe_bulk(n, n_wh, n_items=n_items, seed=W.seed_for(4, 2))
    d = {k: torch.from_numpy(bulk[k]).to(dev) for k in ("ts", "type", "params")}
    for r in range(2):
        b = db.submit(d["ts"] + r * n, d["type"], d["params"])
        b.execute(strategy, conflict_mode=mode, timing=True)
        st = b.sync()
        b.free()
        print(f"{name} run {r}: execute {st['ms_execute']:.3f} ms, analysis {st['ms_analysis']:.3f} ms, "
              f"depth {st['depth']}", flush=True)
    db.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gputx", choices=["gputx", "reference"])
    ap.add_argument("--strategy", default="kset",
                    choices=["kset", "part", "tpl", "auto", "scan", "part_relaxed", "tpl_relaxed"])
    ap.add_argument("--mode", default="paper", choices=["paper", "add"])
    ap.add_argument("--theta", type=float, default=0.0)
    ap.add_argument("--bulk-log2", type=int, default=22)
    ap.add_argument("--sweep", dest="sweep", action="store_true", default=True)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false")
    ap.add_argument("--sweep-budget-s", type=float, default=60.0)
    ap.add_argument("--cpu-baseline", dest="cpu_baseline", action="store_true", default=True)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-budget-s", type=float, default=10.0)
    ap.add_argument("--serve", dest="serve", action="store_true", default=True)
    ap.add_argument("--no-serve", dest="serve", action="store_false")
    ap.add_argument("--serve-rates", default="1e6,5e6,20e6,50e6")
    ap.add_argument("--serve-deadlines-us", default="1000,10000")
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--serve-strategy", default="kset", choices=["kset", "part", "tpl", "auto"])
    ap.add_argument("--serve-subscribers", type=int, default=20_000_000)
    ap.add_argument("--serve-zero-set-max-rate", type=float, default=5e6)
    ap.add_argument("--batched", dest="batched", action="store_true", default=True)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batch-txns", type=int, default=3_000_000)
    ap.add_argument("--subscriber", dest="subscriber", action="store_true", default=True)
    ap.add_argument("--no-subscriber", dest="subscriber", action="store_false")
    ap.add_argument("--sub-subscribers", type=int, default=10_000_000)
    ap.add_argument("--detail-out", default="bench_detail.json",
                    help="file for the sections beside the headline (sweep, serving, batching, "
                         "subscriber schema); '' writes none")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES),
                    help="run one small case twice for a kernel profile and exit (no JSON line)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        # several GPUs: the replicas' timed steps only.  The CPU baseline is an
        # N = 1 figure, and the single-GPU characterisations (sweep, serving,
        # batching, subscriber schema) would hold every GPU for minutes
        args.cpu_baseline = args.sweep = args.serve = args.batched = args.subscriber = False
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_engine(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
