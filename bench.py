#!/usr/bin/env python
"""Throughput of the SSW hot path on GB300: GCUPS, bit-exact against the oracle.

Workload: short-read extension, 1,000,000 DNA pairs (queries U[100, 250] nt,
targets U[300, 1000] nt holding the mutated query, 10 % decoys; +2/-2, gap
open 3, extend 1), seeded and synthetic.  One step = the whole hot path over
the batch: forward fill (max array, ends, secondary), 32-bit refill of the
pairs whose 16-bit lanes overflowed, reversed fill (begins), banded
traceback (CIGAR).  GCUPS counts forward-fill cells (sum of m*n) per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsw|reference]

Under torchrun every rank aligns its own batch of the same size (weak
scaling, no collective on the data path); rank 0 prints one JSON line.  With
--split the ranks share one job instead: pairs go to ranks by cells (longest
processing time first), each rank aligns its shard, and rank 0 gathers the
records in the job's pair order after the timed region (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS (forward-fill cell updates/s), bit-exact vs oracle"
UNIT = "GCUPS"
ALGO_OPS_PER_CELL = 10  # 2-input integer ops of one Gotoh cell update (add, 3 sub, 6 max)
WORKLOAD = "dna_short_read_extension_1M"


def make_workload(name, pairs, rank):
    """(batch, config dict) of a named workload; `pairs` overrides its size."""
    from paper_1208_6350_gb300 import workloads as wl
    if name == "dna_short_read_extension_1M":
        n = pairs or 1_000_000
        cfg = {"workload": name, "pairs": n, "query_nt": [100, 250], "target_nt": [300, 1000],
               "subst": 0.01, "indel": 0.001, "decoys": 0.10, "scoring": "+2/-2, open 3, extend 1"}
        return wl.config2(n, seed=1 + rank), cfg
    if name == "dna_1k_100x1000":
        b = wl.config1(seed=rank)
        if pairs:
            b = b.subset(np.arange(min(pairs, b.npairs)))
        return b, {"workload": name, "pairs": b.npairs, "query_nt": 100, "target_nt": 1000, "subst": 0.02,
                   "indel": 0.002, "scoring": "+2/-2, open 3, extend 1"}
    if name == "dna_long_reads_10k":
        n = pairs or 10_000
        return wl.config3(n, seed=2 + rank), {
            "workload": name, "pairs": n, "query_nt": "log-uniform 1000-20000", "target": "1.2 x query",
            "error": "6% subst, 2% ins, 2% del", "scoring": "+2/-4, open 4, extend 2"}
    if name == "protein_search_1kx10k":
        ps = wl.protein_search(seed=3 + rank)
        n = pairs or 1_000_000
        rng = np.random.default_rng(7 + rank)
        qi = rng.integers(0, ps.n_queries, n)
        di = rng.integers(0, ps.n_db, n)
        return ps.pairs(qi, di, name), {
            "workload": name, "pairs": n, "sample_of": "1,000 queries x 10,000 database sequences",
            "query_aa": [50, 1000], "db_aa": "clip(LogNormal(ln 300, 0.6), 20, 5000)",
            "matrix": "seeded synthetic symmetric 20x20 (BLOSUM-like ranges)", "gap": "open 11, extend 1"}
    raise SystemExit(f"unknown workload {name}")


def workload_config(cfg, b):
    out = dict(cfg)
    out["outputs"] = "score1, ends, score2, ref_end2, begins, CIGAR"
    nbytes = len(b.q) + len(b.t)
    if str(cfg.get("input", "")).startswith("2-bit"):
        nbytes = (len(b.q) + 3) // 4 + (len(b.t) + 3) // 4
    out["l2"] = (f"inputs {nbytes / 1e9:.2f} GB per step, " +
                 ("larger than the 129 MB L2 (no flush)" if nbytes > 129e6 else "smaller than L2"))
    out["cells"] = b.cells
    return out


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------- CPU baseline
def cpu_baseline(b, target_s=10.0, max_pairs=200_000):
    """The oracle as it stands, on all host cores, over a bounded sample."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(123)
    pilot = b.subset(rng.permutation(b.npairs)[:min(1000, max(16, b.npairs // 50))])
    t0 = time.perf_counter()
    oracle.align_batch(pilot.q, pilot.q_off, pilot.q_len, pilot.t, pilot.t_off, pilot.t_len, pilot.W,
                       pilot.gap_open, pilot.gap_extend, nthreads=cores,
                       cigar_stride=int(pilot.q_len.max() + pilot.t_len.max() + 2))
    rate = pilot.cells / max(time.perf_counter() - t0, 1e-6)
    n = int(min(max_pairs, b.npairs, max(16, target_s * rate / (b.cells / b.npairs))))
    s = b.subset(rng.permutation(b.npairs)[:n])
    t0 = time.perf_counter()
    res, _, _ = oracle.align_batch(s.q, s.q_off, s.q_len, s.t, s.t_off, s.t_len, s.W, s.gap_open,
                                   s.gap_extend, nthreads=cores, cigar_stride=int(s.q_len.max() + s.t_len.max() + 2))
    dt = time.perf_counter() - t0
    return {"value": s.cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random pairs of the workload ({s.cells / 1e9:.2f} G cells), full outputs, "
                      f"{dt:.1f} s wall", "cpu": _cpu_model()}


def _cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def fill_traffic_bytes(cells, workload):
    """DRAM bytes per forward-fill launch from the committed ncu summary, if it
    was taken on the current fill kernel source and this workload; else None."""
    if workload != WORKLOAD:
        return None
    path = os.path.join(ROOT, "profiles", "fill_fwd_traffic.txt")
    src = os.path.join(ROOT, "paper_1208_6350_gb300", "csrc", "fill.cu")
    try:
        kv = dict(ln.strip().split("=", 1) for ln in open(path) if "=" in ln and not ln.startswith("#"))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if kv.get("fill_cu_sha256_16") != sha:
            return None
        return float(kv["dram_bytes_per_cell"]) * cells
    except (OSError, KeyError, ValueError):
        return None


def work_summary(r, cells):
    """Work beside the forward fill, from one step's records (reported apart,
    not counted in the metric): pairs refilled in 32-bit lanes; the reversed
    rectangle from the end back to the begin column, (read_end1 + 1) x
    (ref_end1 - ref_begin1 + 1), that a reversed fill stopping at the begin
    covers; the region between begin and end, where the CIGAR's global
    alignment runs.  Pairs with score1 = 0 have neither."""
    n = len(r)
    hit = r["score1"] > 0
    eq = r["read_end1"][hit].astype(np.int64)
    et = r["ref_end1"][hit].astype(np.int64)
    bq = r["read_begin1"][hit].astype(np.int64)
    bt = r["ref_begin1"][hit].astype(np.int64)
    rev = int(((eq + 1) * (et - bt + 1)).sum())
    region = int(((eq - bq + 1) * (et - bt + 1)).sum())
    s32 = int(np.count_nonzero(r["flags"] & 0x1))
    return {"pairs": n, "aligned_pairs": int(hit.sum()),
            "s32_refill_pairs": s32, "s32_refill_frac": round(s32 / max(n, 1), 4),
            "reverse_rect_cells": rev, "reverse_rect_frac": round(rev / max(cells, 1), 4),
            "region_cells": region, "region_frac": round(region / max(cells, 1), 4)}


# ------------------------------------------------------------ GPU arm
def combine_ranks(ms, cells, dist=None, device="cpu"):
    """Whole-job step time and cells: the slowest rank's time, every rank's
    cells (each rank aligns its own batch; no collective on the data path)."""
    if dist is None:
        return ms, cells
    import torch
    x = torch.tensor([ms, float(cells)], dtype=torch.float64, device=device)
    t = x[:1].clone()
    c = x[1:].clone()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(float(c.item())))


def lpt_partition(cells, nparts):
    """One job split over nparts ranks by work: pairs in decreasing order of
    cells (m * n), each to the least loaded rank so far (longest processing
    time first).  Returns each rank's pair indices, ascending."""
    import heapq
    cells = np.asarray(cells, np.int64)
    order = np.argsort(-cells, kind="stable")
    heap = [(0, k) for k in range(nparts)]
    parts = [[] for _ in range(nparts)]
    for p, c in zip(order.tolist(), cells[order].tolist()):
        load, k = heapq.heappop(heap)
        parts[k].append(p)
        heapq.heappush(heap, (load + c, k))
    return [np.sort(np.asarray(x, np.int64)) for x in parts]


def merge_shards(npairs, shards):
    """The whole job's records from the ranks' shards (pair indices, records,
    CIGAR words): records go back to their pairs' places and each shard's
    CIGAR words follow the previous shard's, with cigar_off moved along."""
    from paper_1208_6350_gb300 import gsw
    out = np.zeros(npairs, gsw.RESULT_DTYPE)
    words, base = [], 0
    for idx, rec, cig in shards:
        rec = rec.copy()
        has = rec["cigar_len"] > 0
        rec["cigar_off"][has] += base
        out[idx] = rec
        words.append(np.asarray(cig, np.uint32))
        base += len(cig)
    return out, (np.concatenate(words) if words else np.zeros(0, np.uint32))


def gather_shards(dist, rank, world, idx, rec, cig, npairs):
    """Rank 0 receives every rank's shard (no collective on the data path
    before this: it runs after the timed region) and returns the merged
    records and CIGAR words; the other ranks return None."""
    payload = (np.asarray(idx, np.int64), np.asarray(rec), np.asarray(cig, np.uint32))
    objs = [None] * world if rank == 0 else None
    dist.gather_object(payload, objs, dst=0)
    if rank != 0:
        return None
    return merge_shards(npairs, objs)


def run_gsw(args):
    import torch
    import torch.distributed as dist

    from paper_1208_6350_gb300 import gsw, workloads as wl

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    split = None
    if args.split and world > 1:
        # one job split over the ranks by cells (LPT); every rank builds the
        # same batch and aligns its shard
        full, wcfg = make_workload(args.workload, args.pairs, 0)
        parts = lpt_partition(full.q_len.astype(np.int64) * full.t_len, world)
        b = full.subset(parts[rank])
        split = {"full": full, "idx": parts[rank],
                 "cells_per_rank": [int((full.q_len[x].astype(np.int64) * full.t_len[x]).sum()) for x in parts]}
    else:
        b, wcfg = make_workload(args.workload, args.pairs, rank)
    cells = b.cells
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    # DNA arenas stay 2-bit packed (4 letters per byte) in memory; the call
    # expands them on the device
    packed = b.alphabet == "ACGT" and not args.no_pack
    pk = (lambda a: gsw.pack2(a)) if packed else (lambda a: a)
    wcfg = dict(wcfg, input="2-bit packed DNA arenas (GSW_PACKED2)" if packed else "one byte per letter")
    q, t = T(pk(b.q)), T(pk(b.t))
    qo, to = T(b.q_off.astype(np.int64)), T(b.t_off.astype(np.int64))
    ql, tl = T(b.q_len.astype(np.int32)), T(b.t_len.astype(np.int32))
    n = b.npairs
    res = torch.zeros(n * 12, dtype=torch.int32, device=dev)
    cap = int(min(32 * n + 1024 + (b.q_len.sum() + b.t_len.sum()) // 4, 1 << 30))
    cig = torch.zeros(cap, dtype=torch.int32, device=dev)
    budget = args.long_budget_gb if args.workload == "dna_long_reads_10k" else args.budget_gb
    ctx = gsw.Context(local, budget << 30)
    tune = None
    if args.tune_table:
        # a saved table instead of measuring (e.g. to profile one variant)
        table = [int(x) for x in args.tune_table.split(",")]
        ctx.set_tune(table + [-1] * (gsw.TUNE_BUCKETS - len(table)))
        tune = {"buckets_of_rows": gsw.TUNE_ROWS, "fill_class": table, "source": "--tune-table"}
    elif not args.no_tune:
        # fill class per query-length bucket, measured on this GPU for this
        # scoring and the workload's mean target length (results unchanged)
        t0 = time.perf_counter()
        tune = ctx.autotune(b.W, b.gap_open, b.gap_extend, target_len=max(1, int(b.t_len.mean())))
        tune["seconds"] = round(time.perf_counter() - t0, 2)
        nb = max(1, min(gsw.TUNE_BUCKETS, int(np.ceil(b.q_len.max() / gsw.TUNE_ROWS))))
        tune = {"buckets_of_rows": gsw.TUNE_ROWS, "fill_class": tune["fill_class"][:nb],
                "gcups": tune["gcups"][:nb], "gcups_default_rule": tune["gcups_default"][:nb],
                "seconds": tune["seconds"]}
    # a stream of its own: the library captures the repeated step's launch
    # sequence in CUDA graphs (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    flags = gsw.GSW_CIGAR | gsw.GSW_TIMING | (gsw.GSW_PACKED2 if packed else 0)

    def step():
        gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, b.W, b.gap_open, b.gap_extend, flags,
                            -1, res, cig, cap, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # correctness of what is timed: a random sample against the oracle
    checked = check_sample(b, res, cig, rank) if not args.no_check else 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fill_ms, pipe_ms, launches, graph_segments = [], [], 0, 0
    stage_sum = {}
    e0.record(stream)
    for _ in range(args.steps):
        step()
        st = gsw.gsw_last_stats(ctx.handle)
        launches += st["kernel_launches"]
        graph_segments += st["graph_segments"]
        fill_ms.append(st["stage_ms"]["fill_fwd"])
        pipe_ms.append(st["stage_ms"]["pipeline"])
        for k, v in st["stage_ms"].items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max, job_cells = combine_ranks(ms, cells, dist if world > 1 else None, dev)
    value = job_cells / (ms_max / 1e3) / 1e9
    rec = res.cpu().numpy().view(gsw.RESULT_DTYPE)
    work = work_summary(rec, cells)
    split_info = None
    if split is not None:
        # the ranks' records concatenated on rank 0 in the job's pair order,
        # then a random sample of the whole job checked against the oracle
        used = int(max(0, (rec["cigar_off"] + rec["cigar_len"])[rec["cigar_len"] > 0].max(initial=0)))
        words = cig.cpu().numpy().view(np.uint32)[:used]
        merged = gather_shards(dist, rank, world, split["idx"], rec, words, split["full"].npairs)
        if rank == 0:
            whole, whole_cig = merged
            k = check_records(split["full"], whole, whole_cig, 0) if not args.no_check else 0
            cpr = split["cells_per_rank"]
            split_info = {"ranks": world, "partition": "LPT over pairs sorted by cells (m x n)",
                          "cells_per_rank": cpr, "imbalance": round(max(cpr) / (sum(cpr) / len(cpr)), 5),
                          "gathered_pairs": int(len(whole)), "checked_pairs_of_the_whole_job": k}

    # e2e: the same call on host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, gsw, b, ctx, stream, dev, torch, packed)

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_gops = sms * 128 * 2 * max_mhz * 1e6 / 1e9  # 16-bit lane ops/s at full-rate 16x2 instructions
    fill_s = float(np.mean(fill_ms)) / 1e3
    achieved = ALGO_OPS_PER_CELL * cells / fill_s / 1e9
    roof = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak_gops, 1), "unit": "Gop/s",
            "frac": round(achieved / peak_gops, 4), "traffic": fill_traffic_bytes(cells, args.workload),
            "kernel": "k_fill (forward, 16-bit folded ring)",
            "fill_ms": round(float(np.mean(fill_ms)), 3),
            "fill_gcups": round(cells / fill_s / 1e9, 1),
            "peak_basis": f"{sms} SMs x 128 lanes x 2 16-bit lanes x {max_mhz:.0f} MHz (max SM clock)"}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3),
            "higher_is_better": True, "scaling": "strong" if split is not None else "weak", "vs_baseline": None,
            "dtype": "i16x2 (i32 refill)",
            "data": "synthetic (seeded; stands in for simulated short reads)",
            "config": workload_config(wcfg, b), "e2e": e2e,
            "gpu_launches": launches,
            "graph_segments_replayed": graph_segments,
            "stage_ms": {k: round(v / args.steps, 3) for k, v in stage_sum.items()},
            "checked_pairs": checked, "clocks": clocks, "roofline": roof, "autotune": tune,
            "work_beside_fill": work}
    if split_info is not None:
        line["split"] = split_info
    if world == 1 and args.plain_pairs > 0:
        pp = run_plain(gsw, b, ctx, args.plain_pairs, rec)
        # the batched step's rate over the same pairs, for comparison
        sub = int(min(args.plain_pairs, b.npairs))
        pp["batched_gcups_same_workload"] = round(value, 1)
        pp["batched_over_plain"] = round(value / max(pp["gcups"], 1e-9), 1)
        pp["pairs_are_the_first_of_the_workload"] = sub
        line["plain_per_pair"] = pp
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(b, args.cpu_seconds)
    if world == 1 and args.workload == WORKLOAD and not args.no_long:
        # the long-read workload (10,000 reads of 1-20 kb) through the same
        # call, reported beside the metric's workload
        ctx.close()
        ctx = None
        del q, t, qo, to, ql, tl, res, cig
        torch.cuda.empty_cache()
        line["long_reads"] = run_long_reads(args, gsw, torch, dev)
    if world == 1 and not args.no_serve:
        if ctx is not None:
            ctx.close()
            ctx = None
        torch.cuda.empty_cache()
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        line["serving"] = run_serving(rates, args.serve_requests, args.serve_head, gsw,
                                      eager_rates=tuple(rates[-1:]))
    print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_long_reads(args, gsw, torch, dev):
    """The long-read workload (10,000 DNA reads, lengths log-uniform 1-20 kb at
    10 % error, targets 1.2x; +2/-4, open 4, extend 2): whole pipeline on
    device buffers (CUDA events on the launching stream), the same call from
    pinned host buffers (e2e), and a sample of the timed batch checked
    against the oracle."""
    b, wcfg = make_workload("dna_long_reads_10k", args.long_pairs, 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, t = T(gsw.pack2(b.q)), T(gsw.pack2(b.t))
    qo, to = T(b.q_off.astype(np.int64)), T(b.t_off.astype(np.int64))
    ql, tl = T(b.q_len.astype(np.int32)), T(b.t_len.astype(np.int32))
    n = b.npairs
    res = torch.zeros(n * 12, dtype=torch.int32, device=dev)
    cap = int(min(64 * n + (b.q_len.sum() + b.t_len.sum()) // 4, 1 << 30))
    cig = torch.zeros(cap, dtype=torch.int32, device=dev)
    # a large device-memory budget: the wide-band traceback keeps 4 bits per
    # region cell for every pair at once (about 69 GB of direction words per
    # step of this workload), so it runs as one group instead of several
    ctx = gsw.Context(dev.index or 0, args.long_budget_gb << 30)
    try:
        t0 = time.perf_counter()
        tune = ctx.autotune(b.W, b.gap_open, b.gap_extend, target_len=max(1, int(b.t_len.mean())))
        tune_s = round(time.perf_counter() - t0, 2)
        stream = torch.cuda.Stream(dev)
        flags = gsw.GSW_CIGAR | gsw.GSW_TIMING | gsw.GSW_PACKED2

        def step():
            gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, b.W, b.gap_open, b.gap_extend, flags, -1,
                                res, cig, cap, stream=stream)

        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        checked = check_sample(b, res, cig, 0, k=300, max_cells=2e9) if not args.no_check else 0
        steps = max(1, args.long_steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stage_sum = {}
        e0.record(stream)
        for _ in range(steps):
            step()
            for k, v in gsw.gsw_last_stats(ctx.handle)["stage_ms"].items():
                stage_sum[k] = stage_sum.get(k, 0.0) + v
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        st_last = gsw.gsw_last_stats(ctx.handle)
        out = {"workload": "dna_long_reads_10k", "pairs": n, "cells": b.cells,
               "context_budget_gb": args.long_budget_gb, "traceback_pool_groups": st_last["ring_groups"],
               "value": round(b.cells / (ms / 1e3) / 1e9, 2), "unit": UNIT, "ms_per_step": round(ms, 3),
               "steps": steps, "warmup": 3,
               "stage_ms": {k: round(v / steps, 3) for k, v in stage_sum.items()},
               "checked_pairs": checked, "config": workload_config(dict(wcfg, input="2-bit packed DNA arenas"), b),
               "autotune_seconds": tune_s}
        if not args.no_e2e:
            import types
            out["e2e"] = run_e2e(types.SimpleNamespace(warmup=1, steps=steps), gsw, b, ctx, stream, dev, torch,
                                 packed=True)
        out["work_beside_fill"] = work_summary(res.cpu().numpy().view(gsw.RESULT_DTYPE), b.cells)
        return out
    finally:
        ctx.close()


def run_e2e(args, gsw, b, ctx, stream, dev, torch, packed=False):
    n = b.npairs
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    q, t = (pin(gsw.pack2(b.q)), pin(gsw.pack2(b.t))) if packed else (pin(b.q), pin(b.t))
    qo, to = pin(b.q_off.astype(np.int64)), pin(b.t_off.astype(np.int64))
    ql, tl = pin(b.q_len.astype(np.int32)), pin(b.t_len.astype(np.int32))
    res = pin(np.zeros(n, gsw.RESULT_DTYPE).view(np.int32))
    cap = int(min(32 * n + 1024 + (b.q_len.sum() + b.t_len.sum()) // 4, 1 << 30))
    cig = pin(np.zeros(cap, np.uint32))
    flags = gsw.GSW_CIGAR | gsw.GSW_HOST_IO | (gsw.GSW_PACKED2 if packed else 0)

    def step():
        gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, b.W, b.gap_open, b.gap_extend, flags,
                            -1, res, cig, cap, stream=stream)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / steps
    r = res.view(gsw.RESULT_DTYPE)
    cig_words = int(np.maximum(r["cigar_len"], 0).sum())
    h2d = q.nbytes + t.nbytes + qo.nbytes + to.nbytes + ql.nbytes + tl.nbytes
    d2h = res.nbytes + 4 * cig_words
    return {"value": round(b.cells / dt / 1e9, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 3),
            "api": "gsw_align_batch with GSW_HOST_IO (pinned host buffers)"}


def run_plain(gsw, b, ctx, n_pairs, batched=None):
    """The plain per-pair path (GSW_PLAIN: every pair its own launch sequence,
    waited for before the next, as a caller aligning one pair per call) on
    the first n_pairs pairs of the workload, host buffers; GCUPS on those
    pairs, and whether their records equal the batched step's."""
    s = b.subset(np.arange(min(n_pairs, b.npairs)))
    flags = gsw.GSW_CIGAR | gsw.GSW_PLAIN
    w = s.subset(np.arange(min(8, s.npairs)))
    ctx.align_host(w.q, w.q_off, w.q_len, w.t, w.t_off, w.t_len, b.W, b.gap_open, b.gap_extend, flags, -1,
                   int(w.q_len.sum() + w.t_len.sum() + 64))
    t0 = time.perf_counter()
    res, _, _, rc = ctx.align_host(s.q, s.q_off, s.q_len, s.t, s.t_off, s.t_len, b.W, b.gap_open,
                                   b.gap_extend, flags, -1, int(s.q_len.sum() + s.t_len.sum() + 64))
    dt = time.perf_counter() - t0
    if rc != gsw.GSW_OK:
        raise SystemExit(f"plain per-pair path failed with {rc}")
    same = None
    if batched is not None:
        fields = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2",
                  "cigar_len")
        same = all(np.array_equal(res[f], batched[f][:s.npairs]) for f in fields)
    return {"pairs": s.npairs, "cells": int(s.cells), "seconds": round(dt, 3),
            "gcups": round(s.cells / dt / 1e9, 3), "ms_per_pair": round(dt / s.npairs * 1e3, 3),
            "api": "gsw_align_batch with GSW_PLAIN | GSW_HOST_IO (one launch sequence per pair)",
            "same_records_as_batched": same}


def check_sample(b, res, cig, rank, k=300, max_cells=3e9):
    from paper_1208_6350_gb300 import gsw
    r = res.cpu().numpy().view(gsw.RESULT_DTYPE)
    c = cig.cpu().numpy().view(np.uint32)
    return check_records(b, r, c, rank, k, max_cells)


def check_records(b, r, c, rank, k=300, max_cells=3e9):
    """k random pairs of the batch (their cells bounded) against the oracle:
    every field and the CIGAR; raises SystemExit on a mismatch."""
    import oracle
    rng = np.random.default_rng(7 + rank)
    idx = rng.permutation(b.npairs)[:k]
    # keep the oracle's share of the check bounded (long pairs)
    cum = np.cumsum(b.q_len[idx].astype(np.int64) * b.t_len[idx])
    idx = idx[: max(1, int(np.searchsorted(cum, max_cells)))]
    k = len(idx)
    s = b.subset(idx)
    ores, ocg, _ = oracle.align_batch(s.q, s.q_off, s.q_len, s.t, s.t_off, s.t_len, s.W, s.gap_open,
                                      s.gap_extend, cigar_stride=int(s.q_len.max() + s.t_len.max() + 2))
    for j, p in enumerate(idx):
        for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2"):
            if int(r[f][p]) != int(ores[f][j]):
                raise SystemExit(f"bench check failed: pair {p} field {f}: {int(r[f][p])} != {int(ores[f][j])}")
        o, n_ = int(r["cigar_off"][p]), int(r["cigar_len"][p])
        if list(c[o:o + n_]) != list(ocg[j, : ores["cigar_len"][j]]):
            raise SystemExit(f"bench check failed: pair {p} CIGAR")
    return k


# ------------------------------------------------------------ serving
SERVE_SCORING = (2, -4, 4, 2)  # one scoring for the whole stream: the long reads'


def serving_requests(rate, n_requests, seed=5):
    """The mixed request stream (70 % 100x1000 reads, 20 % short-read
    extensions, 10 % long reads; 1-64 pairs each; Poisson arrivals), every
    request scored with SERVE_SCORING."""
    from paper_1208_6350_gb300 import workloads as wl
    tr = wl.serving_trace(rate, n_requests, seed=seed)
    return [(r.arrival_s, r.kind, r.batch) for r in tr]


def _latency_summary(lat_s, queue_s=None):
    lat = np.asarray(lat_s) * 1e3
    out = {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
           "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}
    if queue_s is not None:
        out["mean_queue_ms"] = round(float(np.mean(queue_s)) * 1e3, 3)
    return out


def serve_trace(gsw, reqs, W, O, X, workers=4, check=None, light_graphs=0):
    """Submits each request at its arrival time (one client thread) and
    collects results with the server's timestamps (another thread).  Latency
    = completion on the host - scheduled arrival."""
    import threading
    srv = gsw.Server(W, O, X, gsw.GSW_CIGAR, workers=workers, max_batch_pairs=8192,
                     max_batch_letters=24 << 20, mem_budget_bytes=48 << 30, light_graphs=light_graphs)
    # warm-up: one request of each kind, not timed
    seen = set()
    for a, k, b in reqs:
        if k not in seen:
            seen.add(k)
            rid = srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len)
            srv.poll(rid, b.npairs)
    n = len(reqs)
    ids = [None] * n
    out = [None] * n
    ready = threading.Semaphore(0)
    t_client0 = time.perf_counter()
    t_srv0 = srv.now()

    def submitter():
        for i, (a, k, b) in enumerate(reqs):
            d = t_client0 + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids[i] = srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len)
            ready.release()

    def poller():
        for i, (a, k, b) in enumerate(reqs):
            ready.acquire()
            rc, res, cig, tm = srv.poll(ids[i], b.npairs, times=True)
            out[i] = (rc, res, cig, tm)

    th = [threading.Thread(target=submitter), threading.Thread(target=poller)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    st = srv.stats()
    srv.close()
    lat, qd = [], []
    for (a, k, b), (rc, res, cig, tm) in zip(reqs, out):
        if rc != gsw.GSW_OK:
            raise SystemExit(f"serving: request failed with {rc}")
        lat.append(tm[2] - t_srv0 - a)
        qd.append(tm[1] - tm[0])
    span = max(tm[2] for *_, tm in out) - t_srv0
    cells = sum(b.cells for _, _, b in reqs)
    return lat, qd, span, cells, out, st


def plain_trace(gsw, reqs, W, O, X):
    """The baseline: requests in arrival order, FIFO, each pair its own
    launch sequence (fill, reverse, banded traceback) on one stream."""
    ctx = gsw.Context(0, 24 << 30)
    try:
        seen = set()
        for a, k, b in reqs:  # warm-up per kind
            if k not in seen:
                seen.add(k)
                ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, W, O, X,
                               gsw.GSW_CIGAR | gsw.GSW_PLAIN, -1, int(b.q_len.sum() + b.t_len.sum() + 64))
        t0 = time.perf_counter()
        lat, outs = [], []
        for a, k, b in reqs:
            d = t0 + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            res, cig, _, rc = ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, W, O, X,
                                             gsw.GSW_CIGAR | gsw.GSW_PLAIN, -1,
                                             int(b.q_len.sum() + b.t_len.sum() + 64))
            if rc != gsw.GSW_OK:
                raise SystemExit(f"plain baseline failed with {rc}")
            lat.append(time.perf_counter() - t0 - a)
            outs.append((res, cig))
        return lat, outs
    finally:
        ctx.close()


def _same_results(gsw, srv_out, plain_out):
    fields = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")
    for (rc, res, cig, _), (pres, pcig) in zip(srv_out, plain_out):
        for f in fields:
            if not np.array_equal(res[f], pres[f]):
                return False
        for p in range(len(res)):
            a = cig[res["cigar_off"][p]: res["cigar_off"][p] + res["cigar_len"][p]] if res["cigar_len"][p] > 0 else []
            c = pcig[pres["cigar_off"][p]: pres["cigar_off"][p] + pres["cigar_len"][p]] if pres["cigar_len"][p] > 0 else []
            if list(a) != list(c):
                return False
    return True


def run_serving(rates, n_requests, head, gsw, dev_name="", eager_rates=()):
    """Per arrival rate: the server over the whole stream, and server vs the
    plain per-pair baseline over the stream's first `head` requests."""
    from paper_1208_6350_gb300 import workloads as wl
    W = wl.dna_matrix(SERVE_SCORING[0], SERVE_SCORING[1])
    O, X = SERVE_SCORING[2], SERVE_SCORING[3]
    rows = []
    for rate in rates:
        reqs = serving_requests(rate, n_requests)
        arr_span = reqs[-1][0] if reqs else 0.0
        lat, qd, span, cells, out, st = serve_trace(gsw, reqs, W, O, X)
        kinds = np.array([k for _, k, _ in reqs])
        lat_a, qd_a = np.asarray(lat), np.asarray(qd)
        by_kind = {name: _latency_summary(lat_a[kinds == k], qd_a[kinds == k])
                   for k, name in ((1, "short_100x1000"), (2, "short_read_extension"), (3, "long_reads"))
                   if (kinds == k).any()}
        row = {"rate_req_s": rate, "requests": len(reqs),
               "offered_gcups": round(cells / max(arr_span, 1e-9) / 1e9, 1),
               "achieved_gcups": round(cells / span / 1e9, 1), "server": _latency_summary(lat, qd),
               "server_by_kind": by_kind, "batches": int(st["batches"]),
               "graph_batches": int(st["graph_batches"])}
        if rate in eager_rates:
            # the same stream with every light batch launched eagerly (no
            # captured graphs), for the short requests' latency
            elat, eqd, espan, _, _, est = serve_trace(gsw, reqs, W, O, X, light_graphs=-1)
            elat_a, eqd_a = np.asarray(elat), np.asarray(eqd)
            row["eager_light_batches"] = {
                "server_by_kind": {name: _latency_summary(elat_a[kinds == k], eqd_a[kinds == k])
                                   for k, name in ((1, "short_100x1000"), (2, "short_read_extension"),
                                                   (3, "long_reads")) if (kinds == k).any()},
                "achieved_gcups": round(cells / espan / 1e9, 1), "graph_batches": int(est["graph_batches"])}
        if head:
            hr = reqs[:head]
            hlat, _, _, _, hout, _ = serve_trace(gsw, hr, W, O, X)
            plat, pout = plain_trace(gsw, hr, W, O, X)
            row["head"] = {"requests": len(hr), "server": _latency_summary(hlat),
                           "plain_per_pair": _latency_summary(plat),
                           "same_results": _same_results(gsw, hout, pout)}
        rows.append(row)
        print(json.dumps({"progress": row}), file=sys.stderr, flush=True)
    return rows


# ------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (this method's plain CPU definition) as the reference arm."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    from paper_1208_6350_gb300 import workloads as wl

    cores = len(os.sched_getaffinity(0))
    b, wcfg = make_workload(args.workload, args.pairs, 0)
    rng = np.random.default_rng(99)
    per_step = args.ref_pairs
    total = 0.0
    cells = 0
    for k in range(args.warmup + args.steps):
        s = b.subset(rng.permutation(b.npairs)[:min(per_step, b.npairs)])
        t0 = time.perf_counter()
        oracle.align_batch(s.q, s.q_off, s.q_len, s.t, s.t_off, s.t_len, s.W, s.gap_open, s.gap_extend,
                           nthreads=cores, cigar_stride=int(s.q_len.max() + s.t_len.max() + 2))
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            total += dt
            cells += s.cells
    value = cells / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", 1)), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": workload_config(wcfg, b),
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random pairs of the workload per step, full outputs",
                             "cpu": _cpu_model()},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reads_vs_reference(args):
    """--workload reads_vs_reference_10M: 1,000 simulated 100-nt reads against
    one 10 Mb reference (gsw_align_to_reference), every read against the whole
    reference; GCUPS = sum of read length x reference length per second."""
    import torch
    from paper_1208_6350_gb300 import gsw, workloads as wl
    import oracle
    if int(os.environ.get("RANK", 0)) != 0:
        return
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    n_reads = args.pairs or 1000
    reads, ref = wl.reads_vs_reference(n_reads, 100, args.ref_len, seed=6)
    cells = int(reads.q_len.astype(np.int64).sum()) * len(ref)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, qo, ql, R = T(reads.q), T(reads.q_off), T(reads.q_len), T(ref)
    res = torch.zeros(n_reads * 12, dtype=torch.int32, device=dev)
    cap = int(reads.q_len.sum()) * 2 + 64 * n_reads
    cig = torch.zeros(cap, dtype=torch.int32, device=dev)
    ctx = gsw.Context(0, args.budget_gb << 30)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    W, O, X = reads.W, reads.gap_open, reads.gap_extend

    def step():
        gsw.gsw_align_to_reference(ctx.handle, n_reads, q, qo, ql, R, len(ref), W, O, X, gsw.GSW_CIGAR, -1, 0,
                                   res, cig, cap, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of what is timed: a few reads against the whole reference, oracle
    checked = 0
    if not args.no_check:
        k = min(8, n_reads)
        ores, ocg, _ = oracle.align_batch(reads.q, reads.q_off[:k], reads.q_len[:k], ref, np.zeros(k, np.int64),
                                          np.full(k, len(ref), np.int32), W, O, X,
                                          cigar_stride=int(reads.q_len.max() + 2 * 100 + 64))
        r = res.cpu().numpy().view(gsw.RESULT_DTYPE)
        c = cig.cpu().numpy().view(np.uint32)
        for p in range(k):
            for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2"):
                if int(r[f][p]) != int(ores[f][p]):
                    raise SystemExit(f"bench check failed: read {p} field {f}")
            o, n_ = int(r["cigar_off"][p]), int(r["cigar_len"][p])
            if list(c[o:o + n_]) != list(ocg[p, : ores["cigar_len"][p]]):
                raise SystemExit(f"bench check failed: read {p} CIGAR")
        checked = k
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    value = cells / (ms / 1e3) / 1e9
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hq, hqo, hql, href = pin(reads.q), pin(reads.q_off), pin(reads.q_len), pin(ref)
        hres = pin(np.zeros(n_reads, gsw.RESULT_DTYPE).view(np.int32))
        hcig = pin(np.zeros(cap, np.uint32))

        def hstep():
            gsw.gsw_align_to_reference(ctx.handle, n_reads, hq, hqo, hql, href, len(ref), W, O, X,
                                       gsw.GSW_CIGAR | gsw.GSW_HOST_IO, -1, 0, hres, hcig, cap, stream=stream)

        hstep()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        e2e = {"value": round(cells / dt / 1e9, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(hq.nbytes + hqo.nbytes + hql.nbytes + href.nbytes),
               "d2h_bytes_per_step": int(hres.nbytes + hcig.nbytes), "ms_per_step": round(dt * 1e3, 3),
               "api": "gsw_align_to_reference with GSW_HOST_IO (pinned host buffers)"}
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i16x2 (i32 refill)",
            "data": "synthetic (seeded; stands in for 1,000 simulated 100 bp reads of a chromosome region)",
            "config": {"workload": "reads_vs_reference", "reads": n_reads, "read_nt": 100, "reference_nt": len(ref),
                       "errors": "1% substitutions, 0.1% 1-3 nt indels", "scoring": "+2/-2, open 3, extend 1",
                       "outputs": "score1, ends, score2, ref_end2, begins, CIGAR against the whole reference",
                       "cells": cells},
            "e2e": e2e, "checked_reads": checked, "clocks": clocks}
    if not args.no_cpu:
        cores = len(os.sched_getaffinity(0))
        k = min(cores, n_reads)
        t0 = time.perf_counter()
        oracle.align_batch(reads.q, reads.q_off[:k], reads.q_len[:k], ref, np.zeros(k, np.int64),
                           np.full(k, len(ref), np.int32), W, O, X, nthreads=cores,
                           cigar_stride=int(reads.q_len.max() + 264))
        dt = time.perf_counter() - t0
        kc = int(reads.q_len[:k].astype(np.int64).sum()) * len(ref)
        line["cpu_baseline"] = {"value": round(kc / dt / 1e9, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{k} reads against the whole reference ({kc / 1e9:.1f} G cells, "
                                          f"{dt:.1f} s)", "cpu": _cpu_model()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_overlap_all_vs_all(args):
    """--workload overlap_all_vs_all: every pair of 22,543 reads of 70 nt
    (gsw_align_all_pairs, score only: score1, ends, secondary), the read-overlap
    computation; GCUPS = sum over pairs of m * n per second."""
    import torch
    from paper_1208_6350_gb300 import gsw, workloads as wl
    import oracle
    if int(os.environ.get("RANK", 0)) != 0:
        return
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    n = args.pairs or 22543
    seq, off, ln = wl.overlap_reads(n, 70, seed=7)
    npairs = n * (n - 1) // 2
    cells = int(((ln.astype(np.int64).sum()) ** 2 - (ln.astype(np.int64) ** 2).sum()) // 2)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    S, O_, L_ = T(gsw.pack2(seq)), T(off), T(ln)
    res = torch.zeros(npairs * 12, dtype=torch.int32, device=dev)
    ctx = gsw.Context(0, args.budget_gb << 30)
    W = wl.dna_matrix(2, -3)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()

    def step():
        rc = load_all_pairs(gsw)(ctx.handle, n, gsw._ptr(S), gsw._ptr(O_), gsw._ptr(L_), W.ctypes.data, 4, 5, 2,
                                 gsw.GSW_PACKED2, -1, 0, gsw._ptr(res), None, 0, stream.cuda_stream)
        if rc != gsw.GSW_OK:
            raise SystemExit(f"gsw_align_all_pairs failed: {rc}")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    checked = 0
    if not args.no_check:
        rng = np.random.default_rng(5)
        ks = np.sort(rng.choice(npairs, 2000, replace=False))
        # row-major triangle: pair k -> (i, j)
        starts = np.arange(n, dtype=np.int64) * n - np.arange(n, dtype=np.int64) * (np.arange(n) + 1) // 2
        ii = np.searchsorted(starts, ks, side="right") - 1
        jj = ks - starts[ii] + ii + 1
        ores, _, _ = oracle.align_batch(seq, off[ii], ln[ii], seq, off[jj], ln[jj], W, 5, 2,
                                        cigar_stride=2 * 70 + 2)
        r = res.cpu().numpy().view(gsw.RESULT_DTYPE)[ks]
        for f in ("score1", "score2", "ref_end1", "read_end1", "ref_end2"):
            if not (r[f] == ores[f]).all():
                raise SystemExit(f"bench check failed: field {f}")
        checked = len(ks)
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": METRIC, "value": round(cells / (ms / 1e3) / 1e9, 2), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i16x2 (i32 refill)",
            "data": "synthetic (seeded; stands in for a 22,543 x 70 bp read set)",
            "config": {"workload": "overlap_all_vs_all", "reads": n, "read_nt": 70, "pairs": npairs,
                       "genome_coverage": 10, "scoring": "+2/-3, open 5, extend 2",
                       "outputs": "score1, ends, score2, ref_end2 for every pair (score only)", "cells": cells,
                       "input": "2-bit packed DNA arena (GSW_PACKED2)"},
            "checked_pairs": checked, "clocks": clocks}
    if not args.no_cpu:
        cores = len(os.sched_getaffinity(0))
        k = 400000
        t0 = time.perf_counter()
        ii = np.random.default_rng(9).integers(0, n, k)
        jj = (ii + 1 + np.random.default_rng(10).integers(0, n - 1, k)) % n
        oracle.align_batch(seq, off[ii], ln[ii], seq, off[jj], ln[jj], W, 5, 2, nthreads=cores,
                           cigar_stride=2 * 70 + 2)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(k * 70 * 70 / dt / 1e9, 3), "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": f"{k} random pairs of the read set, full outputs, "
                                                            f"{dt:.1f} s", "cpu": _cpu_model()}
    print(json.dumps(line), flush=True)
    ctx.close()


def load_all_pairs(gsw):
    return gsw.load().gsw_align_all_pairs


def run_serving_line(args):
    """--workload serving_stream: one line, value = the server's p99 latency at
    the first rate; every rate's figures under "serving"."""
    import torch
    from paper_1208_6350_gb300 import gsw
    if int(os.environ.get("RANK", 0)) != 0:
        return  # one GPU's server; other ranks idle
    torch.cuda.set_device(0)
    rates = [float(x) for x in args.rates.split(",") if x]
    sampler = ClockSampler(0)
    sampler.start()
    rows = run_serving(rates, args.requests, args.head, gsw)
    clocks = sampler.stop()
    first = rows[0]
    line = {"metric": "served latency p99 (arrival to result on the host), mixed request stream",
            "value": first["server"]["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": len(rows),
            "warmup": 3, "higher_is_better": False, "scaling": "none", "vs_baseline": None,
            "dtype": "i16x2 (i32 refill)", "data": "synthetic (seeded request stream)",
            "config": {"workload": "serving_stream", "rates_req_s": rates, "requests_per_rate": args.requests,
                       "mix": "70% 1-64 x (100 vs 1000 nt), 20% 1-64 short-read extensions, "
                              "10% 1-64 long reads (1-20 kb, 1.2x targets)",
                       "scoring": "+2/-4, open 4, extend 2 for every request",
                       "server": "4 workers (2 heavy at 7/8 of the SMs), batches <= 8192 pairs / 24M letters",
                       "baseline": "plain: FIFO, one launch sequence per pair, one stream"},
            "serving": rows, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsw", choices=["gsw", "reference"])
    ap.add_argument("--pairs", type=int, default=0, help="override the workload's pair count")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["dna_short_read_extension_1M", "dna_1k_100x1000", "dna_long_reads_10k",
                             "protein_search_1kx10k", "serving_stream", "reads_vs_reference",
                             "overlap_all_vs_all"])
    ap.add_argument("--ref-len", type=int, default=10_000_000, help="reads_vs_reference: reference letters")
    ap.add_argument("--rates", default="1000,10000,100000,500000",
                    help="serving_stream: Poisson arrival rates (requests/s)")
    ap.add_argument("--requests", type=int, default=2000, help="serving_stream: requests per rate")
    ap.add_argument("--head", type=int, default=100,
                    help="serving_stream: leading requests also run by the plain per-pair baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving runs of the default line")
    ap.add_argument("--serve-rates", default="1000,10000",
                    help="default line: arrival rates of the served stream (one within capacity, one in overload)")
    ap.add_argument("--serve-requests", type=int, default=20000, help="default line: requests per served rate")
    ap.add_argument("--serve-head", type=int, default=60,
                    help="default line: leading requests of each rate also run by the plain per-pair baseline")
    ap.add_argument("--no-long", action="store_true", help="skip the long-read sub-record of the default line")
    ap.add_argument("--long-pairs", type=int, default=0, help="long-read sub-record: pairs (default 10,000)")
    ap.add_argument("--long-steps", type=int, default=3, help="long-read sub-record: timed steps")
    ap.add_argument("--long-budget-gb", type=int, default=160,
                    help="long-read sub-record: context device-memory budget (GB)")
    ap.add_argument("--plain-pairs", type=int, default=2000,
                    help="also time the plain per-pair path (GSW_PLAIN) on this many of the workload's pairs "
                         "(0: skip)")
    ap.add_argument("--no-tune", action="store_true", help="default fill classes instead of the autotuner's")
    ap.add_argument("--tune-table", default="", help="fill class per 32-row bucket, comma-separated (no tuning)")
    ap.add_argument("--no-pack", action="store_true", help="DNA arenas one byte per letter instead of 2-bit packed")
    ap.add_argument("--budget-gb", type=int, default=24)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-pairs", type=int, default=4000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="N>1: split one workload over the ranks by cells (LPT) and gather the records on rank 0 "
                         "(strong scaling) instead of one batch per rank")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving_stream":
        run_serving_line(args)
    elif args.workload == "reads_vs_reference":
        run_reads_vs_reference(args)
    elif args.workload == "overlap_all_vs_all":
        run_overlap_all_vs_all(args)
    else:
        run_gsw(args)


if __name__ == "__main__":
    main()
