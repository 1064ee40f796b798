#!/usr/bin/env python
"""Throughput of the exhaustive all-pairs workload on GB300.

One step = the whole path over one synthetic dictionary of 600,000 words
(lengths round(N(8, 3)) on [1, 25], 40 codes with Zipf(1.1) usage, index =
frequency rank): ingest and length bucketing on the device, every one of the
179,999,700,000 upper-triangle pairs scored by the DPX alignment kernel, the
on-device per-word top-10 and score histogram, list finalisation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--sharded]

Prints one JSON line (rank 0).  `value` is pairs/s with the words already in
HBM; `e2e` is the same metric through the C ABI with host buffers (the H2D copy
of the words and the D2H copy of lists and histogram inside the timed region).
With N > 1 ranks every rank scores its own replica of the workload by default
(the pairs are independent; no collective is on the data path), so `value`
counts the pairs of all ranks over the slowest rank's time ("scaling": "weak").
With --sharded the ranks split one workload's pairs (nw_all_pairs_topk_shard)
and exchange the partial lists on the device (NCCL all-gather, merge kernel,
histogram all-reduce): `value` is that workload's pairs over the slowest
rank's time ("scaling": "strong").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NW pairs/s + GCUPS (% DPX peak); top-10 graph time at ≥0.99 recall vs exact"
UNIT = "pairs/s"
SCORING = (1, -1, -1)
K_NEIGHBOURS = 10
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes (read + write) of one step's alignment launches on the 600k
# workload, from an ncu capture of dram__bytes_read.sum + dram__bytes_write.sum
# (summarised under profiles/); valid only while the kernel sources hash to
# kernel_sha, and reported as null otherwise
TRAFFIC = {"kernel_sha": "e8027e6a77ddc0f4", "bytes_per_step": 441.6e6}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("nw_dp.cuh", "nw_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2509_01654_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def tensor_roofline(flops: float, ms: float, peaks_path: str = os.path.join(ROOT, "MEASURED_PEAKS.json")) -> dict:
    """Roofline of a bf16 tensor-core contraction: `flops` algorithmic FLOPs in
    `ms` milliseconds against the measured bf16 burst peak of MEASURED_PEAKS.json,
    or the 1,900 TFLOP/s fallback when that file is absent."""
    peak, basis = 1900.0, "fallback bf16 dense burst (1,900 TFLOP/s)"
    try:
        with open(peaks_path) as f:
            v = float(json.load(f)["bf16_tflops"])
        if v > 0:
            peak, basis = v, "measured bf16 burst (MEASURED_PEAKS.json bf16_tflops)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    achieved = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_basis": basis}


def workload_config(n, w, info, sharded=False):
    return {
        "workload": f"exhaustive all-pairs NW, {n:,} synthetic words (lengths round(N(8,3)) on [1,25], "
                    f"40 codes Zipf(1.1)), scoring (+1,-1,-1), per-word top-{K_NEIGHBOURS} + score histogram",
        "n_words": n,
        "k": K_NEIGHBOURS,
        "pairs_per_step": int(info["pairs"]),
        "cells_per_step": int(info["cells"]),
        "max_len": int(info["max_len"]),
        "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write); inputs 7 MB < L2",
        "parallelism": ("shards (each rank scores 1/N of the pairs; NCCL all-gather of the partial lists, "
                        "merge on the device, histogram all-reduce)" if sharded
                        else "replicas (one independent workload per rank)"),
    }


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid: str | None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd.insert(1, f"--id=GPU-{uuid}")
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons, power = [], [], set(), []
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------------------
# the oracle on the host cores (bounded sample of the same workload)

def oracle_sample(w, rows_target_s: float, min_rows: int = 8, max_rows: int = 5000):
    """Times the oracle's top-k on sampled words against the whole dictionary;
    returns (pairs/s, rows, seconds, threads)."""
    import oracle
    from paper_2509_01654_gb300 import synth

    threads = oracle.default_threads()
    min_rows = max(min_rows, threads)  # the probe keeps every thread busy, as the sample does
    # a first call warms the threads and the word arrays; the second, on four
    # rows per thread, sets the sample size for about rows_target_s of work
    oracle.topk_rows(w, synth.sample_rows(w.n, min_rows, seed=8), K_NEIGHBOURS, SCORING, nthreads=threads)
    probe = synth.sample_rows(w.n, 4 * min_rows, seed=7)
    t0 = time.perf_counter()
    oracle.topk_rows(w, probe, K_NEIGHBOURS, SCORING, nthreads=threads)
    dt = time.perf_counter() - t0
    rows = int(max(min_rows, min(max_rows, probe.size * rows_target_s / max(dt, 1e-3))))
    rows -= rows % threads if rows > threads else 0
    sample = synth.sample_rows(w.n, rows, seed=6)
    t0 = time.perf_counter()
    oracle.topk_rows(w, sample, K_NEIGHBOURS, SCORING, nthreads=threads)
    dt = time.perf_counter() - t0
    return rows * (w.n - 1) / dt, rows, dt, threads


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_2509_01654_gb300 import synth
    w = synth.exhaustive_words(args.n)
    per_step_s = float(os.environ.get("NW_REF_STEP_S", "10"))
    vals, rows_used, threads = [], 0, 1
    for s in range(args.warmup + args.steps):
        v, rows, dt, threads = oracle_sample(w, per_step_s)
        if s >= args.warmup:
            vals.append((v, rows, dt))
    value = statistics.median(v for v, _, _ in vals)
    rows_used = vals[0][1]
    ms = 1e3 * statistics.median(dt for _, _, dt in vals)
    lens = w.lengths
    cells_per_pair = (lens.sum() ** 2 - (lens ** 2).sum()) / 2 / (w.n * (w.n - 1) / 2)
    sample = (f"per step: top-{K_NEIGHBOURS} of {rows_used} sampled words against all {w.n:,} words "
              f"({rows_used * (w.n - 1):,} pairs), full (la+1)x(lb+1) int32 matrix per pair")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"exhaustive all-pairs NW, {w.n:,} synthetic words, scoring (+1,-1,-1), "
                               f"per-word top-{K_NEIGHBOURS}; each step a bounded sample of rows",
                   "n_words": w.n, "k": K_NEIGHBOURS},
        "gcups": value * cells_per_pair / 1e9,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU path

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_01654_gb300 import build as nw_build
    from paper_2509_01654_gb300 import nw, synth

    nw_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = synth.exhaustive_words(args.n)
    ctx = nw.Context(local_rank, stream=stream)
    codes_d = torch.from_numpy(w.codes).to(dev)
    offs_d = torch.from_numpy(w.offsets.astype(np.int32)).to(dev)
    probe = ctx.load_dictionary(w.codes, w.offsets, 40, SCORING)
    info = probe.info()
    probe.free()
    n, k, nbins = w.n, K_NEIGHBOURS, info["nbins"]
    idx_d = torch.empty((n, k), dtype=torch.int32, device=dev)
    score_d = torch.empty((n, k), dtype=torch.int16, device=dev)
    hist_d = torch.empty(nbins, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx.set_profiling(True)

    sharded = args.sharded
    if sharded:
        from paper_2509_01654_gb300 import dist as nwdist
        part_idx = torch.empty((n, k), dtype=torch.int32, device=dev)
        part_score = torch.empty((n, k), dtype=torch.int16, device=dev)

    def step_device():
        d = ctx.load_dictionary(codes_d, offs_d, 40, SCORING)
        if sharded:  # this rank's shard of the pairs, then the exchange on the device
            d.all_pairs_topk(k, nbr_idx=part_idx, nbr_score=part_score, hist=hist_d, shard=(rank, world))
            prof = ctx.last_profile()
            mi, ms = nwdist.exchange(part_idx, part_score, k, hist=hist_d, ctx=ctx)
            idx_d.copy_(mi)
            score_d.copy_(ms)
        else:
            d.all_pairs_topk(k, nbr_idx=idx_d, nbr_score=score_d, hist=hist_d)
            prof = ctx.last_profile()
        d.free()
        return prof

    # pinned host buffers for the end-to-end leg
    codes_h = torch.from_numpy(w.codes).pin_memory()
    offs_h = torch.from_numpy(w.offsets.view(np.int32)).pin_memory()
    idx_h = torch.empty((n, k), dtype=torch.int32).pin_memory()
    score_h = torch.empty((n, k), dtype=torch.int16).pin_memory()
    hist_h = torch.empty(nbins, dtype=torch.int64).pin_memory()
    codes_np, offs_np = codes_h.numpy(), offs_h.numpy().view(np.uint32)
    idx_np, score_np, hist_np = idx_h.numpy().view(np.uint32), score_h.numpy(), hist_h.numpy()

    def step_e2e():
        if sharded:  # inputs from pinned host memory, the merged lists back to the host
            codes_d.copy_(codes_h, non_blocking=True)
            offs_d.copy_(offs_h, non_blocking=True)
            step_device()
            idx_h.copy_(idx_d, non_blocking=True)
            score_h.copy_(score_d, non_blocking=True)
            hist_h.copy_(hist_d, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
            return
        d = ctx.load_dictionary(codes_np, offs_np, 40, SCORING)
        d.all_pairs_topk(k, nbr_idx=idx_np, nbr_score=score_np, hist=hist_np)
        d.free()

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    rates = ctx.measure_int_rates(300.0)

    sampler = ClockSampler(str(torch.cuda.get_device_properties(dev).uuid)) if rank == 0 else None
    times, dp_ms, launches = [], [], 0
    for _ in range(args.steps):
        flush.fill_(len(times))
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prof = step_device()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        times.append(e0.elapsed_time(e1))
        dp_ms.append(prof["dp_ms"])
        launches += 4 + prof["launches"] + (1 if sharded else 0)  # ingest, alignment, finalisation (+ merge)
    clocks = sampler.stop() if sampler else None

    e2e_times = []
    for _ in range(max(1, args.steps)):
        flush.fill_(len(e2e_times))
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_times.append(e0.elapsed_time(e1))
    # the host leg wrote real results: check them against the device leg
    assert np.array_equal(idx_np, idx_d.cpu().numpy().view(np.uint32))
    assert int(hist_np.sum()) == info["pairs"]

    total_ms = sum(times)
    total_e2e = sum(e2e_times)
    if world > 1:
        t = torch.tensor([total_ms, total_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, total_e2e = t.tolist()
    if rank != 0:
        return
    pairs, cells = info["pairs"], info["cells"]
    # replicas: every rank does the whole workload; shards: the ranks share one
    copies = 1 if sharded else world
    value = copies * pairs * args.steps / (total_ms / 1e3)
    e2e_value = copies * pairs * len(e2e_times) / (total_e2e / 1e3)

    # roofline of the alignment kernel: algorithmic cells over its launches' event time
    # (a shard holds 1/world of the cells: the planner cuts each launch into equal task ranges)
    dp_avg_ms = statistics.mean(dp_ms)
    achieved = (cells / world if sharded else cells) / (dp_avg_ms / 1e3) / 1e9
    c_min = 3.0  # packed instructions per two cells in the fewest-instruction cell update
    peak = 2.0 * rates["viaddmax_s16x2"] / c_min / 1e9
    sha = kernel_sha()
    traffic = TRAFFIC["bytes_per_step"] if TRAFFIC["kernel_sha"] == sha and args.n == 600_000 else None

    # the serving form of the same dictionary: open-loop Poisson load on the query server
    serving_stats = None
    if args.serving_requests > 0:
        from paper_2509_01654_gb300 import serving
        d = ctx.load_dictionary(codes_d, offs_d, 40, SCORING)
        with nw.Server(d, k=k, max_batch_queries=8192, max_inflight=4) as srv:
            serving_stats = serving.run_load(srv, synth.serving_queries(200_000), n_requests=args.serving_requests,
                                             rate_hz=args.serving_rate, max_batch=4096)
        d.free()
        serving_stats["workload"] = (f"Poisson arrivals at {args.serving_rate:g}/s, request sizes log-uniform on "
                                     f"[1, 4096] words of lengths U[1,30], exact top-{k} against the {n:,}-word "
                                     f"dictionary")

    # the batched form: many dictionaries of uneven size in one CUDA-graph launch
    batched_stats = None
    if args.batched_dicts > 0:
        dl = synth.batched_dictionaries(count=args.batched_dicts)
        batch = nw.Batch(ctx, [(x.words.codes, x.words.offsets, x.words.alphabet, x.scoring) for x in dl], k=k)
        binfo = batch.info()
        outs = [(torch.empty((x.words.n, k), dtype=torch.int32, device=dev),
                 torch.empty((x.words.n, k), dtype=torch.int16, device=dev)) for x in dl]
        batch.run(outs)  # warm-up replay
        bt = []
        for _ in range(max(3, args.steps)):
            flush.fill_(len(bt))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch.run(outs)  # one graph launch + per-dictionary copies; synchronous
            bt.append(time.perf_counter() - t0)
        bms = 1e3 * statistics.median(bt)
        batched_stats = {
            "workload": (f"{len(dl)} dictionaries, sizes floor(exp U(ln 1k, ln 50k)), lengths U[1,40], alphabets "
                         f"U{{40..120}}, per-dictionary scoring; exact top-{k} per word; one CUDA-graph launch"),
            "words": int(sum(x.words.n for x in dl)), "pairs": int(binfo["pairs"]), "cells": int(binfo["cells"]),
            "graph_launches_per_run": 1, "alignment_launches_in_graph": int(binfo["launches"]),
            "ms_per_run": bms, "pairs_per_s": binfo["pairs"] / (bms / 1e3),
            "gcups": binfo["cells"] / (bms / 1e3) / 1e9, "autotune_ms": binfo["tune_ms"],
            "words_per_task_by_length": {str(L): t for L, t in enumerate(binfo["words_per_task"]) if t},
            "blocks_per_sm_by_length": {str(L): b for L, b in enumerate(binfo["blocks_per_sm"]) if b},
        }
        batch.free()
        # a second batch of the same shape takes its tile shapes from the autotuner's cache
        again = nw.Batch(ctx, [(x.words.codes, x.words.offsets, x.words.alphabet, x.scoring) for x in dl], k=k)
        ainfo = again.info()
        batched_stats["same_shape_again"] = {"autotune_ms": ainfo["tune_ms"], "tune_cached": int(ainfo["tune_cached"])}
        again.free()
        # the same dictionaries, each with a query set of its own, in one graph
        qsets = synth.batched_query_sets(dl)
        batch = nw.Batch(ctx, [(x.words.codes, x.words.offsets, x.words.alphabet, x.scoring, (q.codes, q.offsets))
                               for x, q in zip(dl, qsets)], k=k)
        binfo = batch.info()
        qouts = [(torch.empty((q.n, k), dtype=torch.int32, device=dev),
                  torch.empty((q.n, k), dtype=torch.int16, device=dev)) for q in qsets]
        batch.run_queries(outs, qouts)  # warm-up replay
        bt = []
        for _ in range(max(3, args.steps)):
            flush.fill_(len(bt))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch.run_queries(outs, qouts)
            bt.append(time.perf_counter() - t0)
        bms = 1e3 * statistics.median(bt)
        batched_stats["with_query_sets"] = {
            "workload": (f"the {len(dl)} dictionaries above, each with a query set of its own (sizes "
                         f"floor(exp U(ln 1, ln 4096)), lengths U[1,40], the dictionary's alphabet); every "
                         f"dictionary's and query set's exact top-{k} in one CUDA-graph launch"),
            "query_words": int(binfo["query_words"]), "query_pairs": int(binfo["query_pairs"]),
            "pairs": int(binfo["pairs"]), "cells": int(binfo["cells"]),
            "alignment_launches_in_graph": int(binfo["launches"]), "ms_per_run": bms,
            "pairs_per_s": binfo["pairs"] / (bms / 1e3), "gcups": binfo["cells"] / (bms / 1e3) / 1e9,
            "autotune_ms": binfo["tune_ms"],
        }
        batch.free()

    # method variants on the same 600k words: a full similarity matrix and the normalised ranking
    variants_stats = None
    if args.variants and rank == 0:
        variants_stats = variants_leg(args, ctx, nw, w, codes_d, offs_d, idx_d, score_d, hist_d, info, flush)

    # the learned candidate proposal against the exhaustive lists of the timed leg
    proposal_stats = None
    if args.proposal_steps > 0 and rank == 0:
        proposal_stats = proposal_leg(args, ctx, nw, w, codes_d, offs_d, idx_d, score_d, total_ms / args.steps, dev)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, rows, dt, threads = oracle_sample(w, float(os.environ.get("NW_CPU_BASELINE_S", "15")))
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"top-{k} of {rows} sampled words against all {n:,} words ({rows * (n - 1):,} pairs) "
                         f"in {dt:.1f} s; full (la+1)x(lb+1) int32 matrix per pair"}

    # issue width implied by the measured rate at the SM clock nvidia-smi reported under load
    lanes_note = ""
    if clocks and clocks.get("sm_mhz"):
        lanes = rates["viaddmax_s16x2"] / (rates["sm_count"] * clocks["sm_mhz"] * 1e6)
        lanes_note = f", {lanes:.1f} lanes/clk/SM at the {clocks['sm_mhz']:.0f} MHz median SM clock under load"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
        "config": workload_config(n, w, info, sharded),
        "gcups": copies * cells * args.steps / (total_ms / 1e3) / 1e9,
        "dp_kernel_ms_per_step": dp_avg_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_basis": "DRAM bytes of one step's alignment launches (all 22), ncu, 600k words",
                     "peak_basis": f"2 cells x measured __viaddmax_s16x2 rate ({rates['viaddmax_s16x2']:.4g}/s "
                                   f"over {rates['sm_count']} SMs{lanes_note}) / {c_min:g} "
                                   f"packed instructions per cell pair; cell-mix microbenchmark "
                                   f"{2 * rates['nw_cell_mix'] / 1e9:.0f} GCUPS",
                     "rates_per_s": {key: rates[key] for key in ("viaddmax_s16x2", "vimax3_s16x2",
                                                                  "vimax_s16x2_relu", "iadd3", "lop3")}},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(codes_np.nbytes + offs_np.nbytes),
                "d2h_bytes_per_step": int(idx_np.nbytes + score_np.nbytes + hist_np.nbytes),
                "ms_per_step": total_e2e / len(e2e_times)},
        "gpu_launches": launches,
        "serving": serving_stats,
        "batched": batched_stats,
        "variants": variants_stats,
        "proposal": proposal_stats,
    }
    print(json.dumps(line), flush=True)


def phoneme_like_matrix(alphabet):
    """A similarity table of the shape Section 6 suggests: 3 for equal codes,
    1 for codes within 2 of each other (similar sounds), -2 otherwise."""
    import numpy as np
    a = np.arange(alphabet)
    d = np.abs(a[:, None] - a[None, :])
    return np.where(d == 0, 3, np.where(d <= 2, 1, -2)).astype(np.int32)


def variants_leg(args, ctx, nw, w, codes_d, offs_d, idx_d, score_d, hist_d, info, flush):
    import torch
    k = K_NEIGHBOURS
    cells = info["cells"]

    def timed(fn, reps):
        fn()  # warm-up
        ts = []
        for _ in range(reps):
            flush.fill_(len(ts))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    reps = max(2, args.steps)
    out = {}
    # own output buffers: the timed leg's lists stay the exhaustive reference of the proposal leg
    idx_d, score_d, hist_d = torch.empty_like(idx_d), torch.empty_like(score_d), torch.empty_like(hist_d)
    S = phoneme_like_matrix(40)
    ds = ctx.load_dictionary_sim(codes_d, offs_d, 40, S, -2)
    hist_s = torch.empty(ds.info()["nbins"], dtype=hist_d.dtype, device=hist_d.device)
    ms = timed(lambda: ds.all_pairs_topk(k, nbr_idx=idx_d, nbr_score=score_d, hist=hist_s), reps)
    out["substitution_matrix"] = {
        "workload": f"{w.n:,} words, top-{k} + histogram, 40 x 40 similarity table (3 equal, 1 within 2 codes, "
                    f"-2 otherwise), gap -2",
        "ms_per_step": round(ms, 2), "gcups": round(cells / (ms / 1e3) / 1e9, 1),
        "pairs_per_s": info["pairs"] / (ms / 1e3)}
    ds.free()
    d = ctx.load_dictionary(codes_d, offs_d, 40, SCORING)
    ms = timed(lambda: d.all_pairs_topk(k, nbr_idx=idx_d, nbr_score=score_d, hist=None, normalised=True), reps)
    out["normalised_ranking"] = {
        "workload": f"{w.n:,} words, top-{k} by s / max(len), match 1, mismatch -1, gap -1",
        "ms_per_step": round(ms, 2), "gcups": round(cells / (ms / 1e3) / 1e9, 1)}
    d.free()
    return out


def recall_vs_exact(ex_i, ex_s, ap_i, ap_s):
    """(strict, tie-aware) recall of approximate top-k lists against exact ones:
    strict = shared neighbours / k; tie-aware also counts a neighbour whose
    (exact) score reaches the exact k-th score."""
    import numpy as np
    ok = ex_i[:, -1] != 0xFFFFFFFF
    e, a = ex_i[ok].astype(np.int64), ap_i[ok].astype(np.int64)
    strict = (e[:, :, None] == a[:, None, :]).any(axis=1).sum(axis=1) / e.shape[1]
    kth = ex_s[ok][:, -1].astype(np.int32)
    tie = np.minimum((ap_s[ok].astype(np.int32) >= kth[:, None]).sum(axis=1), e.shape[1]) / e.shape[1]
    return float(strict.mean()), float(tie.mean())


def proposal_leg(args, ctx, nw, w, codes_d, offs_d, idx_d, score_d, exhaustive_ms, dev):
    import numpy as np
    import torch
    k = K_NEIGHBOURS
    d = ctx.load_dictionary(codes_d, offs_d, 40, SCORING)
    ex_i = idx_d.cpu().numpy().view(np.uint32)
    ex_s = score_d.cpu().numpy()
    n = w.n
    out_i = torch.empty((n, k), dtype=torch.int32, device=dev)
    out_s = torch.empty((n, k), dtype=torch.int16, device=dev)
    train_cfg = dict(batch_pairs=8192, lr=1e-3, lr_final=1e-4, clip_norm=1.0, nbr_fraction=0.5, seed=1,
                     long_len=args.train_long_len, long_fraction=args.train_long_fraction)

    def evaluate(model, C, reps):
        model.proposal_topk(d, C, k, nbr_idx=out_i, nbr_score=out_s)  # warm-up
        profs, walls = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, prof = model.proposal_topk(d, C, k, nbr_idx=out_i, nbr_score=out_s)
            walls.append(1e3 * (time.perf_counter() - t0))
            profs.append(prof)
        ap_i, ap_s = out_i.cpu().numpy().view(np.uint32), out_s.cpu().numpy()
        strict, tie = recall_vs_exact(ex_i, ex_s, ap_i, ap_s)
        by_len = {}
        lens = w.lengths
        for lo, hi in ((1, 4), (5, 8), (9, 12), (13, 16), (17, 25)):
            sel = (lens >= lo) & (lens <= hi)
            if sel.any():
                by_len[f"{lo}-{hi}"] = round(recall_vs_exact(ex_i[sel], ex_s[sel], ap_i[sel], ap_s[sel])[1], 4)
        med = {key: statistics.median(p[key] for p in profs) for key in profs[0]}
        return {"ms": {key: round(v, 3) for key, v in med.items()}, "wall_ms": round(statistics.median(walls), 3),
                "recall_at_10": round(strict, 4), "recall_at_10_tie_aware": round(tie, 4),
                "tie_aware_by_word_length": by_len,
                "speedup_vs_exhaustive": round(exhaustive_ms / med["total_ms"], 2)}

    untrained = nw.Model(ctx, 40, seed=1)
    ablation = {"untrained_C256": evaluate(untrained, 256, 1)}
    untrained.free()
    model = nw.Model(ctx, 40, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = model.train(d, steps=args.proposal_steps, nbr=ex_i, **train_cfg)
    train_s = time.perf_counter() - t0
    # the proposal alone, then with the exhaustive path for long words
    res_proposal_only = {"256": evaluate(model, 256, max(2, args.steps))}
    # the same stages with the candidate sweep in dictionary order (identical lists)
    model.set_sweep_order(False)
    dict_order = evaluate(model, 256, max(2, args.steps))
    model.set_sweep_order(True)
    ablation["dictionary_order_C256"] = {"ms": dict_order["ms"],
                                         "recall_at_10_tie_aware": dict_order["recall_at_10_tie_aware"]}
    model.set_exact_length(args.exact_length)
    res = {str(C): evaluate(model, C, max(2, args.steps)) for C in (256, 384, 512)}
    # the same path trained on the configuration's budget of 2e7 pairs
    budget_pairs = 20_000_000
    budget_steps = -(-budget_pairs // train_cfg["batch_pairs"])
    small = nw.Model(ctx, 40, seed=1)
    t1 = time.perf_counter()
    small.train(d, steps=budget_steps, nbr=ex_i, **train_cfg)
    budget_train_s = time.perf_counter() - t1
    small.set_exact_length(args.exact_length)
    res_budget = {str(C): evaluate(small, C, max(2, args.steps)) for C in (256, 512)}
    small.free()
    model.set_exact_length(args.query_exact_length)
    queries = proposal_queries(args, model, d, k, recall_vs_exact)
    # candidates without a network: the C words nearest in length order (stable by index)
    order = np.argsort(w.lengths, kind="stable")
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    C = 256
    lo = np.clip(pos - C // 2, 0, n - C - 1)
    win = lo[:, None] + np.arange(C + 1)[None, :]
    win = win[win != pos[:, None]].reshape(n, C)
    li, ls = nw.rescore_topk(d, order[win].astype(np.uint32), k)
    st, tt = recall_vs_exact(ex_i, ex_s, li, ls)
    ablation["length_window_C256"] = {"recall_at_10": round(st, 4), "recall_at_10_tie_aware": round(tt, 4)}
    model.free()
    d.free()
    # the metric's second half: top-10 graph time at >= 0.99 (tie-aware) recall
    def graph_at_99(results):
        at99 = [(int(C), r) for C, r in results.items() if r["recall_at_10_tie_aware"] >= 0.99]
        if not at99:
            return None
        C99, r99 = min(at99)
        return {"C": C99, "total_ms": r99["ms"]["total_ms"], "recall_at_10_tie_aware": r99["recall_at_10_tie_aware"],
                "speedup_vs_exhaustive": r99["speedup_vs_exhaustive"]}
    graph99 = graph_at_99(res)
    return {
        "graph_time_at_recall_0.99": graph99,
        "workload": (f"{n:,} words of the exhaustive workload; approximate top-{k} by the learned proposal "
                     f"(embed, quantise, C candidates by exact integer dot product, exact rescoring) against "
                     f"the exhaustive top-{k} lists of the timed leg"),
        "exact_length": args.exact_length,
        "query_exact_length": args.query_exact_length,
        "proposal_only": res_proposal_only,
        "train": {"steps": args.proposal_steps, "pairs": args.proposal_steps * train_cfg["batch_pairs"],
                  "seconds": round(train_s, 2), "target": "s / max(len_i, len_j)",
                  "loss_first_100": round(float(np.mean(losses[:100])), 5),
                  "loss_last_100": round(float(np.mean(losses[-100:])), 5), **train_cfg},
        "exhaustive_ms": round(exhaustive_ms, 3),
        "by_candidates": res,
        "config_training_budget": {
            "pairs": budget_steps * train_cfg["batch_pairs"], "steps": budget_steps,
            "seconds": round(budget_train_s, 2), "by_candidates": res_budget,
            "graph_time_at_recall_0.99": graph_at_99(res_budget)},
        # the candidate kernel: 2 n^2 d FLOP of bf16 products (d = 64) per launch
        "candidates_roofline": {str(C): tensor_roofline(2.0 * n * n * 64, r["ms"]["candidates_ms"])
                                for C, r in res.items()},
        "queries": queries,
        "ablation": ablation,
    }


def proposal_queries(args, model, d, k, recall):
    """A batch of serving-style query words (lengths U[1, 30]) against the
    dictionary: exhaustive nw_query against nw_proposal_query, host buffers
    both ways (each call copies its queries in and its lists out)."""
    import numpy as np
    import torch
    from paper_2509_01654_gb300 import synth
    q = synth.serving_queries(4096, seed=11)
    reps = max(3, args.steps)

    def timed(fn):
        fn()  # warm-up (the proposal's first call also quantises the dictionary)
        ts = []
        out = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts), out

    ex_ms, (ex_i, ex_s) = timed(lambda: d.query(q.codes, q.offsets, k))
    out = {"workload": f"{q.n} query words, lengths U[1,30], against the dictionary; top-{k}",
           "exhaustive_ms": round(ex_ms, 3), "exhaustive_queries_per_s": round(q.n / ex_ms * 1e3, 1)}
    for C in (256, 512):
        ms, (pi, ps) = timed(lambda: model.query(d, q.codes, q.offsets, C, k))
        st, tt = recall(np.asarray(ex_i).view(np.uint32), np.asarray(ex_s), np.asarray(pi).view(np.uint32),
                        np.asarray(ps))
        by_len = {}
        lens = np.asarray(q.lengths)
        for lo, hi in ((1, 10), (11, 20), (21, 25), (26, 30)):  # the dictionary's words are at most 25 long
            sel = (lens >= lo) & (lens <= hi)
            _, t_sel = recall(np.asarray(ex_i).view(np.uint32)[sel], np.asarray(ex_s)[sel],
                              np.asarray(pi).view(np.uint32)[sel], np.asarray(ps)[sel])
            by_len[f"{lo}-{hi}"] = round(t_sel, 4)
        out[str(C)] = {"ms": round(ms, 3), "queries_per_s": round(q.n / ms * 1e3, 1), "recall_at_10": round(st, 4),
                       "recall_at_10_tie_aware": round(tt, 4), "tie_aware_by_query_length": by_len,
                       "speedup_vs_exhaustive": round(ex_ms / ms, 2)}
    if args.serving_requests > 0:
        # the serving leg's open-loop load, answered through the proposal
        from paper_2509_01654_gb300 import nw, serving
        with nw.Server(d, k=k, max_batch_queries=8192, proposal=(model, 256)) as srv:
            ps = serving.run_load(srv, synth.serving_queries(200_000), n_requests=args.serving_requests,
                                  rate_hz=args.serving_rate, max_batch=4096)
        ps["workload"] = ("the serving leg's load (Poisson arrivals, request sizes log-uniform on [1, 4096]) on the "
                          "proposal server, C = 256")
        out["serving"] = ps
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=600_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sharded", action="store_true",
                    help="split one workload's pairs across the ranks (strong scaling) instead of running a replica "
                         "per rank; the exchange (all-gather, device merge, histogram all-reduce) runs even on one GPU")
    ap.add_argument("--serving-requests", type=int, default=150,
                    help="requests of the query-server load (0 skips it)")
    ap.add_argument("--serving-rate", type=float, default=40.0, help="request arrivals per second")
    ap.add_argument("--batched-dicts", type=int, default=64,
                    help="dictionaries of the batched-launch measurement (0 skips it)")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the substitution-matrix and normalised-ranking measurements")
    ap.add_argument("--train-long-len", type=int, default=11,
                    help="training draws --train-long-fraction of its pairs' first words among words this long")
    ap.add_argument("--train-long-fraction", type=float, default=0.4)
    ap.add_argument("--exact-length", type=int, default=17,
                    help="dictionary words of at least this many symbols take the exhaustive path (0: none)")
    ap.add_argument("--query-exact-length", type=int, default=15,
                    help="query words of at least this many symbols take the exhaustive path (0: none)")
    ap.add_argument("--proposal-steps", type=int, default=20000,
                    help="training steps of the learned-proposal measurement (0 skips it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    use_pg = world > 1 or args.sharded  # a sharded run exchanges over NCCL even on one rank
    if use_pg:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29531")
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if use_pg:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
