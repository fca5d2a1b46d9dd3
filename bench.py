#!/usr/bin/env python3
"""Throughput of batched exact matching over a suffix array on one GB300.

Workload (default): a human-genome-sized synthetic reference of 3.1e9 bases
(GC 0.41, 45% repeat families of 300 bp and 6 kb units at 10-20% divergence,
3% tandem repeats) with an int64 suffix array, and 1.1e8 queries of 150 bp
per step (1e8 sampled from the reference with 0-1 substitutions, 1e7
random), locating up to 16 positions per query.  One step = pack the query
batch, search every query (the suffix-array interval) and locate its matches
-- the whole per-batch path -- with the index already built (its build is
timed and reported apart).  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--workload human-sized|repetitive-100m|plain-small|multi-genome|serving|paper-shaped]

--impl reference times the CPU oracle (Alg. 1 on the host cores, the paper's
serial/OpenMP baseline) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact-match queries/s (query bases/s, % HBM roofline alongside)"
UNIT = "queries/s"
WORKLOAD = "repetitive-100Mbp-10M-q100-locate64"

# Algorithmic bytes per query of each phase of a step on this workload
# (m = 100, k = 14), from the oracle's byte model (oracle/bytes_model.py:
# oracle_probe_model_kmer on 20,000 seeded queries: 1.19375 record probes per
# query, 0.41265 of them after the one that comes with the 64-byte k-mer entry,
# 6.58 occurrences on average, 0.51 positions kept at cap 64):
#   pack_batch_kernel: 100 ASCII bytes read + 25 packed bytes written (a batch
#       without a non-base byte needs no validity masks)        = 125
#   search (front_kernel + search_kernel): 8 offset bytes + 25 packed query
#       bytes + one 64-byte k-mer entry + 32 per further record probe + one
#       32-byte result                                          = 142.2
#   locate (3 kernels): 32 result bytes read + 8 offset bytes written + 4.1
#       position bytes (suffix-array entry read and written)   = 44.1
KERNEL_BYTES_PER_QUERY = {
    "pack_batch_kernel": 100 + 25,  # a clean batch: no validity masks written
    "search": 8 + 25 + 64 + 32 * 0.41265 + 32,
    "locate": 32 + 8 + 4.1072,
}
# Random DRAM accesses per query of the search phase (the k-mer entry, further
# record probes, text windows), from the same model: random 32- or 64-byte
# reads are bounded by the DRAM's row activations, not by its bandwidth.
RANDOM_ACCESSES_PER_QUERY = {"search": 1.41265}
BYTES_SOURCE = "oracle/bytes_model.py --workload repetitive-100m (k = 14)"

# DRAM bytes (read + write) per step of the dominant phase from one ncu
# capture (--set full, 100 Mbp workload), valid only while the kernel sources
# hash to kernel_sha (else reported as null).
TRAFFIC = {"kernel_sha": "b52eb447dc121722", "kernel": "search",
           "dram_bytes_per_launch": 2073794048 + 240993536 + 28380672 + 1843712}  # front_kernel + search_kernel


# Sources of each phase's kernels (the traffic figure is tied to them).
PHASE_SOURCES = {
    "pack_batch_kernel": ("pack.cu", "sa_internal.cuh"),
    "search": ("bucket.cu", "front.cu", "search.cu", "sa_internal.cuh"),
    "locate": ("locate.cu", "sa_internal.cuh"),
}


def kernel_sha(phase: str = "search") -> str:
    h = hashlib.sha256()
    for f in PHASE_SOURCES[phase]:
        with open(os.path.join(ROOT, "paper_1303_3692_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while running (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            os.remove(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(seconds: float, dist=None, device=None) -> float:
    """The slowest rank's time: the job ends when it does."""
    if dist is None:
        return seconds
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, n_q_per_rank: int, seconds: float) -> float:
    """Queries per second of the whole job.  The path shards by queries with
    no exchange: every rank holds its own replica of the index and searches
    its own batch of n_q_per_rank queries per step (weak scaling)."""
    return world * steps * n_q_per_rank / seconds


def build_workload(scale: float):
    from paper_1303_3692_gb300 import datagen

    return datagen.repetitive_100m(scale=scale)


def _time_count_steps(idxs, qb_d, qo_d, qr_d, params, args, local):
    """Times args.steps count-only searches (warm-up first, L2 flushed before
    each step): (step ms list, search-kernel ms list, clock summary)."""
    import torch

    import paper_1303_3692_gb300.sa as sa

    dev = qb_d.device
    n_q = qo_d.numel() - 1
    out = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def lib_event():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    params.flags = sa.SA_PARAM_Q_RANGE
    params.q_first, params.q_total = 0, int(qo_d[-1].item())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        sa.sa_search_batch(idxs, qb_d, qo_d, q_ref=qr_d, out=out, params=params)
    starts = [lib_event() for _ in range(args.steps)]
    ends = [lib_event() for _ in range(args.steps)]
    ks = [lib_event() for _ in range(args.steps)]
    ke = [lib_event() for _ in range(args.steps)]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            params.search_events[0], params.search_events[1] = ks[k].cuda_event, ke[k].cuda_event
            starts[k].record(stream)
            sa.sa_search_batch(idxs, qb_d, qo_d, q_ref=qr_d, out=out, params=params)
            ends[k].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    kern_ms = [a.elapsed_time(b) for a, b in zip(ks, ke)]
    return step_ms, kern_ms, clk.summary()


def run_multi_genome(args, world, rank, local):
    """4 references (5, 12, 25, 50 Mbp) and 16,000,000 queries of U[20,250] bp
    in one multi-reference call (count only); the launch shape is autotuned."""
    import torch

    import paper_1303_3692_gb300.sa as sa
    from paper_1303_3692_gb300 import autotune, datagen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    refs, qb, qo, qref, _ = datagen.multi_genome(scale=args.scale)
    t0 = time.perf_counter()
    idxs = [sa.sa_build(torch.from_numpy(r).to(dev)) for r in refs]
    build_s = time.perf_counter() - t0
    n_q = qo.size - 1
    qb_d, qo_d, qr_d = (torch.from_numpy(x).to(dev) for x in (qb, qo, qref))
    params, tune = autotune.autotune(idxs, qb_d, qo_d, q_ref=qr_d, use_cache=False)
    step_ms, kern_ms, clocks = _time_count_steps(idxs, qb_d, qo_d, qr_d, params, args, local)
    total_s = sum(step_ms) / 1e3
    value = args.steps * n_q / total_s
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "multi-genome-4refs-92Mbp-16M-q20to250", "refs_bp": [int(r.size) for r in refs],
                   "queries_per_step": n_q, "mode": "count", "autotuned": tune["best"],
                   "kmer_k": [i.kmer_k for i in idxs], "l2": "flushed between steps"},
        "query_bases_per_s": value * (float(qo[-1]) / n_q),
        "search_kernel_ms": statistics.mean(kern_ms), "step_ms_all": step_ms, "build_s": build_s,
        "gpu_launches": args.steps * 3, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# Table V, suffix-array columns as printed (seconds on a GTX680, 1024-base
# queries against 10^7 bases): batch size -> (SAK kernel, SAT total).  The
# printed SAT at 524,288 (0.13284) exceeds the sum of its parts (0.1284).
PAPER_TABLE5_SA = {
    512: (0.0003, 0.0085), 1024: (0.0004, 0.0086), 2048: (0.0005, 0.0088), 4096: (0.0006, 0.0089),
    8192: (0.0006, 0.0091), 16384: (0.0013, 0.0099), 32768: (0.0063, 0.0152), 65536: (0.0116, 0.0211),
    131072: (0.0398, 0.0505), 262144: (0.0579, 0.0789), 524288: (0.095, 0.13284), 1048576: (0.2716, 0.3214),
    2097152: (0.4762, 0.5545),
}
# Table V's suffix-tree columns: queries -> (STK, STT) in seconds on the GTX680.
PAPER_TABLE5_ST = {
    512: (0.0002, 0.0882), 1024: (0.0004, 0.0894), 2048: (0.0005, 0.0895), 4096: (0.0007, 0.0897),
    8192: (0.0009, 0.091), 16384: (0.0021, 0.0922), 32768: (0.0063, 0.0965), 65536: (0.0081, 0.0985),
    131072: (0.018, 0.1087), 262144: (0.044, 0.1449), 524288: (0.1781, 0.3135), 1048576: (0.22, 0.523),
    2097152: (0.33, 0.929),
}


def run_paper_shaped(args, world, rank, local):
    """The shape of the paper's Table V: 1024-base queries against 10^7 bases in
    batches of 2^9 .. 2^21, count only.  Per batch: the device step (pack +
    search, inputs resident, L2 flushed before each step) and the end-to-end
    call on pinned host queries with the results read back, beside the paper's
    kernel (SAK) and total (SAT) times.  Beside it the flattened suffix tree of
    the same text (Table V's comparison index) searches the same batches, its
    results checked equal to the suffix array's.  The line's value is the
    largest batch's device rate."""
    import torch

    import paper_1303_3692_gb300.sa as sa
    from paper_1303_3692_gb300 import datagen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    w = datagen.paper_shaped(scale=args.scale)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx = sa.sa_build(torch.from_numpy(w.ref).to(dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tree = sa.SuffixTree(idx)
    st_build_s = time.perf_counter() - t0
    m = 1024
    n_max = w.q_offsets.size - 1
    qb_d, qo_d = torch.from_numpy(w.q_bases).to(dev), torch.from_numpy(w.q_offsets).to(dev)
    qb_h, qo_h = torch.from_numpy(w.q_bases).pin_memory(), torch.from_numpy(w.q_offsets).pin_memory()
    out_d = torch.empty((n_max, sa.RESULT_FIELDS), dtype=torch.int64, device=dev)
    out_h = torch.empty((n_max, sa.RESULT_FIELDS), dtype=torch.int64).pin_memory()
    st_out = torch.empty((n_max, sa.RESULT_FIELDS), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    sizes = sorted({q for q in PAPER_TABLE5_SA if q <= n_max} | {n_max})
    sweep = []
    with Clocks(local) as clk:
        for q in sizes:
            tot = int(w.q_offsets[q])
            params = sa.sa_search_params(front_probes=args.front_probes)
            params.flags = sa.SA_PARAM_Q_RANGE
            params.q_first, params.q_total = 0, tot
            qo_q, out_q = qo_d[:q + 1], out_d[:q]
            for _ in range(args.warmup):
                sa.sa_search_batch(idx, qb_d, qo_q, out=out_q, params=params)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            torch.cuda.synchronize()
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                sa.sa_search_batch(idx, qb_d, qo_q, out=out_q, params=params)
                b.record(stream)
            torch.cuda.synchronize()
            dev_ms = statistics.median(a.elapsed_time(b) for a, b in ev)

            def e2e():
                sa.sa_search_batch(idx, qb_h[:tot], qo_h[:q + 1], out=out_q)
                out_h[:q].copy_(out_q, non_blocking=True)
                torch.cuda.synchronize()

            e2e()
            e2e_ms = []
            for _ in range(max(2, args.steps)):
                flush.zero_()
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                e2e()
                e2e_ms.append((time.perf_counter() - t1) * 1e3)
            # the suffix tree on the same batch (its call reads two offsets back first)
            st_q = st_out[:q]
            for _ in range(args.warmup):
                tree.search(qb_d, qo_q, out=st_q)
            torch.cuda.synchronize()
            st_ms = []
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tree.search(qb_d, qo_q, out=st_q)
                b.record(stream)
                torch.cuda.synchronize()
                st_ms.append(a.elapsed_time(b))
            st_equal = bool(torch.equal(st_q, out_q))
            sak, sat = PAPER_TABLE5_SA.get(q, (None, None))
            stk, stt = PAPER_TABLE5_ST.get(q, (None, None))
            sweep.append({"queries": q, "device_ms": dev_ms, "device_queries_per_s": q / dev_ms * 1e3,
                          "e2e_ms": statistics.median(e2e_ms), "paper_sak_s": sak, "paper_sat_s": sat,
                          "st_device_ms": statistics.median(st_ms), "st_over_sa": statistics.median(st_ms) / dev_ms,
                          "st_equals_sa": st_equal, "paper_stk_s": stk, "paper_stt_s": stt})
    if rank != 0:
        return
    top = sweep[-1]
    value = top["device_queries_per_s"]
    paper_top = 2097152 / PAPER_TABLE5_SA[2097152][0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": top["device_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / paper_top if n_max == 2097152 else None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "n": int(w.ref.size), "queries_per_step": n_max, "m": m, "mode": "count",
                   "kmer_k": idx.kmer_k, "l2": "flushed before every timed step; the larger batches exceed L2",
                   "vs_baseline_of": "Table V SAK at 2,097,152 queries (GTX680 kernel time)"},
        "query_bases_per_s": value * m,
        "e2e": {"value": n_max / top["e2e_ms"] * 1e3, "unit": UNIT,
                "h2d_bytes_per_step": int(w.q_offsets[n_max]) + (n_max + 1) * 8,
                "d2h_bytes_per_step": n_max * 32, "ms_per_step": top["e2e_ms"]},
        "sweep": sweep, "build_s": build_s, "datagen_s": gen_s, "gpu_launches": args.steps * 3,
        "suffix_tree": {"nodes": tree.nodes, "node_bytes": tree.device_bytes,
                        "suffix_array_bytes": int(w.ref.size) * 4, "build_s": st_build_s,
                        "all_batches_equal_sa": all(r["st_equals_sa"] for r in sweep),
                        "note": "the tree's descent also reads the text and, at leaves, the suffix array"},
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args)
    print(json.dumps(line), flush=True)


def run_build(args, world, rank, local):
    """Suffix-array construction on the GPU by Section III's method (DC3) and by
    prefix doubling (the library's default builder), on the human-like text at
    10^8 bases (int32 array) and 3.1 * 10^9 bases (int64): wall time of each
    synchronous call with the text resident, the two arrays checked equal.
    The line's value is DC3's rate at the larger size."""
    import torch

    import paper_1303_3692_gb300.sa as sa
    from paper_1303_3692_gb300 import datagen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    warm = torch.from_numpy(datagen.reference(100_000, 7)).to(dev)
    for dc3 in (False, True):  # module load and memory pool, untimed
        sa.sa_suffix_array_gpu(warm, 32, dc3=dc3)
    torch.cuda.synchronize()
    rows = []
    steps = max(1, min(args.steps, 3))
    with Clocks(local) as clk:
        for n_full, width in ((100_000_000, 32), (3_100_000_000, 64)):
            n = max(20_000, int(n_full * args.scale))
            t0 = time.perf_counter()
            ref = datagen.reference(n, datagen.SEED0 + 4, gc=0.41, family_cover=0.45, tandem_cover=0.03)
            gen_s = time.perf_counter() - t0
            d = torch.from_numpy(ref).to(dev)
            del ref
            row = {"n": n, "width_bits": width, "datagen_s": gen_s}
            arrays = {}
            for name, dc3 in (("prefix_doubling", False), ("dc3", True)):
                ts = []
                for _ in range(steps):
                    arrays.pop(name, None)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    arrays[name] = sa.sa_suffix_array_gpu(d, width, dc3=dc3)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                row[name + "_s"] = statistics.median(ts)
                row[name + "_bases_per_s"] = n / row[name + "_s"]
            row["equal"] = bool(torch.equal(arrays["prefix_doubling"], arrays["dc3"]))
            row["dc3_over_doubling"] = row["dc3_s"] / row["prefix_doubling_s"]
            rows.append(row)
            del arrays, d
            torch.cuda.empty_cache()
    if rank != 0:
        return
    top = rows[-1]
    line = {
        "metric": "suffix-array construction rate", "value": top["dc3_bases_per_s"], "unit": "bases/s",
        "n_gpus": world, "steps": steps, "warmup": 1, "ms_per_step": top["dc3_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic",
        "config": {"workload": "sa-build-dc3-vs-doubling", "sizes": [r["n"] for r in rows],
                   "text": "human-like synthetic (GC 0.41, 45% repeat families, 3% tandem repeats)",
                   "timing": "host wall clock around one synchronous call, text resident on the device"},
        "rows": rows, "all_equal": all(r["equal"] for r in rows), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_plain_small(args, world, rank, local):
    """1 Mbp iid reference, 100,000 queries of 32 bp (half copied from the
    reference, half random), count only.  The whole index fits in L2, so the
    number is latency- and launch-bound; L2 is still flushed between steps."""
    import torch

    import paper_1303_3692_gb300.sa as sa
    from paper_1303_3692_gb300 import datagen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = datagen.plain_small()
    t0 = time.perf_counter()
    idx = sa.sa_build(torch.from_numpy(w.ref).to(dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    n_q = w.q_offsets.size - 1
    qb_d, qo_d = torch.from_numpy(w.q_bases).to(dev), torch.from_numpy(w.q_offsets).to(dev)
    step_ms, kern_ms, clocks = _time_count_steps(idx, qb_d, qo_d, None,
                                                 sa.sa_search_params(front_probes=args.front_probes), args, local)
    total_s = sum(step_ms) / 1e3
    value = args.steps * n_q / total_s
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "plain-1Mbp-100k-q32", "n": int(w.ref.size), "queries_per_step": n_q, "m": 32,
                   "mode": "count", "kmer_k": idx.kmer_k, "l2": "flushed between steps; index L2-resident size"},
        "query_bases_per_s": value * 32, "search_kernel_ms": statistics.mean(kern_ms), "step_ms_all": step_ms,
        "build_s": build_s, "gpu_launches": args.steps * 3, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


HUMAN_WORKLOAD = "human-3.1Gbp-int64-q150-locate16"


def _human(args):
    from paper_1303_3692_gb300 import datagen

    nq = args.human_queries
    return datagen.human_sized(scale=args.scale, nq_sampled=nq * 10 // 11, nq_random=nq - nq * 10 // 11)


def verified_suffix_array(idx, ref):
    """The index's suffix array on the host, proven correct by the oracle's
    verifier (a permutation of [0, n) whose adjacent suffixes strictly
    increase is the unique suffix array): at the 3.1 Gbp size the oracle
    verifies the GPU-built array instead of rebuilding it.  Returns (T, sa,
    seconds to verify)."""
    import oracle

    T = oracle.normalize(ref)
    sa_h = idx.suffix_array(device="cpu").numpy()
    t0 = time.perf_counter()
    code, where = oracle.verify_sa(T, sa_h, threads=oracle.cpu_threads())
    dt = time.perf_counter() - t0
    if code != 0:
        raise RuntimeError(f"suffix array fails the oracle's verifier: code {code} at {where}")
    return T, sa_h, dt


def human_byte_model(T, sa_h, w, k: int, cap: int, sample: int = 20000, seed: int = 7, kmer_order: bool = False):
    """Algorithmic bytes and random reads per query of each phase, from the
    oracle's byte model (oracle.probe_model_bracket: the lockstep search over
    each query's k-mer bracket, 32-byte records of 112 bases, text windows
    past them) on a seeded sample of the batch.  The bracket of a query is
    found by the oracle's binary search for its first k bases and their
    successor over the verified suffix array (no 4^k table)."""
    import oracle

    n_q = w.q_offsets.size - 1
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(n_q, size=min(sample, n_q), replace=False))
    n = T.size
    tot = dict(m=0.0, entry=0.0, further=0.0, windows=0.0, kept=0.0, count=0.0, plain_probes=0.0, plain_chunks=0.0)
    for q in pick:
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        if P.size >= k:
            x = oracle.kmer_code(P, k)
            tlo = oracle.kmer_rank(T, sa_h, k, x)
            thi = oracle.kmer_rank(T, sa_h, k, x + 1) if x + 1 < (1 << (2 * k)) else n
            pr, wi, tr, lo, hi = oracle.probe_model_bracket(T, sa_h, (tlo, thi), P, d0=13)
        else:
            pr, wi, tr, lo, hi = oracle.probe_model_bracket(T, sa_h, None, P, d0=13)
        # the plain lockstep search over [-1, n) (no k-mer entries, no records):
        # probes below depth 13 and the 64-base text chunks they compare
        pp, pc, _, _ = oracle.probe_model(T, sa_h, P, d0=13)
        tot["plain_probes"] += pp
        tot["plain_chunks"] += pc
        tot["m"] += P.size
        tot["entry"] += tr
        # the 64-byte k-mer entry carries the bracket's first pivot: that probe costs no record read
        tot["further"] += max(pr - 1, 0) if tr else pr
        tot["windows"] += wi
        tot["kept"] += min(hi - lo, cap)
        tot["count"] += hi - lo
    c = float(len(pick))
    per = {key: v / c for key, v in tot.items()}
    m = per["m"]
    probes = 64 * per["entry"] + 32 * per["further"] + 32 * per["windows"] + 32  # + the 32-byte result
    if kmer_order:
        # sampling pass (offsets and the first two packed words of every 32nd
        # query), scatter pass (offsets and packed bases read -- a batch the
        # packing found clean needs no validity masks -- and a 64-byte record
        # written), first pass reads the record
        reorder = (8 + 16) / 32 + (8 + m / 4 + 64)
        search = reorder + 64 + probes
    else:
        reorder = 0.0
        search = 8 + m / 4 + probes
    return {
        "sample": int(c), "k": k,
        # pack: ASCII read, packed words written (no validity masks for a clean batch)
        "bytes_per_query": {"pack_batch_kernel": m + m / 4, "search": search,
                            "locate": 32 + 8 + 16 * per["kept"]},
        # random sectors per query: 2 for the 64-byte entry, 1 per record, 1 per text window
        "random_sectors_per_query": 2 * per["entry"] + per["further"] + per["windows"],
        "entry_reads_per_query": per["entry"], "record_probes_per_query": per["further"],
        "text_windows_per_query": per["windows"], "mean_count": per["count"], "mean_kept": per["kept"],
        "reorder_bytes_per_query": reorder, "order": "kmer" if kmer_order else "input",
        # packed query + 32 B per probe and per text chunk + 20 B of result + 8 B per kept position
        "plain_lockstep_bytes_per_query": m / 4 + 32 * (per["plain_probes"] + per["plain_chunks"]) + 20
                                          + 8 * per["kept"],
        "plain_lockstep_probes_per_query": per["plain_probes"],
        "source": "oracle.probe_model_bracket over the oracle-verified suffix array",
    }


def run_human_sized(args, world, rank, local):
    """The 3.1 Gbp configuration (the default line): a human-genome-sized
    reference (GC 0.41, 45% repeat families, 3% tandem repeats) with an int64
    suffix array and 1.1e8 queries of 150 bp per step (10:1 sampled with 0-1
    substitutions : random).  One step is one sa_search_locate call: pack the
    batch, search every query and locate up to 16 positions each."""
    import torch

    import paper_1303_3692_gb300.sa as sa

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    cap = 16
    t0 = time.perf_counter()
    w = _human(args)
    gen_s = time.perf_counter() - t0
    n_q = w.q_offsets.size - 1
    m_total = int(w.q_offsets[-1])
    n = int(w.ref.size)

    # Random-read ceiling, measured before the index takes the memory: over
    # 64 GB, and over a buffer the size of the index (whose reads cross many
    # more 2 MB pages than the TLBs cover).
    k_auto = 1
    while k_auto < 15 and (1 << (2 * (k_auto + 1))) <= 3 * n:
        k_auto += 1
    idx_est = n * (8 + 32) + 64 * (1 << (2 * k_auto)) + n // 4
    free_b = torch.cuda.mem_get_info(dev)[0]
    at_index = min(idx_est, free_b - (8 << 30)) & ~((1 << 30) - 1)
    ceiling = {}
    for size in sorted({64 << 30, at_index}):
        if args.no_rr_probe or size <= 0 or size > free_b - (4 << 30):
            continue
        for rb in (32, 64):
            ceiling[f"{size >> 30}GB_{rb}B"] = sa.sa_random_read_rate(size, 1024, 64, read_bytes=rb) / 1e9

    ref_d = torch.from_numpy(w.ref).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = sa.sa_build(ref_d, width=64)
    build_s = time.perf_counter() - t0
    del ref_d
    torch.cuda.empty_cache()

    qb_d = torch.from_numpy(w.q_bases).to(dev)
    qo_d = torch.from_numpy(w.q_offsets).to(dev)
    res = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64, device=dev)
    offs = torch.empty(n_q + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def lib_event():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    tune = None
    if args.autotune:
        from paper_1303_3692_gb300 import autotune

        p, tune = autotune.autotune(idx, qb_d, qo_d, sample=2_000_000, use_cache=False)
    else:
        p = sa.sa_search_params(front_probes=args.front_probes)
    p.flags = sa.SA_PARAM_Q_RANGE | {"auto": 0, "kmer": sa.SA_PARAM_KMER_ORDER,
                                     "input": sa.SA_PARAM_INPUT_ORDER}[args.order]
    p.q_first, p.q_total = 0, m_total
    sa.sa_search_batch(idx, qb_d, qo_d, out=res, params=p)
    o, _ = sa.sa_locate(idx, res, cap, out_pos=torch.empty(1, dtype=torch.int64, device=dev), capacity=0)
    total_pos = int(o[-1].item())
    del o
    pos = torch.empty(max(1, total_pos), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    order = sa.sa_search_order(idx, n_q, p)
    # pack, [bucket count, scan, scatter,] first pass, persistent pass, 3 locate kernels
    launches = 1 + (3 if order == "kmer" else 0) + 2 + 3

    def timed(mode, steps, clk_needed=False):
        ts, ks, pk, lc = [], [], [], []
        for it in range(args.warmup + steps):
            flush.zero_()
            a, b = lib_event(), lib_event()
            k0, k1 = lib_event(), lib_event()
            p.search_events[0], p.search_events[1] = k0.cuda_event, k1.cuda_event
            a.record(stream)
            if mode == "locate16":
                sa.sa_search_locate(idx, qb_d, qo_d, cap, out=res, out_offsets=offs, out_pos=pos,
                                    capacity=total_pos, params=p)
            else:
                sa.sa_search_batch(idx, qb_d, qo_d, out=res, params=p)
            b.record(stream)
            if it >= args.warmup:
                ts.append((a, b, k0, k1))
        torch.cuda.synchronize()
        step = [a.elapsed_time(b) for a, b, _, _ in ts]
        return {"step_ms_all": step, "ms_per_step": statistics.mean(step),
                "pack_ms": statistics.mean(a.elapsed_time(k0) for a, _, k0, _ in ts),
                "search_ms": statistics.mean(k0.elapsed_time(k1) for _, _, k0, k1 in ts),
                "locate_ms": statistics.mean(k1.elapsed_time(b) for _, b, _, k1 in ts)}

    with Clocks(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        main = timed("locate16", args.steps)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    clocks = clk.summary()
    count_only = timed("count", max(3, min(args.steps, 10)))
    total_s = max_over_ranks(sum(main["step_ms_all"]) / 1e3, dist, dev)
    value = job_rate(world, args.steps, n_q, total_s)

    # End to end through the C ABI from pinned host buffers: the batch's
    # bases and offsets go up and results, offsets and positions come back
    # inside the timed region.
    qb_h = torch.from_numpy(w.q_bases).pin_memory()
    qo_h = torch.from_numpy(w.q_offsets).pin_memory()
    res_h = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64).pin_memory()
    offs_h = torch.empty(n_q + 1, dtype=torch.int64).pin_memory()
    pos_h = torch.empty(max(1, total_pos), dtype=torch.int64).pin_memory()
    del qb_d
    torch.cuda.empty_cache()

    def e2e_step():
        sa.sa_search_locate(idx, qb_h, qo_h, cap, out=res_h, out_offsets=offs_h, out_pos=pos_h,
                            capacity=total_pos)
        torch.cuda.synchronize()

    e2e_step()
    e2e_t = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_t)
    h2d = int(qb_h.numel() + qo_h.numel() * 8)
    d2h = int(res_h.numel() * 8 + offs_h.numel() * 8 + total_pos * 8)
    # the plain pinned copy rate of this link, for context
    # (one warm-up copy, then the best of three rounds of four copies)
    probe_n = min(1 << 30, qb_h.numel())
    probe_d = torch.empty(probe_n, dtype=torch.uint8, device=dev)
    probe_d.copy_(qb_h[:probe_n], non_blocking=True)
    h2d_gbs = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(4):
            probe_d.copy_(qb_h[:probe_n], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = max(h2d_gbs, 4 * probe_n / (a.elapsed_time(b) / 1e3) / 1e9)
    del probe_d
    qb_d = torch.from_numpy(w.q_bases).to(dev)

    # The plain one-thread-per-query kernel (Alg. 1) on the first 16M queries.
    n_plain = min(n_q, 16_000_000)
    plain_ms = []
    for _ in range(2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sa.sa_search_batch_plain(idx, qb_d, qo_d[:n_plain + 1], out=res[:n_plain])
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b))
    plain_qps = n_plain / (min(plain_ms) / 1e3)
    del qb_d
    torch.cuda.empty_cache()
    serving = None
    if args.serve_seconds > 0 and world == 1:
        serving = serve_on_index([idx], w.q_bases, w.q_offsets, args.serve_seconds)

    line = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        T, sa_h, verify_s = verified_suffix_array(idx, w.ref)
        model = human_byte_model(T, sa_h, w, idx.kmer_k, cap, kmer_order=order == "kmer")
        phases = {"pack_batch_kernel": main["pack_ms"], "search": main["search_ms"], "locate": main["locate_ms"]}
        per_kernel = {}
        for name, ms in phases.items():
            gbs = model["bytes_per_query"][name] * n_q / (ms / 1e3) / 1e9
            per_kernel[name] = {"ms": ms, "bytes_per_query": model["bytes_per_query"][name], "achieved_gbs": gbs,
                                "frac": gbs / peak}
        dominant = max(phases, key=phases.get)
        traffic = (HUMAN_TRAFFIC["dram_bytes_per_launch"]
                   if HUMAN_TRAFFIC["kernel"] == dominant and HUMAN_TRAFFIC["kernel_sha"] == kernel_sha(dominant)
                   else None)
        sect = model["random_sectors_per_query"] * n_q / (phases["search"] / 1e3) / 1e9
        rr64 = ceiling.get("64GB_32B")
        rrix = ceiling.get(f"{at_index >> 30}GB_32B")
        roof = {"bound": "hbm", "achieved": per_kernel[dominant]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": per_kernel[dominant]["frac"], "traffic": traffic, "kernel": dominant, "peak_kind": peak_kind,
                "bytes_per_query": model["bytes_per_query"][dominant], "bytes_source": model["source"],
                "per_kernel": per_kernel,
                "random_reads": {"kernel": "search", "achieved": sect, "unit": "G sectors/s",
                                 "sectors_per_query": model["random_sectors_per_query"],
                                 "peak_64GB": rr64, "frac_64GB": sect / rr64 if rr64 else None,
                                 "peak_at_index_size": rrix, "index_size_GB": at_index >> 30,
                                 "frac_at_index_size": sect / rrix if rrix else None,
                                 "ceilings_G_reads_per_s": ceiling,
                                 "peak_source": "sa_random_read_rate_ex(size, 1024 threads/SM, 64 dependent reads)"},
                "model": model}
        # For context: the bytes the plain lockstep search would move (every probe
        # below depth 13 a 32-byte read plus 32 bytes per 64-base text chunk it
        # compares), over the whole step's time.  The k-mer entries and records
        # exist to avoid most of them, so this is not the kernel's own roofline.
        pb = model["plain_lockstep_bytes_per_query"]
        step_s = total_s / args.steps
        roof["plain_lockstep_model"] = {"bytes_per_query": pb, "probes_per_query": model["plain_lockstep_probes_per_query"],
                                        "achieved_gbs": pb * n_q / step_s / 1e9,
                                        "frac": pb * n_q / step_s / 1e9 / peak, "over": "whole step"}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_sa(T, sa_h, w, args, f"oracle-verified GPU suffix array ({verify_s:.1f} s to verify)")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": HUMAN_WORKLOAD, "n": n, "queries_per_step": n_q, "m": 150, "locate_cap": cap,
                       "sa_width": 64, "kmer_k": idx.kmer_k, "index_device_bytes": idx.device_bytes,
                       "autotuned": tune["best"] if tune else None,
                       "l2": "flushed between steps (256 MB write, outside the step events); inputs > L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "query_bases_per_s": value * (m_total / n_q),
            "phase_ms": phases, "step_ms_all": main["step_ms_all"],
            "count_only": {"ms_per_step": count_only["ms_per_step"],
                           "queries_per_s": n_q / (count_only["ms_per_step"] / 1e3),
                           "search_ms": count_only["search_ms"]},
            "build_s": build_s, "datagen_s": gen_s, "positions_per_step": total_pos,
            "plain_kernel": {"queries": n_plain, "ms": min(plain_ms), "queries_per_s": plain_qps,
                             "search_speedup": (n_q / ((phases["pack_batch_kernel"] + phases["search"]) / 1e3))
                             / plain_qps},
            "e2e": {"value": n_q / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_s * 1e3, "pinned_h2d_gbs": h2d_gbs,
                    "upload_bound_ms": h2d / (h2d_gbs * 1e9) * 1e3},
            "gpu_launches": args.steps * launches,
            "search_order": order,
            "serving": serving,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serve_on_index(idxs, q_bases, q_offsets, seconds: float, rate: float = 2000.0, pool: int = 2_000_000,
                   caps=(0, 16)):
    """Serving on resident indexes: a Poisson trace (`rate` requests/s for
    `seconds`), each request a log-uniform 1-100,000 queries sliced from a
    pool of the workload's queries, with a locate cap drawn from `caps`;
    served by the continuous-batching server, by one optimized call per
    request, and by one call of the plain Alg. 1 kernel per request."""
    import torch

    from paper_1303_3692_gb300 import serve

    n = min(pool, q_offsets.size - 1)
    qo = np.ascontiguousarray(q_offsets[:n + 1])
    pools = [(torch.from_numpy(np.ascontiguousarray(q_bases[:int(qo[-1])])).pin_memory(), qo)]
    max_cap = max(caps)
    warm = serve.make_trace(pools, rate=rate, duration=0.2, seed=1, caps=caps)
    serve.Server(idxs, slots=3, max_cap=max_cap).run(warm)
    out = {"trace": {"rate_per_s": rate, "seconds": seconds, "queries_per_request": "log-uniform 1-100000",
                     "caps": list(caps)}}
    trace = serve.make_trace(pools, rate=rate, duration=seconds, seed=2, caps=caps)
    out["batched"] = serve.Server(idxs, slots=3, max_cap=max_cap).run(trace)
    for kernel in ("optimized", "plain"):
        t = serve.make_trace(pools, rate=rate, duration=seconds, seed=2, caps=caps)
        serve.run_plain(idxs, t[:2], kernel=kernel)  # warm
        t = serve.make_trace(pools, rate=rate, duration=seconds, seed=2, caps=caps)
        out[f"per_request_{kernel}"] = serve.run_plain(idxs, t, kernel=kernel)
    b = out["batched"]
    for kernel in ("optimized", "plain"):
        o = out[f"per_request_{kernel}"]
        out[f"p99_gain_vs_{kernel}"] = o["p99_ms"] / b["p99_ms"] if b["p99_ms"] else None
        out[f"p50_gain_vs_{kernel}"] = o["p50_ms"] / b["p50_ms"] if b["p50_ms"] else None
    return out


# DRAM bytes (read + write) of one 3.1 Gbp search phase (bucket sample, plan,
# scatter and fill, first pass, persistent pass) from one single-pass ncu capture of the
# default bench command (the median of its 13 full-size steps), valid only
# while the phase's sources hash to kernel_sha.
HUMAN_TRAFFIC = {"kernel_sha": "fc28c78cf4b08d9b", "kernel": "search", "dram_bytes_per_launch": 72_274_846_976}


def cpu_baseline_sa(T, sa_h, w, args, sa_note: str):
    """The oracle (Alg. 1 on all host cores, then on one core) on a bounded
    sample of the batch against a given (verified) suffix array."""
    import oracle

    threads = oracle.cpu_threads()
    n_q = w.q_offsets.size - 1
    probe = min(n_q, 20000)
    t0 = time.perf_counter()
    oracle.search_batch(T, sa_h, w.q_bases, w.q_offsets[:probe + 1], threads=threads)
    rate = probe / max(1e-9, time.perf_counter() - t0)
    sample = int(min(n_q, max(probe, rate * args.cpu_seconds)))
    t0 = time.perf_counter()
    oracle.search_batch(T, sa_h, w.q_bases, w.q_offsets[:sample + 1], threads=threads)
    dt = time.perf_counter() - t0
    sample1 = int(min(n_q, max(1000, (sample / dt) / threads * args.cpu_seconds / 4)))
    t0 = time.perf_counter()
    oracle.search_batch(T, sa_h, w.q_bases, w.q_offsets[:sample1 + 1], threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {sample} of {n_q} queries, search only (Alg. 1), {sa_note}",
            "single_core": {"value": sample1 / dt1, "unit": UNIT, "cores": 1, "sample": f"first {sample1} queries"}}


def run_serving(args, world, rank, local):
    """8 resident references (1, 5, 20, 50, 100, 200, 300, 500 Mbp, 10% segmental
    duplications); a Poisson stream of requests (mean 2,000/s), each targeting a
    random reference with a log-uniform 1-100,000 queries of U[20,300] bp (75%
    sampled); continuous batching against one call per request."""
    import torch

    import paper_1303_3692_gb300.sa as sa
    from paper_1303_3692_gb300 import datagen, serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = [int(x * args.scale) for x in (1e6, 5e6, 20e6, 50e6, 100e6, 200e6, 300e6, 500e6)]
    t0 = time.perf_counter()
    refs = [datagen.reference(max(n, 10_000), datagen.SEED0 + 50 + i, sd_cover=0.10) for i, n in enumerate(sizes)]
    pools = []
    for i, r in enumerate(refs):
        qb, qo, _ = datagen.queries(r, args.pool, datagen.SEED0 + 60 + i, m=(20, 300), frac_sampled=0.75,
                                    subs=(0, 0))
        pools.append((torch.from_numpy(qb).pin_memory(), qo))
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    idxs = [sa.sa_build(torch.from_numpy(r).to(dev)) for r in refs]
    build_s = time.perf_counter() - t0
    warm = serve.make_trace(pools, rate=2000, duration=0.2, seed=1)
    serve.Server(idxs).run(warm)
    trace = serve.make_trace(pools, rate=2000, duration=args.serve_seconds, seed=2)
    with Clocks(local) as clk:
        srv = serve.Server(idxs, slots=3)
        stats = srv.run(trace)
    plain_trace = serve.make_trace(pools, rate=2000, duration=args.serve_seconds, seed=2)
    plain = serve.run_plain(idxs, plain_trace)
    # saturated: the same requests all arriving at once (maximum sustained throughput)
    sat = serve.make_trace(pools, rate=2000, duration=args.serve_seconds, seed=2)
    for r in sat:
        r.arrival = 0.0
    sat_stats = serve.Server(idxs, slots=3).run(sat)
    sat_plain = serve.make_trace(pools, rate=2000, duration=args.serve_seconds, seed=2)
    for r in sat_plain:
        r.arrival = 0.0
    sat_plain_stats = serve.run_plain(idxs, sat_plain)
    if rank != 0:
        return
    line = {
        "metric": "serving p50/p99 latency and queries/s", "value": stats["queries_per_s"], "unit": UNIT,
        "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "serving-8refs-1176Mbp-poisson2000", "refs_bp": [int(r.size) for r in refs],
                   "seconds": args.serve_seconds, "pool_queries_per_ref": args.pool},
        "serving": stats, "plain_per_request": plain,
        "p99_gain": plain["p99_ms"] / stats["p99_ms"] if stats["p99_ms"] else None,
        "saturated": {"batched": sat_stats, "plain_per_request": sat_plain_stats,
                      "throughput_gain": sat_stats["queries_per_s"] / sat_plain_stats["queries_per_s"]},
        "build_s": build_s, "datagen_s": gen_s, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_reference_human(args, world, rank, local):
    """The reference arm on the 3.1 Gbp workload: the oracle as it stands
    (Alg. 1 on this host's cores) on bounded samples of the batch.  The oracle
    cannot sort 3.1e9 suffixes in minutes, so its suffix array is the one the
    GPU builds, proven to be the unique suffix array by the oracle's own
    verifier first; only the oracle's search is timed."""
    import torch

    import oracle
    import paper_1303_3692_gb300.sa as sa

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = _human(args)
    t0 = time.perf_counter()
    idx = sa.sa_build(torch.from_numpy(w.ref).to(dev), width=64)
    build_s = time.perf_counter() - t0
    T, sa_h, verify_s = verified_suffix_array(idx, w.ref)
    del idx
    threads = oracle.cpu_threads()
    n_q = w.q_offsets.size - 1
    probe = min(n_q, 20000)
    t0 = time.perf_counter()
    oracle.search_batch(T, sa_h, w.q_bases, w.q_offsets[:probe + 1], threads=threads)
    rate = probe / max(1e-9, time.perf_counter() - t0)
    sample = int(min(n_q, max(probe, rate * args.ref_step_seconds)))
    qo = w.q_offsets[:sample + 1]
    for _ in range(args.warmup):
        oracle.search_batch(T, sa_h, w.q_bases, qo, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.search_batch(T, sa_h, w.q_bases, qo, threads=threads)
        times.append(time.perf_counter() - t0)
    per_step = statistics.mean(times)
    value = sample / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": HUMAN_WORKLOAD, "n": int(w.ref.size), "queries_per_step": sample, "m": 150,
                   "note": "search only (Alg. 1 on the CPU; the oracle has no locate kernel to time)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {sample} of {n_q} queries per step, against the GPU-built suffix "
                                   f"array after the oracle's verifier proved it ({verify_s:.1f} s; build "
                                   f"{build_s:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """The oracle as it stands, on this host's cores, on bounded query samples."""
    import oracle

    if rank != 0:
        return
    w = build_workload(args.scale)
    T = oracle.normalize(w.ref)
    t0 = time.perf_counter()
    osa = oracle.sa_naive(T)
    build_s = time.perf_counter() - t0
    threads = oracle.cpu_threads()
    n_q = w.q_offsets.size - 1
    # size each step's sample to about a few seconds of CPU work
    probe = min(n_q, 20000)
    t0 = time.perf_counter()
    oracle.search_batch(T, osa, w.q_bases, w.q_offsets[:probe + 1], threads=threads)
    rate = probe / max(1e-9, time.perf_counter() - t0)
    sample = int(min(n_q, max(probe, rate * args.ref_step_seconds)))
    qo = w.q_offsets[:sample + 1]
    for _ in range(args.warmup):
        oracle.search_batch(T, osa, w.q_bases, qo, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.search_batch(T, osa, w.q_bases, qo, threads=threads)
        times.append(time.perf_counter() - t0)
    per_step = statistics.mean(times)
    value = sample / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": int(w.ref.size), "queries_per_step": sample, "m": 100,
                   "note": "search only (Alg. 1 on the CPU; the oracle has no locate kernel to time)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {sample} of {n_q} queries per step, oracle suffix array "
                                   f"(naive sort, {build_s:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    import paper_1303_3692_gb300.sa as sa

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    t0 = time.perf_counter()
    w = build_workload(args.scale)
    gen_s = time.perf_counter() - t0
    n_q = w.q_offsets.size - 1
    m_total = int(w.q_offsets[-1])
    cap = w.cap

    # Index build (timed apart from the search path).
    ref_d = torch.from_numpy(w.ref).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = sa.sa_build(ref_d, width=32)
    build_s = time.perf_counter() - t0
    del ref_d

    qb_d = torch.from_numpy(w.q_bases).to(dev)
    qo_d = torch.from_numpy(w.q_offsets).to(dev)
    res_d = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64, device=dev)
    offs_d = torch.empty(n_q + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    def lib_event():
        # created and marked recorded by torch once; the library re-records it
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    ev_s = [lib_event() for _ in range(2)]
    params = sa.sa_search_params(front_probes=args.front_probes)
    params.search_events[0] = ev_s[0].cuda_event
    params.search_events[1] = ev_s[1].cuda_event
    # the batch's offsets range is known on the host: the call never synchronizes
    params.flags = sa.SA_PARAM_Q_RANGE
    params.q_first = int(w.q_offsets[0])
    params.q_total = int(w.q_offsets[-1] - w.q_offsets[0])

    # size the positions buffer once
    sa.sa_search_batch(idx, qb_d, qo_d, out=res_d, params=params)
    offs_tmp, pos_tmp = sa.sa_locate(idx, res_d, cap)
    total_pos = int(offs_tmp[-1].item())
    pos_d = torch.empty(max(1, total_pos), dtype=torch.int32, device=dev)
    del offs_tmp, pos_tmp
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2

    def step():
        # one call: the search hands each query's first position to the locate
        sa.sa_search_locate(idx, qb_d, qo_d, cap, out=res_d, out_offsets=offs_d, out_pos=pos_d,
                            capacity=total_pos, params=params)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_starts = [lib_event() for _ in range(args.steps)]
    k_ends = [lib_event() for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # evict L2 between steps (outside the step events)
            params.search_events[0] = k_starts[k].cuda_event
            params.search_events[1] = k_ends[k].cuda_event
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
    clocks = clk.summary()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(e) for s, e in zip(k_starts, k_ends)]
    phases = {
        "pack_batch_kernel": statistics.mean(a.elapsed_time(b) for a, b in zip(starts, k_starts)),
        "search": statistics.mean(kern_ms),
        "locate": statistics.mean(a.elapsed_time(b) for a, b in zip(k_ends, ends)),
    }
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = job_rate(world, args.steps, n_q, total_s)

    # End to end through the C ABI with host (pinned) buffers, copies inside.
    qb_h = torch.from_numpy(w.q_bases).pin_memory()
    qo_h = torch.from_numpy(w.q_offsets).pin_memory()
    res_h = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64).pin_memory()
    offs_h = torch.empty(n_q + 1, dtype=torch.int64).pin_memory()
    pos_h = torch.empty(max(1, total_pos), dtype=torch.int32).pin_memory()

    def e2e_step():
        sa.sa_search_locate(idx, qb_h, qo_h, cap, out=res_d, out_offsets=offs_h, out_pos=pos_h, capacity=total_pos)
        res_h.copy_(res_d, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    e2e_times = []
    for _ in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    h2d = int(qb_h.numel() + qo_h.numel() * 8)
    d2h = int(res_h.numel() * 8 + offs_h.numel() * 8 + total_pos * 4)

    # The plain one-thread-per-query kernel (Alg. 1) on the same batch (the
    # call packs the batch first, like the product path).
    plain_ms = []
    for _ in range(2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sa.sa_search_batch_plain(idx, qb_d, qo_d, out=res_d)
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b))
    kern_mean_s = statistics.mean(kern_ms) / 1e3

    peak, peak_kind = measured_peaks()
    per_kernel = {}
    for name, ms in phases.items():
        gbs = KERNEL_BYTES_PER_QUERY[name] * n_q / (ms / 1e3) / 1e9
        per_kernel[name] = {"ms": ms, "bytes_per_query": KERNEL_BYTES_PER_QUERY[name], "achieved_gbs": gbs,
                            "frac": gbs / peak}
    dominant = max(phases, key=phases.get)
    traffic = (TRAFFIC["dram_bytes_per_launch"]
               if TRAFFIC["kernel"] == dominant and TRAFFIC["kernel_sha"] == kernel_sha(dominant) else None)
    roof = {"bound": "hbm", "achieved": per_kernel[dominant]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": per_kernel[dominant]["frac"], "traffic": traffic, "kernel": dominant,
            "peak_kind": peak_kind, "bytes_per_query": KERNEL_BYTES_PER_QUERY[dominant],
            "bytes_source": BYTES_SOURCE, "per_kernel": per_kernel}
    # The search's probes are dependent random reads: their ceiling is the
    # device's random-read rate (DRAM row activations), measured here over a
    # 4 GB buffer with the same resident threads per SM as the first pass.
    rr_peak = sa.sa_random_read_rate(4 << 30, 1024, 64)
    rr_ach = RANDOM_ACCESSES_PER_QUERY["search"] * n_q / (phases["search"] / 1e3)
    roof["random_reads"] = {"kernel": "search", "achieved": rr_ach / 1e9, "peak": rr_peak / 1e9,
                            "unit": "G reads/s", "frac": rr_ach / rr_peak,
                            "reads_per_query": RANDOM_ACCESSES_PER_QUERY["search"],
                            "peak_source": "sa_random_read_rate(4 GB, 1024 threads/SM, 64 dependent reads)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": int(w.ref.size), "queries_per_step": n_q, "m": 100,
                   "locate_cap": cap, "sa_width": 32, "key_depth": idx.key_depth,
                   "l2": "flushed between steps (256 MB write, outside the step events); inputs > L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "query_bases_per_s": value * (m_total / n_q),
        "search_kernel_ms": statistics.mean(kern_ms),
        "phase_ms": phases,
        "step_ms_all": step_ms,
        "wall_s_timed_region": wall,
        "build_s": build_s,
        "datagen_s": gen_s,
        "positions_per_step": total_pos,
        "plain_kernel": {"ms": statistics.mean(plain_ms), "queries_per_s": n_q / (statistics.mean(plain_ms) / 1e3),
                         "search_speedup": statistics.mean(plain_ms) / (phases["pack_batch_kernel"] +
                                                                        phases["search"])},
        "e2e": {"value": n_q / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3},
        "gpu_launches": args.steps * 6,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(w, args):
    """The oracle (Alg. 1 on the host cores) on a bounded sample of the batch."""
    import oracle

    T = oracle.normalize(w.ref)
    t0 = time.perf_counter()
    osa = oracle.sa_naive(T)
    build_s = time.perf_counter() - t0
    threads = oracle.cpu_threads()
    n_q = w.q_offsets.size - 1
    probe = min(n_q, 20000)
    t0 = time.perf_counter()
    oracle.search_batch(T, osa, w.q_bases, w.q_offsets[:probe + 1], threads=threads)
    rate = probe / max(1e-9, time.perf_counter() - t0)
    sample = int(min(n_q, max(probe, rate * args.cpu_seconds)))
    t0 = time.perf_counter()
    oracle.search_batch(T, osa, w.q_bases, w.q_offsets[:sample + 1], threads=threads)
    dt = time.perf_counter() - t0
    # The same oracle on one core, over a quarter of the time budget.
    sample1 = int(min(n_q, max(1000, (sample / dt) / threads * args.cpu_seconds / 4)))
    t0 = time.perf_counter()
    oracle.search_batch(T, osa, w.q_bases, w.q_offsets[:sample1 + 1], threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {sample} of {n_q} queries, search only, oracle suffix array by naive sort "
                      f"({build_s:.1f} s, untimed)",
            "single_core": {"value": sample1 / dt1, "unit": UNIT, "cores": 1, "sample": f"first {sample1} queries"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--workload", choices=["human-sized", "repetitive-100m", "plain-small", "multi-genome",
                                           "serving", "paper-shaped", "build"],
                    default="human-sized")
    ap.add_argument("--autotune", action="store_true", help="tune the launch shape before timing (human-sized)")
    ap.add_argument("--order", choices=["auto", "kmer", "input"], default="auto",
                    help="search order of the human-sized line (auto: the library's choice)")
    ap.add_argument("--no-rr-probe", action="store_true", help="skip the random-read ceiling probes")
    ap.add_argument("--human-queries", type=int, default=110_000_000,
                    help="queries per step of the 3.1 Gbp workload (100M sampled + 10M random)")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--front-probes", type=int, default=0,
                    help="probes per query in the first search pass (0: the library's default)")
    ap.add_argument("--pool", type=int, default=300_000, help="queries pre-generated per reference (serving)")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        if args.workload == "human-sized":
            run_reference_human(args, world, rank, local)
        else:
            run_reference(args, world, rank)
    elif args.workload == "multi-genome":
        run_multi_genome(args, world, rank, local)
    elif args.workload == "plain-small":
        run_plain_small(args, world, rank, local)
    elif args.workload == "serving":
        run_serving(args, world, rank, local)
    elif args.workload == "human-sized":
        run_human_sized(args, world, rank, local)
    elif args.workload == "paper-shaped":
        run_paper_shaped(args, world, rank, local)
    elif args.workload == "build":
        run_build(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
