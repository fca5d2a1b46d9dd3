#!/usr/bin/env python3
"""Throughput of batched exact matching over a suffix array on one GB300.

Workload (default): a 100 Mbp repetitive reference (iid ACGT, 10% segmental
duplications, 2% tandem repeats, int32 suffix array) and 10,000,000 queries of
100 bp (80% sampled from the reference with 0-2 substitutions, 20% random),
locating up to 64 positions per query.  One step = pack the query batch,
search every query (the suffix-array interval) and locate its matches -- the
whole per-batch path -- with the index already built (its build is timed and
reported apart).  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

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

# Algorithmic bytes of the search kernel per query on this workload, from the
# oracle's byte model (oracle_probe_model: lockstep lower/upper-bound search,
# probes below depth 13 -- the levels the shared-memory key table absorbs --
# each one 32-byte suffix-array sector plus one 32-byte text sector per
# 64-base chunk the compare needs, with the LCP-of-bounds skip) on a seeded
# 20,000-query sample, plus ceil(m/4) packed query bytes and 12 result bytes:
#   B_q = 25 + 32 * P_q + 32 * X_q + 12.
# Written by oracle/bytes_model.py.
SEARCH_BYTES_PER_QUERY = 945.7152  # P_q = 13.97, X_q = 14.42 (d0 = 13, 20,000 queries)
SEARCH_BYTES_SOURCE = "oracle/bytes_model.py --workload repetitive-100m"

# DRAM bytes per search-kernel launch from one ncu capture, valid only while
# the kernel sources hash to KERNEL_SHA (else reported as null).
TRAFFIC = {"kernel_sha": "0a098c4064c1bc01", "dram_bytes_per_launch": 7178502000 + 244703232}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("search.cu", "sa_internal.cuh"):
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


def build_workload(scale: float):
    from paper_1303_3692_gb300 import datagen

    return datagen.repetitive_100m(scale=scale)


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
    res_d = torch.empty((n_q, 3), dtype=torch.int64, device=dev)
    offs_d = torch.empty(n_q + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    def lib_event():
        # created and marked recorded by torch once; the library re-records it
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    ev_s = [lib_event() for _ in range(2)]
    params = sa.sa_search_params()
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
        sa.sa_search_batch(idx, qb_d, qo_d, out=res_d, params=params)
        sa.sa_locate(idx, res_d, cap, out_offsets=offs_d, out_pos=pos_d, capacity=total_pos)

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
    total_s = sum(step_ms) / 1e3
    if dist is not None:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * args.steps * n_q / total_s

    # End to end through the C ABI with host (pinned) buffers, copies inside.
    qb_h = torch.from_numpy(w.q_bases).pin_memory()
    qo_h = torch.from_numpy(w.q_offsets).pin_memory()
    res_h = torch.empty((n_q, 3), dtype=torch.int64).pin_memory()
    offs_h = torch.empty(n_q + 1, dtype=torch.int64).pin_memory()
    pos_h = torch.empty(max(1, total_pos), dtype=torch.int32).pin_memory()

    def e2e_step():
        sa.sa_search_batch(idx, qb_h, qo_h, out=res_d)
        sa.sa_locate(idx, res_d, cap, out_offsets=offs_h, out_pos=pos_h, capacity=total_pos)
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

    # The plain one-thread-per-query kernel (Alg. 1) on the same batch.
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
    roof = None
    if SEARCH_BYTES_PER_QUERY:
        achieved = SEARCH_BYTES_PER_QUERY * n_q / kern_mean_s / 1e9
        sha = kernel_sha()
        traffic = TRAFFIC["dram_bytes_per_launch"] if TRAFFIC["kernel_sha"] == sha else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "search_kernel", "peak_kind": peak_kind,
                "bytes_per_query": SEARCH_BYTES_PER_QUERY, "bytes_source": SEARCH_BYTES_SOURCE}

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
        "step_ms_all": step_ms,
        "wall_s_timed_region": wall,
        "build_s": build_s,
        "datagen_s": gen_s,
        "positions_per_step": total_pos,
        "plain_kernel": {"ms": statistics.mean(plain_ms), "queries_per_s": n_q / (statistics.mean(plain_ms) / 1e3),
                         "search_speedup": statistics.mean(plain_ms) / statistics.mean(kern_ms)},
        "e2e": {"value": n_q / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3},
        "gpu_launches": args.steps * 5,
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
    return {"value": sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {sample} of {n_q} queries, search only, oracle suffix array by naive sort "
                      f"({build_s:.1f} s, untimed)"}


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
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
