"""Autotuner for the search's launch shape.

Times sa_search_batch_ex on a sample of a batch for a grid of candidate
(threads per block, blocks per SM, shared-memory key-table depth, queries per
warp chunk of the persistent pass, probes of the first pass), checks that
every candidate returns identical results, and keeps the fastest.  A
candidate of four values leaves the first pass at the library's default.
Results are cached in a JSON file keyed by GPU name, the references' sizes,
the suffix-array width and the batch's length bucket, so a serving process
tunes once per workload shape.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import sa

# (threads per block, blocks per SM, key-table depth, chunk, first-pass probes).
# Every shape keeps 1024 threads per SM: the persistent kernel takes 64
# registers a thread, so more resident threads cannot fit (the library
# reduces such requests) and shapes that forced fewer registers spilled.
DEFAULT_CANDIDATES: Tuple[Tuple[int, ...], ...] = (
    (1024, 1, 13, 64, 3), (1024, 1, 13, 64, 1), (1024, 1, 13, 64, 2), (1024, 1, 13, 64, 4),
    (1024, 1, 12, 64, 3), (1024, 1, 13, 32, 3), (512, 2, 12, 64, 3), (256, 4, 11, 64, 3),
)

LENGTH_BUCKETS = (64, 128, 192, 300, 1 << 62)


def length_bucket(mean_len: float) -> int:
    """Index of the first bucket bound >= the batch's mean query length."""
    for i, b in enumerate(LENGTH_BUCKETS):
        if mean_len <= b:
            return i
    return len(LENGTH_BUCKETS) - 1


def cache_key(gpu: str, refs: Sequence["sa.Index"], mean_len: float) -> str:
    ns = ",".join(str(r.n) for r in refs)
    return f"{gpu}|w{refs[0].width}|k{','.join(str(r.kmer_k) for r in refs)}|n{ns}|b{length_bucket(mean_len)}"


def default_cache_path() -> str:
    base = os.environ.get("SA_AUTOTUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1303_3692_gb300", "autotune.json")


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick_best(timings: Iterable[Tuple[Tuple[int, ...], float]]) -> Tuple[Tuple[int, ...], float]:
    """Fastest candidate; ties go to the earlier one."""
    best = None
    for cand, t in timings:
        if best is None or t < best[1]:
            best = (cand, t)
    if best is None:
        raise ValueError("no candidate timed")
    return best


def params_from(cand: Sequence[int]) -> "sa.sa_search_params":
    th, bps, depth, chunk = cand[:4]
    fp = cand[4] if len(cand) > 4 else 0
    return sa.sa_search_params(threads_per_block=th, blocks_per_sm=bps, key_depth=depth, chunk=chunk,
                               front_probes=fp)


def autotune(refs, q_bases, q_offsets, q_ref=None, sample: int = 1_000_000,
             candidates: Sequence[Tuple[int, ...]] = DEFAULT_CANDIDATES, reps: int = 3,
             cache_path: Optional[str] = None, use_cache: bool = True,
             timer: Optional[Callable] = None) -> Tuple["sa.sa_search_params", dict]:
    """(params, report) for this batch shape; q_bases/q_offsets/q_ref on the device."""
    import torch

    refs = [refs] if isinstance(refs, sa.Index) else list(refs)
    n_q_all = int(q_offsets.numel()) - 1
    n_q = min(n_q_all, sample)
    qo = q_offsets[:n_q + 1]
    mean_len = float((qo[-1] - qo[0]).item()) / max(1, n_q)
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, refs, mean_len)
    path = cache_path or default_cache_path()
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        return params_from(cache[key]["best"]), {"cached": True, **cache[key]}

    stream = torch.cuda.current_stream()

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    first = int(qo[0].item())
    total = int((qo[-1] - qo[0]).item())
    qr = None if q_ref is None else q_ref[:n_q]
    out = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64, device=q_offsets.device)
    ref_result = None
    timings: List[Tuple[Tuple[int, ...], float]] = []
    for cand in candidates:
        p = params_from(cand)
        p.flags = sa.SA_PARAM_Q_RANGE
        p.q_first, p.q_total = first, total
        e0, e1 = ev(), ev()
        p.search_events[0], p.search_events[1] = e0.cuda_event, e1.cuda_event
        ts = []
        for it in range(reps + 1):
            sa.sa_search_batch(refs, q_bases, qo, q_ref=qr, out=out, params=p)
            torch.cuda.synchronize()
            if it:
                ts.append(timer(e0, e1) if timer else e0.elapsed_time(e1))
        if ref_result is None:
            ref_result = out.clone()
        elif not torch.equal(out, ref_result):
            raise RuntimeError(f"candidate {cand} changed the results")
        timings.append((tuple(cand), statistics.median(ts)))
    best, t = pick_best(timings)
    report = {"best": list(best), "ms": t, "sample_queries": n_q,
              "all": [[list(c), ms] for c, ms in timings]}
    if use_cache:
        cache[key] = report
        save_cache(path, cache)
    return params_from(best), {"cached": False, **report}
