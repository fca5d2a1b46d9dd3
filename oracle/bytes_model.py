"""Algorithmic bytes per query of the search, from the oracle's byte model.

Test/measurement infrastructure: runs only the oracle (naive suffix sort and
oracle_probe_model) on a seeded sample of a workload's queries and prints the
per-query byte figure that the benchmark's roofline uses as its numerator:

    B_q = ceil(m/4)              packed query read once
        + 32 * P_q               one 32-byte suffix-array sector per probe
        + 32 * X_q               one 32-byte text sector per 64-base chunk compared
        + 3 * w                  lo, hi, count written (w = suffix-array width in bytes)

P_q counts the probes of the lockstep lower/upper-bound search at depth
>= d0 (the first d0 levels are answered by the shared-memory key table), X_q
the 64-base chunks those probes compare, starting at min(lcp(P,S_L),
lcp(P,S_R)).  Locate adds w * min(count, cap) written plus the same read.

    python -m oracle.bytes_model --workload repetitive-100m [--sample 20000]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1303_3692_gb300 import datagen  # noqa: E402

WORKLOADS = {
    "plain-small": lambda: datagen.plain_small(),
    "repetitive-100m": lambda: datagen.repetitive_100m(),
}


def model(w, sample: int, d0: int, seed: int = 7):
    T = oracle.normalize(w.ref)
    t0 = time.time()
    sa = oracle.sa_naive(T)
    build_s = time.time() - t0
    n_q = w.q_offsets.size - 1
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(n_q, size=min(sample, n_q), replace=False))
    wbytes = 4 if w.width == 32 else 8
    tot = {"query": 0, "sa": 0, "text": 0, "out": 0, "locate": 0, "probes": 0, "chunks": 0, "count": 0}
    for q in pick:
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        pr, ch, lo, hi = oracle.probe_model(T, sa, P, d0=d0)
        tot["query"] += (P.size + 3) // 4
        tot["sa"] += 32 * pr
        tot["text"] += 32 * ch
        tot["out"] += 3 * wbytes
        tot["probes"] += pr
        tot["chunks"] += ch
        k = min(hi - lo, w.cap)
        tot["count"] += hi - lo
        tot["locate"] += 2 * wbytes * k
    k = len(pick)
    per = {key: v / k for key, v in tot.items()}
    per["search_bytes_per_query"] = per["query"] + per["sa"] + per["text"] + per["out"]
    per["sample"] = k
    per["d0"] = d0
    per["oracle_sa_build_s"] = build_s
    return per


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="repetitive-100m")
    ap.add_argument("--sample", type=int, default=20000)
    ap.add_argument("--d0", type=int, default=13)
    a = ap.parse_args()
    w = WORKLOADS[a.workload]()
    print(json.dumps({"workload": w.name, **model(w, a.sample, a.d0)}, indent=1))


if __name__ == "__main__":
    main()
