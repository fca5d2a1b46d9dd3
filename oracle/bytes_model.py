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

The second figure models the search with a k-mer table of plain counts and
32-byte suffix records of 112 bases (oracle_probe_model_kmer):

    B_q = ceil(m/4) + 32 * [m >= k] + 32 * P'_q + 32 * W_q + 3 * w

P'_q probes read one record sector each (below depth d0 only when no k-mer
bracket applies), W_q counts the 32-base text windows of compares that tie on
a record's 112 bases.  The third is the CUDA path's layout, whose 64-byte k-mer
entries carry the bracket's first pivot, so that probe costs no access of its
own:

    B_q = ceil(m/4) + 64 * [m >= k] + 32 * (P'_q - [m >= k and P'_q >= 1]) + 32 * W_q + 3 * w

    python -m oracle.bytes_model --workload repetitive-100m [--sample 20000] [--k 12]
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


def auto_k(n: int) -> int:
    """The largest k with 4^k <= 3n, in 1..15 (the library's automatic choice)."""
    k = 1
    while k < 15 and (1 << (2 * (k + 1))) <= 3 * n:
        k += 1
    return k


def model(w, sample: int, d0: int, k: int = 0, seed: int = 7):
    T = oracle.normalize(w.ref)
    t0 = time.time()
    sa = oracle.sa_naive(T)
    build_s = time.time() - t0
    k = k or auto_k(T.size)
    t0 = time.time()
    table = oracle.kmer_table(T, sa, k)
    table_s = time.time() - t0
    n_q = w.q_offsets.size - 1
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(n_q, size=min(sample, n_q), replace=False))
    wbytes = 4 if w.width == 32 else 8
    tot = {"query": 0, "sa": 0, "text": 0, "out": 0, "locate": 0, "probes": 0, "chunks": 0, "count": 0,
           "k_table": 0, "k_probes": 0, "k_windows": 0, "k_probes_after_entry": 0, "k_with_bracket": 0}
    for q in pick:
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        pr, ch, lo, hi = oracle.probe_model(T, sa, P, d0=d0)
        tot["query"] += (P.size + 3) // 4
        tot["sa"] += 32 * pr
        tot["text"] += 32 * ch
        tot["out"] += 3 * wbytes
        tot["probes"] += pr
        tot["chunks"] += ch
        tot["count"] += hi - lo
        tot["locate"] += 2 * wbytes * min(hi - lo, w.cap)
        kp, kw, kt, klo, khi = oracle.probe_model_kmer(T, sa, table, k, P, d0=d0)
        assert (klo, khi) == (lo, hi)
        tot["k_table"] += 32 * kt
        tot["k_probes"] += kp
        tot["k_with_bracket"] += kt
        # with 64-byte k-mer entries the first probe comes with the entry
        tot["k_probes_after_entry"] += max(kp - 1, 0) if kt else kp
        tot["k_windows"] += kw
    cnt = len(pick)
    per = {key: v / cnt for key, v in tot.items()}
    per["search_bytes_per_query"] = per["query"] + per["sa"] + per["text"] + per["out"]
    per["kmer_record_bytes_per_query"] = (per["query"] + per["k_table"] + 32 * per["k_probes"] +
                                          32 * per["k_windows"] + per["out"])
    # 64-byte k-mer entries carrying the first pivot's record: one random
    # access for the entry, then one per further probe and per text window
    per["krt_random_accesses_per_query"] = (per["k_with_bracket"] + per["k_probes_after_entry"] +
                                            per["k_windows"])
    per["krt_bytes_per_query"] = (per["query"] + 64 * per["k_with_bracket"] + 32 * per["k_probes_after_entry"] +
                                  32 * per["k_windows"] + per["out"])
    per["k"] = k
    per["sample"] = cnt
    per["d0"] = d0
    per["oracle_sa_build_s"] = build_s
    per["oracle_kmer_table_s"] = table_s
    return per


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="repetitive-100m")
    ap.add_argument("--sample", type=int, default=20000)
    ap.add_argument("--d0", type=int, default=13)
    ap.add_argument("--k", type=int, default=0, help="k-mer table k (0: automatic)")
    a = ap.parse_args()
    w = WORKLOADS[a.workload]()
    print(json.dumps({"workload": w.name, **model(w, a.sample, a.d0, a.k)}, indent=1))


if __name__ == "__main__":
    main()
