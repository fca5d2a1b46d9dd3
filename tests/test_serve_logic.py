"""Host-side logic of the serving loop (admission, batch formation, trace
generation, summaries) with fake requests and a fake memory probe.  No GPU."""
import math

import numpy as np
import torch

from paper_1303_3692_gb300 import serve


def _req(rid, n, m=10, arrival=0.0, ref=0):
    offs = np.arange(n + 1, dtype=np.int64) * m
    return serve.Request(rid, ref, None, offs, arrival)


def test_form_batch_respects_query_and_base_limits():
    q = [_req(i, 100) for i in range(5)]
    taken, rest = serve.form_batch(q, max_q=250, max_bases=10**9, budget=10**12)
    assert [r.rid for r in taken] == [0, 1] and [r.rid for r in rest] == [2, 3, 4]
    taken, rest = serve.form_batch(q, max_q=10**9, max_bases=2500, budget=10**12)
    assert [r.rid for r in taken] == [0, 1]


def test_form_batch_respects_memory_budget_and_order():
    q = [_req(0, 10), _req(1, 10**6), _req(2, 10)]
    need_first = serve.scratch_bytes(10, 100)
    taken, rest = serve.form_batch(q, 10**9, 10**12, budget=need_first + 1000)
    assert [r.rid for r in taken] == [0]            # the large one waits, and so does the one behind it
    assert [r.rid for r in rest] == [1, 2]
    taken, rest = serve.form_batch(q, 10**9, 10**12, budget=0)
    assert taken == [] and len(rest) == 3           # nothing admitted without memory


def test_scratch_bytes_grows_with_batch():
    assert serve.scratch_bytes(1000, 100_000) > serve.scratch_bytes(10, 1000) > 0


def test_make_trace_is_poisson_and_slices_pools():
    pools = []
    for r in range(3):
        offs = np.arange(0, 2001 * 7, 7, dtype=np.int64)
        pools.append((torch.zeros(int(offs[-1]), dtype=torch.uint8), offs))
    tr = serve.make_trace(pools, rate=2000, duration=2.0, seed=1, q_range=(1, 1000))
    assert 3600 < len(tr) < 4400                    # ~ rate * duration
    gaps = np.diff([r.arrival for r in tr])
    assert abs(gaps.mean() - 1 / 2000) < 1e-4
    for r in tr[:50]:
        assert 1 <= r.n <= 1000 and r.offsets[0] == 0 and r.bases.numel() == r.nbases
    assert len({r.ref for r in tr}) == 3


def test_summarize_percentiles():
    tr = [_req(i, 5, arrival=0.0) for i in range(100)]
    for i, r in enumerate(tr):
        r.done, r.status = (i + 1) / 1000.0, "done"
    s = serve.summarize(tr, batches=7)
    assert s["served"] == 100 and s["queries"] == 500 and s["batches"] == 7
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and abs(s["p99_ms"] - 99.01) < 1e-6
    assert math.isclose(s["queries_per_s"], 500 / 0.1)


def test_autotune_host_logic(tmp_path):
    from paper_1303_3692_gb300 import autotune

    assert autotune.length_bucket(20) == 0 and autotune.length_bucket(100) == 1
    assert autotune.length_bucket(250) == 3 and autotune.length_bucket(10**6) == 4
    best, t = autotune.pick_best([((1, 1, 1, 1), 3.0), ((2, 2, 2, 2), 1.5), ((3, 3, 3, 3), 1.5)])
    assert best == (2, 2, 2, 2) and t == 1.5
    path = str(tmp_path / "c.json")
    autotune.save_cache(path, {"k": {"best": [1, 2, 3, 4]}})
    assert autotune.load_cache(path) == {"k": {"best": [1, 2, 3, 4]}}
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


def test_split_positions_keeps_each_requests_cap():
    """A batch locates min(count, cap_batch) per query; each request keeps the
    first min(count, its cap), none for an invalid query (count -1)."""
    results = np.array([[0, 3, 3], [5, 5, 0], [-1, -1, -1], [7, 9, 2]], dtype=np.int64)
    offs = np.array([0, 2, 2, 2, 4], dtype=np.int64)  # cap_batch = 2
    pos = np.array([10, 11, 20, 21], dtype=np.int32)
    o1, p1 = serve.split_positions(results, offs, pos, 2, 1)
    assert o1.tolist() == [0, 1, 1, 1, 2] and p1.tolist() == [10, 20]
    o2, p2 = serve.split_positions(results, offs, pos, 2, 2)
    assert o2.tolist() == offs.tolist() and p2.tolist() == pos.tolist()
    assert serve.kept(results[:, 2], 5).tolist() == [3, 0, 0, 2]


def test_make_trace_caps_default_keeps_traces():
    pools = [(np.zeros(100, dtype=np.uint8), np.arange(0, 101, dtype=np.int64))]
    a = serve.make_trace(pools, rate=1000, duration=0.05, seed=3, q_range=(1, 10))
    b = serve.make_trace(pools, rate=1000, duration=0.05, seed=3, q_range=(1, 10), caps=(0, 4))
    assert all(r.cap == 0 for r in a)
    assert {r.cap for r in b} <= {0, 4}
