"""Batching runtime on the GPU: continuous-batching serving (each request's
results are the same alone and in the mix), CUDA-graph capture of the search
and locate calls, and the autotuner."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1303_3692_gb300 import build_lib, sa

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    refs = [datagen.reference(n, 300 + i, sd_cover=0.1, tandem_cover=0.02)
            for i, n in enumerate((20_000, 60_000, 150_000))]
    idxs = [sa.sa_build(torch.from_numpy(r).cuda()) for r in refs]
    pools = []
    for i, r in enumerate(refs):
        qb, qo, _ = datagen.queries(r, 3000, 310 + i, m=(20, 300), frac_sampled=0.75, subs=(0, 1))
        pools.append((torch.from_numpy(qb).pin_memory(), qo))
    return sa, refs, idxs, pools


def _alone(sa, idx, r):
    """The request run by itself: a search, with its own locate cap if it asked for positions."""
    bases = r.bases[:r.nbases].cuda() if r.nbases else torch.zeros(1, dtype=torch.uint8, device="cuda")
    offs = torch.from_numpy(r.offsets).cuda()
    if r.cap:
        return sa.sa_search_locate(idx, bases, offs, r.cap)[0].cpu().numpy()
    return sa.sa_search_batch(idx, bases, offs).cpu().numpy()


def test_serving_results_equal_alone_and_oracle(env):
    from paper_1303_3692_gb300 import serve

    sa, refs, idxs, pools = env
    trace = serve.make_trace(pools, rate=4000, duration=0.05, seed=5, q_range=(1, 600))
    srv = serve.Server(idxs, max_batch_queries=3000, max_batch_bases=3000 * 300, slots=2)
    stats = srv.run(trace)
    assert stats["served"] == len(trace) and stats["rejected"] == 0
    assert stats["batches"] < len(trace)  # requests were coalesced
    osas = [oracle.sa_naive(oracle.normalize(r)) for r in refs]
    for r in trace:
        assert np.array_equal(r.results, _alone(sa, idxs[r.ref], r)), r.rid
    for r in trace[::7]:
        T = oracle.normalize(refs[r.ref])
        lo, hi = oracle.search_batch(T, osas[r.ref], r.bases[:r.nbases].numpy(), r.offsets)
        assert np.array_equal(r.results[:, 0], lo) and np.array_equal(r.results[:, 1], hi)
    # the plain per-request path gives the same answers
    plain_trace = serve.make_trace(pools, rate=4000, duration=0.05, seed=5, q_range=(1, 600))
    serve.run_plain(idxs, plain_trace)
    for a, b in zip(trace, plain_trace):
        assert np.array_equal(a.results, b.results)


def test_serving_mixed_locate_caps(env):
    """Requests with caps 0, 1, 4 and 16 share batches (located up to the
    batch's largest cap); each request's results and positions equal the
    request served alone and the oracle's suffix-array positions."""
    from paper_1303_3692_gb300 import serve

    sa, refs, idxs, pools = env
    trace = serve.make_trace(pools, rate=4000, duration=0.05, seed=9, q_range=(1, 400), caps=(0, 1, 4, 16))
    srv = serve.Server(idxs, max_batch_queries=3000, max_batch_bases=3000 * 300, slots=2, max_cap=16)
    stats = srv.run(trace)
    assert stats["served"] == len(trace) and stats["batches"] < len(trace)
    assert {r.cap for r in trace} == {0, 1, 4, 16}
    osas = [oracle.sa_naive(oracle.normalize(r)) for r in refs]
    for r in trace:
        assert np.array_equal(r.results, _alone(sa, idxs[r.ref], r)), r.rid
        if not r.cap:
            assert r.positions is None
            continue
        bases = r.bases[:r.nbases].cuda() if r.nbases else torch.zeros(1, dtype=torch.uint8, device="cuda")
        _, offs, pos = sa.sa_search_locate(idxs[r.ref], bases, torch.from_numpy(r.offsets).cuda(), r.cap)
        offs = offs.cpu().numpy()
        assert np.array_equal(r.pos_offsets, offs), r.rid
        assert np.array_equal(r.positions, pos[:int(offs[-1])].cpu().numpy()), r.rid
        for q in range(0, r.n, 37):
            lo, hi = int(r.results[q, 0]), int(r.results[q, 1])
            want = osas[r.ref][lo:lo + min(hi - lo, r.cap)]
            assert np.array_equal(r.positions[r.pos_offsets[q]:r.pos_offsets[q + 1]].astype(np.int64), want)


def test_serving_rejects_and_defers(env):
    from paper_1303_3692_gb300 import serve

    sa, refs, idxs, pools = env
    trace = serve.make_trace(pools, rate=2000, duration=0.03, seed=9, q_range=(50, 400))
    big = trace[0]
    # a budget that fits the largest request: everything is served, no batch exceeds it
    one = max(serve.scratch_bytes(r.n, r.nbases) for r in trace)
    srv = serve.Server(idxs, max_batch_queries=1000, max_batch_bases=10**7, slots=2, mem_reserve=0,
                       free_memory=lambda: one)
    stats = srv.run(trace)
    assert stats["served"] == len(trace)
    assert all(serve.scratch_bytes(q, b) <= one for q, b in srv.batch_sizes)
    assert stats["batches"] > 1
    # a request larger than a batch is rejected, the rest are served
    trace2 = serve.make_trace(pools, rate=2000, duration=0.03, seed=9, q_range=(50, 400))
    srv2 = serve.Server(idxs, max_batch_queries=big.n - 1, max_batch_bases=10**7, slots=2)
    stats2 = srv2.run(trace2)
    assert trace2[0].status == "rejected" and stats2["rejected"] >= 1
    assert stats2["served"] + stats2["rejected"] == len(trace2)


def test_cuda_graph_capture_and_replay(env):
    sa, refs, idxs, pools = env
    ref = refs[2]
    n_q = 4000
    qb1, qo, _ = datagen.queries(ref, n_q, 401, m=90, frac_sampled=0.8, subs=(0, 1))
    qb2, _, _ = datagen.queries(ref, n_q, 402, m=90, frac_sampled=0.8, subs=(0, 1))
    bases = torch.from_numpy(qb1).cuda()
    offs = torch.from_numpy(qo).cuda()
    out = torch.empty((n_q, sa.RESULT_FIELDS), dtype=torch.int64, device="cuda")
    loc_off = torch.empty(n_q + 1, dtype=torch.int64, device="cuda")
    loc_pos = torch.empty(n_q * 8, dtype=torch.int32, device="cuda")
    p = sa.sa_search_params()
    p.flags = sa.SA_PARAM_Q_RANGE
    p.q_first, p.q_total = 0, int(qo[-1])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm up (kernel attributes, pool) outside capture
        sa.sa_search_batch(idxs[2], bases, offs, out=out, params=p)
        sa.sa_locate(idxs[2], out, 8, out_offsets=loc_off, out_pos=loc_pos, capacity=loc_pos.numel())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sa.sa_search_batch(idxs[2], bases, offs, out=out, params=p)
        sa.sa_locate(idxs[2], out, 8, out_offsets=loc_off, out_pos=loc_pos, capacity=loc_pos.numel())
    for qb in (qb2, qb1, qb2):
        bases.copy_(torch.from_numpy(qb))
        g.replay()
        torch.cuda.synchronize()
        want = sa.sa_search_batch(idxs[2], torch.from_numpy(qb).cuda(), offs)
        wo, wp = sa.sa_locate(idxs[2], want, 8)
        assert torch.equal(out, want)
        assert torch.equal(loc_off, wo)
        assert torch.equal(loc_pos[:int(wo[-1])], wp[:int(wo[-1])])


def test_autotune_picks_working_params_and_caches(env, tmp_path):
    from paper_1303_3692_gb300 import autotune

    sa, refs, idxs, pools = env
    qb, qo, _ = datagen.queries(refs[2], 20000, 501, m=(20, 200), frac_sampled=0.7, subs=(0, 1))
    bases, offs = torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda()
    cache = str(tmp_path / "tune.json")
    cands = ((1024, 1, 12, 64), (512, 2, 11, 32, 2), (256, 4, 10, 64, 5))
    p, rep = autotune.autotune(idxs[2], bases, offs, candidates=cands, reps=2, cache_path=cache)
    assert not rep["cached"] and tuple(rep["best"]) in cands and len(rep["all"]) == 3
    a = sa.sa_search_batch(idxs[2], bases, offs, params=p)
    b = sa.sa_search_batch(idxs[2], bases, offs)
    assert torch.equal(a, b)
    p2, rep2 = autotune.autotune(idxs[2], bases, offs, candidates=cands, reps=2, cache_path=cache)
    assert rep2["cached"] and rep2["best"] == rep["best"]
