"""Serving at 2.4 Gbp: four resident references of 600 Mbp (10% segmental
duplications, int32 suffix arrays, k = 14 tables), a Poisson trace whose
requests mix locate caps 0/1/4/16 and strands (a quarter search the reverse
complement), coalesced by the continuous-batching server.

* every request's results (and positions) equal the same request run alone;
* a sample of requests is checked against the oracle: the oracle verifies each
  GPU-built suffix array (a permutation whose adjacent suffixes strictly
  increase is the unique one -- rebuilding 600 Mbp by comparison sort would
  take hours), then its Alg. 1 search gives the sampled queries' intervals
  (of the reverse-complemented queries for the other strand) and its locate
  their positions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu

SIZES = (600_000_000,) * 4
CAPS = (0, 1, 4, 16)


@pytest.fixture(scope="module")
def env():
    from paper_1303_3692_gb300 import build_lib, serve
    from paper_1303_3692_gb300 import sa as sa_mod

    build_lib.build()
    torch.cuda.empty_cache()
    refs = [datagen.reference(n, datagen.SEED0 + 80 + i, sd_cover=0.10) for i, n in enumerate(SIZES)]
    idxs = [sa_mod.sa_build(torch.from_numpy(r).cuda(), kmer_k=14) for r in refs]
    pools = []
    for i, r in enumerate(refs):
        qb, qo, _ = datagen.queries(r, 100_000, datagen.SEED0 + 90 + i, m=(20, 300), frac_sampled=0.75, subs=(0, 0))
        pools.append((torch.from_numpy(qb).pin_memory(), qo))
    yield sa_mod, serve, refs, idxs, pools
    for x in idxs:
        x.free()
    torch.cuda.empty_cache()


def _alone(sa, idx, r):
    bases = r.bases[:r.nbases].cuda() if r.nbases else torch.zeros(1, dtype=torch.uint8, device="cuda")
    offs = torch.from_numpy(r.offsets).cuda()
    p = sa.sa_search_params(flags=sa.SA_PARAM_REVERSE_COMPLEMENT if r.rc else 0)
    if r.cap:
        res, o, pos = sa.sa_search_locate(idx, bases, offs, r.cap, params=p)
        return res.cpu().numpy(), o.cpu().numpy(), pos.cpu().numpy()
    return sa.sa_search_batch(idx, bases, offs, params=p).cpu().numpy(), None, None


def test_serving_2gbp_mixed_caps_and_strands(env):
    sa, serve, refs, idxs, pools = env
    trace = serve.make_trace(pools, rate=2000, duration=0.4, seed=31, q_range=(1, 20_000), caps=CAPS, rc_frac=0.25)
    assert any(r.rc for r in trace) and len({r.cap for r in trace}) == len(CAPS)
    srv = serve.Server(idxs, slots=3, max_cap=max(CAPS))
    stats = srv.run(trace)
    assert stats["served"] == len(trace) and stats["rejected"] == 0
    for r in trace:
        res, o, pos = _alone(sa, idxs[r.ref], r)
        assert np.array_equal(r.results, res), r.rid
        if r.cap:
            total = int(o[-1])
            assert np.array_equal(r.pos_offsets, o) and np.array_equal(r.positions, pos[:total]), r.rid

    # the oracle, over each verified suffix array, on sampled requests
    comp = np.zeros(256, dtype=np.uint8)
    for a_, b_ in zip(b"ACGT", b"TGCA"):
        comp[a_] = b_
    rng = np.random.default_rng(32)
    for i, (ref, idx) in enumerate(zip(refs, idxs)):
        T = oracle.normalize(ref)
        sa_h = idx.suffix_array(device="cpu").numpy().astype(np.int64)
        assert oracle.verify_sa(T, sa_h, threads=oracle.cpu_threads()) == (0, -1), i
        mine = [r for r in trace if r.ref == i]
        for r in rng.choice(mine, size=min(12, len(mine)), replace=False):
            bases = r.bases[:r.nbases].numpy()
            for q in rng.choice(r.n, size=min(50, r.n), replace=False):
                P = bases[r.offsets[q]:r.offsets[q + 1]]
                if r.rc:
                    P = comp[P][::-1]
                lo, hi = oracle.search(T, sa_h, P)
                assert r.results[q, :3].tolist() == [lo, hi, hi - lo], (r.rid, q)
                if r.cap:
                    got = r.positions[r.pos_offsets[q]:r.pos_offsets[q + 1]].astype(np.int64)
                    assert np.array_equal(got, oracle.locate(sa_h, lo, hi, r.cap)), (r.rid, q)
