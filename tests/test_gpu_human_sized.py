"""The 3.1 Gbp configuration: a human-genome-sized synthetic reference (GC
0.41, 45% repeat families of 300 bp and 6 kb units at 10-20% divergence, 3%
tandem repeats) with an int64 suffix array, and 150 bp queries (10:1 sampled
with 0-1 substitutions : random).  Parity at full reference size:

* the GPU-built suffix array passes the oracle's verifier (a permutation of
  [0, n) whose adjacent suffixes strictly increase -- which proves it is the
  unique suffix array);
* sampled queries' [lo, hi, count] equal the oracle's definition counts
  (suffixes whose 150-prefix sorts before / not after the query), computed
  without any suffix array;
* their located positions (cap 16) equal the brute-force occurrences put in
  suffix order.

Runs for several minutes and needs ~200 GB of host memory and ~180 GB of
device memory, so it only runs when SA_RUN_HUMAN_SIZED=1."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SA_RUN_HUMAN_SIZED") != "1",
                                 reason="set SA_RUN_HUMAN_SIZED=1 to run the 3.1 Gbp configuration")]


@pytest.fixture(scope="module")
def human():
    from paper_1303_3692_gb300 import build_lib, sa

    build_lib.build()
    w = datagen.human_sized(nq_sampled=2_000_000, nq_random=200_000)
    idx = sa.sa_build(torch.from_numpy(w.ref).cuda(), width=64)
    return sa, w, idx


def test_suffix_array_verified(human):
    sa, w, idx = human
    assert idx.width == 8 and idx.n == 3_100_000_000
    got = idx.suffix_array(device="cpu").numpy()
    T = oracle.normalize(w.ref)
    assert oracle.verify_sa(T, got, threads=oracle.cpu_threads()) == (0, -1)


def test_sampled_queries_and_locate(human):
    sa, w, idx = human
    qb = torch.from_numpy(w.q_bases).cuda()
    qo = torch.from_numpy(w.q_offsets).cuda()
    res = sa.sa_search_batch(idx, qb, qo)
    offs, pos = sa.sa_locate(idx, res, 16)
    res, offs, pos = res.cpu().numpy(), offs.cpu().numpy(), pos.cpu().numpy()
    T = oracle.normalize(w.ref)
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(np.nonzero(w.sampled)[0], 40, replace=False),
                           rng.choice(np.nonzero(~w.sampled)[0], 8, replace=False)])
    sub = np.zeros(pick.size + 1, dtype=np.int64)
    np.cumsum(w.q_offsets[pick + 1] - w.q_offsets[pick], out=sub[1:])
    Q = np.concatenate([w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]] for q in pick])
    lo, hi = oracle.rank_count_batch(T, Q, sub, threads=oracle.cpu_threads())
    assert np.array_equal(res[pick, 0], lo) and np.array_equal(res[pick, 1], hi)
    assert np.array_equal(res[pick, 2], hi - lo)
    for j in (0, 1, 2, 41):  # brute force scans 3.1e9 positions per query
        q = pick[j]
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        cnt, occ = oracle.bruteforce(T, P)
        assert cnt == hi[j] - lo[j]
        want = oracle.sort_positions(T, occ)[:16]
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64), want)
