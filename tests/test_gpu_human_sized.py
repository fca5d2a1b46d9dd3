"""The 3.1 Gbp configuration at full size, in the launch configuration the
benchmark times: a human-genome-sized synthetic reference (GC 0.41, 45% repeat
families of 300 bp and 6 kb units at 10-20% divergence, 3% tandem repeats)
with an int64 suffix array, and 1.1e8 queries of 150 bp (10:1 sampled with
0-1 substitutions : random) searched and located (cap 16) in one
sa_search_locate call.

The oracle cannot sort 3.1e9 suffixes in a test's time, so it verifies the
GPU-built suffix array instead (a permutation of [0, n) whose adjacent
suffixes strictly increase is the unique suffix array) and then:

* its Alg. 1 search over that array gives every one of 1,000,000 sampled
  queries' [lo, hi, count], and its locate their positions -- bit-exact;
* its definition counts, which use no suffix array at all (suffixes whose
  150-prefix sorts before / not after the query), give 48 sampled queries'
  [lo, hi);
* brute-force scanning of all 3.1e9 positions gives four queries' occurrence
  sets;
* every one of the 1.1e8 results satisfies lo <= hi <= n, count = hi - lo, and
  the offsets are the exclusive scan of min(count, 16).

Needs ~230 GB of device memory and ~60 GB of host memory; runs in about two
minutes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu

CAP = 16


@pytest.fixture(scope="module")
def human():
    from paper_1303_3692_gb300 import build_lib, sa

    build_lib.build()
    torch.cuda.empty_cache()
    w = datagen.human_sized()
    idx = sa.sa_build(torch.from_numpy(w.ref).cuda(), width=64)
    qb = torch.from_numpy(w.q_bases).cuda()
    qo = torch.from_numpy(w.q_offsets).cuda()
    capacity = 4 * (qo.numel() - 1)  # about seven times the positions this batch has
    res, offs, pos = sa.sa_search_locate(idx, qb, qo, CAP, capacity=capacity)
    out = (res.cpu().numpy(), offs.cpu().numpy(), pos.cpu().numpy())
    assert out[1][-1] <= capacity
    del qb, qo, res, offs, pos
    T = oracle.normalize(w.ref)
    sa_h = idx.suffix_array(device="cpu").numpy()
    yield w, idx, T, sa_h, out
    idx.free()
    torch.cuda.empty_cache()


def test_suffix_array_verified(human):
    w, idx, T, sa_h, _ = human
    assert idx.width == 8 and idx.n == 3_100_000_000
    assert oracle.verify_sa(T, sa_h, threads=oracle.cpu_threads()) == (0, -1)


def test_all_results_consistent(human):
    w, idx, T, sa_h, (res, offs, pos) = human
    n_q = w.q_offsets.size - 1
    assert res.shape == (n_q, 4) and not (res[:, 3] & 1).any()
    lo, hi, cnt = res[:, 0], res[:, 1], res[:, 2]
    assert np.all(lo >= 0) and np.all(lo <= hi) and np.all(hi <= T.size) and np.array_equal(cnt, hi - lo)
    kept = np.minimum(cnt, CAP)
    assert offs[0] == 0 and np.array_equal(np.diff(offs), kept)
    assert np.array_equal(res[:, 3], np.where(cnt > CAP, 2, 0))  # SA_RESULT_TRUNCATED


def test_sampled_queries_against_oracle_search(human):
    w, idx, T, sa_h, (res, offs, pos) = human
    n_q = w.q_offsets.size - 1
    rng = np.random.default_rng(2024)
    pick = np.sort(rng.choice(n_q, size=1_000_000, replace=False))
    sub = np.zeros(pick.size + 1, dtype=np.int64)
    np.cumsum(w.q_offsets[pick + 1] - w.q_offsets[pick], out=sub[1:])
    Q = w.q_bases.reshape(n_q, 150)[pick].reshape(-1)
    lo, hi = oracle.search_batch(T, sa_h, Q, sub, threads=oracle.cpu_threads())
    assert np.array_equal(res[pick, 0], lo) and np.array_equal(res[pick, 1], hi)
    assert np.array_equal(res[pick, 2], hi - lo)
    # located positions of every sampled query: the first min(count, 16) entries of its interval
    for j in np.nonzero(hi > lo)[0]:
        q = pick[j]
        want = oracle.locate(sa_h, int(lo[j]), int(hi[j]), CAP)
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64), want), q


def test_sampled_queries_against_definition_and_brute_force(human):
    w, idx, T, sa_h, (res, offs, pos) = human
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(np.nonzero(w.sampled)[0], 40, replace=False),
                           rng.choice(np.nonzero(~w.sampled)[0], 8, replace=False)])
    sub = np.zeros(pick.size + 1, dtype=np.int64)
    np.cumsum(w.q_offsets[pick + 1] - w.q_offsets[pick], out=sub[1:])
    Q = np.concatenate([w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]] for q in pick])
    lo, hi = oracle.rank_count_batch(T, Q, sub, threads=oracle.cpu_threads())
    assert np.array_equal(res[pick, 0], lo) and np.array_equal(res[pick, 1], hi)
    for j in (0, 1, 2, 41):  # brute force scans 3.1e9 positions per query
        q = pick[j]
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        cnt, occ = oracle.bruteforce(T, P, cap=1 << 20)
        assert cnt == hi[j] - lo[j]
        want = oracle.sort_positions(T, occ)[:CAP]
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64), want)
