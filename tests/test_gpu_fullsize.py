"""Full-size parity on the 100 Mbp repetitive workload (10,000,000 queries of
100 bp, locate up to 64), in the launch configuration bench.py times: the
suffix array, every query's [lo, hi, count] and every located position equal
the oracle's (naive suffix sort + Alg. 1 on the host cores)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    from paper_1303_3692_gb300 import build_lib, sa

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    w = datagen.repetitive_100m()
    T = oracle.normalize(w.ref)
    osa = oracle.sa_naive(T)
    idx = sa.sa_build(torch.from_numpy(w.ref).cuda())
    return sa, w, T, osa, idx


def test_suffix_array_full_size(c2):
    sa, w, T, osa, idx = c2
    got = idx.suffix_array().cpu().numpy().astype(np.int64)
    assert np.array_equal(got, osa)


def test_search_and_locate_full_size(c2):
    sa, w, T, osa, idx = c2
    qb = torch.from_numpy(w.q_bases).cuda()
    qo = torch.from_numpy(w.q_offsets).cuda()
    res = sa.sa_search_batch(idx, qb, qo)
    offs, pos = sa.sa_locate(idx, res, w.cap)
    got = res.cpu().numpy()
    lo, hi = oracle.search_batch(T, osa, w.q_bases, w.q_offsets, threads=oracle.cpu_threads())
    assert np.array_equal(got[:, 0], lo)
    assert np.array_equal(got[:, 1], hi)
    assert np.array_equal(got[:, 2], hi - lo)
    k = np.minimum(hi - lo, w.cap)
    offs = offs.cpu().numpy()
    assert offs[0] == 0 and np.array_equal(np.diff(offs), k)
    # expected positions: SA[lo_q + j] for j < k_q, queries in order
    starts = np.repeat(lo, k)
    within = np.arange(int(k.sum())) - np.repeat(offs[:-1], k)
    assert np.array_equal(pos.cpu().numpy().astype(np.int64), osa[starts + within])
    # the one-call path that the benchmark times gives the same results and positions
    res2, offs2, pos2 = sa.sa_search_locate(idx, qb, qo, w.cap)
    assert torch.equal(res2[:, :3], res[:, :3])
    # the one call marks each query whose count exceeds the cap as truncated
    assert np.array_equal(res2[:, 3].cpu().numpy(), np.where(got[:, 2] > w.cap, sa.SA_RESULT_TRUNCATED, 0))
    assert np.array_equal(offs2.cpu().numpy(), offs)
    assert torch.equal(pos2[:int(offs[-1])].cpu(), pos[:int(offs[-1])].cpu())
    # every exact copy from the reference occurs; counts agree with brute force on a sample
    rng = np.random.default_rng(3)
    for q in rng.choice(np.nonzero(w.sampled)[0], 8, replace=False):
        P = w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]]
        assert oracle.bruteforce(T, P)[0] == hi[q] - lo[q]


def test_plain_kernel_full_size_sample(c2):
    sa, w, T, osa, idx = c2
    n = 200_000
    qb = torch.from_numpy(w.q_bases[:w.q_offsets[n]]).cuda()
    qo = torch.from_numpy(w.q_offsets[:n + 1]).cuda()
    a = sa.sa_search_batch(idx, qb, qo).cpu()
    b = sa.sa_search_batch_plain(idx, qb, qo).cpu()
    assert torch.equal(a, b)


def test_multi_genome_full_size():
    """4 references (5, 12, 25, 50 Mbp) and 16,000,000 queries of U[20,250] bp,
    each assigned to one reference, searched in one call with q_ref: every
    query's interval equals the oracle's on its own reference."""
    from paper_1303_3692_gb300 import build_lib, sa

    build_lib.build()
    refs, qb, qo, qref, smp = datagen.multi_genome()
    idxs = [sa.sa_build(torch.from_numpy(r).cuda()) for r in refs]
    got = sa.sa_search_batch(idxs, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(),
                             q_ref=torch.from_numpy(qref).cuda()).cpu().numpy()
    for r, ref in enumerate(refs):
        T = oracle.normalize(ref)
        osa = oracle.sa_naive(T)
        assert np.array_equal(idxs[r].suffix_array().cpu().numpy().astype(np.int64), osa)
        sel = np.nonzero(qref == r)[0]
        lens = qo[sel + 1] - qo[sel]
        sub_qo = np.zeros(sel.size + 1, dtype=np.int64)
        np.cumsum(lens, out=sub_qo[1:])
        # gather this reference's queries into one contiguous buffer
        idx = np.repeat(qo[sel], lens) + (np.arange(int(lens.sum())) - np.repeat(sub_qo[:-1], lens))
        lo, hi = oracle.search_batch(T, osa, qb[idx], sub_qo, threads=oracle.cpu_threads())
        assert np.array_equal(got[sel, 0], lo), r
        assert np.array_equal(got[sel, 1], hi), r
        assert np.array_equal(got[sel, 2], hi - lo), r
