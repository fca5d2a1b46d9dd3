"""The k-mer-order search (queries bucketed by their first k bases before the
persistent kernel takes them) against the CPU oracle, bit-exact.  The library
picks that order by itself only for indexes above 48 GB; here
SA_PARAM_KMER_ORDER forces it on small indexes so that every case -- query
lengths around k and the record and window boundaries, empty and invalid
queries, several references with and without k-mer tables, the other strand,
locate, many tiles and buckets -- runs through it, and its results must also
equal the input-order search's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    from paper_1303_3692_gb300 import build_lib
    from paper_1303_3692_gb300 import sa as sa_mod

    build_lib.build()
    return sa_mod


def _both(sa, refs, qb, qo, q_ref=None, flags=0):
    out = []
    for order in (sa.SA_PARAM_KMER_ORDER, sa.SA_PARAM_INPUT_ORDER):
        p = sa.sa_search_params(flags=order | flags)
        r = sa.sa_search_batch(refs, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(),
                               q_ref=None if q_ref is None else torch.from_numpy(q_ref).cuda(), params=p)
        out.append(r.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    return out[0]


@pytest.mark.parametrize("width,k", [(32, None), (64, None), (32, 4), (64, 9)])
def test_kmer_order_repetitive(sa, width, k):
    ref = datagen.reference(200_003, 71 + (k or 0), gc=0.45, sd_cover=0.1, tandem_cover=0.05, family_cover=0.2)
    qb, qo, _ = datagen.queries(ref, 300_000, 72, m=(1, 300), frac_sampled=0.8, subs=(0, 1))
    idx = sa.sa_build(torch.from_numpy(ref).cuda(), width=width, kmer_k=k)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    got = _both(sa, idx, qb, qo)
    lo, hi = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi) and np.array_equal(got[:, 2], hi - lo)


def test_kmer_order_tiny_texts(sa):
    rng = np.random.default_rng(8)
    qs = [""] + ["".join(rng.choice(list("ACGT"), L)) for L in range(1, 9) for _ in range(6)]
    qb = np.frombuffer("".join(qs).encode(), dtype=np.uint8).copy()
    qo = np.zeros(len(qs) + 1, dtype=np.int64)
    np.cumsum([len(q) for q in qs], out=qo[1:])
    for text in ["A", "AC", "ACGTA", "AAAAAAA", "ACGGTACGTAC", "TTTTGGGG"]:
        T = np.frombuffer(text.encode(), dtype=np.uint8)
        idx = sa.sa_build(torch.from_numpy(T.copy()).cuda())
        osa = oracle.sa_naive(T)
        got = _both(sa, idx, qb, qo)
        lo, hi = oracle.search_batch(T, osa, qb, qo)
        assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi), text


def test_kmer_order_multi_reference_mixed_tables(sa):
    refs, qb, qo, qref, _ = datagen.multi_genome(scale=0.004)
    # the second index has no k-mer table: its queries take the key-table descent
    idxs = [sa.sa_build(torch.from_numpy(r).cuda(), kmer_k=0 if i == 1 else None) for i, r in enumerate(refs)]
    got = _both(sa, idxs, qb, qo, qref)
    for i, r in enumerate(refs):
        sel = np.nonzero(qref == i)[0]
        sub = np.zeros(sel.size + 1, dtype=np.int64)
        np.cumsum(qo[sel + 1] - qo[sel], out=sub[1:])
        Q = np.concatenate([qb[qo[q]:qo[q + 1]] for q in sel])
        T = oracle.normalize(r)
        lo, hi = oracle.search_batch(T, oracle.sa_naive(T), Q, sub, threads=oracle.cpu_threads())
        assert np.array_equal(got[sel, 0], lo) and np.array_equal(got[sel, 1], hi), i


def test_kmer_order_invalid_empty_and_other_strand(sa):
    ref = datagen.reference(50_000, 91, sd_cover=0.1, tandem_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 5000, 92, m=(0, 200), frac_sampled=0.7, subs=(0, 1))
    qb = qb.copy()
    bad = [3, 17, 4000]
    for q in bad:
        if qo[q + 1] > qo[q]:
            qb[qo[q]] = ord("N")
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = sa.sa_search_params(flags=sa.SA_PARAM_KMER_ORDER, device_status=st.data_ptr())
    got = sa.sa_search_batch(idx, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(), params=p).cpu().numpy()
    torch.cuda.synchronize()
    assert int(st.item()) == sa.SA_ERR_BASE
    for q in range(qo.size - 1):
        P = qb[qo[q]:qo[q + 1]]
        if q in bad and P.size:
            assert got[q].tolist() == [-1, -1, -1, sa.SA_RESULT_INVALID]
        else:
            lo, hi = oracle.search(T, osa, P)
            assert got[q].tolist() == [lo, hi, hi - lo, 0], q
    # the other strand: the reverse complements, searched in k-mer order
    good = np.array([q for q in range(qo.size - 1) if q not in bad])
    sub = np.zeros(good.size + 1, dtype=np.int64)
    np.cumsum(qo[good + 1] - qo[good], out=sub[1:])
    Q = np.concatenate([qb[qo[q]:qo[q + 1]] for q in good])
    comp = np.zeros(256, dtype=np.uint8)
    for a_, b_ in zip(b"ACGT", b"TGCA"):
        comp[a_] = b_
    RC = np.concatenate([comp[Q[sub[i]:sub[i + 1]]][::-1] for i in range(good.size)])
    got = _both(sa, idx, Q, sub, flags=sa.SA_PARAM_REVERSE_COMPLEMENT)
    lo, hi = oracle.search_batch(T, osa, RC, sub, threads=oracle.cpu_threads())
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi)


def test_kmer_order_search_locate(sa):
    ref = datagen.reference(120_000, 93, sd_cover=0.15, tandem_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 20_000, 94, m=(10, 150), frac_sampled=0.9, subs=(0, 1))
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    p = sa.sa_search_params(flags=sa.SA_PARAM_KMER_ORDER)
    res, offs, pos = sa.sa_search_locate(idx, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(), 8,
                                         params=p)
    res, offs, pos = res.cpu().numpy(), offs.cpu().numpy(), pos.cpu().numpy()
    lo, hi = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
    assert np.array_equal(res[:, 0], lo) and np.array_equal(res[:, 1], hi)
    for q in range(0, qo.size - 1, 7):
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64), oracle.locate(osa, lo[q], hi[q], 8))


@pytest.mark.parametrize("order", ["kmer", "input"])
def test_strand_per_query(sa, order):
    """SA_PARAM_STRAND_PER_QUERY: bit 31 of a query's reference id asks for its
    reverse complement; the others in the same batch search the forward
    strand (two references, both search orders, and the plain kernel)."""
    refs = [datagen.reference(n, 95 + n, sd_cover=0.1, tandem_cover=0.05) for n in (60_000, 35_000)]
    idxs = [sa.sa_build(torch.from_numpy(r).cuda()) for r in refs]
    rng = np.random.default_rng(96)
    n_q = 6000
    q_ref = rng.integers(0, 2, n_q).astype(np.uint32)
    rc = rng.random(n_q) < 0.5
    # each reference's queries, interleaved in the batch by q_ref
    per = [datagen.queries(refs[i], int((q_ref == i).sum()), 97 + i, m=(5, 180), frac_sampled=0.8, subs=(0, 1))
           for i in range(2)]
    nxt = [0, 0]
    parts, lens = [], []
    for q in range(n_q):
        i = q_ref[q]
        b_, o_, _ = per[i]
        j = nxt[i]
        nxt[i] += 1
        parts.append(b_[o_[j]:o_[j + 1]])
        lens.append(o_[j + 1] - o_[j])
    qb = np.concatenate(parts)
    qo = np.zeros(n_q + 1, dtype=np.int64)
    np.cumsum(lens, out=qo[1:])
    flagged = q_ref | np.where(rc, sa.STRAND_BIT, 0).astype(np.uint32)
    fl = sa.SA_PARAM_STRAND_PER_QUERY | (sa.SA_PARAM_KMER_ORDER if order == "kmer" else sa.SA_PARAM_INPUT_ORDER)
    got = sa.sa_search_batch(idxs, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(),
                             q_ref=torch.from_numpy(flagged).cuda(), params=sa.sa_search_params(flags=fl)).cpu().numpy()
    comp = np.zeros(256, dtype=np.uint8)
    for a_, b_ in zip(b"ACGT", b"TGCA"):
        comp[a_] = b_
    Ts = [oracle.normalize(r) for r in refs]
    sas = [oracle.sa_naive(T) for T in Ts]
    for q in range(n_q):
        P = qb[qo[q]:qo[q + 1]]
        if rc[q]:
            P = comp[P][::-1]
        lo, hi = oracle.search(Ts[q_ref[q]], sas[q_ref[q]], P)
        assert got[q, :3].tolist() == [lo, hi, hi - lo], q
    if order == "input":
        # a call without the flag (the plain kernel takes no params) reads bit
        # 31 as part of the id: out of range, so those queries are invalid
        plain = sa.sa_search_batch_plain(idxs, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda(),
                                         q_ref=torch.from_numpy(flagged).cuda())
        assert (plain.cpu().numpy()[rc, 3] == sa.SA_RESULT_INVALID).all()
    # locate ignores the strand bit
    offs, pos = sa.sa_locate(idxs, torch.from_numpy(got).cuda(), 4, q_ref=torch.from_numpy(flagged).cuda())
    offs, pos = offs.cpu().numpy(), pos.cpu().numpy()
    for q in range(0, n_q, 13):
        want = oracle.locate(sas[q_ref[q]], int(got[q, 0]), int(got[q, 1]), 4)
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64), want)


def test_kmer_order_overflow_region(sa):
    """The list's bucket regions are sized from every 32nd query.  Here those
    queries all start with A and every other query with T, so the T buckets
    get the minimum room and most of their records go to the overflow region:
    the results stay bit-exact, with locate too."""
    ref = datagen.reference(300_000, 95, gc=0.5, sd_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 120_000, 96, m=(20, 160), frac_sampled=0.9, subs=(0, 1))
    qs = [bytes(qb[qo[i]:qo[i + 1]]) for i in range(qo.size - 1)]
    a_q = [x for x in qs if x[:1] == b"A"]
    t_q = [x for x in qs if x[:1] == b"T"]
    n = 32 * min(len(a_q), len(t_q) // 31)
    order = []
    ai = ti = 0
    for i in range(n):
        if i % 32 == 0:
            order.append(a_q[ai])
            ai += 1
        else:
            order.append(t_q[ti])
            ti += 1
    qb2 = np.frombuffer(b"".join(order), dtype=np.uint8).copy()
    qo2 = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([len(x) for x in order], out=qo2[1:])
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    got = _both(sa, idx, qb2, qo2)
    T = oracle.normalize(ref)
    lo, hi = oracle.search_batch(T, oracle.sa_naive(T), qb2, qo2, threads=oracle.cpu_threads())
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi)
    # the fused search + locate through the overflow region as well
    for flags in (sa.SA_PARAM_KMER_ORDER, sa.SA_PARAM_INPUT_ORDER):
        p = sa.sa_search_params(flags=flags)
        r, o, pos = sa.sa_search_locate(idx, torch.from_numpy(qb2).cuda(), torch.from_numpy(qo2).cuda(), 4, params=p)
        if flags == sa.SA_PARAM_KMER_ORDER:
            want = (r.cpu().numpy(), o.cpu().numpy(), pos.cpu().numpy())
        else:
            assert np.array_equal(r.cpu().numpy(), want[0]) and np.array_equal(o.cpu().numpy(), want[1])
            assert np.array_equal(pos.cpu().numpy()[:int(want[1][-1])], want[2][:int(want[1][-1])])
