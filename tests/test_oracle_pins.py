"""Pins the CPU oracle to the paper's worked example (Tables I-III, Section IV)
and to brute force, closed forms and invariants.  No GPU."""
import bisect
import itertools

import numpy as np
import pytest

import oracle
from paper_1303_3692_gb300 import datagen


def _t(golden):
    return oracle.normalize(golden["text"][0][0])


def test_table1_suffix_array(golden):
    sa = oracle.sa_naive(_t(golden))
    assert sa.tolist() == [int(x) for x in golden["sa"][0]]


def test_table3_ranks(golden):
    sa = oracle.sa_naive(_t(golden))
    assert oracle.ranks(sa).tolist() == [int(x) for x in golden["rank"][0]]


def test_table2_sample_ranks(golden):
    # Ranks of the suffixes i mod 3 != 0 among themselves follow from the full order.
    sa = oracle.sa_naive(_t(golden))
    samples = [i for i in sa.tolist() if i % 3 != 0]
    got = ["_"] * len(sa)
    for r, i in enumerate(samples, start=1):
        got[i] = str(r)
    assert got == golden["sample_rank"][0]


def test_b0_order(golden):
    sa = oracle.sa_naive(_t(golden))
    assert [i for i in sa.tolist() if i % 3 == 0] == [int(x) for x in golden["b0_order"][0]]


def test_suffix_labels(golden):
    text = golden["text"][0][0]
    for i1, s in golden["suffix1"]:
        assert text[int(i1) - 1:] == s
    sa = oracle.sa_naive(_t(golden))
    for k, s in golden["sa_suffix"]:
        assert text[sa[int(k)]:] == s


def test_section4_search_examples(golden):
    T = _t(golden)
    sa = oracle.sa_naive(T)
    for q, lb, rb in golden["search"]:
        P = oracle.normalize(q)
        lo, hi = oracle.search(T, sa, P)
        assert (lo, hi) == (int(lb), int(rb) + 1), q
        assert oracle.rank_count(T, P) == (lo, hi)
        cnt, _ = oracle.bruteforce(T, P)
        assert cnt == hi - lo


def test_section4_positions(golden):
    T = _t(golden)
    sa = oracle.sa_naive(T)
    for q, *pos in golden["positions"]:
        lo, hi = oracle.search(T, sa, oracle.normalize(q))
        assert oracle.locate(sa, lo, hi, 64).tolist() == [int(p) for p in pos]
        cnt, bf = oracle.bruteforce(T, oracle.normalize(q))
        assert sorted(bf.tolist()) == sorted(int(p) for p in pos)
        assert oracle.sort_positions(T, bf).tolist() == [int(p) for p in pos]


def test_case_folding(golden):
    text = golden["text"][0][0]
    a = oracle.sa_naive(oracle.normalize(text.upper()))
    b = oracle.sa_naive(oracle.normalize(text.lower()))
    assert a.tolist() == b.tolist()


def test_normalize_rejects_non_acgt():
    with pytest.raises(ValueError, match="index 3"):
        oracle.normalize("ACGNT")


def test_empty_query_matches_everything(golden):
    T = _t(golden)
    sa = oracle.sa_naive(T)
    assert oracle.search(T, sa, b"") == (0, T.size)
    assert oracle.rank_count(T, b"") == (0, T.size)


def _bisect_reference(text: str, queries):
    """lo/hi by Python's own string order (library routine) on truncated sorted suffixes."""
    sufs = sorted(text[i:] for i in range(len(text)))
    cache = {}
    out = []
    for q in queries:
        m = len(q)
        if m not in cache:
            cache[m] = [s[:m] for s in sufs]
        keys = cache[m]
        out.append((bisect.bisect_left(keys, q), bisect.bisect_right(keys, q)))
    return sufs, out


def _substring_positions(text: str, maxlen: int):
    occ = {}
    for i in range(len(text)):
        for L in range(1, maxlen + 1):
            if i + L <= len(text):
                occ.setdefault(text[i:i + L], []).append(i)
    return occ


ALL_Q = [""] + ["".join(p) for L in range(1, 5) for p in itertools.product("ACGT", repeat=L)]


@pytest.mark.parametrize("length", [1, 2, 3, 4, 5, 6, 7])
def test_exhaustive_tiny(length):
    """Every text over {A,C,G,T} of the given length x every query of length <= 4
    plus queries longer than the text: SA against Python's sorted(), intervals
    against bisect, occurrence sets against substring enumeration."""
    extra = ["A" * (length + 1), "T" * (length + 2)]
    qs = ALL_Q + extra
    Q = np.frombuffer("".join(qs).encode(), dtype=np.uint8)
    qoff = np.zeros(len(qs) + 1, dtype=np.int64)
    np.cumsum([len(q) for q in qs], out=qoff[1:])
    for tup in itertools.product("ACGT", repeat=length):
        text = "".join(tup)
        T = np.frombuffer(text.encode(), dtype=np.uint8)
        sufs, ref = _bisect_reference(text, qs)
        sa = oracle.sa_naive(T)
        assert [text[i:] for i in sa.tolist()] == sufs
        assert oracle.verify_sa(T, sa)[0] == 0
        lo, hi = oracle.search_batch(T, sa, Q, qoff)
        assert list(zip(lo.tolist(), hi.tolist())) == ref, text
        occ = _substring_positions(text, 4)
        sal = sa.tolist()
        for qi, q in enumerate(qs):
            if 0 < len(q) <= 4:
                exp = occ.get(q, [])
                assert hi[qi] - lo[qi] == len(exp)
                if exp:
                    assert set(sal[lo[qi]:hi[qi]]) == set(exp)
    # definition-based counting agrees on the last text of the sweep
    lo2, hi2 = oracle.rank_count_batch(T, Q, qoff)
    assert lo2.tolist() == lo.tolist() and hi2.tolist() == hi.tolist()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_repetitive_against_bruteforce(seed):
    ref = datagen.reference(3000, seed, gc=0.45, sd_cover=0.0, tandem_cover=0.2)
    # add an exact duplicate block and an all-A run: deep ties and long LCPs
    ref[2000:2400] = ref[100:500]
    ref[2500:2600] = ord("A")
    T = oracle.normalize(ref)
    sa = oracle.sa_naive(T)
    assert oracle.verify_sa(T, sa, threads=4)[0] == 0
    qb, qo, smp = datagen.queries(ref, 400, seed + 7, m=(1, 60), frac_sampled=0.7, subs=(0, 1))
    lo, hi = oracle.search_batch(T, sa, qb, qo, threads=4)
    lo2, hi2 = oracle.rank_count_batch(T, qb, qo, threads=4)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    for q in range(qo.size - 1):
        P = qb[qo[q]:qo[q + 1]]
        cnt, pos = oracle.bruteforce(T, P)
        assert cnt == hi[q] - lo[q]
        assert set(pos.tolist()) == set(sa[lo[q]:hi[q]].tolist())
        assert oracle.sort_positions(T, pos).tolist() == sa[lo[q]:hi[q]].tolist()
    assert (hi - lo)[smp & (np.diff(qo) > 0)].min() >= 0


def test_verify_sa_detects_errors():
    T = oracle.normalize(datagen.reference(500, 9, tandem_cover=0.3))
    sa = oracle.sa_naive(T)
    assert oracle.verify_sa(T, sa) == (0, -1)
    bad = sa.copy()
    bad[[10, 11]] = bad[[11, 10]]
    assert oracle.verify_sa(T, bad) == (3, 10)
    bad = sa.copy()
    bad[5] = bad[6]
    assert oracle.verify_sa(T, bad)[0] == 2
    bad = sa.copy()
    bad[7] = T.size
    assert oracle.verify_sa(T, bad) == (1, 7)


def test_all_same_base_and_period_two():
    for text in ["A" * 40, "AC" * 20, "ACG" * 13 + "A"]:
        T = oracle.normalize(text)
        sa = oracle.sa_naive(T)
        assert [text[i:] for i in sa.tolist()] == sorted(text[i:] for i in range(len(text)))
        _, ref = _bisect_reference(text, ["A", "AA", "AC", "CA", text, text + "A"])
        got = [oracle.search(T, sa, oracle.normalize(q)) for q in
               ["A", "AA", "AC", "CA", text, text + "A"]]
        assert got == ref


def test_probe_model_closed_forms():
    """A query that never splits makes floor or ceil of log2(n+1) probes at d0 = 0
    (a binary search over n+1 gaps); the model's lo/hi equal the search."""
    T = oracle.normalize(datagen.reference(5000, 4))
    sa = oracle.sa_naive(T)
    n = T.size
    rng = np.random.default_rng(0)
    for _ in range(50):
        P = datagen.ASCII[rng.integers(0, 4, 40)]
        pr, ch, lo, hi = oracle.probe_model(T, sa, P, d0=0)
        assert (lo, hi) == oracle.search(T, sa, P)
        if lo == hi:
            assert int(np.floor(np.log2(n + 1))) <= pr <= int(np.ceil(np.log2(n + 1)))
        assert ch >= pr
        pr13, ch13, _, _ = oracle.probe_model(T, sa, P, d0=13)
        assert pr13 == max(0, pr - 13) or lo != hi
    # a split query: counts for both bounds after the split
    P = T[1000:1012]
    pr, ch, lo, hi = oracle.probe_model(T, sa, P, d0=0)
    assert (lo, hi) == oracle.search(T, sa, P) and hi > lo


def _brute_kmer_table(text: str, k: int):
    sufs = [text[i:] for i in range(len(text))]
    out = []
    for x in range(4 ** k):
        s = "".join("ACGT"[(x >> (2 * (k - 1 - t))) & 3] for t in range(k))
        out.append(sum(1 for u in sufs if u < s))  # Python's order: a proper prefix sorts first
    return out + [len(text)]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_kmer_table_against_brute_force(k):
    """table[x] = #suffixes sorting before the k-string x, including short
    suffixes that fall between two k-strings (e.g. AG between ACT and AGA)."""
    rng = np.random.default_rng(k)
    texts = ["ACGTAG", "AG", "A", "TTTT", "ACTAGAAG"] + ["".join(rng.choice(list("ACGT"), L)) for L in (5, 9, 17, 40)]
    for text in texts:
        T = oracle.normalize(text)
        sa = oracle.sa_naive(T)
        assert oracle.kmer_table(T, sa, k).tolist() == _brute_kmer_table(text, k), text


def test_kmer_model_matches_search():
    ref = datagen.reference(6000, 14, tandem_cover=0.1, sd_cover=0.0)
    T = oracle.normalize(ref)
    sa = oracle.sa_naive(T)
    for k in (3, 5):
        tab = oracle.kmer_table(T, sa, k)
        qb, qo, _ = datagen.queries(ref, 300, 15, m=(1, 120), frac_sampled=0.6, subs=(0, 1))
        for q in range(300):
            P = qb[qo[q]:qo[q + 1]]
            pr, wi, tr, lo, hi = oracle.probe_model_kmer(T, sa, tab, k, P, d0=0)
            assert (lo, hi) == oracle.search(T, sa, P)
            if P.size >= k:
                x = int("".join("0123"["ACGT".index(chr(c))] for c in P[:k]), 4)
                s = tab[x + 1] - tab[x]
                assert tr == 1 and pr <= 2 * int(np.ceil(np.log2(s + 2)))
                assert tab[x] - 1 <= lo <= hi <= tab[x + 1]


def test_kmer_rank_and_bracket_model():
    """One k-mer rank by binary search equals the brute-force count of the
    suffixes below that k-string; the bracket form of the byte model, fed
    those two ranks, is the table form (the form used where a 4^k table is
    too large to build)."""
    ref = datagen.reference(4000, 16, tandem_cover=0.1, family_cover=0.3)
    text = bytes(ref).decode()
    T = oracle.normalize(ref)
    sa = oracle.sa_naive(T)
    k = 4
    tab = oracle.kmer_table(T, sa, k)
    brute = _brute_kmer_table(text, k)
    rng = np.random.default_rng(3)
    for x in list(rng.integers(0, 4 ** k, 40)) + [0, 4 ** k - 1]:
        assert oracle.kmer_rank(T, sa, k, int(x)) == brute[int(x)]
    qb, qo, _ = datagen.queries(ref, 200, 17, m=(1, 130), frac_sampled=0.7, subs=(0, 1))
    for q in range(200):
        P = qb[qo[q]:qo[q + 1]]
        want = oracle.probe_model_kmer(T, sa, tab, k, P, d0=5)
        if P.size >= k:
            x = oracle.kmer_code(P, k)
            hi = oracle.kmer_rank(T, sa, k, x + 1) if x + 1 < 4 ** k else T.size
            got = oracle.probe_model_bracket(T, sa, (oracle.kmer_rank(T, sa, k, x), hi), P, d0=5)
        else:
            got = oracle.probe_model_bracket(T, sa, None, P, d0=5)
        assert got == want
        assert got[3:] == oracle.search(T, sa, P)
