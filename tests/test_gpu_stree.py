"""The flattened suffix tree (the paper's comparison index) gives the same
intervals as the suffix-array search: against the oracle on every text of up
to 5 bases and periodic texts, and against both the oracle and the
suffix-array search on repetitive texts with misses, empty and invalid
queries."""
import itertools

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


def _batch(qs):
    qb = np.frombuffer("".join(qs).encode() or b"A", dtype=np.uint8)[: sum(map(len, qs))].copy()
    qo = np.zeros(len(qs) + 1, dtype=np.int64)
    np.cumsum([len(q) for q in qs], out=qo[1:])
    return qb, qo


def _tree_search(sa, tree, qb, qo):
    d = torch.from_numpy(qb).cuda() if qb.size else torch.zeros(1, dtype=torch.uint8, device="cuda")
    return tree.search(d, torch.from_numpy(qo).cuda()).cpu().numpy()


def test_stree_tiny_texts(sa):
    qs = [""] + ["".join(p) for L in range(1, 5) for p in itertools.product("ACGT", repeat=L)] + ["ACGTACGT"]
    qb, qo = _batch(qs)
    texts = ["".join(t) for L in range(1, 6) for t in itertools.product("ACGT", repeat=L)]
    texts += ["A" * 40, "AC" * 20, "ACG" * 13 + "A", "AAC" * 11]
    for text in texts:
        T = np.frombuffer(text.encode(), dtype=np.uint8)
        idx = sa.sa_build(torch.from_numpy(T.copy()).cuda())
        tree = sa.SuffixTree(idx)
        got = _tree_search(sa, tree, qb, qo)
        lo, hi = oracle.search_batch(T, oracle.sa_naive(T), qb, qo)
        assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi), text


@pytest.mark.parametrize("width", [32, 64])
def test_stree_repetitive(sa, width):
    ref = datagen.reference(200_000, 501, gc=0.41, family_cover=0.3, sd_cover=0.1, tandem_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 20_000, 502, m=(0, 200), frac_sampled=0.8, subs=(0, 1))
    qb = qb.copy()
    bad = [5, 77]
    for q in bad:
        if qo[q + 1] > qo[q]:
            qb[qo[q]] = ord("N")
    idx = sa.sa_build(torch.from_numpy(ref).cuda(), width=width)
    tree = sa.SuffixTree(idx)
    assert 0 < tree.nodes < ref.size
    got = _tree_search(sa, tree, qb, qo)
    want = sa.sa_search_batch(idx, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda()).cpu().numpy()
    assert np.array_equal(got, want)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    for q in range(0, qo.size - 1, 41):
        P = qb[qo[q]:qo[q + 1]]
        if q in bad and P.size:
            assert got[q, 3] == sa.SA_RESULT_INVALID
            continue
        assert tuple(got[q, :2]) == oracle.search(T, osa, P), q
