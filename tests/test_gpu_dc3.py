"""The GPU DC3 construction (Section III) against the oracle's naive suffix
sort: every text of up to 6 bases, periodic and Fibonacci texts around every
length mod 3 (the recursion's deepest cases), seeded repetitive texts, both
widths; an index built by it searches like any other; and it equals prefix
doubling."""
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


def _fib(n):
    a, b = "A", "AC"
    while len(b) < n:
        a, b = b, b + a
    return b[:n]


def _texts():
    out = ["".join(t) for L in range(1, 7) for t in itertools.product("ACGT", repeat=L)]
    for n in list(range(7, 40)) + [95, 96, 97, 1000, 3001]:
        out += ["A" * n, ("AC" * n)[:n], ("ACG" * n)[:n], ("AAC" * n)[:n], _fib(n)]
    return out


@pytest.mark.parametrize("width", [32, 64])
def test_dc3_gpu_small_texts(sa, width):
    for text in _texts():
        T = np.frombuffer(text.encode(), dtype=np.uint8)
        got = sa.sa_suffix_array_gpu(torch.from_numpy(T.copy()).cuda(), width=width, dc3=True).cpu().numpy()
        assert np.array_equal(got.astype(np.int64), oracle.sa_naive(T)), text


@pytest.mark.parametrize("n", [200_003, 300_001, 300_002])
def test_dc3_gpu_repetitive(sa, n):
    ref = datagen.reference(n, 400 + n % 7, gc=0.41, family_cover=0.3, sd_cover=0.1, tandem_cover=0.05)
    T = oracle.normalize(ref)
    want = oracle.sa_naive(T)
    d = torch.from_numpy(ref).cuda()
    got = sa.sa_suffix_array_gpu(d, width=32, dc3=True)
    assert np.array_equal(got.cpu().numpy().astype(np.int64), want)
    assert torch.equal(got, sa.sa_suffix_array_gpu(d, width=32))  # prefix doubling: the same array
    # host input, and the lower-case alphabet, give the same array
    low = np.frombuffer(bytes(ref).lower(), dtype=np.uint8).copy()
    assert torch.equal(sa.sa_suffix_array_gpu(low, width=32, dc3=True), got)


def test_dc3_gpu_index_searches(sa):
    ref = datagen.reference(150_000, 411, sd_cover=0.1, tandem_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 5000, 412, m=(5, 160), frac_sampled=0.8, subs=(0, 1))
    idx = sa.sa_build(torch.from_numpy(ref).cuda(), dc3=True)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    got = sa.sa_search_batch(idx, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda()).cpu().numpy()
    lo, hi = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi)


def test_dc3_gpu_errors(sa):
    with pytest.raises(sa.SAError) as e:
        sa.sa_suffix_array_gpu(np.frombuffer(b"ACGNT", dtype=np.uint8).copy(), dc3=True)
    assert e.value.status == sa.SA_ERR_BASE
    with pytest.raises(sa.SAError) as e:  # host DC3 and GPU DC3 at once
        sa.sa_build(torch.from_numpy(np.frombuffer(b"ACGT", dtype=np.uint8).copy()).cuda(), host_build=True, dc3=True)
    assert e.value.status == sa.SA_ERR_ARG
