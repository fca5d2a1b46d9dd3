"""Seeded property tests (hypothesis) on tiny random texts with injected
repeats and tandem runs.  They check the oracle's suffix array against Python's
own byte-string order: it is a permutation, and rank(SA[k]) = k + 1 (Table III's
ranks invert it).  They check the oracle's search against brute-force scanning,
including the insertion point of a miss.  They check the library's host DC3
construction against the oracle.  No GPU."""
import numpy as np
import pytest

pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402

ALPHA = list(b"ACGT")
SETTINGS = settings(max_examples=300, derandomize=True, deadline=None,
                    suppress_health_check=[HealthCheck.too_slow])


@st.composite
def texts(draw):
    n = draw(st.integers(1, 60))
    t = bytearray(draw(st.lists(st.sampled_from(ALPHA), min_size=n, max_size=n)))
    for _ in range(draw(st.integers(0, 3))):  # copied blocks: long shared prefixes
        L = draw(st.integers(1, max(1, len(t) // 2)))
        a = draw(st.integers(0, len(t) - L))
        b = draw(st.integers(0, len(t) - L))
        t[b:b + L] = t[a:a + L]
    if draw(st.booleans()):  # a tandem run
        unit = bytes(draw(st.lists(st.sampled_from(ALPHA), min_size=1, max_size=3)))
        pos = draw(st.integers(0, len(t)))
        t[pos:pos] = unit * draw(st.integers(2, 12))
    return np.frombuffer(bytes(t), dtype=np.uint8).copy()


@st.composite
def text_and_queries(draw):
    T = draw(texts())
    qs = []
    for _ in range(draw(st.integers(1, 8))):
        if draw(st.booleans()):  # a substring, sometimes with one substitution
            a = draw(st.integers(0, T.size - 1))
            q = bytearray(T[a:a + draw(st.integers(0, T.size - a))].tobytes())
            if q and draw(st.booleans()):
                q[draw(st.integers(0, len(q) - 1))] = draw(st.sampled_from(ALPHA))
        else:
            q = bytearray(draw(st.lists(st.sampled_from(ALPHA), max_size=8)))
        qs.append(np.frombuffer(bytes(q), dtype=np.uint8).copy())
    return T, qs


@SETTINGS
@given(texts())
def test_suffix_array_invariants(T):
    sa = oracle.sa_naive(T)
    n = T.size
    assert np.array_equal(np.sort(sa), np.arange(n))
    s = T.tobytes()
    for a, b in zip(sa[:-1], sa[1:]):
        assert s[a:] < s[b:]  # bytes order: A < C < G < T, a proper prefix first
    assert np.array_equal(oracle.ranks(sa)[sa], np.arange(1, n + 1))
    assert oracle.verify_sa(T, sa) == (0, -1)


@SETTINGS
@given(text_and_queries())
def test_search_equals_brute_force(data):
    T, qs = data
    sa = oracle.sa_naive(T)
    s, n = T.tobytes(), T.size
    for P in qs:
        p, m = P.tobytes(), P.size
        lo, hi = oracle.search(T, sa, P)
        if m == 0:
            assert (lo, hi) == (0, n)
            continue
        occ = {i for i in range(n - m + 1) if s[i:i + m] == p}
        assert set(sa[lo:hi].tolist()) == occ and hi - lo == len(occ)
        # Everything before lo sorts below P, everything from hi on above it.
        assert lo == 0 or s[sa[lo - 1]:sa[lo - 1] + m] < p
        assert hi == n or s[sa[hi]:sa[hi] + m] > p


_lib = []


def _sa_module():
    if not _lib:
        from paper_1303_3692_gb300 import build_lib, sa as sa_mod

        build_lib.build()
        _lib.append(sa_mod)
    return _lib[0]


@SETTINGS
@given(texts())
def test_host_dc3_equals_oracle(T):
    got = _sa_module().sa_suffix_array_host(T).astype(np.int64)
    assert np.array_equal(got, oracle.sa_naive(T))
