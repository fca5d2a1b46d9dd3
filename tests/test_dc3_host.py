"""The library's host-side DC3 construction (Section III) against the paper's
Table I, the oracle's naive suffix sort and the suffix-array invariants.
Host code only: runs without a GPU."""
import ctypes
import itertools

import numpy as np
import pytest

import oracle
from paper_1303_3692_gb300 import datagen


@pytest.fixture(scope="module")
def sa():
    from paper_1303_3692_gb300 import build_lib, sa as sa_mod

    build_lib.build()
    return sa_mod


def _dc3(sa, T, width=32):
    return sa.sa_suffix_array_host(np.ascontiguousarray(T, dtype=np.uint8), width).astype(np.int64)


def test_table1(sa, golden):
    T = np.frombuffer(golden["text"][0][0].encode(), dtype=np.uint8)
    assert _dc3(sa, T).tolist() == [int(x) for x in golden["sa"][0]]


def test_every_text_up_to_length_7(sa):
    """All 21,844 texts over {A,C,G,T} of length 1..7, each length's residue
    mod 3 and every pattern of equal triples included."""
    for L in range(1, 8):
        for t in itertools.product(b"ACGT", repeat=L):
            T = np.array(t, dtype=np.uint8)
            assert np.array_equal(_dc3(sa, T), oracle.sa_naive(T)), bytes(T)


@pytest.mark.parametrize("n", [3000, 3001, 3002])
@pytest.mark.parametrize("kind", ["A", "AC", "ACG", "ACGT", "AAC", "binary", "random", "fibonacci"])
def test_periodic_and_random_texts(sa, n, kind):
    """Periodic texts make every triple of a residue class equal, which drives
    the recursion to its full depth; period 3 aligns with the sample."""
    rng = np.random.default_rng(n)
    if kind == "binary":
        T = np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, n)]
    elif kind == "random":
        T = datagen.ASCII[rng.integers(0, 4, n)]
    elif kind == "fibonacci":
        a, b = b"A", b"AC"
        while len(b) < n:
            a, b = b, b + a
        T = np.frombuffer(b[:n], np.uint8)
    else:
        T = np.frombuffer((kind.encode() * n)[:n], np.uint8)
    assert np.array_equal(_dc3(sa, T), oracle.sa_naive(T))


def test_repetitive_reference_against_naive_sort(sa):
    ref = datagen.reference(200_003, 7, gc=0.45, sd_cover=0.10, tandem_cover=0.05)
    assert np.array_equal(_dc3(sa, ref), oracle.sa_naive(oracle.normalize(ref)))


def test_million_bases_are_a_sorted_permutation(sa):
    """A sorted permutation is unique, so the verifier's pass proves the array."""
    ref = datagen.reference(1_000_001, 11, gc=0.41, family_cover=0.3, sd_cover=0.05, tandem_cover=0.03)
    assert oracle.verify_sa(oracle.normalize(ref), _dc3(sa, ref), threads=oracle.cpu_threads()) == (0, -1)


def test_width_case_and_errors(sa):
    ref = datagen.reference(5000, 3, tandem_cover=0.1)
    s32 = _dc3(sa, ref, 32)
    assert np.array_equal(_dc3(sa, ref, 64), s32)
    assert np.array_equal(_dc3(sa, np.char.lower(ref.view("S1")).view(np.uint8)), s32)
    with pytest.raises(sa.SAError) as e:
        sa.sa_suffix_array_host(np.frombuffer(b"ACGNT", np.uint8))
    assert e.value.status == sa.SA_ERR_BASE
    L = sa.lib()
    buf = ctypes.create_string_buffer(b"ACGT")
    out = (ctypes.c_uint32 * 4)()
    assert L.sa_suffix_array_host(ctypes.cast(buf, ctypes.c_void_p), 4, 3, out) == sa.SA_ERR_ARG
    assert L.sa_suffix_array_host(ctypes.cast(buf, ctypes.c_void_p), 0, 4, out) == sa.SA_ERR_ARG
    assert L.sa_suffix_array_host(None, 4, 4, out) == sa.SA_ERR_ARG
    assert L.sa_suffix_array_host(ctypes.cast(buf, ctypes.c_void_p), 4, 4, None) == sa.SA_ERR_ARG
    assert L.sa_suffix_array_host(ctypes.cast(buf, ctypes.c_void_p), 4, 4, out) == sa.SA_OK
    assert list(out) == [0, 1, 2, 3]
