"""Plants plausible mistakes in a copy of the oracle's C source (on the CPU) and
checks that the paper pins or the brute-force sweep reject every one of them.
This shows the pins are strong enough to catch a dropped term, a flipped sign
or a wrong index in the oracle itself."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT, load_golden

SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    # proper prefix sorts after the longer suffix (Table I / reading R3)
    "prefix_last": ("return li < lj ? -1 : 1;", "return li < lj ? 1 : -1;"),
    # lower-bound test made strict (reading R1)
    "lb_strict": ("if (query_cmp(T, n, sa[mid], P, m, NULL) > 0)",
                  "if (query_cmp(T, n, sa[mid], P, m, NULL) >= 0)"),
    # upper-bound test loses its equality case, so hi stops at lo (reading R1)
    "ub_strict": ("if (query_cmp(T, n, sa[mid], P, m, NULL) >= 0)",
                  "if (query_cmp(T, n, sa[mid], P, m, NULL) > 0)"),
    # a suffix that ends early compares larger than the query
    "short_suffix_big": ("            return 1;\n        }\n        if (T[p + k] != P[k]) {",
                         "            return -1;\n        }\n        if (T[p + k] != P[k]) {"),
    # mismatch direction flipped
    "mismatch_sign": ("return P[k] < T[p + k] ? -1 : 1;", "return P[k] < T[p + k] ? 1 : -1;"),
    # the search range leaves out rank 0 (reading R2)
    "left_zero": ("int64_t a = 0, b = n; /* the lower bound lies in [a, b] */",
                  "int64_t a = 1, b = n; /* the lower bound lies in [a, b] */"),
    # comparator skips the first base
    "skip_first_base": ("for (int64_t t = 0; t < k; t++) {", "for (int64_t t = 1; t < k; t++) {"),
}


def _compile(src_text: str, out_dir: str, name: str):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", c, "-o", so])
    lib = ctypes.CDLL(so)
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.oracle_sa_naive.argtypes = [p, i64, p]
    lib.oracle_search.argtypes = [p, i64, p, p, i64, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    return lib


def _sa(lib, text: str):
    T = np.frombuffer(text.encode(), dtype=np.uint8)
    sa = np.empty(len(text), dtype=np.int64)
    lib.oracle_sa_naive(T.ctypes.data_as(ctypes.c_void_p), T.size, sa.ctypes.data_as(ctypes.c_void_p))
    return T, sa


def _search(lib, T, sa, q: str):
    P = np.frombuffer(q.encode(), dtype=np.uint8)
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    lib.oracle_search(T.ctypes.data_as(ctypes.c_void_p), T.size, sa.ctypes.data_as(ctypes.c_void_p),
                      P.ctypes.data_as(ctypes.c_void_p), P.size, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def _pins_hold(lib) -> bool:
    g = load_golden()
    text = g["text"][0][0].upper()
    T, sa = _sa(lib, text)
    if sa.tolist() != [int(x) for x in g["sa"][0]]:
        return False
    for q, lb, rb in g["search"]:
        if _search(lib, T, sa, q.upper()) != (int(lb), int(rb) + 1):
            return False
    for L in range(1, 5):
        for tup in itertools.product("ACGT", repeat=L):
            t = "".join(tup)
            T, sa = _sa(lib, t)
            if [t[i:] for i in sa.tolist()] != sorted(t[i:] for i in range(L)):
                return False
            for q in ["A", "C", "GT", "AAA", t, t + "A"]:
                cnt = sum(1 for i in range(L - len(q) + 1) if t[i:i + len(q)] == q)
                lo, hi = _search(lib, T, sa, q)
                if hi - lo != cnt or set(sa[lo:hi].tolist()) != {i for i in range(L - len(q) + 1)
                                                                  if t[i:i + len(q)] == q}:
                    return False
    return True


def test_unmutated_oracle_passes(tmp_path):
    with open(SRC) as f:
        assert _pins_hold(_compile(f.read(), str(tmp_path), "orig"))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    with open(SRC) as f:
        src = f.read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    assert not _pins_hold(_compile(mutated, str(tmp_path), name))
