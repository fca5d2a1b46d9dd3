"""CPU oracle for exact DNA matching over a suffix array -- test infrastructure.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It loads ``liboracle.so`` compiled from the plain C
in ``oracle.c`` (built by :func:`build`) and exposes numpy-facing wrappers.  It
shares no code with the CUDA library and never imports it.

Texts and queries are numpy ``uint8`` arrays of ASCII bases; call
:func:`normalize` first (case fold + alphabet check, Section III).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p
_pi64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_normalize.argtypes = [_p, _i64, _p, _pi64]
        lib.oracle_normalize.restype = ctypes.c_int
        lib.oracle_sa_naive.argtypes = [_p, _i64, _p]
        lib.oracle_sa_naive.restype = None
        lib.oracle_ranks.argtypes = [_p, _i64, _p]
        lib.oracle_ranks.restype = None
        lib.oracle_verify_sa.argtypes = [_p, _i64, _p, ctypes.c_int, _pi64]
        lib.oracle_verify_sa.restype = ctypes.c_int
        lib.oracle_search.argtypes = [_p, _i64, _p, _p, _i64, _pi64, _pi64]
        lib.oracle_search.restype = None
        lib.oracle_rank_count.argtypes = [_p, _i64, _p, _i64, _pi64, _pi64]
        lib.oracle_rank_count.restype = None
        lib.oracle_bruteforce.argtypes = [_p, _i64, _p, _i64, _p, _i64]
        lib.oracle_bruteforce.restype = _i64
        lib.oracle_sort_positions.argtypes = [_p, _i64, _p, _i64]
        lib.oracle_sort_positions.restype = None
        lib.oracle_search_batch.argtypes = [_p, _i64, _p, _p, _p, _i64, _p, _p, ctypes.c_int]
        lib.oracle_search_batch.restype = None
        lib.oracle_rank_count_batch.argtypes = [_p, _i64, _p, _p, _i64, _p, _p, ctypes.c_int]
        lib.oracle_rank_count_batch.restype = None
        lib.oracle_locate.argtypes = [_p, _i64, _i64, _i64, _p]
        lib.oracle_locate.restype = None
        lib.oracle_probe_model.argtypes = [_p, _i64, _p, _p, _i64, ctypes.c_int,
                                           _pi64, _pi64, _pi64, _pi64]
        lib.oracle_probe_model.restype = None
        lib.oracle_kmer_table.argtypes = [_p, _i64, _p, ctypes.c_int, _p]
        lib.oracle_kmer_table.restype = None
        lib.oracle_probe_model_kmer.argtypes = [_p, _i64, _p, _p, ctypes.c_int, ctypes.c_int, _p, _i64,
                                                _pi64, _pi64, _pi64, _pi64, _pi64]
        lib.oracle_probe_model_kmer.restype = None
        lib.oracle_kmer_rank.argtypes = [_p, _i64, _p, ctypes.c_int, _i64]
        lib.oracle_kmer_rank.restype = _i64
        lib.oracle_probe_model_bracket.argtypes = [_p, _i64, _p, ctypes.c_int, _i64, _i64, ctypes.c_int, _p, _i64,
                                                   _pi64, _pi64, _pi64, _pi64, _pi64]
        lib.oracle_probe_model_bracket.restype = None
        _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, str)):
        a = np.frombuffer(a.encode() if isinstance(a, str) else bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _i64sa(sa) -> np.ndarray:
    """A suffix array as int64 without a copy where it already is 64-bit."""
    if isinstance(sa, np.ndarray) and sa.dtype == np.uint64 and sa.flags.c_contiguous:
        return sa.view(np.int64)
    return np.ascontiguousarray(sa, dtype=np.int64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def cpu_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def normalize(text) -> np.ndarray:
    """Upper-case ACGT bytes; ValueError on a byte outside Sigma (Section III)."""
    t = _u8(text)
    out = np.empty_like(t)
    bad = _i64(-1)
    if _load().oracle_normalize(_ptr(t), t.size, _ptr(out), ctypes.byref(bad)) != 0:
        raise ValueError(f"non-ACGT byte at index {bad.value}")
    return out


def sa_naive(T) -> np.ndarray:
    """Suffix array by comparison-sorting all suffixes (Section III, Table I)."""
    T = _u8(T)
    sa = np.empty(T.size, dtype=np.int64)
    _load().oracle_sa_naive(_ptr(T), T.size, _ptr(sa))
    return sa


def ranks(sa) -> np.ndarray:
    """1-based inverse suffix array (Table III)."""
    sa = _i64sa(sa)
    r = np.empty_like(sa)
    _load().oracle_ranks(_ptr(sa), sa.size, _ptr(r))
    return r


def verify_sa(T, sa, threads: int = 1):
    """(code, index): code 0 iff sa is the suffix array of T (permutation whose
    adjacent suffixes strictly increase); 1 out of range, 2 repeat, 3 order."""
    T = _u8(T)
    sa = _i64sa(sa)
    if sa.size != T.size:
        return (1, -1)
    w = _i64(-1)
    rc = _load().oracle_verify_sa(_ptr(T), T.size, _ptr(sa), int(threads), ctypes.byref(w))
    return (rc, w.value)


def search(T, sa, P):
    """Alg. 1 on the CPU for one query; returns half-open (lo, hi)."""
    T, P = _u8(T), _u8(P)
    sa = _i64sa(sa)
    lo, hi = _i64(), _i64()
    _load().oracle_search(_ptr(T), T.size, _ptr(sa), _ptr(P), P.size,
                          ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def rank_count(T, P):
    """(lo, hi) by definition: counts of suffixes whose m-prefix is < P, <= P."""
    T, P = _u8(T), _u8(P)
    lo, hi = _i64(), _i64()
    _load().oracle_rank_count(_ptr(T), T.size, _ptr(P), P.size, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def search_batch(T, sa, Q, qoff, threads: int = 1):
    """Alg. 1 over a batch; Q concatenated bases, qoff (nq+1) offsets."""
    T, Q = _u8(T), _u8(Q)
    sa = _i64sa(sa)
    qoff = np.ascontiguousarray(qoff, dtype=np.int64)
    nq = qoff.size - 1
    lo = np.empty(nq, dtype=np.int64)
    hi = np.empty(nq, dtype=np.int64)
    _load().oracle_search_batch(_ptr(T), T.size, _ptr(sa), _ptr(Q), _ptr(qoff), nq,
                                _ptr(lo), _ptr(hi), int(threads))
    return lo, hi


def rank_count_batch(T, Q, qoff, threads: int = 1):
    """Definition-based (lo, hi) for a batch, without a suffix array."""
    T, Q = _u8(T), _u8(Q)
    qoff = np.ascontiguousarray(qoff, dtype=np.int64)
    nq = qoff.size - 1
    lo = np.empty(nq, dtype=np.int64)
    hi = np.empty(nq, dtype=np.int64)
    _load().oracle_rank_count_batch(_ptr(T), T.size, _ptr(Q), _ptr(qoff), nq,
                                    _ptr(lo), _ptr(hi), int(threads))
    return lo, hi


def bruteforce(T, P, cap: int = 1 << 30):
    """(count, positions[:min(count,cap)]) of every overlapping occurrence."""
    T, P = _u8(T), _u8(P)
    buf = np.empty(max(0, min(cap, T.size + 1)), dtype=np.int64)
    cnt = _load().oracle_bruteforce(_ptr(T), T.size, _ptr(P), P.size, _ptr(buf), buf.size)
    return int(cnt), buf[:min(cnt, buf.size)].copy()


def sort_positions(T, pos) -> np.ndarray:
    """Positions re-ordered by their suffixes (suffix-array order)."""
    T = _u8(T)
    pos = np.array(pos, dtype=np.int64)
    _load().oracle_sort_positions(_ptr(T), T.size, _ptr(pos), pos.size)
    return pos


def locate(sa, lo: int, hi: int, cap: int) -> np.ndarray:
    sa = _i64sa(sa)
    k = max(0, min(hi - lo, cap))
    out = np.empty(k, dtype=np.int64)
    _load().oracle_locate(_ptr(sa), lo, hi, cap, _ptr(out))
    return out


def probe_model(T, sa, P, d0: int = 13):
    """(probes, chunks, lo, hi) of the lockstep search byte model for one query."""
    T, P = _u8(T), _u8(P)
    sa = _i64sa(sa)
    pr, ch, lo, hi = _i64(), _i64(), _i64(), _i64()
    _load().oracle_probe_model(_ptr(T), T.size, _ptr(sa), _ptr(P), P.size, int(d0),
                               ctypes.byref(pr), ctypes.byref(ch), ctypes.byref(lo), ctypes.byref(hi))
    return pr.value, ch.value, lo.value, hi.value


def kmer_table(T, sa, k: int) -> np.ndarray:
    """table[x] = number of suffixes sorting before the k-base string x; table[4^k] = n."""
    T = _u8(T)
    sa = _i64sa(sa)
    out = np.empty((1 << (2 * k)) + 1, dtype=np.int64)
    _load().oracle_kmer_table(_ptr(T), T.size, _ptr(sa), int(k), _ptr(out))
    return out


def probe_model_kmer(T, sa, table, k: int, P, d0: int = 13):
    """(probes, text windows, table reads, lo, hi) of the k-mer + record search model."""
    T, P = _u8(T), _u8(P)
    sa = _i64sa(sa)
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.int64)
    pr, wi, tr, lo, hi = _i64(), _i64(), _i64(), _i64(), _i64()
    _load().oracle_probe_model_kmer(_ptr(T), T.size, _ptr(sa), None if tab is None else _ptr(tab), int(k), int(d0),
                                    _ptr(P), P.size, ctypes.byref(pr), ctypes.byref(wi), ctypes.byref(tr),
                                    ctypes.byref(lo), ctypes.byref(hi))
    return pr.value, wi.value, tr.value, lo.value, hi.value


def kmer_rank(T, sa, k: int, x: int) -> int:
    """Number of suffixes sorting before the k-base string x (one table entry)."""
    T = _u8(T)
    sa = _i64sa(sa)
    return int(_load().oracle_kmer_rank(_ptr(T), T.size, _ptr(sa), int(k), int(x)))


def kmer_code(P, k: int) -> int:
    """The first k bases of P as a base-4 number (A=0 C=1 G=2 T=3)."""
    x = 0
    for c in bytes(_u8(P)[:k]):
        x = 4 * x + b"ACGT".index(c)
    return x


def probe_model_bracket(T, sa, bracket, P, d0: int = 13):
    """The k-mer + record search model for one query given its bracket
    (tlo, thi) = (table[x], table[x + 1]), or None for a query without one:
    (probes, text windows, table reads, lo, hi)."""
    T, P = _u8(T), _u8(P)
    sa = _i64sa(sa)
    has = bracket is not None
    tlo, thi = bracket if has else (0, 0)
    pr, wi, tr, lo, hi = _i64(), _i64(), _i64(), _i64(), _i64()
    _load().oracle_probe_model_bracket(_ptr(T), T.size, _ptr(sa), int(has), int(tlo), int(thi), int(d0), _ptr(P),
                                       P.size, ctypes.byref(pr), ctypes.byref(wi), ctypes.byref(tr),
                                       ctypes.byref(lo), ctypes.byref(hi))
    return pr.value, wi.value, tr.value, lo.value, hi.value
