"""Thin ctypes binding of libsa.so (C ABI in include/sa.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Buffers may be torch tensors (CUDA or CPU) or numpy arrays;
streams are torch.cuda.Stream objects or raw cudaStream_t integers.  The
binding raises :class:`SAError` with the library's status code on failure and
refuses to run if the compiled library is missing (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported stack
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsa.so")

SA_OK = 0
SA_ERR_ARG = -1
SA_ERR_BASE = -2
SA_ERR_NOMEM = -3
SA_ERR_CUDA = -4
SA_ERR_TIMEOUT = -5
SA_ERR_CAPACITY = -6
SA_ERR_IO = -7
SA_ERR_FORMAT = -8
SA_W32 = 0x1
SA_W64 = 0x2
SA_NO_KMER = 0x4
SA_BUILD_HOST = 0x8
SA_BUILD_DC3 = 0x10
SA_PARAM_Q_RANGE = 0x1
SA_PARAM_REVERSE_COMPLEMENT = 0x2
SA_PARAM_EXPIRE_WAITS = 0x4
SA_PARAM_KMER_ORDER = 0x8
SA_PARAM_INPUT_ORDER = 0x10
SA_PARAM_STRAND_PER_QUERY = 0x20
STRAND_BIT = 0x80000000  # q_ref bit 31 under SA_PARAM_STRAND_PER_QUERY
SA_LOCATE_NOALLOC_MAX_QUERIES = 1 << 26
SA_RESULT_INVALID = 0x1
SA_RESULT_TRUNCATED = 0x2
# int64 fields of one result: lo, hi, count, flags (32 bytes)
RESULT_FIELDS = 4

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p


class SAError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {sa_strerror(status)} ({status})" if what else sa_strerror(status))


class sa_result(ctypes.Structure):
    _fields_ = [("lo", _u64), ("hi", _u64), ("count", _u64), ("flags", _u64)]


class sa_search_params(ctypes.Structure):
    _fields_ = [("threads_per_block", _u32), ("blocks_per_sm", _u32), ("key_depth", _u32), ("chunk", _u32),
                ("search_events", _vp * 2), ("flags", _u32), ("front_probes", _u32), ("q_first", _u64),
                ("q_total", _u64), ("device_status", _vp), ("reserved", _u32 * 2)]


# Every symbol include/sa.h declares, with its ctypes signature.
SIGNATURES = {
    "sa_build": (ctypes.c_int, [_vp, _u64, _u32, _vp, ctypes.POINTER(_vp)]),
    "sa_search_batch": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _vp, _u64, _vp, _vp]),
    "sa_search_batch_ex": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _vp, _u64, _vp, _vp,
                                          ctypes.POINTER(sa_search_params)]),
    "sa_search_batch_plain": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _vp, _u64, _vp, _vp]),
    "sa_locate": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _u64, _u32, _vp, _vp, _u64, _vp]),
    "sa_search_locate": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _vp, _u64, _vp, _u32, _vp, _vp, _u64,
                                        _vp, ctypes.POINTER(sa_search_params)]),
    "sa_locate_noalloc": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _vp, _vp, _u64, _u32, _vp, _vp, _u64, _vp]),
    "sa_save": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp]),
    "sa_load": (ctypes.c_int, [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)]),
    "sa_index_info": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                     ctypes.POINTER(_u32), ctypes.POINTER(_u64)]),
    "sa_copy_kmer_table": (ctypes.c_int, [_vp, _vp, _vp]),
    "sa_copy_suffix_array": (ctypes.c_int, [_vp, _vp, _vp]),
    "sa_free": (None, [_vp]),
    "sa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sa_version": (_u32, []),
    "sa_random_read_rate": (ctypes.c_int, [_u64, _u32, _u32, ctypes.POINTER(ctypes.c_double), _vp]),
    "sa_random_read_rate_ex": (ctypes.c_int, [_u64, _u32, _u32, _u32, ctypes.POINTER(ctypes.c_double), _vp]),
    "sa_suffix_array_host": (ctypes.c_int, [_vp, _u64, _u32, _vp]),
    "sa_suffix_array_gpu": (ctypes.c_int, [_vp, _u64, _u32, _u32, _vp, _vp]),
    "sa_stree_build": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "sa_stree_search": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp, _vp]),
    "sa_stree_info": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "sa_stree_free": (None, [_vp]),
    "sa_search_order": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _u64, ctypes.POINTER(sa_search_params),
                                       ctypes.POINTER(ctypes.c_int)]),
    "sa_scratch_info": (ctypes.c_int, [ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                       ctypes.c_int]),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsa.so is not built ({LIB_PATH}); run "
                               "paper_1303_3692_gb300.build_lib.build() -- there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def sa_strerror(status: int) -> str:
    return lib().sa_strerror(int(status)).decode()


def _check(status: int, what: str):
    if status != SA_OK:
        raise SAError(status, what)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if torch is not None and isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, (bytes, bytearray)):
        raise TypeError("pass bases as a numpy uint8 array or a tensor")
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _stream(s) -> Optional[int]:
    if s is None:
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
        return None
    if torch is not None and isinstance(s, torch.cuda.Stream):
        return s.cuda_stream
    return int(s)


class Index:
    """A reference indexed on the current device: packed text, suffix array and key table."""

    def __init__(self, handle: int):
        self._h = _vp(handle)
        n, w, d, k, b = _u64(), _u32(), _u32(), _u32(), _u64()
        _check(lib().sa_index_info(self._h, ctypes.byref(n), ctypes.byref(w), ctypes.byref(d), ctypes.byref(k),
                                   ctypes.byref(b)), "sa_index_info")
        self.n, self.width, self.key_depth, self.kmer_k, self.device_bytes = n.value, w.value, d.value, k.value, b.value

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("index was freed")
        return self._h

    def free(self):
        if self._h is not None and self._h.value and _lib is not None:
            _lib.sa_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def suffix_array(self, device="cuda"):
        """The suffix array as an int32/int64 tensor (a copy)."""
        dt = torch.int32 if self.width == 4 else torch.int64
        out = torch.empty(self.n, dtype=dt, device=device)
        _check(lib().sa_copy_suffix_array(self.handle, _ptr(out), _stream(None)), "sa_copy_suffix_array")
        if out.is_cuda:
            torch.cuda.current_stream().synchronize()
        return out

    def kmer_table(self, device="cuda"):
        """The k-mer table (4^k + 1 counts) as an int64 tensor (a copy)."""
        if not self.kmer_k:
            raise ValueError("index has no k-mer table")
        out = torch.empty((1 << (2 * self.kmer_k)) + 1, dtype=torch.int32, device=device)
        _check(lib().sa_copy_kmer_table(self.handle, _ptr(out), _stream(None)), "sa_copy_kmer_table")
        if out.is_cuda:
            torch.cuda.current_stream().synchronize()
        return out.to(torch.int64) & 0xFFFFFFFF

    def save(self, path: str):
        sa_save(self, path)


def sa_build(text, width: int = 32, stream=None, kmer_k: Optional[int] = None, host_build: bool = False,
             dc3: bool = False) -> Index:
    """Index one reference (ASCII bases, host or device).  kmer_k: None picks k
    automatically, 0 builds no k-mer table, 1..15 sets k.  host_build: build
    the suffix array on the host by DC3 instead of on the GPU; dc3: build it on
    the GPU by DC3 instead of prefix doubling."""
    flags = SA_W32 if width == 32 else SA_W64 if width == 64 else None
    if flags is None:
        raise ValueError("width must be 32 or 64")
    if host_build:
        flags |= SA_BUILD_HOST
    if dc3:
        flags |= SA_BUILD_DC3
    if kmer_k == 0:
        flags |= SA_NO_KMER
    elif kmer_k is not None:
        if not 1 <= kmer_k <= 15:
            raise ValueError("kmer_k must be 0..15")
        flags |= kmer_k << 8
    n = int(text.numel() if torch is not None and isinstance(text, torch.Tensor) else len(text))
    h = _vp()
    _check(lib().sa_build(_ptr(text), n, flags, _stream(stream), ctypes.byref(h)), "sa_build")
    return Index(h.value)


def sa_save(idx: Index, path: str, stream=None):
    _check(lib().sa_save(idx.handle, os.fsencode(path), _stream(stream)), "sa_save")


def sa_load(path: str, stream=None) -> Index:
    h = _vp()
    _check(lib().sa_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "sa_load")
    return Index(h.value)


def sa_free(idx: Index):
    idx.free()


def sa_index_info(idx: Index):
    return {"n": idx.n, "width": idx.width, "key_depth": idx.key_depth, "kmer_k": idx.kmer_k,
            "device_bytes": idx.device_bytes}


def _refs(refs) -> tuple:
    if isinstance(refs, Index):
        refs = [refs]
    arr = (_vp * len(refs))(*[r.handle.value for r in refs])
    return arr, len(refs)


def _out_like(n_q: int, like):
    dev = like.device if torch is not None and isinstance(like, torch.Tensor) else "cpu"
    return torch.empty((n_q, RESULT_FIELDS), dtype=torch.int64, device=dev)


def _nbytes(x) -> int:
    if torch is not None and isinstance(x, torch.Tensor):
        return x.numel() * x.element_size()
    if isinstance(x, np.ndarray):
        return x.nbytes
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _check_results_buffer(out, n_q: int, what: str):
    """Results are 32 bytes each (lo, hi, count, flags): a smaller buffer
    would be written past its end, so it is refused here."""
    if _nbytes(out) < n_q * ctypes.sizeof(sa_result):
        raise ValueError(f"{what}: results buffer holds {_nbytes(out)} bytes, "
                         f"{n_q} results need {n_q * ctypes.sizeof(sa_result)} (shape (n_q, {RESULT_FIELDS}) int64)")


def _check_locate_buffers(out_offsets, out_pos, n_q: int, capacity: int, width: int, what: str):
    """Offsets take n_q + 1 int64; positions capacity entries of the suffix array's width."""
    if _nbytes(out_offsets) < (n_q + 1) * 8:
        raise ValueError(f"{what}: out_offsets holds {_nbytes(out_offsets)} bytes, needs {(n_q + 1) * 8}")
    if out_pos is not None and _nbytes(out_pos) < capacity * width:
        raise ValueError(f"{what}: out_pos holds {_nbytes(out_pos)} bytes, capacity {capacity} needs "
                         f"{capacity * width}")


def _search(fn, refs, q_bases, q_offsets, q_ref, out, stream, params=None):
    arr, nr = _refs(refs)
    n_q = int((q_offsets.numel() if isinstance(q_offsets, torch.Tensor) else len(q_offsets)) - 1)
    if out is None:
        out = _out_like(n_q, q_offsets)
    _check_results_buffer(out, n_q, fn.__name__)
    args = [arr, nr, _ptr(q_bases), _ptr(q_offsets), _ptr(q_ref), n_q, _ptr(out), _stream(stream)]
    if params is not None:
        args.append(ctypes.byref(params))
    _check(fn(*args), fn.__name__)
    return out


def sa_search_batch(refs, q_bases, q_offsets, q_ref=None, out=None, stream=None, params=None):
    """[lo, hi, count, flags] per query, int64 tensor of shape (n_q, 4); lo = hi =
    count = -1 and flags = SA_RESULT_INVALID mark an invalid query."""
    if params is not None:
        return _search(lib().sa_search_batch_ex, refs, q_bases, q_offsets, q_ref, out, stream, params)
    return _search(lib().sa_search_batch, refs, q_bases, q_offsets, q_ref, out, stream)


def sa_search_batch_plain(refs, q_bases, q_offsets, q_ref=None, out=None, stream=None):
    """Same results by the one-thread-per-query rendering of Alg. 1."""
    return _search(lib().sa_search_batch_plain, refs, q_bases, q_offsets, q_ref, out, stream)


def sa_locate(refs, res, cap: int, q_ref=None, out_offsets=None, out_pos=None, capacity=None, stream=None):
    """(offsets (n_q+1), positions) of the first min(count, cap) matches per query.

    With out_pos None, offsets are computed first and a positions tensor of
    exactly the needed size is allocated on the results' device."""
    arr, nr = _refs(refs)
    n_q = int(res.shape[0])
    _check_results_buffer(res, n_q, "sa_locate")
    dev = res.device if isinstance(res, torch.Tensor) else "cpu"
    dt = torch.int32 if (refs if isinstance(refs, Index) else refs[0]).width == 4 else torch.int64
    if out_offsets is None:
        out_offsets = torch.empty(n_q + 1, dtype=torch.int64, device=dev)
    s = _stream(stream)
    if out_pos is None:
        _check(lib().sa_locate(arr, nr, _ptr(q_ref), _ptr(res), n_q, cap, _ptr(out_offsets), None, 0, s),
               "sa_locate")
        total = int(out_offsets[-1].item())
        out_pos = torch.empty(max(total, 1), dtype=dt, device=dev)
        capacity = total
    if capacity is None:
        capacity = int(out_pos.numel() if isinstance(out_pos, torch.Tensor) else out_pos.size)
    _check_locate_buffers(out_offsets, out_pos, n_q, capacity, 4 if dt == torch.int32 else 8, "sa_locate")
    _check(lib().sa_locate(arr, nr, _ptr(q_ref), _ptr(res), n_q, cap, _ptr(out_offsets), _ptr(out_pos), capacity, s),
           "sa_locate")
    return out_offsets, out_pos


def sa_search_locate(refs, q_bases, q_offsets, cap: int, q_ref=None, out=None, out_offsets=None, out_pos=None,
                     capacity=None, stream=None, params=None):
    """sa_search_batch then sa_locate in one call: (results, offsets, positions).
    The caller gives out_pos (and capacity) or gets positions for at most
    `capacity` (default: cap * n_q) matches on the offsets' device."""
    arr, nr = _refs(refs)
    n_q = int((q_offsets.numel() if isinstance(q_offsets, torch.Tensor) else len(q_offsets)) - 1)
    if out is None:
        out = _out_like(n_q, q_offsets)
    dev = out.device if isinstance(out, torch.Tensor) else "cpu"
    dt = torch.int32 if (refs if isinstance(refs, Index) else refs[0]).width == 4 else torch.int64
    if out_offsets is None:
        out_offsets = torch.empty(n_q + 1, dtype=torch.int64, device=dev)
    if out_pos is None:
        capacity = cap * n_q if capacity is None else capacity
        out_pos = torch.empty(max(capacity, 1), dtype=dt, device=dev)
    if capacity is None:
        capacity = int(out_pos.numel() if isinstance(out_pos, torch.Tensor) else out_pos.size)
    _check_results_buffer(out, n_q, "sa_search_locate")
    _check_locate_buffers(out_offsets, out_pos, n_q, capacity, 4 if dt == torch.int32 else 8, "sa_search_locate")
    p = params if params is not None else sa_search_params()
    _check(lib().sa_search_locate(arr, nr, _ptr(q_bases), _ptr(q_offsets), _ptr(q_ref), n_q, _ptr(out), cap,
                                  _ptr(out_offsets), _ptr(out_pos), capacity, _stream(stream), ctypes.byref(p)),
           "sa_search_locate")
    return out, out_offsets, out_pos


def sa_random_read_rate(buffer_bytes: int = 4 << 30, threads_per_sm: int = 1024, steps: int = 64,
                        stream=None, read_bytes: int = 32) -> float:
    """Dependent random reads per second over a buffer far larger than L2; one
    read is read_bytes contiguous bytes (32 .. 512)."""
    r = ctypes.c_double(0.0)
    _check(lib().sa_random_read_rate_ex(buffer_bytes, threads_per_sm, steps, read_bytes, ctypes.byref(r),
                                        _stream(stream)), "sa_random_read_rate_ex")
    return r.value


def sa_suffix_array_host(text, width: int = 32) -> np.ndarray:
    """The suffix array of host bases (numpy uint8 array or CPU tensor) by the
    library's DC3 construction on the host CPU; needs no GPU."""
    n = int(text.numel() if torch is not None and isinstance(text, torch.Tensor) else len(text))
    if width not in (32, 64):
        raise ValueError("width must be 32 or 64")
    out = np.empty(max(n, 1), dtype=np.uint32 if width == 32 else np.uint64)
    _check(lib().sa_suffix_array_host(_ptr(text), n, width // 8, _ptr(out)), "sa_suffix_array_host")
    return out[:n]


def sa_scratch_info(reset_high: bool = False) -> dict:
    """The library's scratch pool on the current device: bytes reserved, bytes
    in use, and the high-water mark of use (optionally reset)."""
    r, u, h = _u64(), _u64(), _u64()
    _check(lib().sa_scratch_info(ctypes.byref(r), ctypes.byref(u), ctypes.byref(h), int(reset_high)),
           "sa_scratch_info")
    return {"reserved": r.value, "used": u.value, "used_high": h.value}


def sa_search_order(refs, n_q: int, params=None) -> str:
    """'kmer' if a search of n_q queries over refs would run in k-mer order, else 'input'."""
    arr, nr = _refs(refs)
    v = ctypes.c_int(0)
    _check(lib().sa_search_order(arr, nr, n_q, None if params is None else ctypes.byref(params), ctypes.byref(v)),
           "sa_search_order")
    return "kmer" if v.value else "input"


def sa_suffix_array_gpu(text, width: int = 32, dc3: bool = False, stream=None):
    """The suffix array of text (ASCII bases, host or device) built on the GPU,
    by prefix doubling or (dc3=True) by DC3; an int32/int64 CUDA tensor."""
    n = int(text.numel() if torch is not None and isinstance(text, torch.Tensor) else len(text))
    if width not in (32, 64):
        raise ValueError("width must be 32 or 64")
    out = torch.empty(max(n, 1), dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
    _check(lib().sa_suffix_array_gpu(_ptr(text), n, width // 8, SA_BUILD_DC3 if dc3 else 0, _ptr(out),
                                     _stream(stream)), "sa_suffix_array_gpu")
    return out[:n]


class SuffixTree:
    """The flattened suffix tree of an index's text (the paper's comparison
    index); keeps the index alive while it exists."""

    def __init__(self, idx: Index, stream=None):
        h = _vp()
        _check(lib().sa_stree_build(idx.handle, _stream(stream), ctypes.byref(h)), "sa_stree_build")
        self._h, self.index = h, idx
        nodes, b = _u64(), _u64()
        _check(lib().sa_stree_info(self._h, ctypes.byref(nodes), ctypes.byref(b)), "sa_stree_info")
        self.nodes, self.device_bytes = nodes.value, b.value

    def search(self, q_bases, q_offsets, out=None, stream=None):
        """[lo, hi, count, flags] per query (device tensors in and out)."""
        n_q = int(q_offsets.numel() - 1)
        if out is None:
            out = _out_like(n_q, q_offsets)
        _check_results_buffer(out, n_q, "sa_stree_search")
        _check(lib().sa_stree_search(self._h, _ptr(q_bases), _ptr(q_offsets), n_q, _ptr(out), _stream(stream)),
               "sa_stree_search")
        return out

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.sa_stree_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
