"""Continuous-batching serving loop over references resident on one GPU.

Requests (a batch of queries against one of the resident references, and
how many positions to locate per query: 0 for counts only) arrive over time.  The server keeps `slots` batches in flight, each on its own CUDA
stream.  Whenever a slot is free it coalesces the waiting requests, oldest
first, into one batch -- bounded by a query count, a base count and the free
device memory the library's scratch will need -- and runs that batch as one
multi-reference search through the C ABI.
Requests that arrive while other batches run are admitted as soon as a slot
and memory free up, so their work overlaps on the device with the batches
already in flight.  A completed batch's results are scattered back to its
requests and each request's latency (arrival to results on the host) is
recorded.

`run_plain` serves the same trace the simple way for comparison: one
search call per request, in arrival order, each waiting for the previous.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import sa


@dataclass
class Request:
    rid: int
    ref: int
    bases: "object"       # pinned uint8 tensor (host) of the concatenated queries
    offsets: np.ndarray   # int64, n + 1 offsets starting at 0
    arrival: float        # seconds since the start of the trace
    cap: int = 0          # positions to locate per query (0: counts only)
    rc: bool = False      # search the queries' reverse complements (the other strand)
    results: Optional[np.ndarray] = None   # (n, 4) int64: lo, hi, count, flags
    pos_offsets: Optional[np.ndarray] = None  # (n + 1) int64 when cap > 0
    positions: Optional[np.ndarray] = None    # located positions, suffix-array order per query
    done: float = math.nan
    status: str = "pending"

    @property
    def n(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def nbases(self) -> int:
        return int(self.offsets[-1])


def scratch_bytes(n_q: int, n_bases: int, both_strands: bool = False) -> int:
    """Device scratch one search call takes from the library's pool, at most:
    the packed batch (8 bytes per 32 bases) and its validity masks (4 bytes
    per 32 bases), twice when queries name their strands; 64 bytes of worklist
    room per query; in k-mer order the ordered list (64-byte records, room
    for about 2.125 per query plus 257 * 256); small flags, and 256 bytes of
    alignment per allocation."""
    words = ((n_bases + 31) // 32 + 6) * (2 if both_strands else 1)
    listed = ((n_q + 32) * 9 // 8 + 256 * 257 + n_q) * 64
    return 12 * words + 64 * n_q + listed + 1288 * 4 + 80 + 8 * 256


def kept(counts: np.ndarray, cap: int) -> np.ndarray:
    """Positions located per query: min(count, cap), none for an invalid query."""
    return np.where(counts < 0, 0, np.minimum(counts, cap))


def split_positions(results: np.ndarray, offs: np.ndarray, pos: np.ndarray, cap_batch: int, cap: int):
    """A request's positions out of its batch's: the batch located
    min(count, cap_batch) per query at offs; the request keeps the first
    min(count, cap) of each.  Returns (offsets (n + 1), positions)."""
    k = kept(results[:, 2], cap)
    out_offs = np.zeros(k.size + 1, dtype=np.int64)
    np.cumsum(k, out=out_offs[1:])
    idx = np.repeat(offs[:-1], k) + (np.arange(int(out_offs[-1])) - np.repeat(out_offs[:-1], k))
    return out_offs, pos[idx]


def form_batch(queue: List[Request], max_q: int, max_bases: int, budget: int):
    """(taken, rest): the oldest requests whose total queries, bases and
    library scratch stay within max_q, max_bases and the device-memory budget;
    the first request that does not fit ends the batch (no reordering)."""
    nq = nb = 0
    both = False
    i = 0
    while i < len(queue):
        r = queue[i]
        b2 = both or r.rc
        if (nq + r.n > max_q or nb + r.nbases > max_bases
                or scratch_bytes(nq + r.n, nb + r.nbases, both_strands=b2) > budget):
            break
        nq += r.n
        nb += r.nbases
        both = b2
        i += 1
    return queue[:i], queue[i:]


class _Slot:
    def __init__(self, device, max_q: int, max_bases: int, max_cap: int, pos_dtype):
        import torch

        self.stream = torch.cuda.Stream(device=device)
        self.bases = torch.empty(max(1, max_bases), dtype=torch.uint8, device=device)
        self.offsets = torch.empty(max_q + 1, dtype=torch.int64, device=device)
        self.qref = torch.empty(max(1, max_q), dtype=torch.int32, device=device)
        self.out = torch.empty((max(1, max_q), sa.RESULT_FIELDS), dtype=torch.int64, device=device)
        self.h_offsets = torch.empty(max_q + 1, dtype=torch.int64).pin_memory()
        self.h_qref = torch.empty(max(1, max_q), dtype=torch.int32).pin_memory()
        self.h_out = torch.empty((max(1, max_q), sa.RESULT_FIELDS), dtype=torch.int64).pin_memory()
        # located positions (when the server locates): every query's first max_cap
        self.pos_cap = max(1, max_q * max_cap)
        self.loc_offs = torch.empty(max_q + 1, dtype=torch.int64, device=device) if max_cap else None
        self.pos = torch.empty(self.pos_cap, dtype=pos_dtype, device=device) if max_cap else None
        self.h_loc_offs = torch.empty(max_q + 1, dtype=torch.int64).pin_memory() if max_cap else None
        self.cap = 0
        self.event = None
        self.requests: List[Request] = []
        self.n_q = 0


class Server:
    def __init__(self, refs: Sequence["sa.Index"], max_batch_queries: int = 1 << 21,
                 max_batch_bases: int = 1 << 28, slots: int = 2, mem_reserve: int = 1 << 30,
                 params: Optional["sa.sa_search_params"] = None,
                 free_memory: Optional[Callable[[], int]] = None, max_cap: int = 0):
        import torch

        self.refs = list(refs)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.max_q = max_batch_queries
        self.max_bases = max_batch_bases
        self.max_cap = max_cap
        self.mem_reserve = mem_reserve
        self.params = params
        self.free_memory = free_memory or (lambda: torch.cuda.mem_get_info()[0])
        pos_dtype = torch.int32 if self.refs[0].width == 4 else torch.int64
        self.slots = [_Slot(self.device, max_batch_queries, max_batch_bases, max_cap, pos_dtype)
                      for _ in range(slots)]
        self.queue: List[Request] = []
        self.completed: List[Request] = []
        self.batches = 0
        self.batch_sizes: List[tuple] = []  # (queries, bases) of every launched batch

    # -- admission -----------------------------------------------------
    def submit(self, req: Request) -> None:
        if (req.n > self.max_q or req.nbases > self.max_bases or not 0 <= req.ref < len(self.refs)
                or not 0 <= req.cap <= self.max_cap):
            req.status = "rejected"
            req.done = req.arrival
            self.completed.append(req)
            return
        self.queue.append(req)

    def _take_batch(self) -> List[Request]:
        taken, self.queue = form_batch(self.queue, self.max_q, self.max_bases,
                                       self.free_memory() - self.mem_reserve)
        return taken

    # -- one batch -------------------------------------------------------
    def _launch(self, slot: _Slot, reqs: List[Request]) -> None:
        import torch

        nq = sum(r.n for r in reqs)
        nb = sum(r.nbases for r in reqs)
        ho = slot.h_offsets.numpy()
        hr = slot.h_qref.numpy().view(np.uint32)
        both = any(r.rc for r in reqs)
        q, b = 0, 0
        for r in reqs:
            ho[q:q + r.n + 1] = r.offsets + b
            hr[q:q + r.n] = r.ref | (sa.STRAND_BIT if r.rc else 0)
            q += r.n
            b += r.nbases
        with torch.cuda.stream(slot.stream):
            b = 0
            for r in reqs:
                if r.nbases:
                    slot.bases[b:b + r.nbases].copy_(r.bases[:r.nbases], non_blocking=True)
                b += r.nbases
            slot.offsets[:nq + 1].copy_(slot.h_offsets[:nq + 1], non_blocking=True)
            slot.qref[:nq].copy_(slot.h_qref[:nq], non_blocking=True)
            p = sa.sa_search_params() if self.params is None else sa.sa_search_params.from_buffer_copy(self.params)
            p.flags |= sa.SA_PARAM_Q_RANGE
            if both:  # some requests want the other strand: bit 31 of their reference ids
                p.flags |= sa.SA_PARAM_STRAND_PER_QUERY
            p.q_first, p.q_total = 0, nb
            slot.cap = max((r.cap for r in reqs), default=0)
            if nq and slot.cap:  # search and locate in one call, up to the batch's largest cap
                sa.sa_search_locate(self.refs, slot.bases, slot.offsets[:nq + 1], slot.cap, q_ref=slot.qref[:nq],
                                    out=slot.out[:nq], out_offsets=slot.loc_offs[:nq + 1], out_pos=slot.pos,
                                    capacity=slot.pos_cap, stream=slot.stream, params=p)
                slot.h_loc_offs[:nq + 1].copy_(slot.loc_offs[:nq + 1], non_blocking=True)
            elif nq:
                sa.sa_search_batch(self.refs, slot.bases, slot.offsets[:nq + 1], q_ref=slot.qref[:nq],
                                   out=slot.out[:nq], stream=slot.stream, params=p)
            if nq:
                slot.h_out[:nq].copy_(slot.out[:nq], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.requests = reqs
        slot.n_q = nq
        self.batches += 1
        self.batch_sizes.append((nq, nb))

    def _finish(self, slot: _Slot, now: float) -> None:
        out = slot.h_out.numpy()
        pos = offs = None
        if slot.cap and slot.n_q:
            offs = slot.h_loc_offs[:slot.n_q + 1].numpy()
            total = int(offs[-1])
            pos = slot.pos[:total].cpu().numpy()  # the batch's positions (usually few)
        q = 0
        for r in slot.requests:
            r.results = out[q:q + r.n].copy()
            # the batch was located up to its largest cap: truncation is per
            # request, and only a request that asked for positions has it
            valid = r.results[:, 0] != -1
            trunc = (r.results[:, 2] > r.cap) if r.cap else np.zeros(r.n, dtype=bool)
            r.results[:, 3] = np.where(valid, np.where(trunc, sa.SA_RESULT_TRUNCATED, 0), sa.SA_RESULT_INVALID)
            if r.cap:
                r.pos_offsets, r.positions = split_positions(r.results, offs[q:q + r.n + 1], pos, slot.cap, r.cap)
            r.done = now
            r.status = "done"
            q += r.n
            self.completed.append(r)
        slot.requests, slot.event, slot.n_q, slot.cap = [], None, 0, 0

    def poll(self, now: float) -> None:
        for s in self.slots:
            if s.event is not None and s.event.query():
                self._finish(s, now)

    def pump(self, now: float) -> None:
        """Finish completed batches, then launch on every free slot.  A request
        that does not fit even when no batch is in flight is rejected rather
        than allocated for."""
        self.poll(now)
        for s in self.slots:
            if s.event is None and self.queue:
                reqs = self._take_batch()
                if not reqs:
                    if all(x.event is None for x in self.slots):
                        r = self.queue.pop(0)
                        r.status, r.done = "rejected", now
                        self.completed.append(r)
                    break
                self._launch(s, reqs)

    def idle(self) -> bool:
        return not self.queue and all(s.event is None for s in self.slots)

    def run(self, trace: Sequence[Request], clock: Callable[[], float] = time.perf_counter,
            poll_s: float = 50e-6) -> dict:
        """Replays the trace in real time (arrival times relative to the start;
        a trace whose arrivals are all 0 measures the saturated throughput).
        Between events the loop sleeps: until the next arrival when nothing is
        in flight, else for poll_s before it looks at the batches again."""
        pending = sorted(trace, key=lambda r: r.arrival)
        i = 0
        t0 = clock()
        while i < len(pending) or not self.idle():
            now = clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            self.pump(now)
            nxt = pending[i].arrival - (clock() - t0) if i < len(pending) else math.inf
            busy = any(s.event is not None for s in self.slots)
            wait = min(nxt, poll_s) if busy else nxt
            if self.queue and not busy:
                wait = 0.0  # a free slot and a waiting request: no reason to sleep
            if 0 < wait < math.inf:
                time.sleep(wait)
        return summarize(trace, self.batches)


def summarize(trace: Sequence[Request], batches: int) -> dict:
    done = [r for r in trace if r.status == "done"]
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    nq = sum(r.n for r in done)
    span = (max(r.done for r in done) - min(r.arrival for r in trace)) if done else math.nan
    return {
        "requests": len(trace), "served": len(done), "rejected": sum(r.status == "rejected" for r in trace),
        "queries": nq, "batches": batches,
        "p50_ms": float(np.percentile(lat, 50)) if lat.size else math.nan,
        "p99_ms": float(np.percentile(lat, 99)) if lat.size else math.nan,
        "max_ms": float(lat.max()) if lat.size else math.nan,
        "queries_per_s": nq / span if span and span > 0 else math.nan,
        "span_s": span,
    }


def run_plain(refs: Sequence["sa.Index"], trace: Sequence[Request],
              clock: Callable[[], float] = time.perf_counter, kernel: str = "optimized") -> dict:
    """One search call per request, in arrival order, each on the default stream
    and waited for before the next (no coalescing, no overlap).  kernel
    "optimized" makes each call with the library's search (and locate) in one
    call; "plain" with the one-thread-per-query rendering of Alg. 1
    (sa_search_batch_plain), then sa_locate for a request that wants
    positions."""
    import torch

    if kernel not in ("optimized", "plain"):
        raise ValueError("kernel must be 'optimized' or 'plain'")
    dev = torch.device("cuda", torch.cuda.current_device())
    pending = sorted(trace, key=lambda r: r.arrival)
    t0 = clock()
    for r in pending:
        wait = r.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        bases = r.bases[:r.nbases].to(dev, non_blocking=True) if r.nbases else torch.zeros(1, dtype=torch.uint8,
                                                                                             device=dev)
        offs = torch.from_numpy(r.offsets).to(dev, non_blocking=True)
        p = sa.sa_search_params()
        p.flags = sa.SA_PARAM_Q_RANGE | (sa.SA_PARAM_REVERSE_COMPLEMENT if r.rc else 0)
        p.q_first, p.q_total = 0, r.nbases
        if kernel == "plain" and r.rc:
            raise ValueError("the plain kernel searches the forward strand only")
        if kernel == "plain":
            res = sa.sa_search_batch_plain(refs[r.ref], bases, offs)
            if r.cap:
                lo_offs, pos = sa.sa_locate(refs[r.ref], res, r.cap)
                r.pos_offsets = lo_offs.cpu().numpy()
                r.positions = pos[:int(r.pos_offsets[-1])].cpu().numpy()
                res[:, 3] = torch.where(res[:, 2] > r.cap, sa.SA_RESULT_TRUNCATED, res[:, 3])
        elif r.cap:
            res, lo_offs, pos = sa.sa_search_locate(refs[r.ref], bases, offs, r.cap, params=p)
            r.pos_offsets = lo_offs.cpu().numpy()
            r.positions = pos[:int(r.pos_offsets[-1])].cpu().numpy()
        else:
            res = sa.sa_search_batch(refs[r.ref], bases, offs, params=p)
        r.results = res.cpu().numpy()
        r.done = clock() - t0
        r.status = "done"
    return summarize(trace, len(trace))


def make_trace(ref_pools, rate: float, duration: float, seed: int, q_range=(1, 100_000),
               caps: Sequence[int] = (0,), rc_frac: float = 0.0) -> List[Request]:
    """Poisson arrivals (mean `rate` per second over `duration` seconds); each
    request targets a uniformly drawn reference, holds a log-uniform number of
    queries in q_range, sliced from that reference's pool of pinned queries
    (ref_pools[r] = (pinned bases tensor, offsets int64 numpy)), and asks for a
    locate cap drawn uniformly from caps (0: counts only); a fraction rc_frac
    of the requests ask for the other strand.""" 
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        r = int(rng.integers(0, len(ref_pools)))
        bases, offs = ref_pools[r]
        pool_n = offs.size - 1
        n = int(round(math.exp(rng.uniform(math.log(q_range[0]), math.log(q_range[1])))))
        n = max(q_range[0], min(n, pool_n))
        s = int(rng.integers(0, pool_n - n + 1))
        o = offs[s:s + n + 1] - offs[s]
        cap = int(caps[int(rng.integers(0, len(caps)))]) if len(caps) > 1 else int(caps[0])
        rc = bool(rng.random() < rc_frac) if rc_frac > 0 else False
        reqs.append(Request(len(reqs), r, bases[int(offs[s]):int(offs[s + n])], o, t, cap=cap, rc=rc))
    return reqs
