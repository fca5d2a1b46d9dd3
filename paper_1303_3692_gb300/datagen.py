"""Seeded synthetic references and query batches shaped like the paper's workloads.

This module only draws random data; it holds none of the matching method's
arithmetic, so both the CUDA path and the CPU oracle consume its output.
Everything is deterministic in the seed (numpy PCG64).

The paper's own data (the first 10^7 nt of a human chromosome 1 contig and
1024-nt queries mixed from human and mouse contigs, Section V) is not
available; these recipes stand in for it:

* background: iid bases with P(G)=P(C)=gc/2, P(A)=P(T)=(1-gc)/2;
* segmental duplications: a random source block of U[1000,10000] bases is
  copied over a random destination with 1% independent substitutions, until
  the overwritten bases reach the requested cover (overwrite keeps n exact);
* tandem repeats: a random unit of U{2..6} bases repeated U{10..200} times,
  written at a random position, until the cover is reached;
* repeat families: 4 consensus units of 300 bp and 4 of 6 kb; copies with a
  per-copy divergence U[0.10,0.20] are written until the cover is reached,
  about half of the covered bases from each unit size;
* sampled queries start at U[0, n-m] and receive k substitutions at distinct
  uniform positions (k uniform over the stated range), each to one of the
  three other bases; random queries are iid uniform ACGT.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
from dataclasses import dataclass, field

import numpy as np

ASCII = np.frombuffer(b"ACGT", dtype=np.uint8)
_CHUNK = 1 << 24
_POOL = None


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _sub_rng(seed: int, tag: int, chunk: int) -> np.random.Generator:
    """The generator of one chunk of one recipe step: a function of (seed,
    step, chunk index) only, so the output does not depend on how many
    threads draw the chunks."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(tag), int(chunk)])))


def _map(fn, items):
    """Runs fn over items on a thread pool (numpy's random fills, takes and
    ufuncs release the GIL) and returns the results in order."""
    global _POOL
    items = list(items)
    if len(items) <= 1:
        return [fn(x) for x in items]
    if _POOL is None:
        _POOL = _cf.ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1)))
    return list(_POOL.map(fn, items))


def _seed_of(rng: np.random.Generator) -> int:
    return int(rng.integers(0, 1 << 62))


def background(rng: np.random.Generator, n: int, gc: float = 0.5) -> np.ndarray:
    """Codes 0..3 (A,C,G,T) drawn iid with the given GC content."""
    out = np.empty(n, dtype=np.uint8)
    seed = _seed_of(rng)
    t = np.cumsum([(1 - gc) / 2, gc / 2, gc / 2]).astype(np.float32)

    def fill(c):
        s, e = c * _CHUNK, min(n, (c + 1) * _CHUNK)
        r = _sub_rng(seed, 1, c)
        if gc == 0.5:
            out[s:e] = r.integers(0, 4, e - s, dtype=np.uint8)
        else:
            u = r.random(e - s, dtype=np.float32)
            o = out[s:e]
            np.greater_equal(u, t[0], out=o, casting="unsafe")
            o += u >= t[1]
            o += u >= t[2]

    _map(fill, range((n + _CHUNK - 1) // _CHUNK))
    return out


def _mutate(rng: np.random.Generator, block: np.ndarray, rate) -> None:
    """Independent substitutions: each base (with probability rate, a scalar
    or one rate per row of a 2-D block) becomes one of the other three."""
    r = np.asarray(rate, dtype=np.float64)
    if block.ndim == 2 and r.ndim == 1:
        r = r[:, None]
    mask = rng.random(block.shape) < r
    k = int(mask.sum())
    if k:
        block[mask] = (block[mask] + rng.integers(1, 4, k, dtype=np.uint8)) & 3


def segmental_duplications(rng, codes: np.ndarray, cover: float,
                           lmin: int = 1000, lmax: int = 10000, sub_rate: float = 0.01) -> None:
    n = codes.size
    target = int(cover * n)
    done = 0
    if target <= 0 or n <= lmax + 1:
        return
    while done < target:
        L = int(rng.integers(lmin, lmax + 1))
        src = int(rng.integers(0, n - L + 1))
        dst = int(rng.integers(0, n - L + 1))
        block = codes[src:src + L].copy()
        _mutate(rng, block, sub_rate)
        codes[dst:dst + L] = block
        done += L


def tandem_repeats(rng, codes: np.ndarray, cover: float,
                   unit=(2, 6), copies=(10, 200)) -> None:
    n = codes.size
    target = int(cover * n)
    done = 0
    while done < target:
        u = int(rng.integers(unit[0], unit[1] + 1))
        c = int(rng.integers(copies[0], copies[1] + 1))
        L = u * c
        if L >= n:
            break
        dst = int(rng.integers(0, n - L + 1))
        codes[dst:dst + L] = np.tile(rng.integers(0, 4, u, dtype=np.uint8), c)
        done += L


def repeat_families(rng, codes: np.ndarray, cover: float, unit_lens=(300, 6000),
                    n_fam: int = 4, div=(0.10, 0.20)) -> None:
    """Copies of n_fam random consensus units per unit length, each copy with
    its own divergence, written at random destinations (later copies
    overwrite earlier ones) until each unit length covers cover/len(unit_lens)
    of the text.  Copies are drawn in batches of independent chunks and
    written in order."""
    n = codes.size
    cons = {L: np.stack([rng.integers(0, 4, L, dtype=np.uint8) for _ in range(n_fam)]) for L in unit_lens}
    target = int(cover * n)
    seed = _seed_of(rng)
    for li, L in enumerate(unit_lens):
        if L >= n:
            continue
        per = target // len(unit_lens)
        copies = (per + L - 1) // L
        batch = max(1, (1 << 22) // L)
        chunks = [(c, c * batch, min(copies, (c + 1) * batch)) for c in range((copies + batch - 1) // batch)]

        def draw(ch, L=L, li=li):
            c, a, b = ch
            r = _sub_rng(seed, 10 + li, c)
            fam = r.integers(0, n_fam, b - a)
            rate = r.uniform(div[0], div[1], b - a)
            dst = r.integers(0, n - L + 1, b - a)
            block = cons[L][fam]
            _mutate(r, block, rate)
            return dst, block

        # draw a wave of chunks in parallel, write them in chunk order
        wave = 64
        for w0 in range(0, len(chunks), wave):
            for dst, block in _map(draw, chunks[w0:w0 + wave]):
                codes[dst[:, None] + np.arange(L)[None, :]] = block


def to_ascii(codes: np.ndarray) -> np.ndarray:
    out = np.empty(codes.size, dtype=np.uint8)

    def conv(c):
        s, e = c * _CHUNK, min(codes.size, (c + 1) * _CHUNK)
        np.take(ASCII, codes[s:e], out=out[s:e])

    _map(conv, range((codes.size + _CHUNK - 1) // _CHUNK))
    return out


def reference(n: int, seed: int, gc: float = 0.5, sd_cover: float = 0.0,
              tandem_cover: float = 0.0, family_cover: float = 0.0) -> np.ndarray:
    """ASCII reference of n bases built from the recipes above."""
    rng = _rng(seed)
    codes = background(rng, n, gc)
    if family_cover:
        repeat_families(rng, codes, family_cover)
    if sd_cover:
        segmental_duplications(rng, codes, sd_cover)
    if tandem_cover:
        tandem_repeats(rng, codes, tandem_cover)
    return to_ascii(codes)


def queries(ref: np.ndarray, nq: int, seed: int, m=100, frac_sampled: float = 0.5,
            subs=(0, 0)):
    """Query batch against one ASCII reference.

    m is a fixed length or an inclusive (min, max) range drawn uniformly.
    Returns (bases uint8 ASCII concatenated, offsets int64 (nq+1), sampled bool).
    Lengths and the sampled/random choice are drawn first; the bases of each
    chunk of queries then come from that chunk's own generator.
    """
    rng = _rng(seed)
    n = ref.size
    if isinstance(m, (tuple, list)):
        lens = rng.integers(m[0], m[1] + 1, nq).astype(np.int64)
        mmax = int(m[1])
        fixed = False
    else:
        lens = np.full(nq, int(m), dtype=np.int64)
        mmax = int(m)
        fixed = True
    offsets = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    sampled = rng.random(nq) < frac_sampled
    seed2 = _seed_of(rng)
    bases = np.empty(int(offsets[-1]), dtype=np.uint8)
    codes_of = np.full(256, 0, dtype=np.uint8)
    codes_of[ASCII] = np.arange(4, dtype=np.uint8)
    step = max(1, (1 << 22) // max(1, mmax))
    win = np.lib.stride_tricks.sliding_window_view(ref, mmax) if n >= mmax else None

    def chunk(c):
        s, e = c * step, min(nq, (c + 1) * step)
        r = _sub_rng(seed2, 2, c)
        k = e - s
        L = lens[s:e]
        blk = r.integers(0, 4, (k, mmax), dtype=np.uint8)
        smp = sampled[s:e]
        if win is not None:
            starts = (r.random(k) * (n - L + 1)).astype(np.int64)
            starts = np.minimum(starts, n - mmax)
            # sampled queries shorter than mmax near the end still start <= n-m
            blk[smp] = np.take(codes_of, win[starts[smp]])
            nsub = r.integers(subs[0], subs[1] + 1, k)
            first = np.full(k, -1, dtype=np.int64)
            for j in range(int(subs[1])):
                sel = smp & (nsub > j)
                if not sel.any():
                    continue
                rows = np.nonzero(sel)[0]
                # distinct positions: draw position j among the L-j free slots
                p = (r.random(rows.size) * (L[rows] - j)).astype(np.int64)
                if j == 1:
                    p = np.where(p >= first[rows], p + 1, p)
                if j == 0:
                    first[rows] = p
                blk[rows, p] = (blk[rows, p] + r.integers(1, 4, rows.size, dtype=np.uint8)) & 3
        else:
            smp[:] = False
        if fixed:
            np.take(ASCII, blk.reshape(-1), out=bases[offsets[s]:offsets[e]])
        else:
            mask = np.arange(mmax)[None, :] < L[:, None]
            bases[offsets[s]:offsets[e]] = ASCII[blk[mask]]

    _map(chunk, range((nq + step - 1) // step))
    return bases, offsets, sampled


@dataclass
class Workload:
    """One reference plus one query batch (ASCII), with its recipe."""
    name: str
    ref: np.ndarray
    q_bases: np.ndarray
    q_offsets: np.ndarray
    sampled: np.ndarray
    cap: int = 0
    width: int = 32
    meta: dict = field(default_factory=dict)


SEED0 = 1303369200

# The paper-scale workloads (sizes as stated; see the module docstring for
# the recipes).  'scale' shrinks n and the query count for quick tests while
# keeping the recipe.

def plain_small(scale: float = 1.0, seed: int = SEED0 + 1) -> Workload:
    """1 Mbp iid reference; 100,000 queries of 32 bp, half exact copies, half random."""
    n = max(64, int(1_000_000 * scale))
    nq = max(1, int(100_000 * scale))
    ref = reference(n, seed, gc=0.5)
    qb, qo, smp = queries(ref, nq, seed + 1000, m=32, frac_sampled=0.5, subs=(0, 0))
    return Workload("plain-1Mbp-100k-q32", ref, qb, qo, smp, cap=0, width=32,
                    meta={"n": n, "nq": nq, "m": 32})


def repetitive_100m(scale: float = 1.0, seed: int = SEED0 + 2) -> Workload:
    """100 Mbp reference with 10% segmental duplications and 2% tandem repeats;
    10,000,000 queries of 100 bp, 80% sampled with 0-2 substitutions, 20% random;
    locate up to 64 positions."""
    n = max(20_000, int(100_000_000 * scale))
    nq = max(1, int(10_000_000 * scale))
    ref = reference(n, seed, gc=0.5, sd_cover=0.10, tandem_cover=0.02)
    qb, qo, smp = queries(ref, nq, seed + 1000, m=100, frac_sampled=0.8, subs=(0, 2))
    return Workload("repetitive-100Mbp-10M-q100", ref, qb, qo, smp, cap=64, width=32,
                    meta={"n": n, "nq": nq, "m": 100})


def human_sized(scale: float = 1.0, seed: int = SEED0 + 4, nq_sampled: int = 100_000_000,
                nq_random: int = 10_000_000, cap: int = 16) -> Workload:
    """3.1 Gbp reference at GC 0.41 with 45% repeat families and 3% tandem
    repeats, int64 suffix array; 150 bp queries, 10^8 sampled with 0-1
    substitutions plus 10^7 random."""
    n = max(20_000, int(3_100_000_000 * scale))
    nq = max(1, int((nq_sampled + nq_random) * scale))
    ref = reference(n, seed, gc=0.41, family_cover=0.45, tandem_cover=0.03)
    qb, qo, smp = queries(ref, nq, seed + 1000, m=150,
                          frac_sampled=nq_sampled / (nq_sampled + nq_random), subs=(0, 1))
    return Workload("human-3.1Gbp-q150", ref, qb, qo, smp, cap=cap, width=64,
                    meta={"n": n, "nq": nq, "m": 150})


MULTI_REF_SIZES = (5_000_000, 12_000_000, 25_000_000, 50_000_000)
MULTI_REF_GC = (0.38, 0.45, 0.50, 0.62)


def paper_shaped(scale: float = 1.0, seed: int = SEED0 + 6, nq: int = 1 << 21) -> Workload:
    """The shape of the paper's own runs (Section V, Table V): a reference of
    10^7 bases (here human-like: GC 0.41, 45% repeat families, 3% tandem
    repeats) and up to 2^21 queries of 1024 bases, half copied exactly from the
    reference and half random (standing in for the mouse contig's queries,
    which an exact 1024-base match almost never finds in human sequence).
    Every prefix of the batch keeps the half-and-half mix."""
    n = max(20_000, int(10_000_000 * scale))
    nq = max(1, int(nq * scale))
    ref = reference(n, seed, gc=0.41, family_cover=0.45, tandem_cover=0.03)
    qb, qo, smp = queries(ref, nq, seed + 1000, m=1024, frac_sampled=0.5, subs=(0, 0))
    return Workload("paper-shaped-10Mbp-q1024", ref, qb, qo, smp, cap=0, width=32,
                    meta={"n": n, "nq": nq, "m": 1024})


def multi_genome(scale: float = 1.0, seed: int = SEED0 + 3):
    """4 references (5, 12, 25, 50 Mbp; GC 0.38/0.45/0.50/0.62; 5% segmental
    duplications) and 16,000,000 queries of length U[20,250], each assigned
    uniformly to one reference, 70% sampled from it (no substitutions) and 30%
    random.  Returns (refs, q_bases, q_offsets, q_ref, sampled)."""
    refs = [reference(max(2_000, int(s * scale)), seed + 10 * i, gc=g, sd_cover=0.05)
            for i, (s, g) in enumerate(zip(MULTI_REF_SIZES, MULTI_REF_GC))]
    nq = max(4, int(16_000_000 * scale))
    rng = _rng(seed + 999)
    mmin, mmax = 20, 250
    q_ref = rng.integers(0, len(refs), nq).astype(np.uint32)
    lens = rng.integers(mmin, mmax + 1, nq).astype(np.int64)
    sampled = rng.random(nq) < 0.7
    offsets = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    bases = np.empty(int(offsets[-1]), dtype=np.uint8)
    # all references back to back; a sampled query of reference r starts
    # uniformly in [base_r, base_r + n_r - m] and never crosses into the next
    cat = np.concatenate(refs)
    starts_r = np.zeros(len(refs) + 1, dtype=np.int64)
    np.cumsum([r.size for r in refs], out=starts_r[1:])
    win = np.lib.stride_tricks.sliding_window_view(cat, mmax)
    step = 1 << 20
    for s in range(0, nq, step):
        e = min(nq, s + step)
        k = e - s
        L = lens[s:e]
        r = q_ref[s:e]
        blk = ASCII[rng.integers(0, 4, (k, mmax), dtype=np.uint8)]
        smp = sampled[s:e]
        n_r = (starts_r[r + 1] - starts_r[r])
        room = np.maximum(n_r - L + 1, 1)
        st = starts_r[r] + (rng.random(k) * room).astype(np.int64)
        st = np.minimum(st, cat.size - mmax)  # a window of mmax must fit; only bases < L are kept
        blk[smp] = win[st[smp]]
        mask = np.arange(mmax)[None, :] < L[:, None]
        bases[offsets[s]:offsets[e]] = blk[mask]
    return refs, bases, offsets, q_ref, sampled
