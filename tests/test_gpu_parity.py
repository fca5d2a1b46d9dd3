"""GPU parity: libsa (through the C ABI) against the CPU oracle, bit-exact.

Everything here is integer and string work, so the tolerance is zero: suffix
arrays, [lo, hi), counts and located positions must be identical."""
import itertools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def sa():
    from paper_1303_3692_gb300 import build_lib, sa as sa_mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    sa_mod.lib()
    return sa_mod


def _dev(a):
    return torch.from_numpy(np.array(a, copy=True)).to(DEV)


def _batch(queries):
    enc = [q.encode() if isinstance(q, str) else bytes(q) for q in queries]
    qb = np.frombuffer(b"".join(enc) or b"A", dtype=np.uint8)[: sum(len(e) for e in enc)].copy()
    qo = np.zeros(len(enc) + 1, dtype=np.int64)
    np.cumsum([len(e) for e in enc], out=qo[1:])
    return qb, qo


def _check_search(sa, idx, T, osa, qb, qo, plain=True, params=None):
    lo, hi = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
    fns = [lambda *a: sa.sa_search_batch(*a, params=params)]
    if plain:
        fns.append(sa.sa_search_batch_plain)
    for fn in fns:
        got = fn(idx, _dev(qb) if qb.size else torch.zeros(1, dtype=torch.uint8, device=DEV), _dev(qo)).cpu().numpy()
        assert np.array_equal(got[:, 0], lo), np.nonzero(got[:, 0] != lo)[0][:10]
        assert np.array_equal(got[:, 1], hi), np.nonzero(got[:, 1] != hi)[0][:10]
        assert np.array_equal(got[:, 2], hi - lo)
    return lo, hi


def test_paper_example(sa, golden):
    text = golden["text"][0][0]
    idx = sa.sa_build(_dev(np.frombuffer(text.encode(), dtype=np.uint8)))
    assert idx.suffix_array().cpu().tolist() == [int(x) for x in golden["sa"][0]]
    qs = [q for q, _, _ in golden["search"]]
    qb, qo = _batch(qs)
    got = sa.sa_search_batch(idx, _dev(qb), _dev(qo)).cpu().tolist()
    for (q, lb, rb), g in zip(golden["search"], got):
        assert g[:3] == [int(lb), int(rb) + 1, int(rb) - int(lb) + 1], q
    offs, pos = sa.sa_locate(idx, sa.sa_search_batch(idx, _dev(qb), _dev(qo)), 8)
    a = qs.index("a")
    assert pos[offs[a]:offs[a + 1]].cpu().tolist() == [int(p) for p in golden["positions"][0][1:]]


def test_exhaustive_tiny_texts(sa):
    """Every text of length <= 5 (and a sample of length 6-7) x every query of length <= 4."""
    qs = [""] + ["".join(p) for L in range(1, 5) for p in itertools.product("ACGT", repeat=L)] + ["ACGTACGT"]
    qb, qo = _batch(qs)
    rng = np.random.default_rng(5)
    texts = ["".join(t) for L in range(1, 6) for t in itertools.product("ACGT", repeat=L)]
    texts += ["".join(rng.choice(list("ACGT"), L)) for L in (6, 7) for _ in range(100)]
    for text in texts:
        T = np.frombuffer(text.encode(), dtype=np.uint8)
        idx = sa.sa_build(_dev(T))
        osa = oracle.sa_naive(T)
        assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa), text
        _check_search(sa, idx, T, osa, qb, qo, plain=(len(text) <= 3))


LENGTHS = [1, 2, 3, 31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128, 129, 150, 250, 300]


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 1000, 4097, 30011])
@pytest.mark.parametrize("width", [32, 64])
def test_random_references(sa, n, width):
    ref = datagen.reference(n, 100 + n, gc=0.45, sd_cover=0.1 if n > 12000 else 0.0, tandem_cover=0.05)
    if n >= 1000:
        ref[n // 2:n // 2 + n // 5] = ref[0:n // 5]  # long exact repeat: deep ties
    T = oracle.normalize(ref)
    idx = sa.sa_build(_dev(ref), width=width)
    assert idx.width == width // 8
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    qs = []
    rng = np.random.default_rng(n)
    for m in LENGTHS:
        for _ in range(6):
            if m <= n:
                s = int(rng.integers(0, n - m + 1))
                qs.append(ref[s:s + m].tobytes())
            qs.append(datagen.ASCII[rng.integers(0, 4, m)].tobytes())
        qs.append(ref[n - min(m, n):].tobytes())          # ends at the last base
        qs.append(ref[n - min(m, n):].tobytes() + b"A")   # runs past the end
    qs += [b"", ref.tobytes(), ref.tobytes() + b"C"]
    qb, qo = _batch(qs)
    lo, hi = _check_search(sa, idx, T, osa, qb, qo)
    res = sa.sa_search_batch(idx, _dev(qb), _dev(qo))
    for cap in (0, 1, 3, 64):
        offs, pos = sa.sa_locate(idx, res, cap)
        offs, pos = offs.cpu().numpy(), pos.cpu().numpy().astype(np.int64)
        k = np.minimum(hi - lo, cap)
        assert np.array_equal(np.diff(offs), k) and offs[0] == 0
        for q in range(len(qs)):
            assert np.array_equal(pos[offs[q]:offs[q + 1]], oracle.locate(osa, int(lo[q]), int(hi[q]), cap))


@pytest.mark.parametrize("text", ["A" * 5000, "AC" * 2500, "ACGT" * 1000 + "A", "T" * 33],
                         ids=["A5000", "AC2500", "ACGT1000A", "T33"])
def test_degenerate_texts(sa, text):
    T = oracle.normalize(text)
    idx = sa.sa_build(_dev(T))
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    qs = [text[:m] for m in (1, 2, 31, 32, 33, 64, 65, 100, 129)] + ["C", "G" * 3, text, text + "A", "A" * 64 + "C"]
    qb, qo = _batch(qs)
    _check_search(sa, idx, T, osa, qb, qo)


@pytest.mark.parametrize("width", [32, 64])
def test_host_dc3_build(sa, width):
    """SA_BUILD_HOST: the suffix array comes from the host DC3 construction and
    is uploaded; the index (records, k-mer entries) then answers like any other."""
    ref = datagen.reference(30011, 77, gc=0.45, sd_cover=0.1, tandem_cover=0.05)
    ref[15000:21000] = ref[0:6000]  # long exact repeat: deep ties
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    qb, qo, _ = datagen.queries(ref, 3000, 78, m=(1, 200), frac_sampled=0.7, subs=(0, 1))
    for text in (torch.from_numpy(ref.copy()), _dev(ref)):  # host and device text
        idx = sa.sa_build(text, width=width, host_build=True)
        assert idx.width == width // 8
        assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
        assert np.array_equal(idx.kmer_table().cpu().numpy(), oracle.kmer_table(T, osa, idx.kmer_k))
        _check_search(sa, idx, T, osa, qb, qo, plain=False)
    with pytest.raises(sa.SAError) as e:
        sa.sa_build(_dev(np.frombuffer(b"ACGTN", np.uint8)), host_build=True)
    assert e.value.status == sa.SA_ERR_BASE


def test_paper_shaped_1024_base_queries(sa):
    """The paper's query length (Section V): 1024 bases, half copied exactly from
    a repeat-rich reference, half random."""
    w = datagen.paper_shaped(scale=0.1, nq=40960)
    T = oracle.normalize(w.ref)
    osa = oracle.sa_naive(T)
    idx = sa.sa_build(_dev(w.ref))
    lo, hi = _check_search(sa, idx, T, osa, w.q_bases, w.q_offsets)
    assert np.all((hi - lo)[w.sampled] >= 1)


def test_lowercase_equals_uppercase(sa):
    ref = datagen.reference(3000, 3)
    lower = np.frombuffer(ref.tobytes().lower(), dtype=np.uint8)
    a = sa.sa_build(_dev(ref)).suffix_array().cpu()
    b = sa.sa_build(_dev(lower)).suffix_array().cpu()
    assert torch.equal(a, b)
    qb, qo, _ = datagen.queries(ref, 200, 4, m=(5, 40), frac_sampled=0.8)
    idx = sa.sa_build(_dev(ref))
    r1 = sa.sa_search_batch(idx, _dev(qb), _dev(qo)).cpu()
    r2 = sa.sa_search_batch(idx, _dev(np.frombuffer(qb.tobytes().lower(), dtype=np.uint8)), _dev(qo)).cpu()
    assert torch.equal(r1, r2)


def test_host_buffers_match_device_buffers(sa):
    ref = datagen.reference(20000, 21, sd_cover=0.1)
    idx_d = sa.sa_build(_dev(ref))
    idx_h = sa.sa_build(ref)  # host text
    assert torch.equal(idx_d.suffix_array().cpu(), idx_h.suffix_array().cpu())
    qb, qo, _ = datagen.queries(ref, 3000, 22, m=(10, 200), frac_sampled=0.7, subs=(0, 1))
    r_dev = sa.sa_search_batch(idx_d, _dev(qb), _dev(qo)).cpu()
    out_host = torch.empty((qo.size - 1, sa.RESULT_FIELDS), dtype=torch.int64)
    r_host = sa.sa_search_batch(idx_d, qb, qo, out=out_host)
    assert torch.equal(r_dev, r_host)
    pinned = torch.from_numpy(qb).pin_memory()
    r_pin = sa.sa_search_batch(idx_d, pinned, torch.from_numpy(qo).pin_memory(),
                               out=torch.empty((qo.size - 1, sa.RESULT_FIELDS), dtype=torch.int64).pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(r_dev, r_pin)
    offs_d, pos_d = sa.sa_locate(idx_d, r_dev.to(DEV), 16)
    offs_h = np.zeros(qo.size, dtype=np.int64)
    pos_h = np.zeros(int(offs_d[-1].item()) + 5, dtype=np.int32)
    sa.sa_locate(idx_d, r_host, 16, out_offsets=offs_h, out_pos=pos_h)
    assert np.array_equal(offs_h, offs_d.cpu().numpy())
    assert np.array_equal(pos_h[:offs_h[-1]], pos_d.cpu().numpy()[:offs_h[-1]])


@pytest.mark.parametrize("params", [dict(key_depth=1), dict(key_depth=5), dict(key_depth=13),
                                    dict(threads_per_block=128, blocks_per_sm=4, chunk=32),
                                    dict(threads_per_block=512, blocks_per_sm=2, chunk=256),
                                    dict(threads_per_block=512, blocks_per_sm=3, key_depth=12),
                                    dict(threads_per_block=256, blocks_per_sm=6, key_depth=8, chunk=16),
                                    dict(front_probes=1), dict(front_probes=3), dict(front_probes=64)])
def test_tuning_knobs_do_not_change_results(sa, params):
    ref = datagen.reference(200_000, 31, sd_cover=0.1, tandem_cover=0.02)
    T = oracle.normalize(ref)
    idx = sa.sa_build(_dev(ref))
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    qb, qo, _ = datagen.queries(ref, 20000, 32, m=(20, 150), frac_sampled=0.8, subs=(0, 2))
    p = sa.sa_search_params(**params)
    _check_search(sa, idx, T, osa, qb, qo, plain=False, params=p)


def test_multi_reference_batch(sa):
    refs, qb, qo, qref, smp = datagen.multi_genome(scale=0.002)
    idxs = [sa.sa_build(_dev(r)) for r in refs]
    got = sa.sa_search_batch(idxs, _dev(qb), _dev(qo), q_ref=_dev(qref)).cpu().numpy()
    plain = sa.sa_search_batch_plain(idxs, _dev(qb), _dev(qo), q_ref=_dev(qref)).cpu().numpy()
    assert np.array_equal(got, plain)
    for r, ref in enumerate(refs):
        T = oracle.normalize(ref)
        osa = oracle.sa_naive(T)
        sel = np.nonzero(qref == r)[0]
        sub_qo = np.zeros(sel.size + 1, dtype=np.int64)
        np.cumsum(qo[sel + 1] - qo[sel], out=sub_qo[1:])
        sub_qb = np.concatenate([qb[qo[i]:qo[i + 1]] for i in sel]) if sel.size else np.zeros(0, np.uint8)
        lo, hi = oracle.search_batch(T, osa, sub_qb, sub_qo, threads=oracle.cpu_threads())
        assert np.array_equal(got[sel, 0], lo) and np.array_equal(got[sel, 1], hi)
    res = torch.from_numpy(got).to(DEV)
    offs, pos = sa.sa_locate(idxs, res, 5, q_ref=_dev(qref))
    offs, pos = offs.cpu().numpy(), pos.cpu().numpy()
    for q in range(0, qref.size, 37):
        osa = oracle.sa_naive(oracle.normalize(refs[qref[q]]))
        assert np.array_equal(pos[offs[q]:offs[q + 1]].astype(np.int64),
                              oracle.locate(osa, int(got[q, 0]), int(got[q, 1]), 5))


def test_errors(sa):
    with pytest.raises(sa.SAError) as e:
        sa.sa_build(_dev(np.frombuffer(b"ACGTNACGT", dtype=np.uint8)))
    assert e.value.status == sa.SA_ERR_BASE
    idx = sa.sa_build(_dev(np.frombuffer(b"ACGTACGT", dtype=np.uint8)))
    qb, qo = _batch(["ACG", "AXG"])
    with pytest.raises(sa.SAError) as e:
        sa.sa_search_batch(idx, qb, qo, out=torch.empty((2, sa.RESULT_FIELDS), dtype=torch.int64))
    assert e.value.status == sa.SA_ERR_BASE
    # on the device only the query with the bad byte is marked invalid
    got = sa.sa_search_batch(idx, _dev(qb), _dev(qo)).cpu()
    assert got[0].tolist() == [0, 2, 2, 0] and (got[1][:3] == -1).all() and got[1][3] == sa.SA_RESULT_INVALID
    got = sa.sa_search_batch_plain(idx, _dev(qb), _dev(qo)).cpu()
    assert got[0].tolist() == [0, 2, 2, 0] and (got[1][:3] == -1).all() and got[1][3] == sa.SA_RESULT_INVALID
    # out-of-range reference id
    qb, qo = _batch(["ACG", "CG"])
    got = sa.sa_search_batch([idx, idx], _dev(qb), _dev(qo), q_ref=_dev(np.array([0, 2], dtype=np.uint32))).cpu()
    assert got[0].tolist() == [0, 2, 2, 0] and (got[1][:3] == -1).all() and got[1][3] == sa.SA_RESULT_INVALID
    with pytest.raises(sa.SAError) as e:
        sa.sa_search_batch([idx, idx], qb, qo, q_ref=np.array([0, 2], dtype=np.uint32),
                           out=torch.empty((2, sa.RESULT_FIELDS), dtype=torch.int64))
    assert e.value.status == sa.SA_ERR_ARG
    # two references of different widths in one call
    idx64 = sa.sa_build(_dev(np.frombuffer(b"ACGTACGT", dtype=np.uint8)), width=64)
    with pytest.raises(sa.SAError):
        sa.sa_search_batch([idx, idx64], _dev(qb), _dev(qo), q_ref=_dev(np.array([0, 1], dtype=np.uint32)))
    # empty batch
    empty = sa.sa_search_batch(idx, _dev(qb), _dev(np.zeros(1, dtype=np.int64)))
    assert empty.shape == (0, sa.RESULT_FIELDS)


def test_save_load_roundtrip(sa, tmp_path):
    ref = datagen.reference(10000, 41, tandem_cover=0.1)
    idx = sa.sa_build(_dev(ref), width=64)
    p = str(tmp_path / "ref.sai")
    idx.save(p)
    idx2 = sa.sa_load(p)
    assert (idx2.n, idx2.width, idx2.key_depth) == (idx.n, idx.width, idx.key_depth)
    assert torch.equal(idx.suffix_array().cpu(), idx2.suffix_array().cpu())
    qb, qo, _ = datagen.queries(ref, 500, 42, m=(5, 80), frac_sampled=0.5)
    assert torch.equal(sa.sa_search_batch(idx, _dev(qb), _dev(qo)).cpu(),
                       sa.sa_search_batch(idx2, _dev(qb), _dev(qo)).cpu())
    raw = bytearray(open(p, "rb").read())
    raw[200] ^= 0xFF
    bad = str(tmp_path / "bad.sai")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(sa.SAError) as e:
        sa.sa_load(bad)
    assert e.value.status == sa.SA_ERR_FORMAT
    with pytest.raises(sa.SAError) as e:
        sa.sa_load(str(tmp_path / "missing.sai"))
    assert e.value.status == sa.SA_ERR_IO


def test_plain_small_config_full_size(sa):
    """1 Mbp iid reference, 100,000 queries of 32 bp: every query against the oracle."""
    w = datagen.plain_small()
    T = oracle.normalize(w.ref)
    idx = sa.sa_build(_dev(w.ref))
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    lo, hi = _check_search(sa, idx, T, osa, w.q_bases, w.q_offsets)
    # every exact copy occurs at least once; the brute-force count agrees on a sample
    assert (hi - lo)[w.sampled].min() >= 1
    for q in np.nonzero(w.sampled)[0][:100]:
        assert oracle.bruteforce(T, w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]])[0] == hi[q] - lo[q]


@pytest.mark.parametrize("n,k", [(11, 1), (11, 2), (700, 3), (700, 5), (20000, 6), (20000, 0)])
def test_kmer_table_and_search_by_k(sa, n, k):
    ref = datagen.reference(n, 50 + n, tandem_cover=0.1) if n > 11 else np.frombuffer(b"ACGGTACGTAC", np.uint8)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    idx = sa.sa_build(_dev(ref), kmer_k=k)
    assert idx.kmer_k == k
    if k:
        assert np.array_equal(idx.kmer_table().cpu().numpy(), oracle.kmer_table(T, osa, k))
    qb, qo, _ = datagen.queries(ref, 2000, 51, m=(1, 130), frac_sampled=0.6, subs=(0, 1))
    _check_search(sa, idx, T, osa, qb, qo, plain=False)


def test_kmer_table_full_default_k(sa):
    ref = datagen.reference(300_000, 61, sd_cover=0.1, tandem_cover=0.02)
    T = oracle.normalize(ref)
    idx = sa.sa_build(_dev(ref))
    osa = oracle.sa_naive(T)
    assert np.array_equal(idx.suffix_array().cpu().numpy().astype(np.int64), osa)
    assert idx.kmer_k == 9  # largest k with 4^k <= 3n
    assert np.array_equal(idx.kmer_table().cpu().numpy(), oracle.kmer_table(T, osa, idx.kmer_k))


def test_q_range_param_sub_batch(sa):
    """A sub-batch whose offsets start inside a larger buffer, with and without
    the caller-stated range (no host read-back); with a range that is too
    small, the queries reaching past it are marked invalid instead of read."""
    ref = datagen.reference(50_000, 71, sd_cover=0.1)
    T = oracle.normalize(ref)
    idx = sa.sa_build(_dev(ref))
    osa = oracle.sa_naive(T)
    qb, qo, _ = datagen.queries(ref, 1000, 72, m=(10, 140), frac_sampled=0.7, subs=(0, 1))
    sub = qo[100:601]
    qb_d, sub_d = _dev(qb), _dev(sub)
    p = sa.sa_search_params()
    p.flags = sa.SA_PARAM_Q_RANGE
    p.q_first, p.q_total = int(sub[0]), int(sub[-1] - sub[0])
    a = sa.sa_search_batch(idx, qb_d, sub_d, params=p).cpu()
    b = sa.sa_search_batch(idx, qb_d, sub_d).cpu()
    assert torch.equal(a, b)
    lo, hi = oracle.search_batch(T, osa, qb[sub[0]:sub[-1]], sub - sub[0])
    assert np.array_equal(a[:, 0].numpy(), lo) and np.array_equal(a[:, 1].numpy(), hi)
    p.q_total = int(sub[-1] - sub[0]) - 5
    c = sa.sa_search_batch(idx, qb_d, sub_d, params=p).cpu()
    assert (c[-1][:3] == -1).all() and c[-1][3] == sa.SA_RESULT_INVALID and torch.equal(c[:-1], a[:-1])


def _check_positions(res, offs, pos, lo, hi, osa, cap):
    """Offsets are the prefix sum of min(count, cap); query q's positions are
    SA[lo_q], SA[lo_q + 1], ... (suffix-array order)."""
    k = np.minimum(hi - lo, cap)
    assert offs[0] == 0 and np.array_equal(np.diff(offs), k)
    starts = np.repeat(lo, k)
    within = np.arange(int(k.sum())) - np.repeat(offs[:-1], k)
    assert np.array_equal(pos[:int(k.sum())].astype(np.int64), osa[starts + within])


@pytest.mark.parametrize("cap", [1, 16])
def test_search_locate_one_call(sa, cap):
    """sa_search_locate: the search hands each query's SA[lo] to the locate;
    results and positions equal the oracle's, for queries shorter and longer
    than k and repeats with many copies."""
    ref = datagen.reference(300_000, 81, sd_cover=0.1, tandem_cover=0.05)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    idx = sa.sa_build(_dev(ref))
    qb, qo, _ = datagen.queries(ref, 20000, 82, m=(1, 160), frac_sampled=0.8, subs=(0, 1))
    res, offs, pos = sa.sa_search_locate(idx, _dev(qb), _dev(qo), cap)
    lo, hi = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
    got = res.cpu().numpy()
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi) and np.array_equal(got[:, 2], hi - lo)
    _check_positions(got, offs.cpu().numpy(), pos.cpu().numpy(), lo, hi, osa, cap)


def test_search_locate_multi_reference(sa):
    refs, qb, qo, qref, _ = datagen.multi_genome(scale=0.002)
    idxs = [sa.sa_build(_dev(r)) for r in refs]
    res, offs, pos = sa.sa_search_locate(idxs, _dev(qb), _dev(qo), 8, q_ref=_dev(qref))
    got = res.cpu().numpy()
    offs = offs.cpu().numpy()
    pos = pos.cpu().numpy().astype(np.int64)
    k = np.minimum(got[:, 2], 8)
    assert offs[0] == 0 and np.array_equal(np.diff(offs), k)
    for r, ref in enumerate(refs):
        T = oracle.normalize(ref)
        osa = oracle.sa_naive(T)
        for q in np.nonzero(qref == r)[0][:400]:
            P = qb[qo[q]:qo[q + 1]]
            lo, hi = oracle.search(T, osa, P)
            assert (got[q, 0], got[q, 1]) == (lo, hi), q
            assert np.array_equal(pos[offs[q]:offs[q + 1]], osa[lo:lo + min(hi - lo, 8)]), q


def test_random_read_rate_probe(sa):
    """The device's dependent random-read rate (the bench's ceiling for the
    search's probes) is measurable and its arguments are checked."""
    r = sa.sa_random_read_rate(64 << 20, 256, 8)
    assert 1e8 < r < 1e13
    with pytest.raises(sa.SAError):
        sa.sa_random_read_rate(64 << 20, 33, 8)


def _reverse_complement(qb, qo):
    """Each query's reverse complement (A<->T, C<->G, order reversed), in place of it."""
    table = np.arange(256, dtype=np.uint8)
    for a, b in (("A", "T"), ("C", "G"), ("a", "t"), ("c", "g")):
        table[ord(a)], table[ord(b)] = ord(b), ord(a)
    out = np.empty_like(qb)
    for q in range(qo.size - 1):
        out[qo[q]:qo[q + 1]] = table[qb[qo[q]:qo[q + 1]][::-1]]
    return out


def test_reverse_complement_flag(sa):
    """With SA_PARAM_REVERSE_COMPLEMENT every query's reverse complement is
    searched: the results equal the oracle's on the reverse-complemented
    queries, and searching the reverse complements of sampled queries with the
    flag finds the sampled copies again."""
    ref = datagen.reference(200_000, 91, sd_cover=0.1, tandem_cover=0.05)
    T = oracle.normalize(ref)
    osa = oracle.sa_naive(T)
    idx = sa.sa_build(_dev(ref))
    qb, qo, smp = datagen.queries(ref, 5000, 92, m=(1, 200), frac_sampled=0.7, subs=(0, 1))
    rc = _reverse_complement(qb, qo)
    p = sa.sa_search_params()
    p.flags = sa.SA_PARAM_REVERSE_COMPLEMENT
    for fp in (0, 1, 64):  # the first pass alone, and with the persistent pass
        p.front_probes = fp
        got = sa.sa_search_batch(idx, _dev(qb), _dev(qo), params=p).cpu().numpy()
        lo, hi = oracle.search_batch(T, osa, rc, qo, threads=oracle.cpu_threads())
        assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi)
        back = sa.sa_search_batch(idx, _dev(rc), _dev(qo), params=p).cpu().numpy()
        lo2, hi2 = oracle.search_batch(T, osa, qb, qo, threads=oracle.cpu_threads())
        assert np.array_equal(back[:, 0], lo2) and np.array_equal(back[:, 1], hi2)
        assert (back[smp, 2] >= 1).sum() > 0
