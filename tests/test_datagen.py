"""The seeded workload generators: determinism, sizes and recipe statistics."""
import numpy as np

import oracle
from paper_1303_3692_gb300 import datagen


def test_deterministic():
    a = datagen.reference(20000, 5, gc=0.4, sd_cover=0.1, tandem_cover=0.02)
    b = datagen.reference(20000, 5, gc=0.4, sd_cover=0.1, tandem_cover=0.02)
    assert np.array_equal(a, b)
    qa = datagen.queries(a, 100, 3, m=(20, 50), frac_sampled=0.5, subs=(0, 2))
    qb = datagen.queries(a, 100, 3, m=(20, 50), frac_sampled=0.5, subs=(0, 2))
    for x, y in zip(qa, qb):
        assert np.array_equal(x, y)


def test_gc_content():
    for gc in (0.38, 0.5, 0.62):
        r = datagen.reference(400_000, 11, gc=gc)
        frac = np.isin(r, np.frombuffer(b"CG", dtype=np.uint8)).mean()
        assert abs(frac - gc) < 0.005


def test_alphabet_and_lengths():
    r = datagen.reference(50_000, 2, sd_cover=0.1, tandem_cover=0.02, family_cover=0.3)
    assert r.size == 50_000
    assert set(np.unique(r).tolist()) <= set(b"ACGT")
    qb, qo, smp = datagen.queries(r, 1000, 4, m=(20, 250), frac_sampled=0.7)
    lens = np.diff(qo)
    assert lens.min() >= 20 and lens.max() <= 250 and qo[-1] == qb.size
    assert 0.6 < smp.mean() < 0.8


def test_exact_sampled_queries_occur():
    r = datagen.reference(30_000, 8, sd_cover=0.1)
    qb, qo, smp = datagen.queries(r, 200, 9, m=32, frac_sampled=0.5, subs=(0, 0))
    T = oracle.normalize(r)
    for q in np.nonzero(smp)[0][:50]:
        assert oracle.bruteforce(T, qb[qo[q]:qo[q + 1]])[0] >= 1


def test_substitutions_bounded():
    # a sampled query with up to 2 substitutions is within Hamming distance 2 of some window
    r = datagen.reference(5_000, 12)
    qb, qo, smp = datagen.queries(r, 60, 13, m=40, frac_sampled=1.0, subs=(2, 2))
    win = np.lib.stride_tricks.sliding_window_view(r, 40)
    for q in range(60):
        d = (win != qb[qo[q]:qo[q + 1]][None, :]).sum(axis=1).min()
        assert d == 2


def test_multi_genome_shapes():
    refs, qb, qo, qref, smp = datagen.multi_genome(scale=0.0005)
    assert len(refs) == 4 and qo.size == qref.size + 1 and qo[-1] == qb.size
    T = [oracle.normalize(x) for x in refs]
    for q in np.nonzero(smp)[0][:20]:
        assert oracle.bruteforce(T[qref[q]], qb[qo[q]:qo[q + 1]])[0] >= 1


def test_paper_shaped_shape():
    w = datagen.paper_shaped(scale=0.002)
    assert w.ref.size == 20_000 and np.all(np.diff(w.q_offsets) == 1024)
    T = oracle.normalize(w.ref)
    for q in np.nonzero(w.sampled)[0][:10]:
        assert oracle.bruteforce(T, w.q_bases[w.q_offsets[q]:w.q_offsets[q + 1]])[0] >= 1
    assert 0.3 < w.sampled.mean() < 0.7
