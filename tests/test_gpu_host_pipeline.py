"""Host-memory batches large enough for the chunked path (2^21 queries or
more: uploads, kernels and downloads of successive chunks overlap on two
library streams) give exactly the results of the same batch in device memory:
results, located offsets and positions, and the call's status."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu

N_Q = 2_500_000


@pytest.fixture(scope="module")
def env():
    from paper_1303_3692_gb300 import build_lib
    from paper_1303_3692_gb300 import sa as sa_mod

    build_lib.build()
    refs = [datagen.reference(n, 700 + i, sd_cover=0.1, tandem_cover=0.03) for i, n in enumerate((150_000, 90_000))]
    idxs = [sa_mod.sa_build(torch.from_numpy(r).cuda()) for r in refs]
    qb, qo, _ = datagen.queries(refs[0], N_Q, 710, m=(10, 150), frac_sampled=0.8, subs=(0, 1))
    return sa_mod, refs, idxs, qb, qo


def _device(sa, refs, qb, qo, cap=None, q_ref=None):
    args = (refs, torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda())
    kw = {} if q_ref is None else {"q_ref": torch.from_numpy(q_ref).cuda()}
    if cap is None:
        return sa.sa_search_batch(*args, **kw).cpu().numpy()
    r, o, p = sa.sa_search_locate(*args, cap, **kw)
    return r.cpu().numpy(), o.cpu().numpy(), p.cpu().numpy()


@pytest.mark.parametrize("pinned", [False, True])
def test_host_search_equals_device(env, pinned):
    sa, refs, idxs, qb, qo = env
    want = _device(sa, idxs[0], qb, qo)
    qb_h = torch.from_numpy(qb).pin_memory() if pinned else qb
    qo_h = torch.from_numpy(qo).pin_memory() if pinned else qo
    out = np.empty((N_Q, sa.RESULT_FIELDS), dtype=np.int64)
    sa.sa_search_batch(idxs[0], qb_h, qo_h, out=out)
    assert np.array_equal(out, want)
    # and a sample against the oracle
    T = oracle.normalize(refs[0])
    osa = oracle.sa_naive(T)
    pick = np.arange(0, N_Q, 997)
    for q in pick[:400]:
        lo, hi = oracle.search(T, osa, qb[qo[q]:qo[q + 1]])
        assert out[q, 0] == lo and out[q, 1] == hi


@pytest.mark.parametrize("pinned", [False, True])
def test_host_search_locate_equals_device(env, pinned):
    """Pageable buffers get the positions after the last chunk; pinned ones
    receive each chunk's positions as soon as its locate is done."""
    sa, refs, idxs, qb, qo = env
    cap = 8
    q_ref = (np.arange(N_Q) % 3 == 0).astype(np.uint32)  # two references in one call
    want_r, want_o, want_p = _device(sa, idxs, qb, qo, cap, q_ref)
    total = int(want_o[-1])

    def host(shape, dtype):
        t = torch.empty(shape, dtype=dtype)
        return t.pin_memory() if pinned else t

    res = host((N_Q, sa.RESULT_FIELDS), torch.int64)
    offs = host(N_Q + 1, torch.int64)
    pos = host(total, torch.int32)
    pos.fill_(-7)
    qb_h = torch.from_numpy(qb).pin_memory() if pinned else qb
    qo_h = torch.from_numpy(qo).pin_memory() if pinned else qo
    sa.sa_search_locate(idxs, qb_h, qo_h, cap, q_ref=q_ref, out=res, out_offsets=offs, out_pos=pos, capacity=total)
    assert np.array_equal(res.numpy(), want_r)
    assert np.array_equal(offs.numpy(), want_o)
    assert np.array_equal(pos.numpy(), want_p[:total])
    # too small a positions buffer: the positions that fit, nothing past the
    # capacity, and SA_ERR_CAPACITY
    pos.fill_(-7)
    with pytest.raises(sa.SAError) as e:
        sa.sa_search_locate(idxs, qb_h, qo_h, cap, q_ref=q_ref, out=res, out_offsets=offs, out_pos=pos,
                            capacity=total - 5)
    assert e.value.status == sa.SA_ERR_CAPACITY
    p = pos.numpy()
    assert np.array_equal(offs.numpy(), want_o) and np.array_equal(p[:total - 5], want_p[:total - 5])
    assert (p[total - 5:] == -7).all()


def test_host_pipeline_reports_bad_bases(env):
    sa, refs, idxs, qb, qo = env
    bad = qb.copy()
    q = N_Q - 3  # in the last chunk
    bad[qo[q]] = ord("N")
    out = np.empty((N_Q, sa.RESULT_FIELDS), dtype=np.int64)
    with pytest.raises(sa.SAError) as e:
        sa.sa_search_batch(idxs[0], bad, qo, out=out)
    assert e.value.status == sa.SA_ERR_BASE
    assert out[q, 3] == sa.SA_RESULT_INVALID and (out[q, :3] == -1).all()
    assert out[q - 1, 3] != sa.SA_RESULT_INVALID


def test_host_pipeline_kmer_order(env):
    """The chunked host path in k-mer order (forced here; the library takes it
    by itself only for indexes above 48 GB), with locate: every chunk's
    k-mer-ordered list and located positions give the device path's results."""
    sa, refs, idxs, qb, qo = env
    cap = 8
    p = sa.sa_search_params(flags=sa.SA_PARAM_KMER_ORDER)
    want_r, want_o, want_p = _device(sa, idxs[0], qb, qo, cap)
    total = int(want_o[-1])
    res = torch.empty((N_Q, sa.RESULT_FIELDS), dtype=torch.int64).pin_memory()
    offs = torch.empty(N_Q + 1, dtype=torch.int64).pin_memory()
    pos = torch.empty(total, dtype=torch.int32).pin_memory()
    sa.sa_search_locate(idxs[0], torch.from_numpy(qb).pin_memory(), torch.from_numpy(qo).pin_memory(), cap,
                        out=res, out_offsets=offs, out_pos=pos, capacity=total, params=p)
    assert np.array_equal(res.numpy(), want_r)
    assert np.array_equal(offs.numpy(), want_o)
    assert np.array_equal(pos.numpy(), want_p[:total])
