"""The error path of the library's device work (no fault is caused: a wait is
made to expire through a test flag, and bad inputs are plain data).

* A bounded device wait that runs out reaches the caller as SA_ERR_TIMEOUT:
  returned by the call when its output is host memory, and written to the
  caller's device status word when it is device memory.  The context stays
  usable: the next call gives the oracle's results.
* The device status word reports SA_OK, SA_ERR_BASE (a byte that is not a
  base), SA_ERR_ARG (a reference id out of range) and, for the one-call search
  and locate, SA_ERR_CAPACITY (a positions buffer too small).
* sa_locate returns SA_ERR_CAPACITY when the total is read back to the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    from paper_1303_3692_gb300 import build_lib
    from paper_1303_3692_gb300 import sa as sa_mod

    build_lib.build()
    return sa_mod


@pytest.fixture(scope="module")
def case(sa):
    ref = datagen.reference(40_000, 201, sd_cover=0.1, tandem_cover=0.05)
    qb, qo, _ = datagen.queries(ref, 3000, 202, m=(10, 160), frac_sampled=0.7, subs=(0, 1))
    T = oracle.normalize(ref)
    lo, hi = oracle.rank_count_batch(T, qb, qo, threads=oracle.cpu_threads())
    return ref, qb, qo, lo, hi


def _status_word():
    return torch.full((1,), 12345, dtype=torch.int32, device="cuda")


def test_expired_wait_reports_timeout(sa, case):
    ref, qb, qo, lo, hi = case
    # no k-mer table: every query goes through the persistent kernel, whose
    # key-table wait is the one the flag makes expire
    idx = sa.sa_build(torch.from_numpy(ref).cuda(), kmer_k=0)
    qb_d, qo_d = torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda()
    st = _status_word()
    p = sa.sa_search_params(flags=sa.SA_PARAM_EXPIRE_WAITS, device_status=st.data_ptr())
    out = torch.empty((qo.size - 1, sa.RESULT_FIELDS), dtype=torch.int64, device="cuda")
    sa.sa_search_batch(idx, qb_d, qo_d, out=out, params=p)  # device output: queued, returns OK
    torch.cuda.synchronize()
    assert int(st.item()) == sa.SA_ERR_TIMEOUT
    with pytest.raises(sa.SAError) as e:  # host output: the call returns the status itself
        sa.sa_search_batch(idx, qb, qo, out=np.empty((qo.size - 1, sa.RESULT_FIELDS), dtype=np.int64),
                           params=sa.sa_search_params(flags=sa.SA_PARAM_EXPIRE_WAITS))
    assert e.value.status == sa.SA_ERR_TIMEOUT
    # the context is still usable and the next call is right
    st2 = _status_word()
    got = sa.sa_search_batch(idx, qb_d, qo_d, params=sa.sa_search_params(device_status=st2.data_ptr()))
    torch.cuda.synchronize()
    assert int(st2.item()) == sa.SA_OK
    got = got.cpu().numpy()
    assert np.array_equal(got[:, 0], lo) and np.array_equal(got[:, 1], hi)


def test_status_word_codes(sa, case):
    ref, qb, qo, lo, hi = case
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    idx2 = sa.sa_build(torch.from_numpy(ref[:20_000].copy()).cuda())
    n_q = qo.size - 1

    def run(bases, q_ref=None, refs=idx):
        st = _status_word()
        res = sa.sa_search_batch(refs, torch.from_numpy(bases).cuda(), torch.from_numpy(qo).cuda(),
                                 q_ref=None if q_ref is None else torch.from_numpy(q_ref).cuda(),
                                 params=sa.sa_search_params(device_status=st.data_ptr()))
        torch.cuda.synchronize()
        return int(st.item()), res.cpu().numpy()

    code, got = run(qb)
    assert code == sa.SA_OK and np.array_equal(got[:, 0], lo)
    bad = qb.copy()
    bad[qo[5] + 1] = ord("N")
    code, got = run(bad)
    assert code == sa.SA_ERR_BASE and got[5, 0] == -1 and np.array_equal(got[6:, 0], lo[6:])
    q_ref = np.zeros(n_q, dtype=np.uint32)
    q_ref[7] = 2  # only two references in the call
    code, got = run(qb, q_ref, [idx, idx2])
    assert code == sa.SA_ERR_ARG and got[7, 0] == -1 and got[8, 0] == lo[8]


def test_capacity_errors(sa, case):
    ref, qb, qo, lo, hi = case
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    n_q = qo.size - 1
    qb_d, qo_d = torch.from_numpy(qb).cuda(), torch.from_numpy(qo).cuda()
    cap = 8
    need = int(np.minimum(hi - lo, cap).sum())
    assert need > 10
    # one call, device outputs, status word: too small -> SA_ERR_CAPACITY, exact size -> SA_OK
    for capacity, want in ((need - 1, sa.SA_ERR_CAPACITY), (need, sa.SA_OK)):
        st = _status_word()
        pos = torch.empty(need, dtype=torch.int32, device="cuda")
        res, offs, pos = sa.sa_search_locate(idx, qb_d, qo_d, cap, out_pos=pos, capacity=capacity,
                                             params=sa.sa_search_params(device_status=st.data_ptr()))
        torch.cuda.synchronize()
        assert int(st.item()) == want
        assert int(offs[-1].item()) == need
        # each result carries SA_RESULT_TRUNCATED exactly when count > cap
        r = res.cpu().numpy()
        assert np.array_equal(r[:, 3], np.where(r[:, 2] > cap, sa.SA_RESULT_TRUNCATED, 0))
    # separate locate with host offsets: the total is read back, so the call reports it
    res = sa.sa_search_batch(idx, qb_d, qo_d)
    offs_h = np.empty(n_q + 1, dtype=np.int64)
    pos_d = torch.empty(need, dtype=torch.int32, device="cuda")
    with pytest.raises(sa.SAError) as e:
        sa.sa_locate(idx, res, cap, out_offsets=offs_h, out_pos=pos_d, capacity=need - 1)
    assert e.value.status == sa.SA_ERR_CAPACITY and offs_h[-1] == need
    sa.sa_locate(idx, res, cap, out_offsets=offs_h, out_pos=pos_d, capacity=need)
