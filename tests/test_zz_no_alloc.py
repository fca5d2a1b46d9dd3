"""sa_locate_noalloc: locate for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- their device memory is owned up front
by another allocator, or they run a latency-critical loop where an allocation
could block or fail.  sa_locate_noalloc keeps its scan scratch in a static
device array instead.  This test calls it through the C ABI twice in a row
(the array keeps the previous call's contents), requires both results to
equal sa_locate's exactly, the tolerance of every integer test here, and
checks around each call that nothing was allocated: the library's scratch
pool, torch's allocator and the device's free memory are unchanged.  The file
is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    from paper_1303_3692_gb300 import build_lib, sa as sa_mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    sa_mod.lib()
    return sa_mod


def _noalloc(sa, idxs, res, cap, q_ref, offs, pos, capacity):
    arr = (ctypes.c_void_p * len(idxs))(*[i.handle.value for i in idxs])
    return sa.lib().sa_locate_noalloc(arr, len(idxs), None if q_ref is None else q_ref.data_ptr(), res.data_ptr(),
                                      res.shape[0], cap, offs.data_ptr(),
                                      None if pos is None else pos.data_ptr(), capacity,
                                      torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("width", [32, 64])
def test_noalloc_matches_sa_locate_twice(sa, width):
    refs, qb, qo, qref, _ = datagen.multi_genome(scale=0.002)
    idxs = [sa.sa_build(torch.from_numpy(r).cuda(), width=width) for r in refs]
    qb_d, qo_d, qref_d = (torch.from_numpy(x).cuda() for x in (qb, qo, qref))
    res = sa.sa_search_batch(idxs, qb_d, qo_d, q_ref=qref_d)
    n_q = res.shape[0]
    assert n_q > 4096 * 2  # several scan tiles
    for cap in (3, 64):
        offs_ref, pos_ref = sa.sa_locate(idxs, res, cap, q_ref=qref_d)
        total = int(offs_ref[-1].item())
        dt = torch.int32 if width == 32 else torch.int64
        for call in range(2):
            offs = torch.full((n_q + 1,), -7, dtype=torch.int64, device="cuda")
            pos = torch.full((max(total, 1),), -7, dtype=dt, device="cuda")
            # the call must allocate nothing: the library's scratch pool sees no
            # allocation (its high-water mark stays 0 after a reset), torch's
            # allocator and the device's free memory do not change
            torch.cuda.synchronize()
            before = sa.sa_scratch_info(reset_high=True)
            torch_before = torch.cuda.memory_allocated()
            free_before = torch.cuda.mem_get_info()[0]
            assert _noalloc(sa, idxs, res, cap, qref_d, offs, pos, total) == sa.SA_OK
            torch.cuda.synchronize()
            after = sa.sa_scratch_info()
            assert after["used_high"] == 0 and after["used"] == 0, (before, after)
            assert after["reserved"] == before["reserved"]
            assert torch.cuda.memory_allocated() == torch_before
            assert torch.cuda.mem_get_info()[0] == free_before
            assert torch.equal(offs, offs_ref), (cap, call)
            assert torch.equal(pos[:total], pos_ref[:total]), (cap, call)


def test_noalloc_rejects_too_many_queries_and_host_buffers(sa):
    ref = datagen.reference(5000, 3)
    idx = sa.sa_build(torch.from_numpy(ref).cuda())
    res = torch.zeros((4, sa.RESULT_FIELDS), dtype=torch.int64, device="cuda")
    offs = torch.zeros(5, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * 1)(idx.handle.value)
    L = sa.lib()
    big = sa.SA_LOCATE_NOALLOC_MAX_QUERIES + 1
    assert L.sa_locate_noalloc(arr, 1, None, res.data_ptr(), big, 4, offs.data_ptr(), None, 0, None) == \
        sa.SA_ERR_CAPACITY
    host_offs = np.zeros(5, dtype=np.int64)
    assert L.sa_locate_noalloc(arr, 1, None, res.data_ptr(), 4, 4, host_offs.ctypes.data, None, 0, None) == \
        sa.SA_ERR_ARG
