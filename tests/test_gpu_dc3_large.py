"""The GPU DC3 construction at the 3.1 Gbp size: the int64 suffix array of the
human-sized synthetic reference passes the oracle's verifier (a permutation of
[0, n) whose adjacent suffixes strictly increase is the unique suffix array),
and prefix doubling builds the same array.  Both build times are printed."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1303_3692_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_dc3_gpu_3100mbp():
    from paper_1303_3692_gb300 import build_lib
    from paper_1303_3692_gb300 import sa

    build_lib.build()
    torch.cuda.empty_cache()
    ref = datagen.reference(3_100_000_000, datagen.SEED0 + 4, gc=0.41, family_cover=0.45, tandem_cover=0.03)
    d = torch.from_numpy(ref).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dc3 = sa.sa_suffix_array_gpu(d, width=64, dc3=True)
    t_dc3 = time.perf_counter() - t0
    t0 = time.perf_counter()
    pd = sa.sa_suffix_array_gpu(d, width=64)
    t_pd = time.perf_counter() - t0
    print(f"3.1 Gbp suffix array: DC3 {t_dc3:.2f} s, prefix doubling {t_pd:.2f} s")
    assert torch.equal(dc3, pd)
    del pd, d
    torch.cuda.empty_cache()
    T = oracle.normalize(ref)
    assert oracle.verify_sa(T, dc3.cpu().numpy(), threads=oracle.cpu_threads()) == (0, -1)
