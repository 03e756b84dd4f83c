"""The allocation-free fixed-partition encode (leco_encode_fixed_noalloc) against leco_encode.

That entry point serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or paths that cannot take an allocation's synchronization); its scratch is a fixed
__device__ array shared by all calls. Here two calls in a row, on different inputs, must give the
records and residual words of the allocating entry point byte for byte, the second call must leave
the device's free memory unchanged, and sizes past the fixed scratch must be refused. This file is
collected last so a failure here comes after every other test.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_15374_gb300 as pkg

    pkg.build()
    from paper_2306_15374_gb300 import leco

    return leco


def _via_allocating(lc, v, L, model, bits):
    col = lc.leco_encode(to_dev(v, bits), lc.fixed(L), model)
    rec, words, _ = lc.leco_column_export(col)
    col.free()
    return rec, words


def test_noalloc_matches_allocating_encode_twice(lc):
    import torch

    cases = [(W.cfg1(1_000_000), 1024, 1, 64),
             (W.timestamps_u32(300_001, seed=3), 4096, 0, 32),
             (W.adversarial_u64(70_001, seed=4), 33, 1, 64)]
    for v, L, model, bits in cases:
        want_rec, want_words = _via_allocating(lc, v, L, model, bits)
        m = (len(v) + L - 1) // L
        rec = torch.zeros(4 * max(m, 1), dtype=torch.int64, device="cuda")
        words = torch.full((len(want_words) // 8 + 64,), -1, dtype=torch.int64, device="cuda")
        dv = to_dev(v, bits)
        torch.cuda.synchronize()
        for call in range(2):  # two calls in a row share the scratch array
            free_before = torch.cuda.mem_get_info()[0]
            nw = lc.leco_encode_fixed_noalloc(dv, L, rec, words, model)
            torch.cuda.synchronize()
            if call == 1:  # the first call may load kernels; the second must take no device memory
                assert torch.cuda.mem_get_info()[0] == free_before
            assert nw * 8 == len(want_words)
            assert rec.cpu().numpy().tobytes()[: 32 * m] == want_rec
            assert words.cpu().numpy().tobytes()[: 8 * nw] == want_words


def test_noalloc_refuses_what_does_not_fit(lc):
    import torch

    v = W.cfg1(100_000)
    rec = torch.zeros(4 * 100, dtype=torch.int64, device="cuda")
    small = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(lc.LecoError) as e:
        lc.leco_encode_fixed_noalloc(to_dev(v), 1024, rec, small)
    assert e.value.status == lc.LECO_ERR_INVALID_ARG and e.value.nwords > 4
    # more partitions than the fixed scratch holds (2^18)
    big = torch.zeros((1 << 18) + 1, dtype=torch.int64, device="cuda")
    big_rec = torch.zeros(4 * big.numel(), dtype=torch.int64, device="cuda")
    with pytest.raises(lc.LecoError) as e:
        lc.leco_encode_fixed_noalloc(big, 1, big_rec, small)
    assert e.value.status == lc.LECO_ERR_INVALID_ARG
    # a records buffer too small for ceil(n / L) records is refused before the call
    with pytest.raises(ValueError):
        lc.leco_encode_fixed_noalloc(big, 1, torch.zeros(1, dtype=torch.int64, device="cuda"), small)
