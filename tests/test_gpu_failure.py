"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes (an
mbarrier no thread arrives at) gives up after its limit, reports LECO_ERR_TIMEOUT through the status
path the scan and pack kernels use, and the device stays usable for the next calls."""
import time

import pytest

import workloads as W
from gpu_util import from_dev, to_dev

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


@pytest.mark.parametrize("limit_us", [1_000, 20_000])
def test_bounded_wait_gives_up_and_reports(lc, limit_us):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert lc.leco_selftest_wait_timeout(limit_us) == lc.LECO_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= limit_us * 1e-6  # it waited its full limit, then returned
    v = W.cfg1(200_000)  # the context is intact: encode, decode and sync still work
    col = lc.leco_encode(to_dev(v), lc.fixed(1024), 1)
    out = torch.empty(len(v), dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == v).all()
    assert lc.leco_sync(col) == lc.LECO_OK
