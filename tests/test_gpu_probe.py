"""The execution-unit probes run on the device and return plausible rates: every kind positive, the
32-bit integer units well ahead of the binary64 ones (GB300's FP64 rate is a small fraction of its
integer rate), and a rate below what the device's clock and SM count allow for 128 lanes per SM."""
import pytest

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


def test_probe_rates_are_plausible(lc):
    import torch

    props = torch.cuda.get_device_properties(0)
    rates = {k: lc.leco_probe_throughput(k) for k in lc.PROBE_KINDS}
    assert all(r > 0 for r in rates.values()), rates
    assert rates[0] > 4 * rates[3], rates
    # no SM issues more than 4 warps x 32 lanes of simple integer work per clock (2.2 GHz is above
    # any clock of the part)
    assert rates[0] < props.multi_processor_count * 128 * 2.2e9, rates
