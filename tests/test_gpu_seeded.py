"""Seeded variable partitioning (LECO_PART_VAR_SEEDED: each chunk's split grows from its smoothest
point in both directions) on the GPU against the CPU oracle: identical boundaries after split and
round-synchronous merge, identical columns, exact decode and lookups."""
import numpy as np
import pytest

import oracle
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
    oracle.build()
    from paper_2306_15374_gb300 import leco

    return leco


CASES = [
    ("piecewise_300k", lambda: W.piecewise_linear(300_000, segments=10, mean_len=30_000, seed=4), 64),
    ("timestamps_200k", lambda: W.timestamps_u32(200_000, seed=5), 32),
    ("adversarial_20k", lambda: W.adversarial_u64(20_000, seed=3), 64),
    ("sine_150k", lambda: W.sine_mixture(150_000, seed=6), 64),
    ("random_70k", lambda: W.random_u64(70_001, 7), 64),
    ("line_140k", lambda: (np.arange(140_000, dtype=np.uint64) * np.uint64(977) + np.uint64(5)), 64),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("tau", [0.0, 0.03, 0.1])
def test_seeded_partition_matches_oracle(lc, case, tau):
    import torch

    _, gen, bits = case
    v = gen()
    starts = torch.empty(len(v) + 1, dtype=torch.int64, device="cuda")
    for model in (1, 0):
        m = lc.leco_var_partition(to_dev(v, bits), starts, lc.variable(tau, seeded=True), model)
        got = from_dev(starts)[: m + 1]
        expect = oracle.var_partition(v, tau, model, variant="round", seeded=True)
        assert got.tolist() == expect.tolist(), model


def test_seeded_partition_with_a_small_cap(lc):
    import torch

    v = W.piecewise_linear(150_000, segments=8, mean_len=20_000, seed=8)
    starts = torch.empty(len(v) + 1, dtype=torch.int64, device="cuda")
    m = lc.leco_var_partition(to_dev(v), starts, lc.variable(0.1, cap=300, seeded=True), 1)
    got = from_dev(starts)[: m + 1]
    expect = oracle.var_partition(v, 0.1, 1, variant="round", cap=300, seeded=True)
    assert got.tolist() == expect.tolist()
    assert np.diff(got.astype(np.int64)).max() <= 300


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_seeded_column_parity(lc, case):
    import torch

    _, gen, bits = case
    v = gen()
    n = len(v)
    for model in (1, 2):
        col = lc.leco_encode(to_dev(v, bits), lc.variable(0.1, seeded=True), model)
        assert col.stats()["kind"] == lc.LECO_PART_VAR
        rec_b, words_b, starts_b = lc.leco_column_export(col)
        st = oracle.var_partition(v, 0.1, 1, variant="round", seeded=True)
        rec, words = oracle.encode(v, st, model)
        assert starts_b == st.tobytes() and rec_b == rec.tobytes() and words_b == words.tobytes()
        tdt = torch.int32 if bits == 32 else torch.int64
        out = torch.empty(n, dtype=tdt, device="cuda")
        lc.leco_decode_all(col, out)
        assert (from_dev(out) == v).all()
        idx = W.uniform_indices(20_000, n, seed=2)
        o2 = torch.empty(len(idx), dtype=tdt, device="cuda")
        lc.leco_random_access(col, to_dev(idx), o2)
        assert (from_dev(o2) == v[idx]).all()
