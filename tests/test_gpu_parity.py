"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Integer work is bit-exact: decoded values, lookups, sums, and for the encoder the records and the
residual words byte for byte. Sizes span several tiles and ragged tails; the full-size cases run
the 200M-value columns in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import exact_sum, from_dev, make_blob, parse_blob, to_dev

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


def _cases():
    yield "cfg1_1M_L1024", W.cfg1(), 1024, 1, 64
    yield "linear_ragged_L4096", W.linear_noise(300_007, 1 << 20, 53, 4096, seed=3), 4096, 1, 64
    yield "normal_L4096", W.sorted_normal(200_003, 2.0 ** 40, 2.0 ** 36, seed=4), 4096, 1, 64
    yield "lognormal_L4096", W.sorted_lognormal(200_003, 1e9, 2.0, seed=5), 4096, 1, 64
    yield "adversarial_L37", W.adversarial_u64(50_001, seed=6), 37, 1, 64
    yield "adversarial_const_L1000", W.adversarial_u64(20_000, seed=7), 1000, 0, 64
    yield "random_L1", W.random_u64(5_000, 8), 1, 1, 64
    yield "random_L5000_gt_n", W.random_u64(3_333, 9), 5000, 1, 64
    yield "runs_L256", W.runs(100_000, 300, seed=10), 256, 1, 64
    yield "sorted63_L100", np.sort(W.random_u64(80_000, 11, bits=63)), 100, 1, 64
    yield "for_L1024", W.cfg1(100_000), 1024, 0, 64
    yield "ts_u32_L512", W.timestamps_u32(150_001, seed=12), 512, 1, 32
    yield "ts_u32_const_L33", W.timestamps_u32(70_001, seed=13), 33, 0, 32
    # model ranges that cross zero as signed numbers (64-bit: values on both sides of 2^64 = 0)
    # and 32-bit ranges whose residual band dips below zero (clamped bounds)
    yield "wrap_zero_u64_L512", W.linear_noise(100_003, -(1 << 30), 21_000, 4096, seed=14), 512, 1, 64
    yield "low_u64_L1024", W.random_u64(60_001, 15, bits=20), 1024, 1, 64
    yield "low_u32_L1024", W.random_u64(60_001, 16, bits=20), 1024, 1, 32
    # ramps falling to 0 and staying there: the fitted line dips below zero (negative predictions)
    # on a fine grid (s > 32), so the 32-bit decode must floor with an arithmetic shift; partitions
    # of 32, 64 and 96 values reach the one-group, the paired and the mixed decode loops
    def ramp(period, top, step, seed):
        x = np.arange(70_001) % period
        return np.maximum(0, top - step * x).astype(np.uint64) + W.random_u64(70_001, seed, bits=2)
    yield "neg_pred_u32_L32", ramp(32, 100, 8, 17), 32, 1, 32
    yield "neg_pred_u32_L96", ramp(96, 300, 8, 18), 96, 1, 32
    yield "neg_pred_u64_L64", ramp(64, 200, 8, 19), 64, 1, 64


CASES = list(_cases())
IDS = [c[0] for c in CASES]


def _gpu_encode(lc, v, L, model, bits):
    return lc.leco_encode(to_dev(v, bits), lc.fixed(L), model)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_encode_is_byte_identical_to_oracle(lc, case):
    _, v, L, model, bits = case
    col = _gpu_encode(lc, v, L, model, bits)
    rec_b, words_b, _ = lc.leco_column_export(col)
    rec, words = oracle.encode_fixed(v, L, model)
    assert rec_b == rec.tobytes()
    assert words_b == words.tobytes()
    st = col.stats()
    assert st["partitions"] == len(rec) and st["residual_bytes"] == 8 * len(words)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_decode_of_oracle_column(lc, case):
    import torch

    _, v, L, model, bits = case
    rec, words = oracle.encode_fixed(v, L, model)
    col = lc.leco_deserialize(make_blob(rec, words, len(v), L, 0 if bits == 32 else 1, 0, model))
    out = torch.empty(len(v), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    got = from_dev(out)
    assert (got == oracle.decode(rec, words, len(v), bits)).all()
    assert (got == v).all()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_decode_range_lookup_filter(lc, case):
    import torch

    _, v, L, model, bits = case
    n = len(v)
    col = _gpu_encode(lc, v, L, model, bits)
    tdt = torch.int32 if bits == 32 else torch.int64
    g = W.rng(99)
    ranges = [(0, n), (0, 0), (n, 0), (n - 1, 1), (0, 1)]
    for _ in range(6):
        a, b = sorted(int(x) for x in g.integers(0, n + 1, size=2))
        ranges.append((a, b - a))
    for a, cnt in ranges:
        out = torch.empty(max(cnt, 1), dtype=tdt, device="cuda")
        lc.leco_decode_range(col, a, cnt, out)
        assert (from_dev(out)[:cnt] == v[a:a + cnt]).all()
    idx = np.concatenate([W.uniform_indices(20_000, n, seed=1), np.array([0, n - 1, 0, n - 1], np.uint64)])
    out = torch.empty(len(idx), dtype=tdt, device="cuda")
    lc.leco_random_access(col, to_dev(idx), out)
    assert (from_dev(out) == v[idx]).all()
    assert lc.leco_sync(col) == lc.LECO_OK
    rec, words = oracle.encode_fixed(v, L, model)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    top = (1 << 64) - 1
    bounds = [W.filter_bounds(v), (0, top), (5, 4), (int(v[n // 2]), int(v[n // 2])),
              (0, 1 << 20), (top - (1 << 20), top), (1 << 40, 1 << 50), (1 << 31, (1 << 32) - 1)]
    for lo, hi in bounds:
        want = oracle.filter_sum(rec, words, n, lo, hi, bits)
        assert want == exact_sum(v, lo, hi)
        for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL, 3):
            lc.leco_filter_sum(col, lo, hi, res, flags=flags)
            r = from_dev(res)
            assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == want, flags


def test_out_of_range_lookup_sets_status(lc):
    import torch

    v = W.cfg1(10_000)
    col = _gpu_encode(lc, v, 1024, 1, 64)
    idx = np.array([5, 10_000, 1 << 63, 9_999, (1 << 64) - 1], dtype=np.uint64)
    out = torch.full((5,), 7, dtype=torch.int64, device="cuda")
    lc.leco_random_access(col, to_dev(idx), out)
    got = from_dev(out)
    assert got[0] == v[5] and got[3] == v[9999] and got[1] == 0 and got[2] == 0 and got[4] == 0
    assert lc.leco_sync(col) == lc.LECO_ERR_INDEX_RANGE
    assert lc.leco_sync(col) == lc.LECO_OK  # cleared


def test_non_exact_records_use_binary64(lc):
    """Records with arbitrary theta (exact flag clear, or set but false) decode by the binary64
    definition, exactly like the oracle."""
    import torch

    g = W.rng(21)
    n, L, b = 4096 * 3 + 17, 4096, 20
    m = (n + L - 1) // L
    rec = np.zeros(m, dtype=oracle.RECORD_DTYPE)
    total = n * b
    big = 0
    for i in range(n):
        big |= int(g.integers(0, 1 << b)) << (i * b)
    nwords = oracle.words_for_bits(total)
    words = np.array([(big >> (64 * w)) & ((1 << 64) - 1) for w in range(nwords)], dtype=np.uint64)
    for p in range(m):
        rec[p]["theta0"] = float(g.uniform(-1e15, 1e15))
        rec[p]["theta1"] = float(g.uniform(-1e9, 1e9)) / 3.0
        rec[p]["start"] = p * L
        exact_claim = 1 if p == 1 else 0  # a false claim must be caught by the device table
        rec[p]["word3"] = (p * L * b) | (b << 48) | (exact_claim << 62)
    col = lc.leco_deserialize(make_blob(rec, words, n, L, 1, 0, 1))
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == oracle.decode(rec, words, n)).all()
    idx = W.uniform_indices(5000, n, seed=3)
    o2 = torch.empty(len(idx), dtype=torch.int64, device="cuda")
    lc.leco_random_access(col, to_dev(idx), o2)
    assert (from_dev(o2) == oracle.lookup(rec, words, n, idx, L=L)[0]).all()


def test_empty_and_single(lc):
    import torch

    for v in (np.zeros(0, dtype=np.uint64), np.array([12345678901234], dtype=np.uint64)):
        col = lc.leco_encode(to_dev(v) if v.size else torch.empty(0, dtype=torch.int64, device="cuda"),
                             lc.fixed(1024), 1)
        out = torch.empty(max(v.size, 1), dtype=torch.int64, device="cuda")
        lc.leco_decode_all(col, out)
        assert (from_dev(out)[: v.size] == v).all()
        res = torch.ones(3, dtype=torch.int64, device="cuda")
        lc.leco_filter_sum(col, 0, (1 << 64) - 1, res)
        assert from_dev(res).tolist() == [v.size, int(v.sum()) if v.size else 0, 0]
        blob = lc.leco_serialize(col)
        col2 = lc.leco_deserialize(blob)
        assert lc.leco_serialize(col2) == blob


def test_serialize_round_trip_and_corruption(lc):
    import torch

    v = W.cfg1(50_000)
    col = _gpu_encode(lc, v, 1024, 1, 64)
    blob = lc.leco_serialize(col)
    d = parse_blob(blob)
    rec, words = oracle.encode_fixed(v, 1024, 1)
    assert d["records"].tobytes() == rec.tobytes() and (d["words"] == words).all()
    col2 = lc.leco_deserialize(blob)
    out = torch.empty(len(v), dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col2, out)
    assert (from_dev(out) == v).all()
    for pos in (0, 70, 64 + 32 * 3 + 24, len(blob) - 1):
        bad = bytearray(blob)
        bad[pos] ^= 0x10
        with pytest.raises(lc.LecoError) as e:
            lc.leco_deserialize(bytes(bad))
        assert e.value.status == lc.LECO_ERR_CORRUPT


# ----------------------------------------------------------------------------- variable partitions

VAR_CASES = [
    ("piecewise_300k", lambda: W.piecewise_linear(300_000, segments=10, mean_len=30_000, seed=4), 64),
    ("timestamps_200k", lambda: W.timestamps_u32(200_000, seed=5), 32),
    ("adversarial_20k", lambda: W.adversarial_u64(20_000, seed=3), 64),
    ("cfg1_150k", lambda: W.cfg1(150_000), 64),
    ("mixed_chunks_394k", lambda: W.mixed_chunks_u64(seed=6), 64),
]


@pytest.mark.parametrize("case", VAR_CASES, ids=[c[0] for c in VAR_CASES])
@pytest.mark.parametrize("tau", [0.0, 0.03, 0.1])
def test_var_partition_matches_round_oracle(lc, case, tau):
    import torch

    _, gen, bits = case
    v = gen()
    for model in (1, 0):
        starts = torch.empty(len(v) + 1, dtype=torch.int64, device="cuda")
        m = lc.leco_var_partition(to_dev(v, bits), starts, lc.variable(tau), model)
        got = from_dev(starts)[: m + 1]
        expect = oracle.var_partition(v, tau, model, variant="round")
        assert got.tolist() == expect.tolist()


@pytest.mark.parametrize("case", VAR_CASES, ids=[c[0] for c in VAR_CASES])
def test_var_column_parity(lc, case):
    import torch

    _, gen, bits = case
    v = gen()
    n = len(v)
    col = lc.leco_encode(to_dev(v, bits), lc.variable(0.03), 1)
    rec_b, words_b, starts_b = lc.leco_column_export(col)
    st = oracle.var_partition(v, 0.03, 1, variant="round")
    rec, words = oracle.encode(v, st, 1)
    assert starts_b == st.tobytes() and rec_b == rec.tobytes() and words_b == words.tobytes()
    tdt = torch.int32 if bits == 32 else torch.int64
    out = torch.empty(n, dtype=tdt, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == v).all()
    idx = W.uniform_indices(30_000, n, seed=2)
    o2 = torch.empty(len(idx), dtype=tdt, device="cuda")
    lc.leco_random_access(col, to_dev(idx), o2)
    assert (from_dev(o2) == v[idx]).all()
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    lo, hi = W.filter_bounds(v)
    for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL):
        lc.leco_filter_sum(col, lo, hi, res, flags=flags)
        r = from_dev(res)
        assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == exact_sum(v, lo, hi)
    # ranges crossing partition and tile boundaries
    g = W.rng(5)
    for _ in range(10):
        a, b = sorted(int(x) for x in g.integers(0, n + 1, size=2))
        o3 = torch.empty(max(b - a, 1), dtype=tdt, device="cuda")
        lc.leco_decode_range(col, a, b - a, o3)
        assert (from_dev(o3)[: b - a] == v[a:b]).all()
    # the blob of a variable column round-trips as well
    col2 = lc.leco_deserialize(lc.leco_serialize(col))
    lc.leco_decode_all(col2, out)
    assert (from_dev(out) == v).all()


def test_var_compression_close_to_sequential_merge(lc):
    """GPU boundaries compress within 2% of the paper's sequential split/merge reading."""
    for gen, bits in ((lambda: W.piecewise_linear(200_000, segments=8, mean_len=25_000, seed=7), 64),
                      (lambda: W.timestamps_u32(200_000, seed=8), 32)):
        v = gen()
        col = lc.leco_encode(to_dev(v, bits), lc.variable(0.03), 1)
        gpu_bytes = col.stats()["record_bytes"] + col.stats()["residual_bytes"]
        st = oracle.var_partition(v, 0.03, 1, variant="seq")
        rec, words = oracle.encode(v, st, 1)
        seq_bytes = oracle.compressed_bytes(rec, words)
        assert gpu_bytes <= 1.02 * seq_bytes


# ----------------------------------------------------------------------------- partition-size search (§3.2.1)

def _search_cases():
    x = np.arange(600_000, dtype=np.float64)
    yield "cfg1_2M", W.cfg1(2_000_000), 64, 10000, 0.01
    yield "quadratic", (x * x * 2e-5).astype(np.uint64) + W.random_u64(600_000, 5, bits=6), 64, 4096, 0.02
    yield "lognormal", W.sorted_lognormal(2_000_000, 1e9, 2.0, seed=3), 64, 10000, 0.01
    yield "timestamps_u32", W.timestamps_u32(1_000_000, seed=4), 32, 2000, 0.05
    yield "random", W.random_u64(300_000, 6), 64, 1000, 0.01
    yield "short_column", W.cfg1(700), 64, 10000, 0.01
    yield "adversarial", W.adversarial_u64(100_000, seed=7), 64, 300, 0.2


SEARCH = list(_search_cases())


@pytest.mark.parametrize("case", SEARCH, ids=[c[0] for c in SEARCH])
def test_partition_size_search_matches_oracle(lc, case):
    """Same sample, same sizes, same search path: the GPU picks the oracle's L with the same sample
    size in bits and the same number of sizes evaluated; the auto policy then encodes byte for byte
    like the fixed policy at that L."""
    _, v, bits, N, frac = case
    for model in (1, 0):
        want = oracle.search_partition_size(v, N, frac, 11, model)
        got = lc.leco_search_partition_size(to_dev(v, bits), model, max_len=N, sample_frac=frac, seed=11)
        assert got == want, model
    if N <= 10000 and frac == 0.01:
        L = oracle.search_partition_size(v, N, 0.01, 0, 1)[0]
        col = lc.leco_encode(to_dev(v, bits), lc.auto(N), 1)
        rec_b, words_b, _ = lc.leco_column_export(col)
        rec, words = oracle.encode_fixed(v, L, 1)
        assert rec_b == rec.tobytes() and words_b == words.tobytes()
        assert col.stats()["partitions"] == (len(v) + L - 1) // L


# ----------------------------------------------------------------------------- full size

@pytest.mark.parametrize("dist", ["a", "b", "c"])
def test_full_size_cfg2(lc, dist):
    """200M uint64, L = 4096, in the benchmark's launch configuration: encode byte-identical to the
    oracle, full decode equal to the input, 10M lookups, filter-sum at ~1% selectivity."""
    import torch

    v = W.cfg2(dist)
    n = len(v)
    dv = to_dev(v)
    col = lc.leco_encode(dv, lc.fixed(W.L_CFG2), 1)
    rec_b, words_b, _ = lc.leco_column_export(col)
    rec, words = oracle.encode_fixed(v, W.L_CFG2, 1)
    assert rec_b == rec.tobytes() and words_b == words.tobytes()
    del rec_b, words_b
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert torch.equal(out, dv)
    del out
    idx = W.uniform_indices(10_000_000, n, seed=2)
    o2 = torch.empty(len(idx), dtype=torch.int64, device="cuda")
    lc.leco_random_access(col, to_dev(idx), o2)
    assert (from_dev(o2) == v[idx]).all()
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    lo, hi = W.filter_bounds(v)
    want = exact_sum(v, lo, hi)
    for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL):
        lc.leco_filter_sum(col, lo, hi, res, flags=flags)
        r = from_dev(res)
        assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == want
    assert lc.leco_sync(col) == lc.LECO_OK


# ----------------------------------------------------------------------------- tiny columns, concurrency

@pytest.mark.parametrize("bits", [64, 32])
def test_tiny_columns(lc, bits):
    """n in {2, L-1, L, L+1, 2L+1} with L = 37, both models: fixed encode byte-identical to the
    oracle, variable boundaries equal to the oracle's round variant, decode, lookups and the full-range
    sum exact. 64-bit columns include the extremes (width-64 partitions)."""
    import torch

    L = 37
    tdt = torch.int32 if bits == 32 else torch.int64
    for n in (2, L - 1, L, L + 1, 2 * L + 1):
        v = W.random_u64(n, seed=n, bits=bits) if bits == 32 else W.adversarial_u64(n, seed=n)
        for model in (0, 1):
            col = lc.leco_encode(to_dev(v, bits), lc.fixed(L), model)
            rec_b, words_b, _ = lc.leco_column_export(col)
            rec, words = oracle.encode_fixed(v, L, model)
            assert rec_b == rec.tobytes() and words_b == words.tobytes(), (n, model)
            vcol = lc.leco_encode(to_dev(v, bits), lc.variable(0.03), model)
            starts = np.frombuffer(lc.leco_column_export(vcol)[2], dtype=np.uint64)
            assert (starts == oracle.var_partition(v, 0.03, model)).all(), (n, model)
            for c in (col, vcol):
                out = torch.empty(n, dtype=tdt, device="cuda")
                lc.leco_decode_all(c, out)
                assert (from_dev(out) == v).all()
                idx = np.array([0, n - 1, n // 2, 1], dtype=np.uint64)
                o2 = torch.empty(len(idx), dtype=tdt, device="cuda")
                lc.leco_random_access(c, to_dev(idx), o2)
                assert (from_dev(o2) == v[idx]).all()
                res = torch.zeros(3, dtype=torch.int64, device="cuda")
                lc.leco_filter_sum(c, 0, (1 << 64) - 1, res)
                r = from_dev(res)
                assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == exact_sum(v, 0, (1 << 64) - 1)
                assert lc.leco_sync(c) == lc.LECO_OK


def test_concurrent_host_threads_on_separate_streams(lc):
    """Columns are immutable after encode and the library's shared state (memory pool, tuning table)
    is locked: four host threads, each on its own stream, encode, decode, look up and filter their
    own columns at the same time and get exact results."""
    import threading

    import torch

    errors = []

    def worker(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                v = W.linear_noise(2_000_000 + 1000 * k, 1 << 20, 5 + k, 300, seed=20 + k)
                dv = to_dev(v)
                for policy in (lc.fixed(1024), lc.variable(0.03)):
                    col = lc.leco_encode(dv, policy, 1)
                    out = torch.empty_like(dv)
                    lc.leco_decode_all(col, out)
                    idx = to_dev(W.uniform_indices(100_000, len(v), seed=k))
                    o2 = torch.empty(idx.numel(), dtype=torch.int64, device="cuda")
                    lc.leco_random_access(col, idx, o2)
                    res = torch.zeros(3, dtype=torch.int64, device="cuda")
                    lo, hi = W.filter_bounds(v)
                    lc.leco_filter_sum(col, lo, hi, res)
                    s.synchronize()
                    if not torch.equal(out, dv) or not torch.equal(o2, dv[idx]):
                        errors.append((k, "values"))
                    r = from_dev(res)
                    if (int(r[0]), int(r[1]) | (int(r[2]) << 64)) != exact_sum(v, lo, hi):
                        errors.append((k, "sum"))
                    if lc.leco_sync(col, s) != lc.LECO_OK:
                        errors.append((k, "status"))
                    col.free()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append((k, repr(e)))

    th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
