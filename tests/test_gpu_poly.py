"""Parity of the polynomial model (LECO_MODEL_POLY: per partition the smallest of constant, linear,
quadratic and cubic) between the CUDA path, through the C ABI, and the CPU oracle.

The encoder is byte-identical to the oracle's (records, coefficient blocks and residual words);
decode, range decode, lookups and every filter mode return the input exactly, also on columns the
oracle encoded (the CUDA decoder checked independently of the CUDA encoder). Cases mix all four
kinds, cross the polynomial length limits (64 and 16384 values), wrap through zero as signed
numbers, and cover 32-bit columns and variable partitions.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import exact_sum, from_dev, make_blob, parse_blob, to_dev

pytestmark = pytest.mark.gpu

POLY = 2


@pytest.fixture(scope="module")
def lc():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_15374_gb300 as pkg

    pkg.build()
    oracle.build()
    from paper_2306_15374_gb300 import leco

    assert leco.LECO_MODEL_POLY == POLY
    return leco


def _exact_cubic(n, N):
    x = np.arange(n, dtype=np.int64) % N
    return ((1 << 40) - 1000 * x + 3 * x * x + x * x * x // 7).astype(np.uint64)


def _cases():
    yield "sine_L4096", W.sine_mixture(300_007, seed=1), 4096, 64
    yield "sine_L1000", W.sine_mixture(200_003, p2=1e4, seed=2), 1000, 64
    yield "sine_L64", W.sine_mixture(50_001, p2=2e3, noise=4, seed=3), 64, 64
    yield "sine_L63_no_poly", W.sine_mixture(50_001, p2=2e3, noise=4, seed=3), 63, 64
    yield "sine_L16384", W.sine_mixture(100_000, seed=4), 16384, 64
    yield "sine_L16385_no_poly", W.sine_mixture(4 * 16385, seed=5), 16385, 64
    yield "sine_wrap_zero", W.sine_mixture(120_001, base=0, seed=6), 2048, 64
    yield "sine_u32_L4096", W.sine_mixture(200_001, base=1 << 31, a1=1e9, a2=1e7, seed=7), 4096, 32
    yield "sine_u32_L777", W.sine_mixture(100_003, base=1 << 31, a1=1e9, a2=1e7, p2=9e3, seed=8), 777, 32
    yield "exact_cubic_L2048", _exact_cubic(40_000, 2048), 2048, 64
    yield "cfg1_L1024", W.cfg1(200_000), 1024, 64
    yield "random_L100", W.random_u64(30_000, 6), 100, 64
    yield "adversarial_L128", W.adversarial_u64(30_001, seed=7), 128, 64
    yield "runs_L256", W.runs(50_000, 300, seed=8), 256, 64


CASES = list(_cases())
IDS = [c[0] for c in CASES]


def _encode(lc, v, L, bits):
    return lc.leco_encode(to_dev(v, bits), lc.fixed(L), POLY)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_poly_encode_is_byte_identical_to_oracle(lc, case):
    name, v, L, bits = case
    col = _encode(lc, v, L, bits)
    rec_b, words_b, _ = lc.leco_column_export(col)
    rec, words = oracle.encode_fixed(v, L, POLY)
    assert rec_b == rec.tobytes()
    assert words_b == words.tobytes()
    npoly = int(oracle.rec_poly(rec["word3"]).sum())
    if name.startswith(("sine", "exact")) and "no_poly" not in name:
        assert npoly > 0
    if "no_poly" in name:
        assert npoly == 0
    assert col.stats()["residual_bytes"] == 8 * len(words)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_poly_decode_range_lookup_filter(lc, case):
    import torch

    _, v, L, bits = case
    n = len(v)
    col = _encode(lc, v, L, bits)
    tdt = torch.int32 if bits == 32 else torch.int64
    g = W.rng(98)
    ranges = [(0, n), (n - 1, 1), (0, 1)]
    for _ in range(6):
        a, b = sorted(int(x) for x in g.integers(0, n + 1, size=2))
        ranges.append((a, b - a))
    for a, cnt in ranges:
        out = torch.empty(max(cnt, 1), dtype=tdt, device="cuda")
        lc.leco_decode_range(col, a, cnt, out)
        assert (from_dev(out)[:cnt] == v[a:a + cnt]).all(), (a, cnt)
    idx = np.concatenate([W.uniform_indices(20_000, n, seed=1), np.array([0, n - 1], np.uint64)])
    out = torch.empty(len(idx), dtype=tdt, device="cuda")
    lc.leco_random_access(col, to_dev(idx), out)
    assert (from_dev(out) == v[idx]).all()
    assert lc.leco_sync(col) == lc.LECO_OK
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    top = (1 << 64) - 1
    for lo, hi in (W.filter_bounds(v), (0, top), (int(v[n // 2]), int(v[n // 2])), (1 << 40, 1 << 41)):
        want = exact_sum(v, lo, hi)
        for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL):
            lc.leco_filter_sum(col, lo, hi, res, flags=flags)
            r = from_dev(res)
            assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == want, flags


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in ("sine_L4096", "sine_u32_L777", "sine_L64")],
                         ids=["sine_L4096", "sine_u32_L777", "sine_L64"])
def test_poly_decode_of_oracle_column(lc, case):
    """The CUDA decoder on a column the oracle encoded (no CUDA encoder involved)."""
    import torch

    _, v, L, bits = case
    n = len(v)
    rec, words = oracle.encode_fixed(v, L, POLY)
    blob = make_blob(rec, words, n, L, 0 if bits == 32 else 1, 0, POLY)
    col = lc.leco_deserialize(blob)
    assert lc.leco_serialize(col) == blob
    out = torch.empty(n, dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == v).all()
    idx = W.uniform_indices(10_000, n, seed=3)
    o2 = torch.empty(len(idx), dtype=out.dtype, device="cuda")
    lc.leco_random_access(col, to_dev(idx), o2)
    assert (from_dev(o2) == v[idx]).all()


def test_poly_corrupt_blocks_are_rejected(lc):
    v = W.sine_mixture(20_000, seed=9)
    rec, words = oracle.encode_fixed(v, 1000, POLY)
    poly = np.flatnonzero(oracle.rec_poly(rec["word3"]))
    assert poly.size
    p = int(poly[0])
    off = int(oracle.rec_offset(rec["word3"][p]))

    big0 = int.from_bytes(words.tobytes(), "little")

    def field(pos):
        return (big0 >> pos) & ((1 << 64) - 1)

    def with_field(pos, value):  # the stream with the 64-bit field at bit pos replaced
        big = (big0 & ~(((1 << 64) - 1) << pos)) | ((value & ((1 << 64) - 1)) << pos)
        return np.frombuffer(big.to_bytes(8 * len(words), "little"), dtype=np.uint64).copy()

    E = field(off + 256)
    bad = [
        (rec, with_field(off + 256, E | (1 << 30))),   # exponent word: bits above the three exponents
        (rec, with_field(off + 256, (E & ~0xFF) | 63)),  # exponent 63 > 62
        (rec, with_field(off + 64, 1 << 62)),          # |K1| > 2^61
        (rec, with_field(off + 64, -(1 << 62))),
    ]
    r2 = rec.copy()
    r2["word3"][p] |= np.uint64(1 << 62)             # exact flag on a polynomial record
    bad.append((r2, words))
    r3 = rec.copy()
    r3["theta0"][p] = 1.0                            # theta of a polynomial record must be 0
    bad.append((r3, words))
    for r, w in bad:
        with pytest.raises(lc.LecoError) as e:
            lc.leco_deserialize(make_blob(r, w, len(v), 1000, 1, 0, POLY))
        assert e.value.status == lc.LECO_ERR_CORRUPT
    # a polynomial record inside a column whose header names the linear model
    with pytest.raises(lc.LecoError):
        lc.leco_deserialize(make_blob(rec, words, len(v), 1000, 1, 0, 1))
    col = lc.leco_deserialize(make_blob(rec, words, len(v), 1000, 1, 0, POLY))
    assert lc.leco_serialize(col) == make_blob(rec, words, len(v), 1000, 1, 0, POLY)


def test_poly_variable_partitions_and_given_starts(lc):
    """Variable partitions under the polynomial model: boundaries from the linear sizes (the same
    as LECO_MODEL_LINEAR's), then the per-partition choice; also with caller-given starts."""
    import torch

    v = W.sine_mixture(300_000, p2=2e4, seed=10)
    n = len(v)
    col = lc.leco_encode(to_dev(v), lc.variable(0.03), POLY)
    rec_b, words_b, starts_b = lc.leco_column_export(col)
    st = oracle.var_partition(v, 0.03, 1, variant="round")
    rec, words = oracle.encode(v, st, POLY)
    assert starts_b == st.tobytes() and rec_b == rec.tobytes() and words_b == words.tobytes()
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == v).all()
    g = W.rng(12)
    cuts = np.unique(np.concatenate([[0, n], g.integers(1, n, size=150)])).astype(np.uint64)
    col2 = lc.leco_encode_with_starts(to_dev(v), to_dev(cuts), len(cuts) - 1, POLY)
    rec_b, words_b, _ = lc.leco_column_export(col2)
    rec, words = oracle.encode(v, cuts, POLY)
    assert rec_b == rec.tobytes() and words_b == words.tobytes()
    idx = W.uniform_indices(20_000, n, seed=4)
    o2 = torch.empty(len(idx), dtype=torch.int64, device="cuda")
    lc.leco_random_access(col2, to_dev(idx), o2)
    assert (from_dev(o2) == v[idx]).all()


def test_poly_auto_partition_size(lc):
    """LECO_PART_AUTO under the polynomial model searches L with the linear sizes, then encodes
    fixed partitions of that L with the per-partition choice."""
    v = W.sine_mixture(400_000, seed=11)
    col = lc.leco_encode(to_dev(v), lc.auto(4096), POLY)
    L = col.stats()["part_size"]
    assert L == oracle.search_partition_size(v, 4096, 0.01, 0, 1)[0]
    rec_b, words_b, _ = lc.leco_column_export(col)
    rec, words = oracle.encode_fixed(v, L, POLY)
    assert rec_b == rec.tobytes() and words_b == words.tobytes()


def test_poly_model_limits(lc):
    """The allocation-free encode takes constant and linear columns only."""
    import torch

    v = W.sine_mixture(10_000, seed=12)
    rec_out = torch.empty(4 * 10, dtype=torch.int64, device="cuda")
    words_out = torch.empty(20_000, dtype=torch.int64, device="cuda")
    with pytest.raises(lc.LecoError) as e:
        lc.leco_encode_fixed_noalloc(to_dev(v), 1024, rec_out, words_out, POLY)
    assert e.value.status == lc.LECO_ERR_INVALID_ARG


@pytest.mark.parametrize("bits", [64, 32])
def test_poly_batched_encode(lc, bits):
    """The batched encode over columns of all three models: each column byte-identical to the
    oracle's encoding with its model and L, and every filter mode exact (the polynomial columns'
    tiles carry their exact bounds)."""
    import torch

    g = W.rng(40 + bits)
    vals, models, Ls = [], [], []
    for c in range(24):
        n = int(np.exp(g.uniform(np.log(50), np.log(120_000)))) if c % 7 else 0
        base = 1 << 31 if bits == 32 else 1 << 40
        v = W.sine_mixture(n, base=base, a1=1e9, a2=1e7, p2=float(g.choice([3e3, 2e4])), seed=c)
        vals.append(v)
        models.append(int(c % 3))
        Ls.append(int(g.choice([64, 100, 1024, 4096])))
    dvals = [to_dev(v, bits) for v in vals]
    cols = lc.leco_batch_encode(dvals, models, Ls)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    for v, m, L, col in zip(vals, models, Ls, cols):
        rec_b, words_b, _ = lc.leco_column_export(col)
        rec, words = oracle.encode_fixed(v, L, m)
        assert rec_b == rec.tobytes() and words_b == words.tobytes(), (m, L, len(v))
        out = torch.empty(max(len(v), 1), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
        lc.leco_decode_all(col, out)
        assert (from_dev(out)[: len(v)] == v).all()
        if len(v):
            lo, hi = W.filter_bounds(v)
            for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL):
                lc.leco_filter_sum(col, lo, hi, res, flags=flags)
                r = from_dev(res)
                assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == exact_sum(v, lo, hi)
    outs = [torch.empty(max(len(v), 1), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda") for v in vals]
    lc.leco_batch_decode(cols, outs)
    torch.cuda.synchronize()
    for v, o in zip(vals, outs):
        assert (from_dev(o)[: len(v)] == v).all()


def test_poly_never_larger_than_linear(lc):
    for v, L in ((W.sine_mixture(100_000, seed=13), 4096), (W.cfg1(100_000), 1024),
                 (W.random_u64(20_000, 14), 500)):
        a = lc.leco_encode(to_dev(v), lc.fixed(L), POLY).stats()
        b = lc.leco_encode(to_dev(v), lc.fixed(L), 1).stats()
        c = lc.leco_encode(to_dev(v), lc.fixed(L), 0).stats()
        assert a["total_bytes"] <= min(b["total_bytes"], c["total_bytes"])


def test_poly_columns_in_batched_decode_and_server(lc):
    """A batch plan (and its CUDA graph) over polynomial and linear columns takes the batched scan
    with the polynomial loop; a server with a polynomial column answers lookups and range decodes
    with the column's values."""
    import torch

    vals = [W.sine_mixture(150_001, seed=20), W.cfg1(120_000), W.sine_mixture(90_000, p2=7e3, seed=21)]
    cols = [lc.leco_encode(to_dev(vals[0]), lc.fixed(4096), POLY), lc.leco_encode(to_dev(vals[1]), lc.fixed(1024), 1),
            lc.leco_encode(to_dev(vals[2]), lc.variable(0.03), POLY)]
    outs = [torch.full((len(v),), -1, dtype=torch.int64, device="cuda") for v in vals]
    plan = lc.leco_batch_plan_create(cols, outs)
    for runner in (lc.leco_batch_plan_run, lc.leco_batch_plan_run_graph):
        for o in outs:
            o.fill_(-1)
        runner(plan)
        torch.cuda.synchronize()
        for v, o in zip(vals, outs):
            assert (from_dev(o) == v).all()
    plan.free()
    s = lc.leco_server_create(4 << 30, max_batch_values=1 << 20, max_batch_lookups=1 << 14)
    ids = [lc.leco_server_admit(s, c) for c in cols]
    g = W.rng(22)
    reqs = []
    for k in range(200):
        c = int(g.integers(0, 3))
        n = len(vals[c])
        if k % 2:
            idx = g.integers(0, n, size=int(g.integers(1, 2000)), dtype=np.uint64)
            out = np.empty(len(idx), dtype=np.uint64)
            reqs.append((lc.leco_server_submit_lookup(s, ids[c], idx, out), out, vals[c][idx]))
        else:
            cnt = int(g.integers(1, 50_000))
            b = int(g.integers(0, n - cnt + 1))
            out = np.empty(cnt, dtype=np.uint64)
            reqs.append((lc.leco_server_submit_range(s, ids[c], b, cnt, out), out, vals[c][b:b + cnt]))
    for rid, out, want in reqs:
        assert lc.leco_server_wait(s, rid) == lc.LECO_OK
        assert np.array_equal(out, want)
    s.destroy()


@pytest.mark.parametrize("n", [0, 1, 2, 63, 64, 65, 127, 4096, 4097])
def test_poly_tiny_columns(lc, n):
    """Empty and tiny columns under the polynomial model (one partition below, at and above the
    64-value minimum, a ragged second partition): byte parity, decode, lookups, sums, round trip."""
    import torch

    v = W.sine_mixture(max(n, 1), p2=500.0, noise=2, seed=30)[:n]
    dv = to_dev(v) if n else torch.empty(0, dtype=torch.int64, device="cuda")
    col = lc.leco_encode(dv, lc.fixed(4096), POLY)
    rec_b, words_b, _ = lc.leco_column_export(col)
    rec, words = oracle.encode_fixed(v, 4096, POLY)
    assert rec_b == rec.tobytes() and words_b == words.tobytes()
    out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out)[:n] == v).all()
    if n:
        idx = np.array([0, n - 1, n // 2], dtype=np.uint64)
        o2 = torch.empty(3, dtype=torch.int64, device="cuda")
        lc.leco_random_access(col, to_dev(idx), o2)
        assert (from_dev(o2) == v[idx]).all()
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    lc.leco_filter_sum(col, 0, (1 << 64) - 1, res, flags=lc.LECO_FILTER_PRUNE)
    r = from_dev(res)
    assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == exact_sum(v, 0, (1 << 64) - 1)
    blob = lc.leco_serialize(col)
    assert lc.leco_serialize(lc.leco_deserialize(blob)) == blob
    assert lc.leco_sync(col) == lc.LECO_OK
