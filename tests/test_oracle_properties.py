"""Properties of the oracle on arbitrary inputs (hypothesis; skipped where it is not installed).

For any column of 64- or 32-bit values, any partition size and either model, the encoding is
lossless (§3.3: value = prediction + zigzag residual, mod 2^64), point lookups return the stored
values, and the filter-sum over any closed interval equals the count and exact sum taken from the
values themselves. Variable partitions tile the column and are lossless as well. Extreme values
(0, 2^63 - 1, 2^63, 2^64 - 1) and long runs are drawn on purpose: they exercise the width-64 and
the exact-grid fallbacks."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import HealthCheck, given, settings  # noqa: E402

EDGES = [0, 1, (1 << 63) - 1, 1 << 63, (1 << 64) - 1, (1 << 53) + 1, (1 << 32) - 1]


@st.composite
def columns(draw, bits):
    top = (1 << bits) - 1
    n = draw(st.integers(0, 300))
    kind = draw(st.sampled_from(["uniform", "walk", "runs", "edges"]))
    if kind == "uniform":
        vals = draw(st.lists(st.integers(0, top), min_size=n, max_size=n))
    elif kind == "walk":
        start = draw(st.integers(0, top))
        steps = draw(st.lists(st.integers(-1000, 100_000), min_size=n, max_size=n))
        vals, x = [], start
        for s in steps:
            x = (x + s) & top  # wraps through zero and the top
            vals.append(x)
    elif kind == "runs":
        pool = draw(st.lists(st.integers(0, top), min_size=1, max_size=4))
        vals = [pool[(i // 17) % len(pool)] for i in range(n)]
    else:
        vals = draw(st.lists(st.sampled_from([e & top for e in EDGES]), min_size=n, max_size=n))
    return np.array(vals, dtype=np.uint64)


def _check_queries(orc, rec, words, v, bits, L, draw):
    n = v.size
    assert (orc.decode(rec, words, n, bits) == v).all()
    if n:
        idx = np.array(draw(st.lists(st.integers(0, n - 1), min_size=1, max_size=20)), dtype=np.uint64)
        got, bad = orc.lookup(rec, words, n, idx, L=L, dtype_bits=bits)
        assert bad == 0 and (got == v[idx]).all()
    top = (1 << bits) - 1
    lo = draw(st.integers(0, top))
    hi = draw(st.integers(0, top))
    sel = [int(x) for x in v if lo <= int(x) <= hi]
    assert orc.filter_sum(rec, words, n, lo, hi, bits) == (len(sel), sum(sel))


@settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(data=st.data(), bits=st.sampled_from([64, 32]), model=st.sampled_from([0, 1]),
       L=st.sampled_from([1, 2, 3, 7, 64, 100, 1000]))
def test_fixed_partitions_are_lossless(orc, data, bits, model, L):
    v = data.draw(columns(bits))
    rec, words = orc.encode_fixed(v, L, model)
    assert len(rec) == (v.size + L - 1) // L
    assert (orc.rec_width(rec["word3"]) <= 64).all()
    _check_queries(orc, rec, words, v, bits, L, data.draw)


@settings(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(data=st.data(), bits=st.sampled_from([64, 32]), tau=st.sampled_from([0.0, 0.03, 0.15]))
def test_variable_partitions_tile_and_are_lossless(orc, data, bits, tau):
    v = data.draw(columns(bits))
    starts = orc.var_partition(v, tau)
    assert starts[0] == 0 and starts[-1] == v.size
    assert (np.diff(starts.astype(np.int64)) > 0).all() or v.size == 0
    rec, words = orc.encode(v, starts, orc.MODEL_LINEAR)
    _check_queries(orc, rec, words, v, bits, 0, data.draw)


@settings(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(data=st.data(), bits=st.sampled_from([64, 32]), L=st.sampled_from([63, 64, 65, 128, 300]))
def test_polynomial_model_is_lossless(orc, data, bits, L):
    """The per-partition choice among constant, linear, quadratic and cubic (§3.1, §4) on arbitrary
    columns, also sampled smooth ones where higher degrees win: lossless, with lookups and sums."""
    if data.draw(st.booleans()):
        v = data.draw(columns(bits))
    else:  # an integer cubic plus small noise: the polynomial candidates apply
        n = data.draw(st.integers(0, 400))
        c = [data.draw(st.integers(-50, 50)) for _ in range(4)]
        noise = data.draw(st.lists(st.integers(0, 3), min_size=n, max_size=n))
        top = (1 << bits) - 1
        v = np.array([(c[0] * i ** 3 + c[1] * i ** 2 + c[2] * i + (1 << (bits - 2)) + noise[i]) & top
                      for i in range(n)], dtype=np.uint64)
    rec, words = orc.encode_fixed(v, L, 2)
    _check_queries(orc, rec, words, v, bits, L, data.draw)


@settings(max_examples=80, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(data=st.data(), bits=st.sampled_from([64, 32]), model=st.sampled_from([0, 1, 2]),
       L=st.sampled_from([1, 5, 64, 100, 300]))
def test_partition_size_is_what_the_encoder_stores(orc, data, bits, model, L):
    """The size the partitioner minimises (§3.2.2: the model's bits plus len * b) is what the encoder
    stores for that partition: the 256-bit record, len * b residual bits, and the 320-bit coefficient
    block of a polynomial partition; and the stream's offsets add up to those bits."""
    v = data.draw(columns(bits))
    rec, words = orc.encode_fixed(v, L, model)
    b = orc.rec_width(rec["word3"])
    poly = orc.rec_poly(rec["word3"])
    off = orc.rec_offset(rec["word3"])
    total = 0
    for p in range(len(rec)):
        a = int(rec["start"][p])
        e = min(a + L, v.size)
        stored = (e - a) * int(b[p]) + (320 if poly[p] else 0)
        assert int(off[p]) == total
        total += stored
        assert orc.partition_size_bits(v[a:e], model) == 256 + stored
    assert len(words) == orc.words_for_bits(total)
