"""Host-side validation of self-describing blobs (leco_deserialize), no GPU needed.

A blob whose CRC-32 matches can still describe a stream the decoders must not run on: a field
width above 64, offsets that are not dense, starts that do not tile [0, n), a stream whose size does
not match its fields, bits set in the padding. Every such blob is refused with LECO_ERR_CORRUPT on
the host, before anything reaches the device, so the decode kernels only ever read fields inside the
stream. Each case below takes a valid column encoded by the oracle, breaks one thing, and rebuilds
the blob with a correct CRC (the layout of include/leco.h, restated in tests/gpu_util.py)."""
import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_util import make_blob

U64 = np.uint64


@pytest.fixture(scope="module")
def lc():
    import paper_2306_15374_gb300 as pkg

    pkg.build()
    from paper_2306_15374_gb300 import leco

    return leco


def _status(lc, blob):
    h = ctypes.c_void_p()
    s = lc.lib().leco_deserialize(blob, len(blob), None, ctypes.byref(h))
    if s == lc.LECO_OK:  # on a machine with a GPU a valid blob becomes a column
        lc.lib().leco_column_free(h)
    return s


def _w3(off, b, s=0, exact=0, poly=0):
    return U64(off | (b << 48) | ((s & 0x7F) << 55) | (exact << 62) | (poly << 63))


def _fields(rec):
    w3 = rec["word3"].astype(U64)
    return (w3 & U64((1 << 48) - 1)).astype(np.int64), ((w3 >> U64(48)) & U64(0x7F)).astype(np.int64)


@pytest.fixture(scope="module")
def fixed_col(orc):
    v = W.cfg1(5000)
    rec, words = orc.encode_fixed(v, 256, orc.MODEL_LINEAR)
    return v, rec, words


@pytest.fixture(scope="module")
def var_col(orc):
    v = W.piecewise_linear(6000, segments=6, mean_len=1000, seed=7)
    st = orc.var_partition(v, 0.03)
    rec, words = orc.encode(v, st, orc.MODEL_LINEAR)
    return v, st, rec, words


def test_valid_blobs_pass_validation(lc, orc, fixed_col, var_col):
    v, rec, words = fixed_col
    assert _status(lc, make_blob(rec, words, len(v), 256, 1, 0, 1)) != lc.LECO_ERR_CORRUPT
    v, st, rec, words = var_col
    assert _status(lc, make_blob(rec, words, len(v), 0, 1, 1, 1, starts=st)) != lc.LECO_ERR_CORRUPT
    # a one-partition column of zero-width fields (an exact line): the stream is padding only
    line = np.arange(10, 10 + 3 * 1000, 3, dtype=U64)
    rec1, words1 = orc.encode_fixed(line, 1000, orc.MODEL_LINEAR)
    assert len(words1) == 2 and _fields(rec1)[1].tolist() == [0]
    assert _status(lc, make_blob(rec1, words1, 1000, 1000, 1, 0, 1)) != lc.LECO_ERR_CORRUPT


def test_header_fields_out_of_range(lc, fixed_col):
    v, rec, words = fixed_col
    n = len(v)
    for dtype, kind, model, L in ((3, 0, 1, 256), (1, 2, 1, 256), (1, 0, 3, 256), (1, 0, 1, 0)):
        assert _status(lc, make_blob(rec, words, n, L, dtype, kind, model)) == lc.LECO_ERR_CORRUPT
    # records for a different partition size; one record missing; n with no records
    assert _status(lc, make_blob(rec, words, n, 128, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    assert _status(lc, make_blob(rec[:-1], words, n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    assert _status(lc, make_blob(rec[:0], words[:2] * U64(0), n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    # a byte more or less than the header says
    blob = make_blob(rec, words, n, 256, 1, 0, 1)
    assert _status(lc, blob + b"\0") == lc.LECO_ERR_CORRUPT
    assert _status(lc, blob[:-1]) == lc.LECO_ERR_CORRUPT


def test_record_fields_that_would_read_outside_the_stream(lc, fixed_col):
    v, rec, words = fixed_col
    n = len(v)
    off, b = _fields(rec)
    assert (b > 0).all() and (b < 64).all()

    def with_word3(p, w3):
        r = rec.copy()
        r["word3"][p] = w3
        return make_blob(r, words, n, 256, 1, 0, 1)

    assert _status(lc, with_word3(3, _w3(int(off[3]), 65))) == lc.LECO_ERR_CORRUPT  # width above 64
    assert _status(lc, with_word3(5, _w3(int(off[5]) + 1, int(b[5])))) == lc.LECO_ERR_CORRUPT  # gap
    assert _status(lc, with_word3(5, _w3(int(off[5]) - 1, int(b[5])))) == lc.LECO_ERR_CORRUPT  # overlap
    # a polynomial block flag in a linear-model column
    assert _status(lc, with_word3(2, _w3(int(off[2]), int(b[2]), poly=1))) == lc.LECO_ERR_CORRUPT
    # a start that is not p * L
    r = rec.copy()
    r["start"][2] += 1
    assert _status(lc, make_blob(r, words, n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    # the last partition one bit wider: the fields end past the stream's bit count
    r = rec.copy()
    last = len(rec) - 1
    r["word3"][last] = _w3(int(off[last]), int(b[last]) + 1)
    assert _status(lc, make_blob(r, words, n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT


def test_stream_size_and_padding(lc, fixed_col):
    v, rec, words = fixed_col
    n = len(v)
    off, b = _fields(rec)
    total = int(off[-1] + b[-1] * (n - int(rec["start"][-1])))
    assert total % 64  # the last field word has unused high bits
    w = words.copy()
    w[-1] = U64(1)  # padding word not zero
    assert _status(lc, make_blob(rec, w, n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    w = words.copy()
    w[total // 64] |= U64(1) << U64(63)  # a bit after the last field
    assert _status(lc, make_blob(rec, w, n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    # one padding word more or less than the stream's size calls for
    assert _status(lc, make_blob(rec, np.append(words, [U64(0), U64(0)]), n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT
    assert _status(lc, make_blob(rec, words[:-1], n, 256, 1, 0, 1)) == lc.LECO_ERR_CORRUPT


def test_variable_starts_must_tile_the_column(lc, var_col):
    v, st, rec, words = var_col
    n = len(v)
    assert len(st) > 3

    def blob_with(starts, r=rec):
        return make_blob(r, words, n, 0, 1, 1, 1, starts=starts)

    s = st.copy()
    s[-1] = U64(n - 1)  # does not end at n
    assert _status(lc, blob_with(s)) == lc.LECO_ERR_CORRUPT
    s = st.copy()
    s[0] = U64(1)  # does not begin at 0
    assert _status(lc, blob_with(s)) == lc.LECO_ERR_CORRUPT
    s = st.copy()
    s[2] = s[1]  # an empty partition
    assert _status(lc, blob_with(s)) == lc.LECO_ERR_CORRUPT
    s = st.copy()
    s[2] = s[3] + U64(1)  # starts out of order
    assert _status(lc, blob_with(s)) == lc.LECO_ERR_CORRUPT
    # a record's start disagreeing with the starts array
    r = rec.copy()
    r["start"][1] += 1
    assert _status(lc, blob_with(st, r)) == lc.LECO_ERR_CORRUPT


def test_partition_longer_than_the_length_cap(lc):
    """One variable partition of 2^24 + 1 zero-width fields: every field lies inside the stream, but
    partitions are capped at 2^24 values, so the blob is refused; at 2^24 it passes."""
    import oracle

    for n, want_corrupt in ((1 << 24, False), ((1 << 24) + 1, True)):
        rec = np.zeros(1, dtype=oracle.RECORD_DTYPE)
        rec["theta0"] = 7.0
        rec["word3"] = _w3(0, 0, exact=1)
        words = np.zeros(2, dtype=U64)
        blob = make_blob(rec, words, n, 0, 1, 1, 1, starts=np.array([0, n], dtype=U64))
        assert (_status(lc, blob) == lc.LECO_ERR_CORRUPT) == want_corrupt


def test_polynomial_blocks_must_be_evaluable(lc, orc):
    """A polynomial partition's 320-bit block (T, K1..K3, exponent word) is checked on the host:
    exponents at most 62 in the low three bytes, |K_j| <= 2^61, and the exponent spread behind each
    nonzero K_j within the room its Gram term leaves in 124 bits (49, 34 and 20 for j = 1, 2, 3).
    A spread exactly at the room passes; one more is refused."""
    POLY = 2
    v = W.sine_mixture(20_000, seed=9)
    rec, words = orc.encode_fixed(v, 1000, POLY)
    n = len(v)
    poly = np.flatnonzero(orc.rec_poly(rec["word3"]))
    assert poly.size
    big0 = int.from_bytes(words.tobytes(), "little")

    def field(pos):
        return (big0 >> pos) & ((1 << 64) - 1)

    def blob(fields):
        big = big0
        for pos, value in fields.items():
            big = (big & ~(((1 << 64) - 1) << pos)) | ((value & ((1 << 64) - 1)) << pos)
        w = np.frombuffer(big.to_bytes(8 * len(words), "little"), dtype=U64).copy()
        return make_blob(rec, w, n, 1000, 1, 0, POLY)

    assert _status(lc, blob({})) != lc.LECO_ERR_CORRUPT
    # a partition whose block has a nonzero K_j, for each j that has one somewhere
    room = (49, 34, 20)
    tested = set()
    for p in poly:
        off = int(orc.rec_offset(rec["word3"][int(p)]))
        E = field(off + 256)
        assert _status(lc, blob({off + 256: E | (1 << 30)})) == lc.LECO_ERR_CORRUPT  # bits above the exponents
        assert _status(lc, blob({off + 256: (E & ~0xFF) | 63})) == lc.LECO_ERR_CORRUPT  # exponent 63
        assert _status(lc, blob({off + 64: 1 << 62})) == lc.LECO_ERR_CORRUPT  # |K1| > 2^61
        assert _status(lc, blob({off + 64: -(1 << 62)})) == lc.LECO_ERR_CORRUPT
        assert _status(lc, blob({off + 64: 1 << 61})) != lc.LECO_ERR_CORRUPT  # |K1| = 2^61 is allowed
        for j in range(3):
            if j in tested or field(off + 64 * (j + 1)) == 0:
                continue
            tested.add(j)
            for spread, corrupt in ((room[j], False), (room[j] + 1, True)):
                # s_j = 0 and the other two exponents = spread: S - s_j = spread; every other term
                # has S - s_i = 0
                e = sum((0 if i == j else spread) << (8 * i) for i in range(3))
                assert (_status(lc, blob({off + 256: e})) == lc.LECO_ERR_CORRUPT) == corrupt, (j, spread)
        if len(tested) == 3:
            break
    assert tested == {0, 1, 2}  # every Gram term is used by some partition of this column
