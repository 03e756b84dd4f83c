"""Full-size parity in the launch configurations the benchmark times: the variable-partition columns
(200M piecewise-linear uint64 and 500M uint32 timestamps), the 10,000-column batch (3B values) and
the 2,000-column serving workload (2.5B values).

The oracle cannot encode columns of this size in seconds, so every output is compared element by
element with the input values (decode(encode(x)) == x, lookups, exact filter sums), sampled
partitions are compared with the oracle's own fit (parameters, width, residual bits), sampled
whole columns of the batch are compared byte for byte with the oracle's encoding, and variable
partitions are checked for what holds at any size: the boundaries inside each sampled chunk are a
subset of the oracle's split of that chunk (merges only remove boundaries), and no adjacent pair of
final partitions has a positive merge gain under the oracle's size function (the merge stopped at a
fixpoint)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import exact_sum, from_dev, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CHUNK = 1 << 16
CAP = 1 << 24
TAU = 0.03


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


def _bits(words: np.ndarray, off: int, nbits: int) -> int:
    """Bits [off, off + nbits) of an LSB-first stream of little-endian 64-bit words."""
    if nbits == 0:
        return 0
    w0, w1 = off // 64, (off + nbits) // 64 + 1
    x = int.from_bytes(words[w0:w1].tobytes(), "little")
    return (x >> (off - 64 * w0)) & ((1 << nbits) - 1)


def _check_partition(v, rec, words, s, e, model):
    """One GPU partition against the oracle's encoding of the same values as a lone partition."""
    r_o, w_o = oracle.encode(v[s:e], np.array([0, e - s], dtype=np.uint64), model)
    got, want = rec.view(np.uint64).reshape(4), r_o.view(np.uint64).reshape(4)
    assert got[0] == want[0] and got[1] == want[1], (s, e)  # theta0, theta1 bit patterns
    assert got[2] == s
    g3, o3 = int(got[3]), int(want[3])
    assert g3 >> 48 == o3 >> 48, (s, e)  # width, grid exponent, exact flag
    b = (g3 >> 48) & 0x7F
    assert _bits(words, g3 & ((1 << 48) - 1), b * (e - s)) == _bits(w_o, 0, b * (e - s)), (s, e)


def _check_queries(lc, col, v, dv, bits):
    import torch

    n = len(v)
    out = torch.empty_like(dv)
    lc.leco_decode_all(col, out)
    assert torch.equal(out, dv)
    del out
    idx = W.uniform_indices(10_000_000, n, seed=2)
    didx = to_dev(idx)
    o2 = torch.empty(len(idx), dtype=dv.dtype, device="cuda")
    lc.leco_random_access(col, didx, o2)
    assert torch.equal(o2, dv[didx])
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    for lo, hi in (W.filter_bounds(v), (0, (1 << 64) - 1)):
        want = exact_sum(v, lo, hi)
        for flags in (0, lc.LECO_FILTER_PRUNE, lc.LECO_FILTER_DECODE_ALL):
            lc.leco_filter_sum(col, lo, hi, res, flags=flags)
            r = from_dev(res)
            assert (int(r[0]), int(r[1]) | (int(r[2]) << 64)) == want, flags
    assert lc.leco_sync(col) == lc.LECO_OK


_CFG3 = {}


def _cfg3(dist):
    """The full variable-partition column, generated once per test session."""
    if dist not in _CFG3:
        _CFG3[dist] = W.cfg3(dist)
    return _CFG3[dist]


# Contiguous slices of the two full columns, each partitioned as a column of its own: 8M piecewise
# values (about 120 chunks of 2^16 and, from the split's ~4M partitions, the merge's full round
# count) and 16M timestamps (about 250 chunks, partitions merged across chunk edges).
SLICES = [("a", 60_000_000, 8_000_000), ("b", 200_000_000, 16_000_000)]


@pytest.mark.parametrize("dist,off,n", SLICES, ids=["piecewise_8M", "timestamps_16M"])
def test_variable_partition_slice_matches_round_oracle(lc, dist, off, n):
    """The whole boundary list of the GPU split/merge equals the oracle's round reading (§3.2.2,
    chunked split and round-synchronous merge) on a multi-million-value slice; the column built on it
    is lossless."""
    import torch

    v = _cfg3(dist)[off:off + n].copy()
    bits = 64 if dist == "a" else 32
    dv = to_dev(v, bits)
    starts = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    m = lc.leco_var_partition(dv, starts, lc.variable(TAU), lc.LECO_MODEL_LINEAR)
    got = from_dev(starts)[: m + 1]
    want = oracle.var_partition(v, TAU, lc.LECO_MODEL_LINEAR, variant="round")
    assert len(got) == len(want) and np.array_equal(got, want)
    col = lc.leco_encode(dv, lc.variable(TAU), lc.LECO_MODEL_LINEAR)
    out = torch.empty_like(dv)
    lc.leco_decode_all(col, out)
    assert torch.equal(out, dv)
    col.free()


# Slices of the full columns where the oracle's sequential merge finishes in seconds (two 2M-value
# timestamp slices, ~1-2 s each) or tens of seconds (one 500K-value piecewise slice).
SEQ_SLICES = [("b", 33_703_774, 2_000_000), ("b", 285_115_043, 2_000_000), ("a", 114_217_773, 500_000)]


@pytest.mark.parametrize("dist,off,n", SEQ_SLICES, ids=["timestamps_2M_a", "timestamps_2M_b", "piecewise_500K"])
def test_variable_partition_slice_within_2pct_of_sequential_merge(lc, dist, off, n):
    """The compressed size of the GPU partitioning of a slice (the round reading, §3.2.2) is within
    2% of the oracle's sequential split/merge (one best pair merged at a time) on the same slice."""
    v = _cfg3(dist)[off:off + n].copy()
    bits = 64 if dist == "a" else 32
    col = lc.leco_encode(to_dev(v, bits), lc.variable(TAU), lc.LECO_MODEL_LINEAR)
    rec_b, words_b, _ = lc.leco_column_export(col)
    col.free()
    gpu_bytes = len(rec_b) + len(words_b)
    seq = oracle.var_partition(v, TAU, lc.LECO_MODEL_LINEAR, variant="seq")
    srec, swords = oracle.encode(v, seq, lc.LECO_MODEL_LINEAR)
    seq_bytes = oracle.compressed_bytes(srec, swords)
    assert gpu_bytes <= 1.02 * seq_bytes, (gpu_bytes, seq_bytes)


@pytest.mark.parametrize("dist", ["a", "b"])
def test_full_size_variable_partitions(lc, dist):
    """200M piecewise-linear uint64 / 500M uint32 timestamps, GPU split/merge at tau = 0.03."""
    v = _cfg3(dist)
    bits = 64 if dist == "a" else 32
    n = len(v)
    dv = to_dev(v, bits)
    col = lc.leco_encode(dv, lc.variable(TAU), lc.LECO_MODEL_LINEAR)
    rec_b, words_b, starts_b = lc.leco_column_export(col)
    rec = np.frombuffer(rec_b, dtype=oracle.RECORD_DTYPE)
    words = np.frombuffer(words_b, dtype=np.uint64)
    starts = np.frombuffer(starts_b, dtype=np.uint64)
    m = len(rec)
    lens = np.diff(starts.astype(np.int64))
    assert starts[0] == 0 and int(starts[-1]) == n and (lens > 0).all() and lens.max() <= CAP
    assert (rec["start"] == starts[:-1]).all()
    g = W.rng(17)
    for p in np.unique(np.concatenate([[0, m - 1], g.integers(0, m, size=300)])):
        _check_partition(v, rec[p:p + 1], words, int(starts[p]), int(starts[p + 1]), lc.LECO_MODEL_LINEAR)
    for p in g.integers(0, m - 1, size=200):  # the merge reached a fixpoint
        s0, s1, s2 = int(starts[p]), int(starts[p + 1]), int(starts[p + 2])
        if s2 - s0 <= CAP:
            whole = oracle.partition_size_bits(v[s0:s2])
            assert whole >= oracle.partition_size_bits(v[s0:s1]) + oracle.partition_size_bits(v[s1:s2]), p
    for ch in g.integers(0, (n + CHUNK - 1) // CHUNK, size=20):  # merges only removed split boundaries
        a, e = int(ch) * CHUNK, min(int(ch) * CHUNK + CHUNK, n)
        split = oracle.var_split(v[a:e], TAU, chunk=CHUNK) + np.uint64(a)
        inside = starts[(starts >= a) & (starts < e)]
        assert np.isin(inside, split).all(), ch
    _check_queries(lc, col, v, dv, bits)


def _generate(gen, spec, ncols, keep):
    """Columns generated on host threads (numpy releases the GIL), uploaded as they complete; host
    copies kept only for the columns in `keep`."""
    dvals, host = [], {}
    with ThreadPoolExecutor(max(2, os.cpu_count() or 2)) as ex:
        for c, v in enumerate(ex.map(lambda c: gen(spec, c), range(ncols))):
            dvals.append(to_dev(v))
            if c in keep:
                host[c] = v
    return dvals, host


def test_full_size_batch(lc):
    """10,000 columns, 3B values: one batched encode (byte-identical to the oracle on sampled
    columns), the same encode replayed as one CUDA graph (identical to it), and one persistent
    decode launch and its CUDA graph (equal to the input)."""
    import torch

    spec = W.batch_spec()
    ncols = len(spec["lens"])
    g = W.rng(19)
    sample = set(g.choice(ncols, size=12, replace=False).tolist())
    sample |= {int(np.argmin(spec["lens"])), int(np.argmax(spec["lens"]))}
    dvals, host = _generate(W.batch_column, spec, ncols, sample)
    models, Ls = spec["model"].tolist(), spec["L"].tolist()
    cols = lc.leco_batch_encode(dvals, models, Ls)
    for c, v in host.items():
        rec_b, words_b, _ = lc.leco_column_export(cols[c])
        rec, words = oracle.encode_fixed(v, Ls[c], models[c])
        assert rec_b == rec.tobytes() and words_b == words.tobytes(), c
    # the same batch prepared once and replayed as one CUDA graph: the sampled columns byte for byte,
    # every column the same size
    eplan = lc.leco_batch_encode_plan_create(dvals, models, Ls)
    lc.leco_batch_encode_plan_run(eplan)
    gcols = lc.leco_batch_encode_plan_columns(eplan)
    eplan.free()
    for c in host:
        assert lc.leco_column_export(gcols[c]) == lc.leco_column_export(cols[c]), c
    assert all(a.stats()["residual_bytes"] == b.stats()["residual_bytes"] for a, b in zip(gcols, cols))
    for c in gcols:
        c.free()
    outs = [torch.empty_like(d) for d in dvals]
    plan = lc.leco_batch_plan_create(cols, outs)
    for runner in (lc.leco_batch_plan_run, lc.leco_batch_plan_run_graph):
        for o in outs:
            o.fill_(-1)
        runner(plan)
        torch.cuda.synchronize()
        assert all(torch.equal(d, o) for d, o in zip(dvals, outs))
    plan.free()


def test_full_size_serving(lc):
    """2,000 resident columns (2.5B values, half variable) in a server with a 40 GB budget: a mixed
    burst of lookups and range decodes, all in flight together, each result equal to the input."""
    import torch

    spec = W.serve_spec()
    ncols = len(spec["lens"])
    dvals, _ = _generate(W.serve_column, spec, ncols, set())
    s = lc.leco_server_create(int(40e9), max_batch_values=1 << 24, max_batch_lookups=1 << 17)
    ids = []
    for c, d in enumerate(dvals):
        pol = lc.variable(TAU) if spec["variable"][c] else lc.fixed(4096)
        ids.append(lc.leco_server_admit(s, lc.leco_encode(d, pol, lc.LECO_MODEL_LINEAR)))
    g = W.rng(23)
    reqs = []
    for k in range(3000):
        c = int(g.integers(0, ncols))
        n = int(spec["lens"][c])
        pinned = k % 2 == 0
        if g.random() < 0.5:
            idx = g.integers(0, n, size=int(np.exp(g.uniform(0, np.log(4096)))), dtype=np.uint64)
            out = torch.empty(len(idx), dtype=torch.int64).pin_memory().numpy().view(np.uint64) if pinned \
                else np.empty(len(idx), dtype=np.uint64)
            rid = lc.leco_server_submit_lookup(s, ids[c], idx, out)
            reqs.append((rid, out, c, ("lookup", idx)))
        else:
            cnt = int(min(n, np.exp(g.uniform(np.log(1000), np.log(1_000_000)))))
            b = int(g.integers(0, n - cnt + 1))
            out = torch.empty(cnt, dtype=torch.int64).pin_memory().numpy().view(np.uint64) if pinned \
                else np.empty(cnt, dtype=np.uint64)
            rid = lc.leco_server_submit_range(s, ids[c], b, cnt, out)
            reqs.append((rid, out, c, ("range", b, cnt)))
    for rid, out, c, what in reqs:
        assert lc.leco_server_wait(s, rid) == lc.LECO_OK
        if what[0] == "lookup":
            want = from_dev(dvals[c][to_dev(what[1])])
        else:
            want = from_dev(dvals[c][what[1]:what[1] + what[2]])
        assert np.array_equal(out, want), (c, what[0])
    st = lc.leco_server_stats_get(s)
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["max_batch_size"] > 1
    s.destroy()
