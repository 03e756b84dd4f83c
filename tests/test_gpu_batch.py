"""Batched forms against the single-column path and the input (GPU): one persistent launch (and its
CUDA graph) decoding many columns of uneven lengths, mixed widths, models and partition kinds; the
scan autotuner's table and its effect on results (none)."""
import numpy as np
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


def _columns(lc, count=60, seed=3):
    g = W.rng(seed)
    out = []
    for c in range(count):
        n = int(np.exp(g.uniform(np.log(1), np.log(300_000))))
        kind = c % 5
        if kind == 0:
            v, bits = W.linear_noise(n, 1000, int(g.integers(0, 100)), int(g.integers(0, 500)), seed=c), 64
        elif kind == 1:
            v, bits = W.timestamps_u32(n, seed=c), 32
        elif kind == 2:
            v, bits = W.adversarial_u64(n, seed=c), 64
        elif kind == 3:
            v, bits = np.sort(W.random_u64(n, c, bits=50)), 64
        else:
            v, bits = W.piecewise_linear(n, segments=max(1, n // 20000), mean_len=20000, seed=c), 64
        L = int(g.choice([37, 256, 1024, 4096]))
        model = int(g.integers(0, 2))
        policy = lc.variable(0.03) if (c % 7 == 0 and n > 10) else lc.fixed(L)
        col = lc.leco_encode(to_dev(v, bits), policy, model)
        out.append((v, bits, col))
    return out


def test_batch_plan_decodes_every_column(lc):
    import torch

    cols = _columns(lc)
    outs = [torch.full((max(len(v), 1),), -1, dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
            for v, bits, _ in cols]
    plan = lc.leco_batch_plan_create([c for _, _, c in cols], outs)
    assert lc.leco_batch_plan_jobs(plan) == sum((len(v) + 4095) // 4096 for v, _, _ in cols)
    for runner in (lc.leco_batch_plan_run, lc.leco_batch_plan_run_graph, lc.leco_batch_plan_run_graph):
        for o in outs:
            o.fill_(-1)
        runner(plan)
        torch.cuda.synchronize()
        for (v, bits, _), o in zip(cols, outs):
            assert (from_dev(o)[: len(v)] == v).all()
    assert lc.leco_batch_plan_sync(plan) == lc.LECO_OK
    best = lc.leco_batch_plan_tune(plan)  # a new shape recaptures the graph; results are unchanged
    assert best["stages"] in (2, 3, 4, 6, 8) and best["consumer_warps"] in (4, 8) and best["ms"] > 0
    for runner in (lc.leco_batch_plan_run, lc.leco_batch_plan_run_graph):
        for o in outs:
            o.fill_(-1)
        runner(plan)
        torch.cuda.synchronize()
        for (v, bits, _), o in zip(cols, outs):
            assert (from_dev(o)[: len(v)] == v).all()
    plan.free()
    for o in outs:
        o.fill_(-1)
    lc.leco_batch_decode([c for _, _, c in cols], outs)
    for (v, bits, _), o in zip(cols, outs):
        assert (from_dev(o)[: len(v)] == v).all()


@pytest.mark.parametrize("bits", [64, 32])
def test_batch_encode_matches_single_column_encode(lc, bits):
    import torch

    g = W.rng(17 + bits)
    vals, models, Ls = [], [], []
    for c in range(40):
        n = int(np.exp(g.uniform(0, np.log(200_000)))) if c % 9 else 0
        if bits == 32:
            v = W.timestamps_u32(n, seed=c)
        else:
            v = W.linear_noise(n, 1 << 30, int(g.integers(0, 60)), int(g.integers(0, 3000)), seed=c) if c % 2 \
                else W.adversarial_u64(n, seed=c)
        vals.append(v)
        models.append(int(g.integers(0, 2)))
        Ls.append(int(g.choice([1, 37, 256, 1024, 4096])))
    dvals = [to_dev(v, bits) for v in vals]
    cols = lc.leco_batch_encode(dvals, models, Ls)
    for v, dv, m, L, col in zip(vals, dvals, models, Ls, cols):
        ref = lc.leco_encode(dv, lc.fixed(L), m)
        assert lc.leco_column_export(col) == lc.leco_column_export(ref)
        assert lc.leco_serialize(col) == lc.leco_serialize(ref)
        out = torch.empty(max(len(v), 1), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
        lc.leco_decode_all(col, out)
        assert (from_dev(out)[: len(v)] == v).all()
    # freeing in any order keeps the others valid until the last one goes
    for col in cols[::2]:
        col.free()
    for v, col in list(zip(vals, cols))[1::2]:
        out = torch.empty(max(len(v), 1), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
        lc.leco_decode_all(col, out)
        assert (from_dev(out)[: len(v)] == v).all()


@pytest.mark.parametrize("bits", [64, 32])
def test_batch_encode_plan_graph_matches_batch_encode(lc, bits):
    """The batched encode prepared once and replayed as one CUDA graph: each run's columns are byte
    for byte those of leco_batch_encode on the same values (constant, linear and polynomial models,
    empty, tiny and multi-tile columns); a run after the inputs change in place encodes the new
    contents; the columns taken out stay valid after the plan runs again and after it is freed."""
    import torch

    g = W.rng(41 + bits)
    models, Ls, lens = [], [], []
    for c in range(36):
        lens.append(int(np.exp(g.uniform(0, np.log(150_000)))) if c % 8 else 0)
        models.append(c % 3)
        Ls.append(int(g.choice([1, 37, 256, 1024, 4096])))

    def values(seed):
        out = []
        for c, n in enumerate(lens):
            if bits == 32:
                out.append(W.timestamps_u32(n, seed=seed + c))
            elif c % 2:
                out.append(W.linear_noise(n, 1 << 30, int(g.integers(0, 60)), int(g.integers(0, 3000)), seed=seed + c))
            else:
                out.append(W.adversarial_u64(n, seed=seed + c))
        return out

    vals = values(100)
    dvals = [to_dev(v, bits) for v in vals]
    plan = lc.leco_batch_encode_plan_create(dvals, models, Ls)
    assert lc.leco_batch_encode_plan_reserved_bytes(plan) >= sum(8 * n for n in lens)
    with pytest.raises(lc.LecoError):  # nothing encoded before the first run
        lc.leco_batch_encode_plan_columns(plan)
    kept = []
    for rnd in range(2):
        if rnd == 1:  # same shapes, new contents, same device buffers
            vals = values(900)
            for dv, v in zip(dvals, vals):
                dv.copy_(to_dev(v, bits))
        lc.leco_batch_encode_plan_run(plan)
        cols = lc.leco_batch_encode_plan_columns(plan)
        refs = lc.leco_batch_encode(dvals, models, Ls)
        for v, col, ref in zip(vals, cols, refs):
            assert lc.leco_column_export(col) == lc.leco_column_export(ref)
            assert lc.leco_serialize(col) == lc.leco_serialize(ref)
        kept.append((vals, cols))
    plan.free()
    for vs, cols in kept:
        for v, col in zip(vs, cols):
            out = torch.empty(max(len(v), 1), dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
            lc.leco_decode_all(col, out)
            assert lc.leco_sync(col) == lc.LECO_OK
            assert (from_dev(out)[: len(v)] == v).all()


def test_encode_tuner_keeps_results_identical(lc, tmp_path):
    """Every batched-encode shape the tuner tries gives the same bytes; the chosen one is stored and
    saved with the scan configurations."""
    g = W.rng(29)
    vals, models, Ls = [], [], []
    for c in range(24):
        n = int(np.exp(g.uniform(np.log(100), np.log(400_000))))
        vals.append(W.linear_noise(n, 1 << 30, int(g.integers(0, 60)), int(g.integers(0, 3000)), seed=c))
        models.append(c % 2)
        Ls.append(int(g.choice([37, 256, 1024, 4096])))
    dvals = [to_dev(v) for v in vals]
    before = [lc.leco_column_export(c) for c in lc.leco_batch_encode(dvals, models, Ls)]
    best = lc.leco_tune_batch_encode(dvals, models, Ls)
    assert best["item_values"] in (1024, 2048, 4096) and best["fit_ctas"] in (2, 3, 4) and best["ms"] > 0
    after = [lc.leco_column_export(c) for c in lc.leco_batch_encode(dvals, models, Ls)]
    assert before == after
    path = str(tmp_path / "tune_enc.json")
    lc.leco_tune_save(path)
    assert '"item_values"' in open(path).read()
    lc.leco_tune_load(path)


def test_tuner_keeps_results_identical(lc, tmp_path):
    import torch

    v = W.cfg1(2_000_000)
    col = lc.leco_encode(to_dev(v), lc.fixed(1024), 1)
    best = lc.leco_tune_scan(col, 0)
    assert best["stages"] in (2, 3, 4, 6, 8) and best["consumer_warps"] in (4, 8) and best["ms"] > 0
    lo, hi = W.filter_bounds(v)
    bf = lc.leco_tune_scan(col, 1, lo, hi)
    assert bf["ms"] > 0
    out = torch.empty(len(v), dtype=torch.int64, device="cuda")
    lc.leco_decode_all(col, out)
    assert (from_dev(out) == v).all()
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    lc.leco_filter_sum(col, lo, hi, res)
    sel = v[(v >= lo) & (v <= hi)]
    r = from_dev(res)
    assert int(r[0]) == sel.size and int(r[1]) == int(sel.sum())
    path = str(tmp_path / "tune.json")
    lc.leco_tune_save(path)
    text = open(path).read()
    assert '"stages"' in text and '"consumer_warps"' in text
    lc.leco_tune_load(path)


def test_trim_memory_keeps_live_columns(lc):
    """Freed columns' memory stays cached in the library's pool until trimmed; trimming leaves live
    columns intact."""
    import torch

    v = W.cfg1(500_000)
    keep = lc.leco_encode(to_dev(v), lc.fixed(1024), 1)
    for _ in range(3):
        lc.leco_encode(to_dev(v), lc.fixed(1024), 1).free()
    lc.leco_trim_memory()
    out = torch.empty(len(v), dtype=torch.int64, device="cuda")
    lc.leco_decode_all(keep, out)
    assert (from_dev(out) == v).all()
