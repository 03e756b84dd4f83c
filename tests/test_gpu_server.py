"""The serving loop on the GPU: every request's result is identical alone and in a concurrent mix,
and equals the column's values (lookups and range decodes over fixed and variable columns of 32-
and 64-bit values); the one-launch-per-request mode returns the same; the budget refuses columns
that do not fit."""
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


def _server_with_columns(lc, **kw):
    s = lc.leco_server_create(8 << 30, max_batch_values=1 << 22, max_batch_lookups=1 << 16, **kw)
    data = [(W.cfg1(300_000), 64, lc.fixed(1024)),
            (W.timestamps_u32(250_000, seed=2), 32, lc.variable(0.03)),
            (W.piecewise_linear(200_000, segments=5, mean_len=40_000, seed=3), 64, lc.variable(0.03)),
            (W.sorted_lognormal(100_000, 1e9, 2.0, seed=4), 64, lc.fixed(4096))]
    cols = {}
    for v, bits, pol in data:
        col = lc.leco_encode(to_dev(v, bits), pol, 1)
        cols[lc.leco_server_admit(s, col)] = (v, bits)
    return s, cols


def _requests(cols, count=300, seed=9):
    g = np.random.default_rng(seed)
    out = []
    ids = list(cols)
    for _ in range(count):
        cid = ids[int(g.integers(0, len(ids)))]
        n = len(cols[cid][0])
        if g.random() < 0.5:
            out.append(("lookup", cid, g.integers(0, n, size=int(np.exp(g.uniform(0, np.log(4096)))), dtype=np.uint64)))
        else:
            cnt = int(min(n, np.exp(g.uniform(np.log(1000), np.log(200_000)))))
            out.append(("range", cid, (int(g.integers(0, n - cnt + 1)), cnt)))
    return out


def _out(size, dt, pinned):
    """Result buffer: pageable numpy (staged delivery) or pinned host memory (direct delivery)."""
    if not pinned:
        return np.zeros(size, dtype=dt)
    import torch

    t = torch.zeros(size, dtype=torch.int32 if dt == np.uint32 else torch.int64).pin_memory()
    return t.numpy().view(dt)  # the array keeps the pinned tensor alive through its base


_count = [0]


def _submit(lc, s, cols, req):
    kind, cid, arg = req
    dt = np.uint32 if cols[cid][1] == 32 else np.uint64
    _count[0] += 1
    pinned = _count[0] % 2 == 0
    if kind == "lookup":
        out = _out(arg.size, dt, pinned)
        return lc.leco_server_submit_lookup(s, cid, arg, out), out
    out = _out(arg[1], dt, pinned)
    return lc.leco_server_submit_range(s, cid, arg[0], arg[1], out), out


def _expected(cols, req):
    kind, cid, arg = req
    v = cols[cid][0]
    return v[arg] if kind == "lookup" else v[arg[0]:arg[0] + arg[1]]


@pytest.mark.parametrize("per_request", [False, True])
def test_results_identical_alone_and_in_the_mix(lc, per_request):
    s, cols = _server_with_columns(lc, max_batch_requests=1 if per_request else 0)
    reqs = _requests(cols)
    mixed = [_submit(lc, s, cols, r) for r in reqs]  # all in flight together
    for rid, _ in mixed:
        assert lc.leco_server_wait(s, rid) == lc.LECO_OK
    alone = []
    for r in reqs:  # one at a time
        rid, out = _submit(lc, s, cols, r)
        assert lc.leco_server_wait(s, rid) == lc.LECO_OK
        alone.append(out)
    for r, (_, m), a in zip(reqs, mixed, alone):
        assert np.array_equal(m, a)
        assert np.array_equal(m.astype(np.uint64), _expected(cols, r))
    st = lc.leco_server_stats_get(s)
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    if not per_request:
        assert st["max_batch_size"] > 1
    else:
        assert st["max_batch_size"] == 1
    s.destroy()


def test_budget_refuses_what_does_not_fit(lc):
    import torch

    s = lc.leco_server_create(1 << 30, max_batch_values=1 << 20, max_batch_lookups=1 << 12)
    reserved = lc.leco_server_stats_get(s)["reserved_bytes"]
    assert 0 < reserved < 1 << 30
    v = torch.arange(100_000_000, dtype=torch.int64, device="cuda") * 7919 % 1000003
    col = lc.leco_encode(v, lc.fixed(4096), 1)  # incompressible noise: ~0.25 GB
    big = lc.leco_encode(torch.cat([v] * 4), lc.fixed(4096), 1)  # ~1 GB: over the budget
    cid = lc.leco_server_admit(s, col)
    with pytest.raises(lc.LecoError) as e:
        lc.leco_server_admit(s, big)
    assert e.value.status == lc.LECO_ERR_BUDGET
    assert big.stats()["n"] == 400_000_000  # the caller still owns the refused column
    out = np.zeros(10, dtype=np.uint64)
    rid = lc.leco_server_submit_range(s, cid, 12345, 10, out)
    assert lc.leco_server_wait(s, rid) == lc.LECO_OK
    assert out.tolist() == (torch.arange(12345, 12355, device="cuda") * 7919 % 1000003).tolist()
    lc.leco_server_evict(s, cid)
    assert lc.leco_server_stats_get(s)["resident_bytes"] == 0
    s.destroy()
