"""The serving loop's scheduling, admission and bookkeeping on the host (no GPU): the server's
mock executor runs batches on the CPU after a fixed delay and fills results with a fixed function
of (column, position), so routing, continuous batching, budgets and latency stats are checked
without touching a device."""
import threading
import time

import numpy as np
import pytest

GOLD = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def mock_value(col, i, bits):
    v = ((col << 40) ^ ((i * GOLD) & M64)) & M64
    return v & 0xFFFFFFFF if bits == 32 else v


@pytest.fixture(scope="module")
def lc():
    import paper_2306_15374_gb300 as pkg

    pkg.build()
    from paper_2306_15374_gb300 import leco

    leco.lib()
    return leco


def test_budget_admission(lc):
    s = lc.leco_server_create(1000, mock=True, mock_batch_us=100)
    a = lc.leco_server_admit_mock(s, 100, lc.LECO_U64, 600)
    with pytest.raises(lc.LecoError) as e:
        lc.leco_server_admit_mock(s, 100, lc.LECO_U64, 500)
    assert e.value.status == lc.LECO_ERR_BUDGET
    b = lc.leco_server_admit_mock(s, 100, lc.LECO_U32, 400)
    assert a != b
    assert lc.leco_server_stats_get(s)["resident_bytes"] == 1000
    lc.leco_server_evict(s, a)
    assert lc.leco_server_stats_get(s)["resident_bytes"] == 400
    c = lc.leco_server_admit_mock(s, 10, lc.LECO_U64, 500)  # fits again after the eviction
    assert lc.leco_server_stats_get(s)["columns"] == 2
    s.destroy()


def test_results_route_to_the_right_requests(lc):
    s = lc.leco_server_create(1 << 30, mock=True, mock_batch_us=2000)
    cols = {lc.leco_server_admit_mock(s, 100_000, lc.LECO_U64, 1000): 64,
            lc.leco_server_admit_mock(s, 50_000, lc.LECO_U32, 1000): 32}
    g = np.random.default_rng(5)
    reqs = []
    for _ in range(200):  # submitted back to back: arrivals outpace the slots, so batches form
        cid = list(cols)[int(g.integers(0, 2))]
        bits = cols[cid]
        n = 100_000 if bits == 64 else 50_000
        if g.random() < 0.5:
            idx = g.integers(0, n, size=int(g.integers(1, 300)), dtype=np.uint64)
            out = np.zeros(idx.size, dtype=np.uint64 if bits == 64 else np.uint32)
            rid = lc.leco_server_submit_lookup(s, cid, idx, out)
            reqs.append((rid, out, cid, bits, [int(i) for i in idx]))
        else:
            b = int(g.integers(0, n - 10))
            cnt = int(g.integers(1, min(5000, n - b)))
            out = np.zeros(cnt, dtype=np.uint64 if bits == 64 else np.uint32)
            rid = lc.leco_server_submit_range(s, cid, b, cnt, out)
            reqs.append((rid, out, cid, bits, range(b, b + cnt)))
    for rid, out, cid, bits, pos in reqs:
        assert lc.leco_server_wait(s, rid) == lc.LECO_OK
        assert out.tolist() == [mock_value(cid, i, bits) for i in pos]
    st = lc.leco_server_stats_get(s)
    assert st["completed"] == 200 and st["failed"] == 0
    assert st["batches"] < 200 and st["max_batch_size"] > 1  # requests arriving together share batches
    assert st["p99_us"] >= st["p50_us"] > 0
    s.destroy()


def test_one_request_per_launch_mode(lc):
    s = lc.leco_server_create(1 << 30, max_batch_requests=1, mock=True, mock_batch_us=50)
    cid = lc.leco_server_admit_mock(s, 1000, lc.LECO_U64, 10)
    outs = [np.zeros(10, dtype=np.uint64) for _ in range(20)]
    rids = [lc.leco_server_submit_range(s, cid, 7 * k, 10, o) for k, o in enumerate(outs)]
    for rid in rids:
        lc.leco_server_wait(s, rid)
    st = lc.leco_server_stats_get(s)
    assert st["batches"] == st["completed"] == 20 and st["max_batch_size"] == 1
    s.destroy()


def test_continuous_batching_admits_arrivals_while_busy(lc):
    """With one slot and slow batches, requests submitted while a batch runs all join the next
    batch rather than queueing one by one."""
    s = lc.leco_server_create(1 << 30, max_inflight=1, mock=True, mock_batch_us=30_000)
    cid = lc.leco_server_admit_mock(s, 10_000, lc.LECO_U64, 10)
    first = lc.leco_server_submit_range(s, cid, 0, 10, np.zeros(10, dtype=np.uint64))
    time.sleep(0.005)  # the first batch is now running
    outs = [np.zeros(5, dtype=np.uint64) for _ in range(50)]
    rids = [lc.leco_server_submit_range(s, cid, k, 5, o) for k, o in enumerate(outs)]
    for rid in [first] + rids:
        lc.leco_server_wait(s, rid)
    st = lc.leco_server_stats_get(s)
    assert st["batches"] == 2 and st["max_batch_size"] == 50
    s.destroy()


def test_submit_validation(lc):
    s = lc.leco_server_create(1 << 30, max_batch_lookups=100, max_batch_values=1000, mock=True)
    cid = lc.leco_server_admit_mock(s, 500, lc.LECO_U64, 10)
    out = np.zeros(1000, dtype=np.uint64)
    for call, status in [
        (lambda: lc.leco_server_submit_lookup(s, cid, np.array([500], np.uint64), out), lc.LECO_ERR_INDEX_RANGE),
        (lambda: lc.leco_server_submit_lookup(s, cid, np.zeros(101, np.uint64), out), lc.LECO_ERR_INVALID_ARG),
        (lambda: lc.leco_server_submit_range(s, cid, 400, 101, out), lc.LECO_ERR_INDEX_RANGE),
        (lambda: lc.leco_server_submit_range(s, cid, 0, 0, out), lc.LECO_ERR_INVALID_ARG),
        (lambda: lc.leco_server_submit_range(s, cid + 1, 0, 1, out), lc.LECO_ERR_INVALID_ARG),
    ]:
        with pytest.raises(lc.LecoError) as e:
            call()
        assert e.value.status == status
    rid = lc.leco_server_submit_range(s, cid, 0, 1, out)
    lc.leco_server_wait(s, rid)
    with pytest.raises(lc.LecoError):
        lc.leco_server_wait(s, rid)  # already collected
    s.destroy()


def test_evict_waits_for_pending_requests(lc):
    s = lc.leco_server_create(1 << 30, max_inflight=1, mock=True, mock_batch_us=20_000)
    cid = lc.leco_server_admit_mock(s, 1000, lc.LECO_U64, 10)
    out = np.zeros(10, dtype=np.uint64)
    rid = lc.leco_server_submit_range(s, cid, 0, 10, out)
    t0 = time.time()
    lc.leco_server_evict(s, cid)
    assert time.time() - t0 >= 0.01  # returned only after the request's batch finished
    assert lc.leco_server_wait(s, rid) == lc.LECO_OK
    assert out.tolist() == [mock_value(cid, k, 64) for k in range(10)]
    s.destroy()


def test_concurrent_submitters_and_poisson_driver(lc):
    s = lc.leco_server_create(1 << 30, mock=True, mock_batch_us=500)
    ids = [lc.leco_server_admit_mock(s, 200_000, lc.LECO_U64, 100) for _ in range(4)]
    errors = []

    def worker(seed):
        g = np.random.default_rng(seed)
        for _ in range(50):
            cid = ids[int(g.integers(0, 4))]
            idx = g.integers(0, 200_000, size=16, dtype=np.uint64)
            out = np.zeros(16, dtype=np.uint64)
            rid = lc.leco_server_submit_lookup(s, cid, idx, out)
            lc.leco_server_wait(s, rid)
            if out.tolist() != [mock_value(cid, int(i), 64) for i in idx]:
                errors.append(seed)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    lc.leco_server_reset_stats(s)
    sent = lc.leco_server_drive_poisson(s, ids, rate=2000, seconds=0.3, seed=1, max_range=5000)
    st = lc.leco_server_stats_get(s)
    assert sent > 100 and st["completed"] == sent and st["failed"] == 0
    s.destroy()


def test_binding_refuses_short_host_outputs(lc):
    """The server writes each request's values, at the column's width, into the caller's host array:
    the binding refuses an array that is too short, strided or read-only before the request is
    queued; an array of exactly the right size is served."""
    s = lc.leco_server_create(1 << 30, mock=True)
    a = lc.leco_server_admit_mock(s, 1000, lc.LECO_U64, 10)
    b = lc.leco_server_admit_mock(s, 1000, lc.LECO_U32, 10)
    idx = np.array([1, 2, 3, 4], dtype=np.uint64)
    with pytest.raises(ValueError, match="needs 32"):
        lc.leco_server_submit_lookup(s, a, idx, np.zeros(3, dtype=np.uint64))
    with pytest.raises(ValueError, match="needs 32"):
        lc.leco_server_submit_lookup(s, a, idx, np.zeros(4, dtype=np.uint32))  # 32-bit slots, 64-bit column
    with pytest.raises(ValueError, match="needs 80"):
        lc.leco_server_submit_range(s, a, 0, 10, np.zeros(9, dtype=np.uint64))
    with pytest.raises(ValueError, match="contiguous"):
        lc.leco_server_submit_range(s, a, 0, 10, np.zeros(20, dtype=np.uint64)[::2])
    ro = np.zeros(10, dtype=np.uint64)
    ro.flags.writeable = False
    with pytest.raises(ValueError, match="writable"):
        lc.leco_server_submit_range(s, a, 0, 10, ro)
    # exact sizes: 4 x 4 bytes for the 32-bit column, 10 x 8 for the 64-bit one
    out32, out64 = np.zeros(4, dtype=np.uint32), np.zeros(10, dtype=np.uint64)
    r1 = lc.leco_server_submit_lookup(s, b, idx, out32)
    r2 = lc.leco_server_submit_range(s, a, 5, 10, out64)
    assert lc.leco_server_wait(s, r1) == lc.LECO_OK and lc.leco_server_wait(s, r2) == lc.LECO_OK
    assert out32.tolist() == [mock_value(b, int(i), 32) for i in idx]
    assert out64.tolist() == [mock_value(a, i, 64) for i in range(5, 15)]
    # after eviction the id is unknown: the library refuses it
    lc.leco_server_evict(s, a)
    with pytest.raises(lc.LecoError) as e:
        lc.leco_server_submit_range(s, a, 0, 1, np.zeros(1, dtype=np.uint64))
    assert e.value.status == lc.LECO_ERR_INVALID_ARG
    s.destroy()
