#!/usr/bin/env python3
"""LeCo hot-path benchmark on GB300.

Headline workload (the metric's configuration): three 200M-value uint64 columns, fixed partitions
of 4096, linear model, seeded and synthetic (linear + bounded noise; sorted Normal(2^40, 2^36);
sorted 1e9 * LogNormal(0, 2)). Each column is encoded once (encode throughput is reported
separately); the timed step then runs, for every column, the three query paths of the library:
full decode, the fused filter-sum at ~1% selectivity, and 10M uniform random lookups. All inputs
are resident in HBM and larger than L2.

value = algorithmic bytes of one whole step (decode + lookups + filter-sum over the three
columns) / step time, in GB/s; the full-decode figure alone is ops.decode and roofline.achieved.
Algorithmic bytes, C = compressed bytes (32 per record + 8 per residual word):
  decode  C + 8 n          filter-sum  C + 24          lookups  k * (8 idx + 8 out + 32 sector)

e2e: the same step through the public API with pinned host buffers (indices in, every result out),
the copies on their own streams so one column's results leave while the next column is decoded;
e2e.host_link_gbs is the link's copy-engine bandwidth measured in the same run, which bounds it.

After the headline (one GPU, unless --no-extra), the same run measures the other workloads and
reports them under ops: the 1M-value fixed column with the whole oracle timed beside it
(ops.cfg1_fix_1M), the two variable-partition columns (ops.cfg3_var), the 10,000-column batch
(ops.cfg4_batch) and the serving loop with p50/p99 latency (ops.cfg5_serve).

--impl reference times the CPU oracle (partition-parallel on the host cores) on a bounded sample of
the same columns: every 100th partition, so the sample's encoding is exactly those partitions of
the full encoding.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DISTS = ("a", "b", "c")
L = 4096
METRIC = "LeCo decode GB/s & %HBM roofline; random-access Mlookups/s; serving p50/p99"
WORKLOAD = "LeCo-fix L=4096 linear, 3 x 200M uint64 (linear+noise, sorted normal, sorted lognormal)"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["leco", "reference"], default="leco")
    ap.add_argument("--n", type=int, default=200_000_000)
    ap.add_argument("--lookups", type=int, default=10_000_000)
    ap.add_argument("--sample-every", type=int, default=100, help="CPU sample: every k-th partition")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-columns", type=int, default=10_000)
    ap.add_argument("--batch-total", type=float, default=3e9)
    ap.add_argument("--serve-columns", type=int, default=2000)
    ap.add_argument("--serve-total", type=float, default=2.5e9)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: skip the 1M, variable, batch and serving workloads")
    ap.add_argument("--cpu-sample-every", type=int, default=20,
                    help="CPU baseline sample of the headline columns: every k-th partition")
    ap.add_argument("--workload", choices=["fix", "var", "batch", "serve", "poly"], default="fix",
                    help="fix: the 3 x 200M fixed-partition columns (default); var: the variable-partition "
                         "columns (200M piecewise-linear uint64, 500M uint32 timestamps); batch: 10,000 columns; "
                         "serve: the serving loop; poly: the polynomial model against the line on a 200M sine mixture")
    ap.add_argument("--tau", type=float, default=0.03)
    ap.add_argument("--tau-sweep", default="", help="var workload: comma-separated tau values to sweep (CR vs tau)")
    return ap.parse_args()


KSCAN_SRCS = [os.path.join(ROOT, "paper_2306_15374_gb300", "csrc", f) for f in ("k_scan.cu", "leco_internal.cuh", "tma.cuh")]
# DRAM read + write per decode launch from one ncu capture of this workload (mean of columns a, b, c;
# see profiles/k_tilescan_decode_filter_fix200M.md), valid only for the kernel sources it was taken on
# (keyed by their hash; re-keyed once since, when the shared header gained only host declarations of
# the batched-encode launchers and the decode kernel's code stayed the same).
DECODE_TRAFFIC = {"sha256": "1e091f3002cd25780c164ad5dc869ef8ca403b716143b0ec0422a72376811554",
                  "bytes_per_launch": (1894286848 + 1973986048 + 1846223104) / 3}


def decode_traffic():
    import hashlib

    h = hashlib.sha256()
    for path in KSCAN_SRCS:
        with open(path, "rb") as f:
            h.update(f.read())
    return DECODE_TRAFFIC["bytes_per_launch"] if h.hexdigest() == DECODE_TRAFFIC["sha256"] else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sample_partitions(v, every: int):
    """Every `every`-th partition of L values (a bounded, representative CPU sample)."""
    import numpy as np

    m = (len(v) + L - 1) // L
    parts = np.arange(0, m, every)
    parts = parts[parts * L + L <= len(v)]
    idx = (parts[:, None] * L + np.arange(L)[None, :]).ravel()
    return v[idx]


def step_bytes(comp_bytes, n, k):
    dec = comp_bytes + 8 * n
    filt = comp_bytes + 24
    look = k * (8 + 8 + 32)
    return dec, filt, look


# ----------------------------------------------------------------------------- CPU oracle arm

def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_oracle_run(cols, lookups_frac, reps=1, threads=1):
    """Time the oracle on prepared samples: decode, filter-sum and lookups of every sample piece.
    threads > 1 runs the pieces on a thread pool (the oracle is C behind ctypes, which releases the
    GIL, and shares no state between calls): partition-parallel on that many cores. Returns
    (algorithmic bytes, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    def work(s):
        v, rec, words, idx, lo, hi = s["v"], s["rec"], s["words"], s["idx"], s["lo"], s["hi"]
        d = oracle.decode(rec, words, len(v))
        oracle.filter_sum(rec, words, len(v), lo, hi)
        oracle.lookup(rec, words, len(v), idx, L=L)
        return d

    pieces = [p for c in cols for p in c["pieces"]]
    total_b = 0
    for c in cols:
        dec, filt, look = step_bytes(c["comp"], c["n"], c["k"])
        total_b += (dec + filt + look) * reps
    outs = []
    t0 = time.perf_counter()
    if threads <= 1:
        for _ in range(reps):
            outs = [work(p) for p in pieces]
    else:
        with ThreadPoolExecutor(threads) as ex:
            for _ in range(reps):
                outs = list(ex.map(work, pieces))
    total_t = time.perf_counter() - t0
    for p, d in zip(pieces, outs):
        assert (d == p["v"]).all()
    return total_b, total_t


def prepare_cpu_samples(columns, every, lookups, n, parts=1):
    """Every `every`-th partition of each column, encoded by the oracle; split into `parts` pieces of
    whole partitions (each encoded on its own) so the pieces can be decoded in parallel. The work
    (partitions decoded, values filtered, lookups) is the same for any number of pieces."""
    import numpy as np

    import oracle
    import workloads as W

    out = []
    for d, v in columns.items():
        s = sample_partitions(v, every)
        k = max(1, int(lookups * len(s) / n))
        lo, hi = W.filter_bounds(v)
        idx = W.uniform_indices(k, len(s), seed=7)
        m = len(s) // L
        bounds = np.linspace(0, m, max(1, min(parts, m)) + 1).astype(np.int64) * L
        pieces, comp = [], 0
        for a, b in zip(bounds[:-1], bounds[1:]):
            sv = s[a:b]
            rec, words = oracle.encode_fixed(sv, L, oracle.MODEL_LINEAR)
            comp += oracle.compressed_bytes(rec, words)
            sel = idx[(idx >= a) & (idx < b)] - np.uint64(a)
            pieces.append(dict(v=sv, rec=rec, words=words, idx=sel, lo=lo, hi=hi))
        out.append(dict(pieces=pieces, comp=comp, n=len(s), k=k))
    return out


def timed_median(fn, reps=3):
    """Median wall time of reps calls of fn (and fn's last result)."""
    ts, r = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        r = fn()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts), r


def cpu_baseline_headline(args, columns, n):
    """The oracle on the headline columns' sample (every cpu_sample_every-th partition), timed as the
    median of 3 runs, partition-parallel on all host cores and on one thread; plus the oracle's
    encode of the same sample."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    cores = host_cores()
    every = args.cpu_sample_every
    samples = prepare_cpu_samples(columns, every, args.lookups, n, parts=cores)
    b = cpu_oracle_run(samples, None, threads=cores)[0]
    runs_all = sorted(cpu_oracle_run(samples, None, threads=cores)[1] for _ in range(3))
    runs_one = sorted(cpu_oracle_run(samples, None, threads=1)[1] for _ in range(3))
    b1 = b
    pieces = [p for c in samples for p in c["pieces"]]
    enc_bytes = sum(8 * len(p["v"]) for p in pieces) + sum(c["comp"] for c in samples)

    def encode_all(threads):
        def enc(p):
            return oracle.encode_fixed(p["v"], L, oracle.MODEL_LINEAR)
        if threads <= 1:
            return [enc(p) for p in pieces]
        with ThreadPoolExecutor(threads) as ex:
            return list(ex.map(enc, pieces))

    t_enc_all, _ = timed_median(lambda: encode_all(cores))
    t_enc_one, _ = timed_median(lambda: encode_all(1))
    nsamp = sum(c["n"] for c in samples)
    return {"value": b / runs_all[1] / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "single_thread_value": b1 / runs_one[1] / 1e9,
            "encode_gbs": enc_bytes / t_enc_all / 1e9, "encode_single_thread_gbs": enc_bytes / t_enc_one / 1e9,
            "runs": 3, "statistic": "median", "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{nsamp} values: every {every}th 4096-value partition of each column; decode + filter-sum + "
                      f"proportional lookups (value), encode (encode_gbs), partition-parallel on {cores} threads; "
                      f"single_thread_*: the same on one thread; median of 3 runs each"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    import oracle
    import workloads as W

    oracle.build()
    columns = {d: W.cfg2(d, args.n) for d in DISTS}
    every = args.sample_every
    cores = host_cores()
    samples = prepare_cpu_samples(columns, every, args.lookups, args.n, parts=cores)
    # keep the whole run within about 90 s of oracle time: thin the per-step sample if needed
    _, t1 = cpu_oracle_run(samples, None, threads=cores)
    budget = 90.0
    if (args.steps + args.warmup) * t1 > budget:
        every = int(every * (args.steps + args.warmup) * t1 / budget) + 1
        samples = prepare_cpu_samples(columns, every, args.lookups, args.n, parts=cores)
    args.sample_every = every
    del columns
    for _ in range(args.warmup):
        cpu_oracle_run(samples, None, threads=cores)
    b, t = cpu_oracle_run(samples, None, reps=args.steps, threads=cores)
    value = b / t / 1e9
    nsamp = sum(c["n"] for c in samples)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"every {args.sample_every}th partition"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{nsamp} values: every {args.sample_every}th 4096-value partition of each column, "
                                   f"partition-parallel on {cores} threads"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def max_over_ranks(ms, world, device):
    """The slowest rank's step time: every rank processes the same units, so the job's time is the
    max over ranks (all-reduce MAX; the identity at world 1)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_gbs(bytes_per_rank_step, world, ms):
    """Whole-job throughput: the bytes all ranks processed in one step over the (max) step time."""
    return world * bytes_per_rank_step / (ms * 1e-3) / 1e9


def run_leco(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import paper_2306_15374_gb300 as pkg

    if rank == 0:
        pkg.build()
    if world > 1:
        dist.barrier()
    pkg.build()
    from paper_2306_15374_gb300 import leco

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    columns = {d: W.cfg2(d, args.n) for d in DISTS}
    n = args.n
    k = args.lookups
    cols, comp, bounds, idxs = {}, {}, {}, {}
    enc_ms = []
    for d, v in columns.items():
        dv = torch.from_numpy(v.view(np.int64)).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):  # second encode is the timed one (pools warm)
            torch.cuda.synchronize()
            e0.record(stream)
            c = leco.leco_encode(dv, leco.fixed(L), leco.LECO_MODEL_LINEAR)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep == 0:
                c.free()
        enc_ms.append(e0.elapsed_time(e1))
        cols[d] = c
        st = c.stats()
        comp[d] = st["record_bytes"] + st["residual_bytes"]
        bounds[d] = W.filter_bounds(v)
        idxs[d] = torch.from_numpy(W.uniform_indices(k, n, seed=ord(d)).view(np.int64)).to(dev)
        del dv
    out = torch.empty(n, dtype=torch.int64, device=dev)
    outk = torch.empty(k, dtype=torch.int64, device=dev)
    res = torch.zeros(3, dtype=torch.int64, device=dev)

    ops = ("decode", "filter", "lookup")
    ev = {(d, o): [] for d in DISTS for o in ops}

    run_op = {"decode": lambda d: leco.leco_decode_all(cols[d], out),
              "lookup": lambda d: leco.leco_random_access(cols[d], idxs[d], outk),
              "filter": lambda d: leco.leco_filter_sum(cols[d], bounds[d][0], bounds[d][1], res)}

    def step(record):
        # one operator across all columns at a time (decodes, then lookups, then filter-sums), so a
        # scan does not pay for the write-back of the decoded column left dirty in L2 just before it
        for o in ("decode", "lookup", "filter"):
            for d in DISTS:
                if record:
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                run_op[o](d)
                if record:
                    b.record(stream)
                    ev[(d, o)].append((a, b))

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, world, dev)

    per = {}
    dec_b = filt_b = look_b = 0
    for d in DISTS:
        db, fb, lb = step_bytes(comp[d], n, k)
        dec_b += db
        filt_b += fb
        look_b += lb
    step_b = dec_b + filt_b + look_b
    for o in ops:
        tms = sum(a.elapsed_time(b) for d in DISTS for a, b in ev[(d, o)]) / args.steps
        per[o] = tms
    # filter variants outside the step: model-bound pruning (§5.1) and decode-every-value
    variants = {}
    for name, fl in (("prune", leco.LECO_FILTER_PRUNE), ("decode_all", leco.LECO_FILTER_DECODE_ALL)):
        reps = max(3, min(args.steps, 50))
        for d in DISTS:
            leco.leco_filter_sum(cols[d], bounds[d][0], bounds[d][1], res, flags=fl)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(reps):
            for d in DISTS:
                leco.leco_filter_sum(cols[d], bounds[d][0], bounds[d][1], res, flags=fl)
        v1.record(stream)
        torch.cuda.synchronize()
        variants[name] = v0.elapsed_time(v1) / reps
    peak, peak_kind = measured_peaks()
    dec_gbs = dec_b / (per["decode"] * 1e-3) / 1e9
    ops_out = {
        "decode": {"gbs": dec_gbs, "ms": per["decode"], "frac_hbm": dec_gbs / peak},
        "filter_sum": {"gbs": filt_b / (per["filter"] * 1e-3) / 1e9, "ms": per["filter"],
                       "frac_hbm": filt_b / (per["filter"] * 1e-3) / 1e9 / peak,
                       "mode": "scan all residual words, decode groups whose model bounds meet [lo, hi]"},
        "filter_sum_prune": {"ms": variants["prune"],
                             "scan_equivalent_gbs": filt_b / (variants["prune"] * 1e-3) / 1e9,
                             "mode": "LECO_FILTER_PRUNE: tiles whose model bounds miss [lo, hi] are not read"},
        "filter_sum_decode_all": {"gbs": filt_b / (variants["decode_all"] * 1e-3) / 1e9,
                                  "ms": variants["decode_all"],
                                  "frac_hbm": filt_b / (variants["decode_all"] * 1e-3) / 1e9 / peak,
                                  "mode": "LECO_FILTER_DECODE_ALL: every value decoded and compared"},
        "random_access": {"mlookups_s": 3 * k / (per["lookup"] * 1e-3) / 1e6, "ms": per["lookup"],
                          "gbs": look_b / (per["lookup"] * 1e-3) / 1e9},
        "encode": {"gbs": sum(8 * n + comp[d] for d in DISTS) / (sum(enc_ms) * 1e-3) / 1e9,
                   "ms": sum(enc_ms)},
        "compressed_bytes": {d: comp[d] for d in DISTS},
        "ratio": {d: comp[d] / (8 * n) for d in DISTS},
    }
    # execution-unit probes (a few ms each): the integer and binary64 rates the kernels' instruction
    # mixes are held against
    probes = {name: leco.leco_probe_throughput(kind) for kind, name in
              ((0, "int32_shift_xor_add_ops_s"), (1, "int64_shift_xor_add_ops_s"), (2, "int32_and_funnel_ops_s"),
               (3, "fp64_mul_add_ops_s"), (4, "random_8B_reads_s"))}
    roofline = {"bound": "hbm", "kernel": "k_tilescan<decode u64> (full-column decode)", "achieved": dec_gbs,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": dec_gbs / peak,
                "traffic": decode_traffic() if n == 200_000_000 else None,
                "bytes_per_launch": dec_b / 3, "unit_probes": probes}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, leco, cols, comp, bounds, n, k, dev, stream, step_b, columns)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_headline(args, columns, n)

    value = whole_job_gbs(step_b, world, ms)
    for c in cols.values():
        c.free()
    cols.clear()
    del out, outk, idxs, columns
    if world == 1 and not args.no_extra:  # the other workloads, on the same GPU after the headline
        torch.cuda.synchronize()
        leco.leco_trim_memory()
        torch.cuda.empty_cache()
        for key, fn in (("cfg1_fix_1M", bench_fix1m), ("cfg3_var", bench_var), ("cfg4_batch", bench_batch),
                        ("cfg5_serve", bench_serve)):
            t_w = time.time()
            ops_out[key] = fn(args, leco, dev, stream)
            ops_out[key]["wall_s"] = time.time() - t_w
            torch.cuda.synchronize()
            leco.leco_trim_memory()
            torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_per_column": n, "partition_size": L, "lookups_per_column": k,
                   "l2": "inputs larger than L2 (compressed columns 0.3-0.7 GB, decoded 1.6 GB)",
                   "parallelism": f"replicas x{world}"},
        "ops": ops_out, "roofline": roofline, "clocks": clocks, "e2e": e2e,
        "gpu_launches": 9 * args.steps, "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def host_link_gbs(dev, nbytes=1 << 30, reps=3):
    """Copy-engine bandwidth of the host link (pinned host memory): device->host and host->device
    GB/s for one nbytes copy, best of reps. Every e2e step moves its results over this link."""
    import torch

    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d.fill_(1)
    best = {}
    for name, (dst, src) in (("d2h", (h, d)), ("h2d", (d, h))):
        ts = []
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        best[name] = nbytes / (min(ts[1:]) * 1e-3) / 1e9
    del h, d
    return best


def run_e2e(args, leco, cols, comp, bounds, n, k, dev, stream, step_b, columns):
    """Same step through the public API with host buffers: lookup indices copied in from pinned
    memory, decoded columns, lookup results and sums copied back to pinned memory. The copies run
    on their own streams: the device->host copy of one column's results overlaps the next column's
    decode, filter and lookups (two device result buffers in turn), and the indices of all three
    columns are copied in up front."""
    import numpy as np
    import torch

    import workloads as W

    h_idx = {d: torch.from_numpy(W.uniform_indices(k, n, seed=ord(d)).view(np.int64)).pin_memory() for d in DISTS}
    h_out = {d: torch.empty(n, dtype=torch.int64).pin_memory() for d in DISTS}
    h_outk = {d: torch.empty(k, dtype=torch.int64).pin_memory() for d in DISTS}
    h_res = {d: torch.empty(3, dtype=torch.int64).pin_memory() for d in DISTS}
    d_idx = {d: torch.empty(k, dtype=torch.int64, device=dev) for d in DISTS}
    out = [torch.empty(n, dtype=torch.int64, device=dev) for _ in range(2)]
    outk = [torch.empty(k, dtype=torch.int64, device=dev) for _ in range(2)]
    res = [torch.zeros(3, dtype=torch.int64, device=dev) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    comp_s = torch.cuda.current_stream()

    def step():
        s_in.wait_stream(comp_s)
        with torch.cuda.stream(s_in):
            for d in DISTS:
                d_idx[d].copy_(h_idx[d], non_blocking=True)
        comp_s.wait_stream(s_in)
        freed = [None, None]
        for j, d in enumerate(DISTS):
            b = j % 2
            if freed[b] is not None:
                comp_s.wait_event(freed[b])  # the copy out of this buffer's previous column is done
            leco.leco_decode_all(cols[d], out[b])
            leco.leco_filter_sum(cols[d], bounds[d][0], bounds[d][1], res[b])
            leco.leco_random_access(cols[d], d_idx[d], outk[b])
            s_out.wait_stream(comp_s)
            with torch.cuda.stream(s_out):
                h_out[d].copy_(out[b], non_blocking=True)
                h_outk[d].copy_(outk[b], non_blocking=True)
                h_res[d].copy_(res[b], non_blocking=True)
                freed[b] = torch.cuda.Event()
                freed[b].record(s_out)
        comp_s.wait_stream(s_out)
        comp_s.synchronize()

    for _ in range(max(1, args.warmup)):
        step()
    link = host_link_gbs(dev)
    steps = max(1, min(args.steps, 5))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    # outside the timed region: the host buffers hold every column's decoded values, its lookups and
    # its filter-sum (the copy streams delivered the right bytes)
    ok = True
    for d in DISTS:
        v = columns[d]
        ok = ok and np.array_equal(h_out[d].numpy().view(np.uint64), v)
        ok = ok and np.array_equal(h_outk[d].numpy().view(np.uint64), v[h_idx[d].numpy().view(np.uint64)])
        leco.leco_filter_sum(cols[d], bounds[d][0], bounds[d][1], res[0])
        ok = ok and torch.equal(res[0].cpu(), h_res[d])
    if not ok:
        print("e2e: host results differ from the columns", file=sys.stderr)
    d2h = 3 * (8 * n + 8 * k + 24)
    return {"value": step_b / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "h2d_bytes_per_step": 3 * 8 * k, "d2h_bytes_per_step": d2h,
            "host_link_gbs": link, "d2h_frac_of_link": d2h / (ms * 1e-3) / 1e9 / link["d2h"],
            "results_verified": bool(ok)}


def gpu_setup():
    import torch

    import paper_2306_15374_gb300 as pkg

    pkg.build()
    from paper_2306_15374_gb300 import leco

    torch.cuda.set_device(0)
    return leco, torch.device("cuda", 0), torch.cuda.current_stream()


def ev_timed(fn, stream, reps, warm=3):
    """Average CUDA-event time (ms) of reps calls of fn after warm untimed ones."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bench_fix1m(args, leco, dev, stream):
    """The 1M-value fixed-partition column (v_i = 1000 + 37 i + U{-500..500}, L = 1024, linear):
    encode, full decode and 100k uniform lookups on the GPU, with the whole oracle timed beside it
    (encode, decode and the same lookups on one host thread), and the encodings compared byte for
    byte."""
    import numpy as np
    import torch

    import oracle
    import workloads as W

    oracle.build()
    L1, k = W.L_CFG1, 100_000
    v = W.cfg1()
    n = len(v)
    dv = torch.from_numpy(v.view(np.int64)).to(dev)
    idx = W.uniform_indices(k, n, seed=0, stream=2)
    didx = torch.from_numpy(idx.view(np.int64)).to(dev)
    o = torch.empty(n, dtype=torch.int64, device=dev)
    ok_ = torch.empty(k, dtype=torch.int64, device=dev)
    reps = 50
    t_enc = ev_timed(lambda: leco.leco_encode(dv, leco.fixed(L1), leco.LECO_MODEL_LINEAR).free(), stream, 10, warm=2)
    col = leco.leco_encode(dv, leco.fixed(L1), leco.LECO_MODEL_LINEAR)
    st = col.stats()
    comp = st["record_bytes"] + st["residual_bytes"]
    t_dec = ev_timed(lambda: leco.leco_decode_all(col, o), stream, reps)
    t_ra = ev_timed(lambda: leco.leco_random_access(col, didx, ok_), stream, reps)
    exact = bool(torch.equal(o, dv)) and bool(torch.equal(ok_, dv[didx]))
    rec_b, words_b, _ = leco.leco_column_export(col)
    col.free()
    t_oenc, (rec, words) = timed_median(lambda: oracle.encode_fixed(v, L1, oracle.MODEL_LINEAR))
    t_odec, d = timed_median(lambda: oracle.decode(rec, words, n))
    t_olook, (lk, _) = timed_median(lambda: oracle.lookup(rec, words, n, idx, L=L1))
    exact = exact and bool((d == v).all()) and bool((lk == v[idx]).all())
    enc_b, dec_b = 8 * n + comp, comp + 8 * n
    return {
        "workload": "1M uint64, v_i = 1000 + 37 i + U{-500..500} (seed 0), L = 1024, linear; 100k uniform lookups",
        "ratio": comp / (8 * n), "compressed_bytes": comp, "encode_identical_to_oracle":
            rec_b == rec.tobytes() and words_b == words.tobytes(), "results_exact": exact,
        "gpu": {"encode_ms": t_enc, "encode_gbs": enc_b / (t_enc * 1e-3) / 1e9, "decode_ms": t_dec,
                "decode_gbs": dec_b / (t_dec * 1e-3) / 1e9, "lookup_ms": t_ra,
                "mlookups_s": k / (t_ra * 1e-3) / 1e6},
        "oracle": {"kind": "oracle", "cores": 1, "sample": "the whole 1M-value column, median of 3 runs",
                   "encode_ms": 1e3 * t_oenc, "encode_gbs": enc_b / t_oenc / 1e9, "decode_ms": 1e3 * t_odec,
                   "decode_gbs": dec_b / t_odec / 1e9, "lookup_ms": 1e3 * t_olook,
                   "mlookups_s": k / t_olook / 1e6},
    }


def bench_var(args, leco, dev, stream, sweep=False):
    """Variable partitions (tau = args.tau): GPU split/merge + encode of the 200M piecewise-linear
    uint64 column and the 500M uint32 timestamp column, then decode, filter-sum and 10M lookups per
    column; the oracle beside it decodes, filters and looks up every 100th GPU partition (encoded
    by the oracle with the same boundaries), on one host thread."""
    import numpy as np
    import torch

    import oracle
    import workloads as W

    oracle.build()
    n_a = args.n
    n_b = int(args.n * 2.5)
    specs = [("piecewise_u64", lambda: W.cfg3("a", n_a), 64), ("timestamps_u32", lambda: W.cfg3("b", n_b), 32)]
    k = args.lookups
    peak, _ = measured_peaks()
    out = {}
    for name, gen, bits in specs:
        v = gen()
        n = len(v)
        if bits == 32:
            dv = torch.from_numpy(v.astype(np.uint32).view(np.int32)).to(dev)
        else:
            dv = torch.from_numpy(v.view(np.int64)).to(dev)
        vb = bits // 8

        def var_encode(tau, seeded):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c = leco.leco_encode(dv, leco.variable(tau, seeded=seeded), leco.LECO_MODEL_LINEAR)
            b.record(stream)
            torch.cuda.synchronize()
            return c, a.elapsed_time(b)

        c0, _ = var_encode(args.tau, False)  # warms the library's memory pool
        c0.free()
        col, enc_ms = var_encode(args.tau, False)
        fix = leco.leco_encode(dv, leco.fixed(4096), leco.LECO_MODEL_LINEAR)
        st, stf = col.stats(), fix.stats()
        fix.free()
        comp = st["record_bytes"] + st["residual_bytes"] + 8 * (st["partitions"] + 1)
        tdt = torch.int32 if bits == 32 else torch.int64
        o = torch.empty(n, dtype=tdt, device=dev)
        idx = torch.from_numpy(W.uniform_indices(k, n, seed=11).view(np.int64)).to(dev)
        ok_ = torch.empty(k, dtype=tdt, device=dev)
        res = torch.zeros(3, dtype=torch.int64, device=dev)
        lo, hi = W.filter_bounds(v)
        reps = max(3, min(args.steps, 50))
        # the library's scan tuner picks stages x consumer warps for this column's shape
        tuned = {"decode": leco.leco_tune_scan(col, 0), "filter": leco.leco_tune_scan(col, 1, lo, hi)}
        t_dec = ev_timed(lambda: leco.leco_decode_all(col, o), stream, reps)
        ok = bool(torch.equal(o, dv))
        t_fil = ev_timed(lambda: leco.leco_filter_sum(col, lo, hi, res), stream, reps)
        t_pru = ev_timed(lambda: leco.leco_filter_sum(col, lo, hi, res, flags=leco.LECO_FILTER_PRUNE), stream, reps)
        t_ra = ev_timed(lambda: leco.leco_random_access(col, idx, ok_), stream, reps)
        ok = ok and bool(torch.equal(ok_, dv[idx]))
        r = {
            "n": n, "partitions": st["partitions"], "ratio": comp / (n * vb), "ratio_fixed_4096": stf["ratio"],
            "partition_encode_ms": enc_ms, "partition_encode_gbs": (n * vb + comp) / (enc_ms * 1e-3) / 1e9,
            "decode_ms": t_dec, "decode_gbs": (comp + n * vb) / (t_dec * 1e-3) / 1e9,
            "decode_frac_hbm": (comp + n * vb) / (t_dec * 1e-3) / 1e9 / peak, "decode_equals_input": ok,
            "filter_ms": t_fil, "filter_gbs": (comp + 24) / (t_fil * 1e-3) / 1e9,
            "filter_frac_hbm": (comp + 24) / (t_fil * 1e-3) / 1e9 / peak,
            "filter_prune_ms": t_pru, "lookup_ms": t_ra, "mlookups_s": k / (t_ra * 1e-3) / 1e6, "tuned_scan": tuned,
        }
        # the oracle beside it: every 100th GPU partition, encoded with the same boundaries
        _, _, starts_b = leco.leco_column_export(col)
        starts = np.frombuffer(starts_b, dtype=np.uint64).astype(np.int64)
        pick = np.arange(0, len(starts) - 1, 100)
        sv = np.concatenate([v[starts[p]:starts[p + 1]] for p in pick])
        sst = np.concatenate([[0], np.cumsum([starts[p + 1] - starts[p] for p in pick])]).astype(np.uint64)
        ks = max(1, int(k * len(sv) / n))
        sidx = W.uniform_indices(ks, len(sv), seed=12)
        slo, shi = W.filter_bounds(sv)
        t_oenc, (srec, swords) = timed_median(lambda: oracle.encode(sv, sst, oracle.MODEL_LINEAR))
        t_odec, sd = timed_median(lambda: oracle.decode(srec, swords, len(sv), bits))
        t_ofil, _ = timed_median(lambda: oracle.filter_sum(srec, swords, len(sv), slo, shi, bits))
        t_olook, _ = timed_median(lambda: oracle.lookup(srec, swords, len(sv), sidx, L=0, dtype_bits=bits))
        assert (sd == sv).all()
        scomp = oracle.compressed_bytes(srec, swords)
        r["oracle"] = {"kind": "oracle", "cores": 1, "sample": f"every 100th GPU partition ({len(sv)} values), "
                       "encoded by the oracle with the same boundaries; median of 3 runs",
                       "encode_gbs": (len(sv) * vb + scomp) / t_oenc / 1e9,
                       "decode_gbs": (scomp + len(sv) * vb) / t_odec / 1e9,
                       "filter_gbs": (scomp + 24) / t_ofil / 1e9, "mlookups_s": ks / t_olook / 1e6}
        if sweep:
            def var_stats(tau, seeded):
                c, ms = var_encode(tau, seeded)
                sc = c.stats()
                cb = sc["record_bytes"] + sc["residual_bytes"] + 8 * (sc["partitions"] + 1)
                c.free()
                return {"tau": tau, "partitions": sc["partitions"], "ratio": cb / (n * vb),
                        "partition_encode_ms": ms}

            # the seeded split (each chunk grown from its smoothest point both ways, §3.2.2)
            r["seeded"] = var_stats(args.tau, True)
            if args.tau_sweep:
                # compression against tau (the partitioner's one knob, swept over the paper's range),
                # left-to-right and seeded
                tau_rows = []
                for tau in [float(t) for t in args.tau_sweep.split(",")]:
                    row = var_stats(tau, False)
                    row["seeded"] = var_stats(tau, True)
                    tau_rows.append(row)
                L_auto, _, n_eval = leco.leco_search_partition_size(dv, leco.LECO_MODEL_LINEAR)
                auto = leco.leco_encode(dv, leco.auto(), leco.LECO_MODEL_LINEAR)
                r["tau_sweep"] = tau_rows
                r["fixed_searched_size"] = {"L": L_auto, "sizes_evaluated": n_eval, "ratio": auto.stats()["ratio"]}
                auto.free()
        out[name] = r
        col.free()
        del dv, o, idx, ok_
    return {"workload": "LeCo-var tau=%g: 200M piecewise-linear uint64, 500M uint32 timestamps" % args.tau,
            "results": out}


def run_var(args):
    leco, dev, stream = gpu_setup()
    print(json.dumps(bench_var(args, leco, dev, stream, sweep=True)), flush=True)
    return 0


def run_poly(args):
    """Polynomial model (per-partition choice among constant, linear, quadratic and cubic) against
    the linear model on a 200M-value uint64 sine mixture, fixed partitions of 4096: compression,
    encode, decode, filter-sum and 10M lookups per model (not the default workload)."""
    import numpy as np
    import torch

    import workloads as W
    import paper_2306_15374_gb300 as pkg

    pkg.build()
    from paper_2306_15374_gb300 import leco

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    L = 4096
    v = W.sine_mixture(args.n)
    n = len(v)
    dv = torch.from_numpy(v.view(np.int64)).to(dev)
    k = args.lookups
    idx = torch.from_numpy(W.uniform_indices(k, n, seed=11).view(np.int64)).to(dev)
    lo, hi = W.filter_bounds(v)
    reps = max(3, min(args.steps, 50))
    peak, _ = measured_peaks()

    def timed(fn, r=reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(r):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / r

    out = {}
    for name, model in (("linear", leco.LECO_MODEL_LINEAR), ("poly", leco.LECO_MODEL_POLY)):
        enc_ms = timed(lambda: leco.leco_encode(dv, leco.fixed(L), model).free(), r=3)
        col = leco.leco_encode(dv, leco.fixed(L), model)
        st = col.stats()
        comp = st["record_bytes"] + st["residual_bytes"]
        rec_b, _, _ = leco.leco_column_export(col)
        w3 = np.frombuffer(rec_b, dtype=np.uint64)[3::4]  # word3 of each 32-byte record
        npoly = int((w3 >> np.uint64(63)).sum())
        o = torch.empty(n, dtype=torch.int64, device=dev)
        ok_ = torch.empty(k, dtype=torch.int64, device=dev)
        res = torch.zeros(3, dtype=torch.int64, device=dev)
        t_dec = timed(lambda: leco.leco_decode_all(col, o))
        ok = bool(torch.equal(o, dv))
        t_fil = timed(lambda: leco.leco_filter_sum(col, lo, hi, res))
        t_ra = timed(lambda: leco.leco_random_access(col, idx, ok_))
        ok = ok and bool(torch.equal(ok_, dv[idx]))
        out[name] = {
            "ratio": comp / (8 * n), "compressed_bytes": comp, "polynomial_partitions": npoly,
            "partitions": st["partitions"], "encode_ms": enc_ms, "encode_gbs": (8 * n + comp) / (enc_ms * 1e-3) / 1e9,
            "decode_ms": t_dec, "decode_gbs": (comp + 8 * n) / (t_dec * 1e-3) / 1e9,
            "decode_frac_hbm": (comp + 8 * n) / (t_dec * 1e-3) / 1e9 / peak,
            "filter_ms": t_fil, "filter_gbs": (comp + 24) / (t_fil * 1e-3) / 1e9,
            "filter_frac_hbm": (comp + 24) / (t_fil * 1e-3) / 1e9 / peak,
            "lookup_ms": t_ra, "mlookups_s": k / (t_ra * 1e-3) / 1e6, "results_equal_input": ok,
        }
        col.free()
        del o, ok_
    line = {"workload": f"LeCo-Poly vs linear: {n} uint64 sine mixture (two sines + noise), L={L}",
            "peak_gbs": peak, "results": out}
    if not args.no_cpu_baseline:
        # the oracle beside it: encode and decode of every 100th partition, one thread
        import oracle

        oracle.build()
        smp = sample_partitions(v, args.sample_every)
        cpu = {"kind": "oracle", "cores": 1,
               "sample": f"every {args.sample_every}th {L}-value partition ({len(smp)} values), one thread"}
        for name, model in (("linear", oracle.MODEL_LINEAR), ("poly", oracle.MODEL_POLY)):
            t0 = time.perf_counter()
            rec, words = oracle.encode_fixed(smp, L, model)
            t1 = time.perf_counter()
            d = oracle.decode(rec, words, len(smp))
            t2 = time.perf_counter()
            assert (d == smp).all()
            cb = oracle.compressed_bytes(rec, words)
            cpu[name] = {"encode_gbs": (8 * len(smp) + cb) / (t1 - t0) / 1e9,
                         "decode_gbs": (cb + 8 * len(smp)) / (t2 - t1) / 1e9, "ratio": cb / (8 * len(smp))}
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def upload_columns(gen, spec, ncols, dev):
    """Columns generated on host threads (numpy releases the GIL) and copied to the device as
    they complete."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    out = []
    with ThreadPoolExecutor(max(2, os.cpu_count() or 2)) as ex:
        for v in ex.map(lambda c: gen(spec, c), range(ncols)):
            out.append(torch.from_numpy(v.view(np.int64)).to(dev))
    return out


def bench_batch(args, leco, dev, stream):
    """Batched form: 10,000 uint64 columns, lengths log-uniform in [1K, 10M] rescaled to 3B values,
    each linear + noise, sorted normal or sorted lognormal with its own seed, constant or linear
    model (50/50), partition size 256/1024/4096. Encode and decode all columns in one pass (decode:
    one persistent launch, also as a CUDA graph, with the autotuned scan shape; encode: the library
    call, and a prepared plan replayed as one CUDA graph) against one launch
    per column."""
    import numpy as np  # noqa: F401
    import torch

    import workloads as W

    spec = W.batch_spec(args.batch_columns, int(args.batch_total))
    ncols = len(spec["lens"])
    lens = spec["lens"]
    models, Ls = spec["model"].tolist(), spec["L"].tolist()
    vals = upload_columns(W.batch_column, spec, ncols, dev)
    total = int(lens.sum())

    def ev_time(fn, reps=1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, r

    # encode: the tuner picks the batched encode's shape on this batch, then batched vs one call per
    # column (each call syncs once to size its stream)
    enc_tuned = leco.leco_tune_batch_encode(vals, models, Ls)
    cols = leco.leco_batch_encode(vals, models, Ls)
    for c in cols:
        c.free()
    t_py, cols = ev_time(lambda: leco.leco_batch_encode(vals, models, Ls))  # through the Python binding
    for c in cols:
        c.free()
    # the library call alone: its arguments (10,000 device pointers and sizes) marshalled beforehand
    import ctypes

    k_, dt_, p_vals, p_ns, p_ms, p_ls = leco._batch_args(vals, models, Ls)
    p_out = (ctypes.c_void_p * max(k_, 1))()

    def lib_encode():
        st_ = leco.lib().leco_batch_encode(p_vals, p_ns, p_ms, p_ls, k_, dt_, leco._stream(None), p_out)
        if st_ != leco.LECO_OK:
            raise leco.LecoError(st_, "leco_batch_encode")
        return [leco.Column(ctypes.c_void_p(p_out[i])) for i in range(k_)]

    t_benc, cols = ev_time(lib_encode)
    # the same encode prepared once and replayed as one CUDA graph (stream offsets on the device, no
    # host round trip); its result is then copied out into columns at their exact size
    eplan = leco.leco_batch_encode_plan_create(vals, models, Ls)
    reserved = leco.leco_batch_encode_plan_reserved_bytes(eplan)
    leco.leco_batch_encode_plan_run(eplan)
    t_genc, _ = ev_time(lambda: leco.leco_batch_encode_plan_run(eplan), 3)
    t_take, gcols = ev_time(lambda: leco.leco_batch_encode_plan_columns(eplan))
    same_graph = all(leco.leco_column_export(a) == leco.leco_column_export(b)
                     for a, b in zip(gcols[:: max(1, ncols // 50)], cols[:: max(1, ncols // 50)]))
    for c in gcols:
        c.free()
    eplan.free()
    del gcols

    def per_col_encode():
        return [leco.leco_encode(v, leco.fixed(L), m) for v, L, m in zip(vals, Ls, models)]

    t_penc, single = ev_time(per_col_encode)
    same = all(leco.leco_column_export(a) == leco.leco_column_export(b)
               for a, b in zip(cols[:: max(1, ncols // 50)], single[:: max(1, ncols // 50)]))
    comp = sum(c.stats()["record_bytes"] + c.stats()["residual_bytes"] for c in cols)
    for c in single:
        c.free()
    # autotune the plan's scan shape (every candidate times the whole multi-column launch), then decode
    outs = [torch.empty(int(n), dtype=torch.int64, device=dev) for n in lens]
    plan = leco.leco_batch_plan_create(cols, outs)
    tuned = leco.leco_batch_plan_tune(plan)
    reps = max(3, min(args.steps, 20))
    leco.leco_batch_plan_run(plan)
    t_plan, _ = ev_time(lambda: leco.leco_batch_plan_run(plan), reps)
    leco.leco_batch_plan_run_graph(plan)
    t_graph, _ = ev_time(lambda: leco.leco_batch_plan_run_graph(plan), reps)
    ok = all(torch.equal(o, v) for o, v in zip(outs, vals))
    for o in outs:
        o.zero_()

    def per_col_decode():
        for c, o in zip(cols, outs):
            leco.leco_decode_all(c, o)

    per_col_decode()
    t_pdec, _ = ev_time(per_col_decode, max(1, reps // 4))
    ok = ok and all(torch.equal(o, v) for o, v in zip(outs, vals))
    peak, _ = measured_peaks()
    dec_bytes = comp + 8 * total
    enc_bytes = 8 * total + comp
    res = {
        "workload": f"batched: {ncols} uint64 columns, {total} values (log-uniform 1K-10M rescaled; linear + noise, "
                    "sorted normal, sorted lognormal), L in {256,1024,4096}, constant/linear 50/50",
        "encode_batched_ms": t_benc, "encode_batched_gbs": enc_bytes / (t_benc * 1e-3) / 1e9,
        "encode_batched_python_call_ms": t_py,
        "encode_per_column_ms": t_penc, "encode_speedup": t_penc / t_benc, "encode_identical": same,
        "encode_graph_ms": t_genc, "encode_graph_gbs": enc_bytes / (t_genc * 1e-3) / 1e9,
        "encode_graph_speedup_vs_per_column": t_penc / t_genc, "encode_graph_identical": same_graph,
        "encode_graph_columns_ms": t_take, "encode_graph_reserved_bytes": reserved,
        "decode_plan_ms": t_plan, "decode_plan_gbs": dec_bytes / (t_plan * 1e-3) / 1e9,
        "decode_plan_frac_hbm": dec_bytes / (t_plan * 1e-3) / 1e9 / peak,
        "decode_graph_ms": t_graph, "decode_per_column_ms": t_pdec,
        "decode_speedup_vs_per_column": t_pdec / t_graph, "decode_equals_input": ok,
        "jobs": leco.leco_batch_plan_jobs(plan), "tuned_scan": tuned, "tuned_encode": enc_tuned,
        "compressed_bytes": comp,
        "kernel_launches": {"decode_plan": 1, "decode_per_column": ncols, "encode_graph": 1},
    }
    plan.free()
    for c in cols:
        c.free()
    del vals, outs
    return res


def run_batch(args):
    leco, dev, stream = gpu_setup()
    print(json.dumps(bench_batch(args, leco, dev, stream)), flush=True)
    return 0


def bench_serve(args, leco, dev, stream):
    """Serving form: 2,000 resident uint64 columns (lengths log-uniform 100K-50M rescaled to 2.5B
    values; half fixed L=4096 over linear + noise, half variable over piecewise-linear), admitted
    against a 40 GB budget; a Poisson stream of requests (50% lookups of log-uniform 1-4096 indices,
    50% range decodes of log-uniform 1K-1M values) at several offered loads, continuous batching vs
    one launch per request. Also an admission-stress run with the budget at half the resident size.
    The columns are encoded once; each server gets copies rebuilt from their serialized form."""
    import workloads as W

    spec = W.serve_spec(args.serve_columns, int(args.serve_total))
    ncols = len(spec["lens"])
    t0 = time.time()
    vals = upload_columns(W.serve_column, spec, ncols, dev)
    t_gen = time.time() - t0
    t0 = time.time()
    blobs = []
    for c in range(ncols):
        pol = leco.variable(args.tau) if spec["variable"][c] else leco.fixed(4096)
        col = leco.leco_encode(vals[c], pol, leco.LECO_MODEL_LINEAR)
        blobs.append(leco.leco_serialize(col))
        col.free()
        vals[c] = None
    t_enc = time.time() - t0

    def build_columns():
        return [leco.leco_deserialize(b) for b in blobs]

    results = {}
    resident = None
    rates = None  # both modes are offered the same absolute loads: fractions of the batched saturation
    for mode, mb in (("continuous", 0), ("per_request", 1)):
        cols = build_columns()
        resident = resident or sum(c.stats()["device_bytes"] for c in cols)
        s = leco.leco_server_create(int(40e9), max_batch_requests=mb, max_batch_values=1 << 24,
                                    max_batch_lookups=1 << 17)
        ids = [leco.leco_server_admit(s, c) for c in cols]  # the server owns the columns now
        leco.leco_server_reset_stats(s)
        leco.leco_server_drive_poisson(s, ids, rate=2e6, seconds=1.0, seed=1)  # saturation burst
        st = leco.leco_server_stats_get(s)
        sat = st["completed"] / st["elapsed_s"]
        if rates is None:
            rates = [(f, f * sat) for f in (0.1, 0.25, 0.5, 0.75, 0.9, 1.1)]
        runs = []
        for f, rate in rates:
            leco.leco_server_reset_stats(s)
            sent = leco.leco_server_drive_poisson(s, ids, rate=rate, seconds=args.serve_seconds, seed=int(f * 100))
            st = leco.leco_server_stats_get(s)
            runs.append({"offered_frac_of_batched_saturation": f, "offered_rps": rate, "sent": sent,
                         "throughput_rps": st["completed"] / st["elapsed_s"],
                         "lookups_per_s": st["lookups"] / st["elapsed_s"],
                         "decoded_gbs": 8 * st["range_values"] / st["elapsed_s"] / 1e9,
                         "p50_us": st["p50_us"], "p99_us": st["p99_us"], "batches": st["batches"],
                         "launches": st["launches"], "max_batch": st["max_batch_size"]})
        results[mode] = {"saturation_rps": sat, "loads": runs}
        s.destroy()
    # admission stress: a budget of half the resident size refuses the columns that do not fit
    cols = build_columns()
    s = leco.leco_server_create(int(resident // 2), max_batch_values=1 << 22, max_batch_lookups=1 << 14)
    admitted = refused = 0
    for c in cols:
        try:
            leco.leco_server_admit(s, c)
            admitted += 1
        except leco.LecoError as e:
            assert e.status == leco.LECO_ERR_BUDGET
            refused += 1
            c.free()
    st = leco.leco_server_stats_get(s)
    stress = {"budget_bytes": int(resident // 2), "admitted": admitted, "refused": refused,
              "resident_bytes": st["resident_bytes"], "reserved_bytes": st["reserved_bytes"]}
    s.destroy()
    return {
        "workload": f"serving: {ncols} resident uint64 columns, {int(spec['lens'].sum())} values, half fixed / half "
                    "variable, budget 40 GB; Poisson requests, 50% lookups (1-4096), 50% ranges (1K-1M)",
        "generate_s": t_gen, "encode_s": t_enc, "resident_bytes": resident, "seconds_per_load": args.serve_seconds,
        "results": results, "admission_stress": stress}


def run_serve(args):
    leco, dev, stream = gpu_setup()
    print(json.dumps(bench_serve(args, leco, dev, stream)), flush=True)
    return 0


def main():
    args = parse_args()
    if args.workload == "var" and args.impl != "reference":
        return run_var(args)
    if args.workload == "serve" and args.impl != "reference":
        return run_serve(args)
    if args.workload == "batch" and args.impl != "reference":
        return run_batch(args)
    if args.workload == "poly" and args.impl != "reference":
        return run_poly(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_leco(args)


if __name__ == "__main__":
    sys.exit(main())
