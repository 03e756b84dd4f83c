"""Seeded synthetic columns for the LeCo path.

The only module that both the CUDA-path tests/bench and the CPU oracle consume. It holds no part of
the method's arithmetic (no fitting, packing or decoding): only value generators, index batches
and filter bounds. Every generator is numpy on the host with a PCG64 stream keyed by
(seed, stream), so one call yields the same array for both sides in one run.

The paper's integer datasets are not available; these stand in for them with the shapes of the
paper's synthetic and real workloads (§4.1): near-linear sequences with bounded noise, sorted
samples of a normal and a log-normal, piecewise-linear series with slope changes, and
timestamp-like increasing counters with jitter and jumps.
"""
from __future__ import annotations

import numpy as np

U64_MAX = (1 << 64) - 1


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


# ----------------------------------------------------------------------------- value columns

def linear_noise(n: int, base: int, slope: int, noise: int, seed: int = 0,
                 stream: int = 0) -> np.ndarray:
    """v_i = base + slope*i + U{-noise..noise}, as uint64 (base must keep values >= 0)."""
    g = rng(seed, stream)
    v = np.arange(n, dtype=np.int64)
    v *= slope
    v += base
    if noise:
        v += g.integers(-noise, noise + 1, size=n, dtype=np.int64)
    return v.astype(np.uint64)


def _sorted_standard_normal(n: int, g: np.random.Generator) -> np.ndarray:
    """n sorted N(0,1) samples without a sort: uniform order statistics from normalised
    exponential spacings, pushed through the inverse normal CDF."""
    from scipy.special import ndtri

    e = g.standard_exponential(n + 1)
    c = np.cumsum(e)
    u = c[:-1]
    u /= c[-1]
    return ndtri(u)


def _to_u64_sorted(x: np.ndarray) -> np.ndarray:
    x = np.rint(x)
    np.clip(x, 0.0, 1.8446744073709550e19, out=x)
    v = x.astype(np.uint64)
    np.maximum.accumulate(v, out=v)
    return v


def sorted_normal(n: int, mean: float, sd: float, seed: int = 0, stream: int = 0) -> np.ndarray:
    """Sorted samples of Normal(mean, sd) rounded to uint64."""
    z = _sorted_standard_normal(n, rng(seed, stream))
    z *= sd
    z += mean
    return _to_u64_sorted(z)


def sorted_lognormal(n: int, scale: float, sigma: float, seed: int = 0,
                     stream: int = 0) -> np.ndarray:
    """Sorted samples of scale * LogNormal(0, sigma) rounded to uint64."""
    z = _sorted_standard_normal(n, rng(seed, stream))
    z *= sigma
    np.exp(z, out=z)
    z *= scale
    return _to_u64_sorted(z)


def piecewise_linear(n: int, segments: int = 1000, mean_len: float = 200_000,
                     slope_range=(1.0, 1e4), max_k: int = 20, seed: int = 0,
                     stream: int = 0) -> np.ndarray:
    """Continuous piecewise-linear uint64 series: geometric segment lengths (mean mean_len,
    rescaled so they sum to n), slope U[slope_range] per segment, noise U{-2^k..2^k} with
    k ~ U{0..max_k} per segment; each segment starts where the previous one ended."""
    g = rng(seed, stream)
    segments = max(1, min(segments, n)) if n else 0
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    lens = g.geometric(1.0 / mean_len, size=segments).astype(np.float64)
    lens = np.maximum(1, np.rint(lens * (n / lens.sum()))).astype(np.int64)
    diff = n - int(lens.sum())
    i = segments - 1
    while diff != 0:  # put the rounding remainder on the last segments, keeping lengths >= 1
        take = diff if diff > 0 else max(diff, 1 - int(lens[i]))
        lens[i] += take
        diff -= take
        i = (i - 1) % segments
    slopes = g.uniform(slope_range[0], slope_range[1], size=segments)
    ks = g.integers(0, max_k + 1, size=segments)
    seg = np.repeat(np.arange(segments), lens)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    j = np.arange(n, dtype=np.int64) - offs[seg]
    rise = np.floor(slopes[seg] * j).astype(np.int64)
    seg_rise = np.floor(slopes * lens).astype(np.int64)
    starts = (1 << (max_k + 2)) + np.concatenate([[0], np.cumsum(seg_rise)[:-1]])
    amp = (np.int64(1) << ks.astype(np.int64))[seg]
    noise = g.integers(0, 2 * amp + 1, dtype=np.int64) - amp
    v = starts[seg] + rise + noise
    return v.astype(np.uint64)


def timestamps_u32(n: int, step: int = 1000, period: int = 86400, amp: int = 300,
                   jump_p: float = 0.001, jump_max: int = 1_000_000, seed: int = 0,
                   stream: int = 0) -> np.ndarray:
    """Increasing timestamp-like counter stored mod 2^32 (a wrapping 32-bit column):
    t_i = step*i + round(amp*sin(2 pi i/period)) + sum of Bernoulli(jump_p) x U{1..jump_max} jumps.
    Returned zero-extended as uint64."""
    g = rng(seed, stream)
    i = np.arange(n, dtype=np.int64)
    table = np.rint(amp * np.sin(2 * np.pi * np.arange(period) / period)).astype(np.int64)
    t = i * step + table[i % period]
    jumps = (g.random(n) < jump_p) * g.integers(1, jump_max + 1, size=n, dtype=np.int64)
    t += np.cumsum(jumps)
    return (t & 0xFFFFFFFF).astype(np.uint64)


def sine_mixture(n: int, base: int = 1 << 40, a1: float = 1e9, p1: float = 1e6, a2: float = 1e7,
                 p2: float = 4e4, noise: int = 128, seed: int = 0, stream: int = 0) -> np.ndarray:
    """Two superposed sine signals plus uniform noise, the sensor-like shape where higher-order
    models pay (§4's mixture-of-sines data set): v_i = base + floor(a1 sin(2 pi i/p1) +
    a2 sin(2 pi i/p2)) + U{-noise..noise}. Generated in chunks of 2^24 values."""
    g = rng(seed, stream)
    out = np.empty(n, dtype=np.uint64)
    step = 1 << 24
    for a in range(0, n, step):
        i = np.arange(a, min(n, a + step), dtype=np.float64)
        s = np.floor(a1 * np.sin(2 * np.pi * i / p1) + a2 * np.sin(2 * np.pi * i / p2)).astype(np.int64)
        out[a:a + i.size] = (base + s + g.integers(-noise, noise + 1, size=i.size, dtype=np.int64)).astype(np.uint64)
    return out


# ----------------------------------------------------------------------------- small / adversarial

def random_u64(n: int, seed: int = 0, stream: int = 0, bits: int = 64) -> np.ndarray:
    g = rng(seed, stream)
    hi = (1 << bits) - 1
    if bits == 64:
        return g.integers(0, 1 << 64, size=n, dtype=np.uint64, endpoint=False)
    return g.integers(0, hi, size=n, dtype=np.uint64, endpoint=True)


def adversarial_u64(n: int, seed: int = 0) -> np.ndarray:
    """Extremes: 0, 2^64-1, 2^63, 2^63-1 and alternations of them, mixed with random values."""
    g = rng(seed, 7)
    pool = np.array([0, U64_MAX, 1 << 63, (1 << 63) - 1, 1, U64_MAX - 1, 1 << 53, (1 << 53) + 1],
                    dtype=np.uint64)
    v = pool[g.integers(0, pool.size, size=n)]
    mask = g.random(n) < 0.25
    v[mask] = random_u64(int(mask.sum()), seed, 8)
    return v


def runs(n: int, run_len: int, seed: int = 0) -> np.ndarray:
    """Constant runs (the RLE case): each run of run_len equal values."""
    g = rng(seed, 9)
    vals = g.integers(0, 1 << 40, size=(n + run_len - 1) // max(run_len, 1), dtype=np.uint64)
    return np.repeat(vals, run_len)[:n]


def mixed_chunks_u64(seed: int = 0, chunk: int = 1 << 16) -> np.ndarray:
    """Six chunk-sized regions of different shape and a partial seventh, so that one column holds
    both split schedules and the decoder's zero-width runs: smooth (a line), noisy (noise 2^20),
    smooth with a noisy middle window, a line with rare jumps, constant runs, values near 2^63 (a
    chunk whose values leave (-2^62, 2^62)), then 1000 values of a line."""
    g = rng(seed, 10)
    i = np.arange(chunk, dtype=np.int64)
    parts = [
        1_000_000 + 37 * i,
        5_000_000 + 1000 * i + g.integers(-(1 << 20), (1 << 20) + 1, size=chunk),
        9_000_000 + 11 * i + np.where((i >= 40_000) & (i < 41_000), g.integers(0, 1 << 18, size=chunk), 0),
        20_000_000 + 1000 * i + np.cumsum((g.random(chunk) < 0.002) * g.integers(1, 100_000, size=chunk)),
        np.repeat(g.integers(0, 1 << 30, size=chunk // 700 + 1), 700)[:chunk],
    ]
    out = [p.astype(np.uint64) for p in parts]
    out.append(((1 << 63) - (1 << 40) + 3 * i + g.integers(0, 8, size=chunk)).astype(np.uint64))
    out.append((7 + 5 * np.arange(1000, dtype=np.int64)).astype(np.uint64))
    return np.concatenate(out)


# ----------------------------------------------------------------------------- queries

def uniform_indices(k: int, n: int, seed: int = 0, stream: int = 2) -> np.ndarray:
    if n == 0:
        return np.zeros(k, dtype=np.uint64)
    return rng(seed, stream).integers(0, n, size=k, dtype=np.uint64)


def filter_bounds(values: np.ndarray, frac_lo: float = 0.495, frac_hi: float = 0.505):
    """(lo, hi) = the values of rank floor(frac_lo*n) and floor(frac_hi*n) of the sorted column:
    an inclusive range selecting about 1% of the rows."""
    n = values.size
    if n == 0:
        return 0, 0
    a, b = int(frac_lo * n), min(int(frac_hi * n), n - 1)
    part = np.partition(values, [a, b])
    return int(part[a]), int(part[b])


# ----------------------------------------------------------------------------- named configs

L_CFG1 = 1024
L_CFG2 = 4096


def cfg1(n: int = 1_000_000) -> np.ndarray:
    """1M values v_i = 1000 + 37 i + U{-500..500}, seed 0 (partition size 1024)."""
    return linear_noise(n, 1000, 37, 500, seed=0)


def cfg2(dist: str, n: int = 200_000_000) -> np.ndarray:
    """200M-value fixed-partition columns (partition size 4096): 'a' linear 2^20 + 53 i +
    U{-4096..4096}; 'b' sorted Normal(2^40, 2^36); 'c' sorted 1e9 * LogNormal(0, 2)."""
    if dist == "a":
        return linear_noise(n, 1 << 20, 53, 4096, seed=1)
    if dist == "b":
        return sorted_normal(n, float(1 << 40), float(1 << 36), seed=2)
    if dist == "c":
        return sorted_lognormal(n, 1e9, 2.0, seed=3)
    raise ValueError(dist)


def cfg3(dist: str, n: int | None = None) -> np.ndarray:
    """Variable-partition columns: 'a' 200M piecewise-linear uint64; 'b' 500M uint32 timestamps."""
    if dist == "a":
        return piecewise_linear(200_000_000 if n is None else n, seed=4)
    if dist == "b":
        return timestamps_u32(500_000_000 if n is None else n, seed=5)
    raise ValueError(dist)


# ----------------------------------------------------------------------------- many-column workloads

def batch_spec(ncols: int = 10_000, total: int = 3_000_000_000, seed: int = 41) -> dict:
    """The many-column batch: lengths log-uniform in [1K, 10M], rescaled so they sum to `total`
    (each at least 1K); each column one of the three fixed-partition distributions (0: linear +
    noise as the 1M-value column, 1: sorted normal, 2: sorted lognormal, as the 200M-value ones),
    the constant or linear model (50/50) and a partition size in {256, 1024, 4096}."""
    g = rng(seed)
    lens = np.exp(g.uniform(np.log(1e3), np.log(1e7), size=ncols))
    lens = np.maximum(1000, np.rint(lens * (total / lens.sum()))).astype(np.int64)
    return {"lens": lens, "dist": g.integers(0, 3, size=ncols), "model": g.integers(0, 2, size=ncols),
            "L": g.choice(np.array([256, 1024, 4096]), size=ncols)}


def batch_column(spec: dict, c: int) -> np.ndarray:
    n, d = int(spec["lens"][c]), int(spec["dist"][c])
    if d == 0:
        return linear_noise(n, 1000, 37, 500, seed=1000 + c)
    if d == 1:
        return sorted_normal(n, float(1 << 40), float(1 << 36), seed=1000 + c)
    return sorted_lognormal(n, 1e9, 2.0, seed=1000 + c)


def serve_spec(ncols: int = 2_000, total: int = 2_500_000_000, seed: int = 53) -> dict:
    """The resident columns of the serving workload: lengths log-uniform in [100K, 50M], rescaled
    so they sum to `total` (each at least 100K); even columns fixed partitions (L = 4096) over
    linear + noise values, odd columns variable partitions over piecewise-linear values."""
    g = rng(seed)
    lens = np.exp(g.uniform(np.log(1e5), np.log(5e7), size=ncols))
    lens = np.maximum(100_000, np.rint(lens * (total / lens.sum()))).astype(np.int64)
    return {"lens": lens, "slope": g.integers(1, 100, size=ncols), "noise": g.integers(1, 4000, size=ncols),
            "variable": np.arange(ncols) % 2 == 1}


def serve_column(spec: dict, c: int) -> np.ndarray:
    n = int(spec["lens"][c])
    if spec["variable"][c]:
        return piecewise_linear(n, segments=max(1, n // 200_000), mean_len=200_000, seed=7000 + c)
    return linear_noise(n, 1 << 32, int(spec["slope"][c]), int(spec["noise"][c]), seed=7000 + c)
