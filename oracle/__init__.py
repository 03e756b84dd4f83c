"""LeCo CPU oracle: ctypes wrapper around ``leco_oracle.c``.

TEST INFRASTRUCTURE ONLY. The product path (the CUDA library and its Python binding) never imports
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
do. It shares no code with the CUDA path: the C source restates the algorithm from the paper
(Liu, Zeng & Zhang, LeCo, §3.1-§3.3) in plain loops, compiled with ``-ffp-contract=off``.

Arrays are numpy; values are passed as ``uint64`` (32-bit columns zero-extended).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leco_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

MODEL_CONSTANT = 0
MODEL_LINEAR = 1
MODEL_POLY = 2  # per-partition choice among constant, linear, quadratic and cubic (R10)
POLY_MIN_LEN = 64
POLY_MAX_LEN = 16384
METRIC_TILDE = 0
METRIC_DELTA = 1
SM_BITS = 256  # model size S_M: one 32-byte record
DEFAULT_CAP = 1 << 24
DEFAULT_CHUNK = 1 << 16

RECORD_DTYPE = np.dtype(
    [("theta0", "<f8"), ("theta1", "<f8"), ("start", "<u8"), ("word3", "<u8")]
)
assert RECORD_DTYPE.itemsize == 32


class _Fit(ctypes.Structure):
    _fields_ = [
        ("theta0", ctypes.c_double),
        ("theta1", ctypes.c_double),
        ("A", ctypes.c_int64),
        ("B", ctypes.c_int64),
        ("s", ctypes.c_int32),
        ("exact", ctypes.c_int32),
        ("b", ctypes.c_int32),
        ("fallback", ctypes.c_int32),
        ("shift", ctypes.c_int64),
    ]


class _PolyFit(ctypes.Structure):
    _fields_ = [
        ("c", ctypes.c_double * 4),
        ("K", ctypes.c_int64 * 4),
        ("sj", ctypes.c_int32 * 4),
        ("T", ctypes.c_int64),
        ("S", ctypes.c_int32),
        ("b", ctypes.c_int32),
        ("valid", ctypes.c_int32),
        ("degree", ctypes.c_int32),
        ("size", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (
        not force
        and os.path.exists(_SO)
        and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
    ):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
        "-fPIC", "-shared", _SRC, "-o", tmp, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    L = ctypes.CDLL(build())
    u64, i64, i32, dbl, vp = (
        ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
    )
    sig = {
        "orc_clamp_floor": (i64, [dbl]),
        "orc_predict": (i64, [dbl, dbl, u64]),
        "orc_fit_partition": (None, [vp, u64, i32, ctypes.POINTER(_Fit)]),
        "orc_partition_size_bits": (u64, [vp, u64, i32]),
        "orc_fit_poly": (None, [vp, u64, i32, ctypes.POINTER(_PolyFit)]),
        "orc_choose_kind": (i32, [vp, u64, ctypes.POINTER(u64)]),
        "orc_gram_p_parts": (None, [i32, u64, u64, ctypes.POINTER(u64), ctypes.POINTER(i64)]),
        "orc_gram_norm_parts": (None, [i32, u64, ctypes.POINTER(u64), ctypes.POINTER(i64)]),
        "orc_words_for_bits": (u64, [u64]),
        "orc_encode": (u64, [vp, u64, vp, u64, i32, vp, vp, u64]),
        "orc_decode": (None, [vp, u64, vp, u64, i32, vp]),
        "orc_lookup": (u64, [vp, u64, vp, u64, ctypes.c_uint32, i32, vp, u64, vp]),
        "orc_filter_sum": (None, [vp, u64, vp, u64, i32, u64, u64, vp]),
        "orc_delta_tilde": (i32, [vp, u64, u64]),
        "orc_delta_bits": (i32, [vp, u64, u64]),
        "orc_split_cost": (i64, [vp, u64, u64, i32]),
        "orc_var_split": (u64, [vp, u64, dbl, u64, u64, u64, i32, vp]),
        "orc_var_split_seeded": (u64, [vp, u64, dbl, u64, u64, u64, i32, vp]),
        "orc_chunk_seed": (u64, [vp, u64, u64]),
        "orc_var_merge_seq": (u64, [vp, vp, u64, i32, u64, u64, vp]),
        "orc_var_merge_round": (u64, [vp, vp, u64, i32, u64, u64, vp]),
        "orc_splitmix64": (u64, [u64]),
        "orc_search_samples": (u64, [u64, u64, dbl, u64, vp]),
        "orc_sample_size_bits": (u64, [vp, vp, u64, u64, u64, i32]),
        "orc_search_partition_size": (u64, [vp, u64, u64, dbl, u64, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _u64(a) -> np.ndarray:
    if not isinstance(a, np.ndarray):
        a = np.array(a, dtype=np.uint64)
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint64:
        a = a.astype(np.uint64)
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


# ------------------------------------------------------------------ prediction (§3.3)

def clamp_floor(y: float) -> int:
    return int(lib().orc_clamp_floor(float(y)))


def predict(theta0: float, theta1: float, x: int) -> int:
    """pred(i') = clamp_floor(fl(fl(theta1 * i') + theta0)) in binary64 without FMA."""
    return int(lib().orc_predict(float(theta0), float(theta1), int(x)))


# ------------------------------------------------------------------ regressor (§3.1)

def fit(values, model: int = MODEL_LINEAR) -> dict:
    v = _u64(values)
    f = _Fit()
    lib().orc_fit_partition(_p(v), v.size, model, ctypes.byref(f))
    return {k: getattr(f, k) for k, _ in _Fit._fields_}


def partition_size_bits(values, model: int = MODEL_LINEAR) -> int:
    v = _u64(values)
    return int(lib().orc_partition_size_bits(_p(v), v.size, model))


def fit_poly(values, degree: int) -> dict:
    """One polynomial candidate (R10): c (least-squares coefficients on p1..p3), K and sj (grid
    coefficients and their exponents), S, T, b, valid, size."""
    v = _u64(values)
    f = _PolyFit()
    lib().orc_fit_poly(_p(v), v.size, degree, ctypes.byref(f))
    return {"c": list(f.c), "K": list(f.K), "sj": list(f.sj), "S": f.S, "T": f.T, "b": f.b,
            "valid": f.valid, "degree": f.degree, "size": f.size}


def choose_model(values) -> tuple[int, int]:
    """(kind, size in bits) the polynomial model picks for one partition: kind 0 constant,
    1 linear, 2 quadratic, 3 cubic."""
    v = _u64(values)
    size = ctypes.c_uint64(0)
    k = lib().orc_choose_kind(_p(v), v.size, ctypes.byref(size))
    return int(k), int(size.value)


def _i128(lo, hi) -> int:
    return (int(hi.value) << 64) | int(lo.value)


def gram_p(j: int, N: int, x: int) -> int:
    lo, hi = ctypes.c_uint64(0), ctypes.c_int64(0)
    lib().orc_gram_p_parts(j, N, x, ctypes.byref(lo), ctypes.byref(hi))
    return _i128(lo, hi)


def gram_norm(j: int, N: int) -> int:
    lo, hi = ctypes.c_uint64(0), ctypes.c_int64(0)
    lib().orc_gram_norm_parts(j, N, ctypes.byref(lo), ctypes.byref(hi))
    return _i128(lo, hi)


# ------------------------------------------------------------------ partitions (§3.2)

def fixed_starts(n: int, L: int) -> np.ndarray:
    """Fixed-length partitioning (§3.2.1): partition j covers [jL, min((j+1)L, n))."""
    if L < 1:
        raise ValueError("partition size must be >= 1")
    m = (n + L - 1) // L
    s = np.arange(m + 1, dtype=np.uint64) * np.uint64(L)
    s[-1] = n
    return s


def var_split(values, tau: float = 0.1, sm_bits: int = SM_BITS, cap: int = DEFAULT_CAP,
              chunk: int = DEFAULT_CHUNK, metric: int = METRIC_TILDE, seeded: bool = False) -> np.ndarray:
    """Split phase (§3.2.2, R7); seeded: partitions grow from each chunk's seed both ways (R11)."""
    v = _u64(values)
    out = np.zeros(v.size + 1, dtype=np.uint64)
    f = lib().orc_var_split_seeded if seeded else lib().orc_var_split
    m = f(_p(v), v.size, float(tau), sm_bits, cap, chunk, metric, _p(out))
    return out[: m + 1].copy()


def chunk_seed(values, a: int, e: int) -> int:
    v = _u64(values)
    return int(lib().orc_chunk_seed(_p(v), a, e))


def var_merge_seq(values, starts, model: int = MODEL_LINEAR, sm_bits: int = SM_BITS,
                  cap: int = DEFAULT_CAP):
    v = _u64(values)
    st = _u64(starts).copy()
    passes = ctypes.c_uint64(0)
    m = lib().orc_var_merge_seq(_p(v), _p(st), max(st.size - 1, 0), model, sm_bits, cap,
                                ctypes.byref(passes))
    return st[: m + 1].copy(), int(passes.value)


def var_merge_round(values, starts, model: int = MODEL_LINEAR, sm_bits: int = SM_BITS,
                    cap: int = DEFAULT_CAP):
    v = _u64(values)
    st = _u64(starts).copy()
    rounds = ctypes.c_uint64(0)
    m = lib().orc_var_merge_round(_p(v), _p(st), max(st.size - 1, 0), model, sm_bits, cap,
                                  ctypes.byref(rounds))
    return st[: m + 1].copy(), int(rounds.value)


def var_partition(values, tau: float = 0.1, model: int = MODEL_LINEAR, variant: str = "round",
                  cap: int = DEFAULT_CAP, chunk: int = DEFAULT_CHUNK, seeded: bool = False) -> np.ndarray:
    """Split then merge (§3.2.2). variant 'round' uses chunked split + round merge; 'seq' the
    paper's literal single sweep + sequential merge passes. seeded: the seeded split (R11)."""
    if variant == "round":
        st = var_split(values, tau, SM_BITS, cap, chunk, seeded=seeded)
        st, _ = var_merge_round(values, st, model, SM_BITS, cap)
    elif variant == "seq":
        st = var_split(values, tau, SM_BITS, cap, 0)
        st, _ = var_merge_seq(values, st, model, SM_BITS, cap)
    else:
        raise ValueError(variant)
    return st


def search_samples(n: int, N: int, frac: float = 0.01, seed: int = 0) -> np.ndarray:
    """Starts of the subsequences of length N sampled for the partition-size search (§3.2.1)."""
    kmax = max(1, int(frac * n / N)) if n > N else 1
    out = np.zeros(kmax, dtype=np.uint64)
    k = lib().orc_search_samples(n, N, float(frac), int(seed), _p(out))
    return out[:k].copy()


def sample_size_bits(values, starts, N: int, L: int, model: int = MODEL_LINEAR) -> int:
    v = _u64(values)
    st = _u64(starts)
    return int(lib().orc_sample_size_bits(_p(v), _p(st), st.size, N, L, model))


def search_partition_size(values, N: int = 10000, frac: float = 0.01, seed: int = 0,
                          model: int = MODEL_LINEAR):
    """Fixed partition size search (§3.2.1): (L, sample size in bits at L, sizes evaluated)."""
    v = _u64(values)
    bits = ctypes.c_uint64(0)
    ne = ctypes.c_uint64(0)
    L = lib().orc_search_partition_size(_p(v), v.size, N, float(frac), int(seed), model, ctypes.byref(bits),
                                        ctypes.byref(ne))
    return int(L), int(bits.value), int(ne.value)


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(int(x)))


def delta_tilde(values, i: int, j: int) -> int:
    v = _u64(values)
    return int(lib().orc_delta_tilde(_p(v), i, j))


def delta_bits(values, i: int, j: int) -> int:
    v = _u64(values)
    return int(lib().orc_delta_bits(_p(v), i, j))


def split_cost(values, i: int, j: int, metric: int = METRIC_TILDE) -> int:
    v = _u64(values)
    return int(lib().orc_split_cost(_p(v), i, j, metric))


# ------------------------------------------------------------------ encoder / decoder (§3.3)

def words_for_bits(total_bits: int) -> int:
    return int(lib().orc_words_for_bits(total_bits))


def encode(values, starts, model: int = MODEL_LINEAR):
    """Fit and pack every partition [starts[p], starts[p+1]). Returns (records, words)."""
    v = _u64(values)
    st = _u64(starts)
    m = max(st.size - 1, 0)
    rec = np.zeros(m, dtype=RECORD_DTYPE)
    cap = words_for_bits(64 * v.size + 320 * m)
    words = np.zeros(cap, dtype=np.uint64)
    nw = lib().orc_encode(_p(v), v.size, _p(st), m, model, _p(rec), _p(words), cap)
    if nw == 0:
        raise RuntimeError("oracle encode: word buffer too small")
    return rec, words[:nw].copy()


def encode_fixed(values, L: int, model: int = MODEL_LINEAR):
    return encode(values, fixed_starts(len(values), L), model)


def decode(records, words, n: int, dtype_bits: int = 64) -> np.ndarray:
    rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
    w = _u64(words)
    out = np.zeros(n, dtype=np.uint64)
    lib().orc_decode(_p(rec), rec.size, _p(w), n, dtype_bits, _p(out))
    return out


def lookup(records, words, n: int, idx, L: int = 0, dtype_bits: int = 64):
    """Point lookups; L > 0 fixed partitions, L == 0 variable. Returns (values, n_out_of_range)."""
    rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
    w = _u64(words)
    ix = _u64(idx)
    out = np.zeros(ix.size, dtype=np.uint64)
    bad = lib().orc_lookup(_p(rec), rec.size, _p(w), n, L, dtype_bits, _p(ix), ix.size, _p(out))
    return out, int(bad)


def filter_sum(records, words, n: int, lo: int, hi: int, dtype_bits: int = 64):
    """(count, sum) over lo <= v <= hi (unsigned); sum is a Python int, exact mod 2^128."""
    rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
    w = _u64(words)
    out = np.zeros(3, dtype=np.uint64)
    lib().orc_filter_sum(_p(rec), rec.size, _p(w), n, dtype_bits, int(lo), int(hi), _p(out))
    return int(out[0]), int(out[1]) | (int(out[2]) << 64)


# ------------------------------------------------------------------ record fields (format R6)

def rec_offset(word3) -> np.ndarray:
    return np.asarray(word3, dtype=np.uint64) & np.uint64((1 << 48) - 1)


def rec_width(word3) -> np.ndarray:
    return (np.asarray(word3, dtype=np.uint64) >> np.uint64(48)) & np.uint64(0x7F)


def rec_grid(word3) -> np.ndarray:
    s = ((np.asarray(word3, dtype=np.uint64) >> np.uint64(55)) & np.uint64(0x7F)).astype(np.int64)
    return np.where(s >= 64, s - 128, s)


def rec_exact(word3) -> np.ndarray:
    return (np.asarray(word3, dtype=np.uint64) >> np.uint64(62)) & np.uint64(1)


def rec_poly(word3) -> np.ndarray:
    return (np.asarray(word3, dtype=np.uint64) >> np.uint64(63)) & np.uint64(1)


def compressed_bytes(records, words) -> int:
    return 32 * len(records) + 8 * len(words)
