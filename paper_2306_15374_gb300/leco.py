"""Python binding of libleco (include/leco.h): argument marshalling only.

Every function has the name of the C entry point it calls. Device buffers are torch CUDA tensors
(their data pointers are passed through); streams are torch CUDA streams (default: the current
one). Values are stored in 8- or 4-byte integer tensors holding the unsigned bit patterns
(torch.int64/uint64 for 64-bit columns, torch.int32/uint32 for 32-bit ones). All compute runs in
the CUDA library; there is no CPU fallback: if libleco.so is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

from . import builder as _build

LECO_OK = 0
LECO_ERR_INVALID_ARG = 1
LECO_ERR_OOM = 2
LECO_ERR_INDEX_RANGE = 3
LECO_ERR_CUDA = 4
LECO_ERR_CORRUPT = 5
LECO_ERR_TIMEOUT = 6
LECO_ERR_BUDGET = 7

LECO_U32 = 0
LECO_U64 = 1
LECO_MODEL_CONSTANT = 0
LECO_MODEL_LINEAR = 1
LECO_MODEL_POLY = 2  # per partition: constant, linear, quadratic or cubic, by exact size
LECO_PART_FIXED = 0
LECO_PART_VAR = 1
LECO_PART_AUTO = 2
LECO_PART_VAR_SEEDED = 3  # variable, each chunk's split grown from its smoothest point both ways
LECO_FILTER_PRUNE = 1
LECO_FILTER_DECODE_ALL = 2


class LecoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {leco_status_string(status)} ({status})" if what else
                         f"{leco_status_string(status)} ({status})")


class PartitionPolicy(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("part_size", ctypes.c_uint32), ("tau", ctypes.c_double)]


class SumResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("sum_lo", ctypes.c_uint64), ("sum_hi", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64), ("partitions", ctypes.c_uint64), ("record_bytes", ctypes.c_uint64),
        ("residual_bytes", ctypes.c_uint64), ("total_bytes", ctypes.c_uint64), ("ratio", ctypes.c_double),
        ("dtype", ctypes.c_int32), ("kind", ctypes.c_int32), ("model", ctypes.c_int32),
        ("part_size", ctypes.c_uint32), ("residual_bits", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
    ]


class ScanConfig(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_uint32), ("consumer_warps", ctypes.c_uint32), ("ms", ctypes.c_double)]


class EncodeConfig(ctypes.Structure):
    _fields_ = [("item_values", ctypes.c_uint32), ("fit_ctas", ctypes.c_uint32), ("ms", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("max_batch_requests", ctypes.c_uint32),
        ("max_batch_lookups", ctypes.c_uint64), ("max_batch_values", ctypes.c_uint64), ("max_columns", ctypes.c_uint32),
        ("mock", ctypes.c_uint32), ("mock_batch_us", ctypes.c_uint32),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
        ("lookups", ctypes.c_uint64), ("range_values", ctypes.c_uint64), ("batches", ctypes.c_uint64),
        ("launches", ctypes.c_uint64), ("max_batch_size", ctypes.c_uint64), ("p50_us", ctypes.c_double),
        ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
        ("elapsed_s", ctypes.c_double), ("resident_bytes", ctypes.c_uint64), ("reserved_bytes", ctypes.c_uint64),
        ("columns", ctypes.c_uint32),
    ]


def fixed(L: int) -> PartitionPolicy:
    return PartitionPolicy(LECO_PART_FIXED, int(L), 0.0)


def variable(tau: float = 0.03, cap: int = 0, seeded: bool = False) -> PartitionPolicy:
    return PartitionPolicy(LECO_PART_VAR_SEEDED if seeded else LECO_PART_VAR, int(cap), float(tau))


def auto(max_len: int = 0) -> PartitionPolicy:
    """Fixed partitions of the size the §3.2.1 search picks over 1 .. max_len (0 = 10000)."""
    return PartitionPolicy(LECO_PART_AUTO, int(max_len), 0.0)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libleco.so from the package's _build directory (build it first with build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        raise RuntimeError(f"libleco.so is not built ({_build.SO}); run paper_2306_15374_gb300.build()")
    L = ctypes.CDLL(_build.SO)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    col_pp = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "leco_status_string": (ctypes.c_char_p, [i32]),
        "leco_version": (u32, []),
        "leco_encode": (i32, [vp, u64, i32, PartitionPolicy, i32, vp, col_pp]),
        "leco_var_partition": (i32, [vp, u64, i32, PartitionPolicy, i32, vp, ctypes.POINTER(u64), vp]),
        "leco_encode_with_starts": (i32, [vp, u64, i32, vp, u64, i32, vp, col_pp]),
        "leco_decode_all": (i32, [vp, vp, vp]),
        "leco_decode_range": (i32, [vp, u64, u64, vp, vp]),
        "leco_random_access": (i32, [vp, vp, u64, vp, vp]),
        "leco_filter_sum": (i32, [vp, u64, u64, u32, vp, vp]),
        "leco_sync": (i32, [vp, vp]),
        "leco_stats_get": (i32, [vp, ctypes.POINTER(Stats)]),
        "leco_column_export": (i32, [vp, vp, vp, vp]),
        "leco_serialize": (i32, [vp, vp, u64, ctypes.POINTER(u64)]),
        "leco_deserialize": (i32, [vp, u64, vp, col_pp]),
        "leco_column_free": (None, [vp]),
        "leco_column_free_async": (None, [vp, vp]),
        "leco_encode_fixed_noalloc": (i32, [vp, u64, i32, u32, i32, vp, vp, u64, ctypes.POINTER(u64), vp]),
        "leco_tune_scan": (i32, [vp, u32, u64, u64, vp, ctypes.POINTER(ScanConfig)]),
        "leco_tune_save": (i32, [ctypes.c_char_p]),
        "leco_tune_load": (i32, [ctypes.c_char_p]),
        "leco_batch_plan_create": (i32, [ctypes.POINTER(vp), ctypes.POINTER(vp), u32, col_pp]),
        "leco_batch_plan_run": (i32, [vp, vp]),
        "leco_batch_plan_run_graph": (i32, [vp, vp]),
        "leco_batch_plan_jobs": (u64, [vp]),
        "leco_batch_plan_sync": (i32, [vp, vp]),
        "leco_trim_memory": (i32, []),
        "leco_search_partition_size": (i32, [vp, u64, i32, i32, u32, ctypes.c_double, u64, vp,
                                             ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "leco_selftest_wait_timeout": (i32, [u32, vp]),
        "leco_probe_throughput": (i32, [i32, ctypes.POINTER(ctypes.c_double), vp]),
        "leco_batch_plan_tune": (i32, [vp, vp, ctypes.POINTER(ScanConfig)]),
        "leco_batch_plan_free": (None, [vp]),
        "leco_batch_decode": (i32, [ctypes.POINTER(vp), ctypes.POINTER(vp), u32, vp]),
        "leco_batch_encode": (i32, [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(i32),
                                    ctypes.POINTER(u32), u32, i32, vp, ctypes.POINTER(vp)]),
        "leco_tune_batch_encode": (i32, [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(i32),
                                         ctypes.POINTER(u32), u32, i32, vp, ctypes.POINTER(EncodeConfig)]),
        "leco_batch_encode_plan_create": (i32, [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(i32),
                                                ctypes.POINTER(u32), u32, i32, vp, col_pp]),
        "leco_batch_encode_plan_run": (i32, [vp, vp]),
        "leco_batch_encode_plan_columns": (i32, [vp, vp, ctypes.POINTER(vp)]),
        "leco_batch_encode_plan_reserved_bytes": (u64, [vp]),
        "leco_batch_encode_plan_free": (None, [vp]),
        "leco_server_create": (i32, [ctypes.POINTER(ServerConfig), col_pp]),
        "leco_server_admit": (i32, [vp, vp, ctypes.POINTER(u32)]),
        "leco_server_admit_mock": (i32, [vp, u64, i32, u64, ctypes.POINTER(u32)]),
        "leco_server_evict": (i32, [vp, u32]),
        "leco_server_submit_lookup": (i32, [vp, u32, vp, u64, vp, ctypes.POINTER(u64)]),
        "leco_server_submit_range": (i32, [vp, u32, u64, u64, vp, ctypes.POINTER(u64)]),
        "leco_server_wait": (i32, [vp, u64, u32, ctypes.POINTER(i32)]),
        "leco_server_drive_poisson": (i32, [vp, ctypes.POINTER(u32), u32, ctypes.c_double, ctypes.c_double, u64,
                                            ctypes.c_double, u64, u64, u64, ctypes.POINTER(u64)]),
        "leco_server_stats_get": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "leco_server_reset_stats": (i32, [vp]),
        "leco_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    """Names of the leco_* entry points this binding resolves from the library."""
    L = lib()
    return [n for n in dir(L) if n.startswith("leco_")]


# ------------------------------------------------------------------------------ helpers

def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dtype_of(t) -> int:
    import torch

    if t.element_size() == 8:
        return LECO_U64
    if t.element_size() == 4:
        return LECO_U32
    raise ValueError(f"values must be 4- or 8-byte integers, got {t.dtype}")


def _dev(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _room(t, nbytes: int, what: str) -> None:
    """A device buffer the call writes must hold nbytes: the library cannot see its size, and a
    short one would be written past its end on the device."""
    if t is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{what}: buffer of {t.numel() * t.element_size()} bytes, needs {nbytes}")


def _indices(t, what: str) -> None:
    if t.element_size() != 8:
        raise ValueError(f"{what}: indices must be 8-byte integers, got {t.dtype}")


def _check(status: int, what: str):
    if status != LECO_OK:
        raise LecoError(status, what)


class Column:
    """Owning handle of a leco_column (freed with leco_column_free when collected)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        self._shape = None  # (n, value bytes), read once: a column is immutable after encode

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("column already freed")
        return self._h

    def free(self):
        if self._h:
            lib().leco_column_free(self._h)
            self._h = None

    def free_async(self, stream=None):
        if self._h:
            lib().leco_column_free_async(self._h, _stream(stream))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = Stats()
        _check(lib().leco_stats_get(self.handle, ctypes.byref(s)), "leco_stats_get")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    @property
    def n(self) -> int:
        return self.stats()["n"]

    @property
    def dtype(self) -> int:
        return self.stats()["dtype"]

    def shape(self) -> tuple:
        """(values, bytes per value) of the column."""
        if self._shape is None:
            st = self.stats()
            self._shape = (int(st["n"]), 4 if st["dtype"] == LECO_U32 else 8)
        return self._shape


# ------------------------------------------------------------------------------ entry points

def leco_status_string(status: int) -> str:
    return lib().leco_status_string(int(status)).decode()


def leco_version() -> int:
    return int(lib().leco_version())


def leco_encode(values, policy: PartitionPolicy, model: int = LECO_MODEL_LINEAR, stream=None,
                dtype: int | None = None) -> Column:
    h = ctypes.c_void_p()
    dt = _dtype_of(values) if dtype is None else dtype
    _check(lib().leco_encode(_dev(values), values.numel(), dt, policy, model, _stream(stream),
                             ctypes.byref(h)), "leco_encode")
    return Column(h)


def leco_var_partition(values, starts_out, policy: PartitionPolicy, model: int = LECO_MODEL_LINEAR,
                       stream=None) -> int:
    """Split + merge on the device; starts_out (int64 CUDA tensor of n+1) gets m+1 starts; returns m."""
    m = ctypes.c_uint64(0)
    _room(starts_out, 8 * (values.numel() + 1), "leco_var_partition")
    _check(lib().leco_var_partition(_dev(values), values.numel(), _dtype_of(values), policy, model,
                                    _dev(starts_out), ctypes.byref(m), _stream(stream)),
           "leco_var_partition")
    return int(m.value)


def leco_encode_with_starts(values, starts, m: int, model: int = LECO_MODEL_LINEAR,
                            stream=None) -> Column:
    _indices(starts, "leco_encode_with_starts")
    if starts.numel() < int(m) + 1:
        raise ValueError(f"leco_encode_with_starts: {starts.numel()} starts, needs m + 1 = {int(m) + 1}")
    h = ctypes.c_void_p()
    _check(lib().leco_encode_with_starts(_dev(values), values.numel(), _dtype_of(values), _dev(starts),
                                         int(m), model, _stream(stream), ctypes.byref(h)),
           "leco_encode_with_starts")
    return Column(h)


def leco_decode_all(col: Column, out, stream=None) -> None:
    n, vb = col.shape()
    _room(out, n * vb, "leco_decode_all")
    _check(lib().leco_decode_all(col.handle, _dev(out), _stream(stream)), "leco_decode_all")


def leco_decode_range(col: Column, begin: int, count: int, out, stream=None) -> None:
    _room(out, int(count) * col.shape()[1], "leco_decode_range")
    _check(lib().leco_decode_range(col.handle, int(begin), int(count), _dev(out), _stream(stream)),
           "leco_decode_range")


def leco_random_access(col: Column, idx, out, stream=None) -> None:
    _indices(idx, "leco_random_access")
    _room(out, idx.numel() * col.shape()[1], "leco_random_access")
    _check(lib().leco_random_access(col.handle, _dev(idx), idx.numel(), _dev(out), _stream(stream)),
           "leco_random_access")


def leco_filter_sum(col: Column, lo: int, hi: int, out, flags: int = 0, stream=None) -> None:
    """out: CUDA tensor of >= 3 int64 (count, sum_lo, sum_hi)."""
    _room(out, 24, "leco_filter_sum")
    _check(lib().leco_filter_sum(col.handle, int(lo), int(hi), int(flags), _dev(out), _stream(stream)),
           "leco_filter_sum")


def leco_sync(col: Column, stream=None) -> int:
    """Returns the status code (LECO_OK or the first device-side error) without raising."""
    return int(lib().leco_sync(col.handle, _stream(stream)))


def leco_stats_get(col: Column) -> dict:
    return col.stats()


def leco_column_export(col: Column):
    """(records bytes, words bytes, starts bytes or None) copied to host as Python bytes."""
    st = col.stats()
    m, nw = st["partitions"], st["residual_bytes"] // 8
    rec = ctypes.create_string_buffer(max(32 * m, 1))
    words = ctypes.create_string_buffer(max(8 * nw, 1))
    starts = ctypes.create_string_buffer(8 * (m + 1)) if st["kind"] == LECO_PART_VAR else None
    _check(lib().leco_column_export(col.handle, rec, words, starts), "leco_column_export")
    return rec.raw[: 32 * m], words.raw[: 8 * nw], (starts.raw if starts is not None else None)


def leco_serialize(col: Column) -> bytes:
    need = ctypes.c_uint64(0)
    _check(lib().leco_serialize(col.handle, None, 0, ctypes.byref(need)), "leco_serialize")
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().leco_serialize(col.handle, buf, need.value, ctypes.byref(need)), "leco_serialize")
    return buf.raw[: need.value]


def leco_deserialize(blob: bytes, stream=None) -> Column:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().leco_deserialize(buf, len(blob), _stream(stream), ctypes.byref(h)), "leco_deserialize")
    return Column(h)


def leco_column_free(col: Column) -> None:
    col.free()


def leco_encode_fixed_noalloc(values, L: int, records_out, words_out, model: int = LECO_MODEL_LINEAR,
                              stream=None) -> int:
    """Fixed-partition encode into caller buffers with no device allocation (see include/leco.h).
    records_out: CUDA tensor of >= 32 * ceil(n / L) bytes; words_out: CUDA tensor whose byte size
    / 8 is the word capacity. Returns the stream's word count; raises LecoError (INVALID_ARG) when
    the capacity is too small, with the needed count in the exception's .nwords."""
    n = values.numel()
    m = (n + int(L) - 1) // int(L) if int(L) >= 1 else 0
    for name, t in (("records_out", records_out), ("words_out", words_out)):
        if not t.is_cuda or not t.is_contiguous() or t.device != values.device:
            raise ValueError(f"{name} must be a contiguous CUDA tensor on the values' device")
    if records_out.numel() * records_out.element_size() < 32 * m:
        raise ValueError(f"records_out holds fewer than 32 * {m} bytes")
    nw = ctypes.c_uint64(0)
    cap = words_out.numel() * words_out.element_size() // 8
    st = lib().leco_encode_fixed_noalloc(_dev(values), values.numel(), _dtype_of(values), int(L), model,
                                         _dev(records_out), _dev(words_out), cap, ctypes.byref(nw),
                                         _stream(stream))
    if st != LECO_OK:
        err = LecoError(st, "leco_encode_fixed_noalloc")
        err.nwords = int(nw.value)
        raise err
    return int(nw.value)


# ------------------------------------------------------------------------------ batch / tuning (leco_batch.h)

def leco_tune_scan(col: Column, op: int = 0, lo: int = 0, hi: int = (1 << 64) - 1, stream=None) -> dict:
    """Time the scan configurations on this column (op 0 decode, 1 filter-sum) and keep the best."""
    cfg = ScanConfig()
    _check(lib().leco_tune_scan(col.handle, int(op), int(lo), int(hi), _stream(stream), ctypes.byref(cfg)),
           "leco_tune_scan")
    return {"stages": cfg.stages, "consumer_warps": cfg.consumer_warps, "ms": cfg.ms}


def leco_selftest_wait_timeout(limit_us: int, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (LECO_ERR_TIMEOUT is the expected one)."""
    return int(lib().leco_selftest_wait_timeout(int(limit_us), _stream(stream)))


def leco_search_partition_size(values, model: int = 1, max_len: int = 0, sample_frac: float = 0.0, seed: int = 0,
                               stream=None):
    """Fixed partition-size search (§3.2.1) on a device column: (L, sample bits at L, sizes evaluated)."""
    L, bits, ne = ctypes.c_uint32(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().leco_search_partition_size(_dev(values), values.numel(), _dtype_of(values), int(model), int(max_len),
                                            float(sample_frac), int(seed),
                                            _stream(stream), ctypes.byref(L), ctypes.byref(bits), ctypes.byref(ne)),
           "leco_search_partition_size")
    return int(L.value), int(bits.value), int(ne.value)


PROBE_KINDS = {0: "int32 shift+xor+add", 1: "int64 shift+xor+add", 2: "int32 and+funnel shift", 3: "fp64 mul+add",
               4: "random 8-byte reads"}


def leco_probe_throughput(kind: int, stream=None) -> float:
    """Measured operations per second of one execution-unit probe (kinds in PROBE_KINDS)."""
    r = ctypes.c_double(0.0)
    _check(lib().leco_probe_throughput(int(kind), ctypes.byref(r), _stream(stream)), "leco_probe_throughput")
    return float(r.value)


def leco_trim_memory() -> None:
    """Return the device memory the library's pool keeps cached to the driver (current device)."""
    _check(lib().leco_trim_memory(), "leco_trim_memory")


def leco_tune_save(path: str) -> None:
    _check(lib().leco_tune_save(path.encode()), "leco_tune_save")


def leco_tune_load(path: str) -> None:
    _check(lib().leco_tune_load(path.encode()), "leco_tune_load")


def _handles(cols):
    return (ctypes.c_void_p * max(len(cols), 1))(*[c.handle for c in cols])


def _ptrs(outs):
    return (ctypes.c_void_p * max(len(outs), 1))(*[o.data_ptr() for o in outs])


def _outs_room(cols, outs, what: str) -> None:
    """outs[c] receives every value of cols[c]: one contiguous device buffer of at least n * value
    bytes per column."""
    if len(outs) != len(cols):
        raise ValueError(f"{what}: {len(cols)} columns but {len(outs)} outputs")
    for c, o in zip(cols, outs):
        n, vb = c.shape()
        _room(o, n * vb, what)
        if not o.is_cuda or not o.is_contiguous():
            raise ValueError(f"{what}: outputs must be contiguous CUDA tensors")


class BatchPlan:
    """Owning handle of a leco_batch_plan; keeps its columns and outputs alive."""

    def __init__(self, handle, cols, outs):
        self._h, self._cols, self._outs = handle, list(cols), list(outs)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("plan already freed")
        return self._h

    def free(self):
        if self._h:
            lib().leco_batch_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def leco_batch_plan_create(cols, outs) -> BatchPlan:
    _outs_room(cols, outs, "leco_batch_plan_create")
    h = ctypes.c_void_p()
    _check(lib().leco_batch_plan_create(_handles(cols), _ptrs(outs), len(cols), ctypes.byref(h)),
           "leco_batch_plan_create")
    return BatchPlan(h, cols, outs)


def leco_batch_plan_run(plan: BatchPlan, stream=None) -> None:
    _check(lib().leco_batch_plan_run(plan.handle, _stream(stream)), "leco_batch_plan_run")


def leco_batch_plan_run_graph(plan: BatchPlan, stream=None) -> None:
    _check(lib().leco_batch_plan_run_graph(plan.handle, _stream(stream)), "leco_batch_plan_run_graph")


def leco_batch_plan_tune(plan: BatchPlan, stream=None) -> dict:
    """Time the plan under every scan shape and keep the fastest for this plan."""
    cfg = ScanConfig()
    _check(lib().leco_batch_plan_tune(plan.handle, _stream(stream), ctypes.byref(cfg)), "leco_batch_plan_tune")
    return {"stages": cfg.stages, "consumer_warps": cfg.consumer_warps, "ms": cfg.ms}


def leco_batch_plan_sync(plan: BatchPlan, stream=None) -> int:
    """Synchronize and return (and clear) the first device error of the plan's runs (LECO_OK if none)."""
    return int(lib().leco_batch_plan_sync(plan.handle, _stream(stream)))


def leco_batch_plan_jobs(plan: BatchPlan) -> int:
    return int(lib().leco_batch_plan_jobs(plan.handle))


def leco_batch_plan_free(plan: BatchPlan) -> None:
    plan.free()


def leco_batch_decode(cols, outs, stream=None) -> None:
    _outs_room(cols, outs, "leco_batch_decode")
    _check(lib().leco_batch_decode(_handles(cols), _ptrs(outs), len(cols), _stream(stream)), "leco_batch_decode")


class Server:
    """Owning handle of a leco_server. Keeps each pending request's output buffer alive."""

    def __init__(self, handle):
        self._h = handle
        self._pending = {}
        self._width = {}  # bytes per value of each admitted column, for the output checks

    @property
    def handle(self):
        if not self._h:
            raise ValueError("server already destroyed")
        return self._h

    def destroy(self):
        if self._h:
            lib().leco_server_destroy(self._h)
            self._h = None
            self._pending.clear()
            self._width.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def leco_server_create(budget_bytes: int, max_inflight: int = 0, max_batch_requests: int = 0,
                       max_batch_lookups: int = 0, max_batch_values: int = 0, max_columns: int = 0,
                       mock: bool = False, mock_batch_us: int = 0) -> Server:
    cfg = ServerConfig(int(budget_bytes), int(max_inflight), int(max_batch_requests), int(max_batch_lookups),
                       int(max_batch_values), int(max_columns), 1 if mock else 0, int(mock_batch_us))
    h = ctypes.c_void_p()
    _check(lib().leco_server_create(ctypes.byref(cfg), ctypes.byref(h)), "leco_server_create")
    return Server(h)


def leco_server_admit(server: Server, col: Column) -> int:
    """The server takes ownership of the column (the Column handle is emptied)."""
    cid = ctypes.c_uint32(0)
    vb = col.shape()[1]
    _check(lib().leco_server_admit(server.handle, col.handle, ctypes.byref(cid)), "leco_server_admit")
    col._h = None
    server._width[int(cid.value)] = vb
    return int(cid.value)


def leco_server_admit_mock(server: Server, n: int, dtype: int, nbytes: int) -> int:
    cid = ctypes.c_uint32(0)
    _check(lib().leco_server_admit_mock(server.handle, int(n), int(dtype), int(nbytes), ctypes.byref(cid)),
           "leco_server_admit_mock")
    server._width[int(cid.value)] = 4 if int(dtype) == LECO_U32 else 8
    return int(cid.value)


def leco_server_evict(server: Server, col_id: int) -> None:
    _check(lib().leco_server_evict(server.handle, int(col_id)), "leco_server_evict")
    server._width.pop(int(col_id), None)


def _host_room(server: Server, col_id: int, out, count: int, what: str) -> None:
    """The server writes count values of the column's width into out, a host array it cannot
    size: a short or non-contiguous one would be written past its end. Unknown columns are left to
    the library, which refuses them."""
    vb = server._width.get(int(col_id))
    if vb is None:
        return
    if not out.flags["C_CONTIGUOUS"] or not out.flags["WRITEABLE"]:
        raise ValueError(f"{what}: out must be a writable C-contiguous array")
    if out.nbytes < int(count) * vb:
        raise ValueError(f"{what}: out of {out.nbytes} bytes, needs {int(count) * vb}")


def leco_server_submit_lookup(server: Server, col_id: int, idx, out) -> int:
    """idx: numpy uint64 array (copied); out: numpy array of the column's width (filled on completion)."""
    import numpy as np

    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    _host_room(server, col_id, out, idx.size, "leco_server_submit_lookup")
    rid = ctypes.c_uint64(0)
    _check(lib().leco_server_submit_lookup(server.handle, int(col_id), idx.ctypes.data_as(ctypes.c_void_p), idx.size,
                                           out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rid)),
           "leco_server_submit_lookup")
    server._pending[rid.value] = out
    return int(rid.value)


def leco_server_submit_range(server: Server, col_id: int, begin: int, count: int, out) -> int:
    _host_room(server, col_id, out, count, "leco_server_submit_range")
    rid = ctypes.c_uint64(0)
    _check(lib().leco_server_submit_range(server.handle, int(col_id), int(begin), int(count),
                                          out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rid)),
           "leco_server_submit_range")
    server._pending[rid.value] = out
    return int(rid.value)


def leco_server_wait(server: Server, req_id: int, timeout_ms: int = 60_000) -> int:
    """Returns the request's status; raises LecoError(TIMEOUT) if it is still pending."""
    res = ctypes.c_int(0)
    _check(lib().leco_server_wait(server.handle, int(req_id), int(timeout_ms), ctypes.byref(res)), "leco_server_wait")
    server._pending.pop(req_id, None)
    return int(res.value)


def leco_server_drive_poisson(server: Server, col_ids, rate: float, seconds: float, seed: int = 0,
                              lookup_frac: float = 0.5, max_lookup: int = 4096, min_range: int = 1000,
                              max_range: int = 1_000_000) -> int:
    ids = (ctypes.c_uint32 * len(col_ids))(*[int(c) for c in col_ids])
    sent = ctypes.c_uint64(0)
    _check(lib().leco_server_drive_poisson(server.handle, ids, len(col_ids), float(rate), float(seconds), int(seed),
                                           float(lookup_frac), int(max_lookup), int(min_range), int(max_range),
                                           ctypes.byref(sent)), "leco_server_drive_poisson")
    return int(sent.value)


def leco_server_stats_get(server: Server) -> dict:
    st = ServerStats()
    _check(lib().leco_server_stats_get(server.handle, ctypes.byref(st)), "leco_server_stats_get")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def leco_server_reset_stats(server: Server) -> None:
    _check(lib().leco_server_reset_stats(server.handle), "leco_server_reset_stats")


def leco_server_destroy(server: Server) -> None:
    server.destroy()


def _batch_args(values, models, Ls):
    k = len(values)
    if len(models) != k or len(Ls) != k:
        raise ValueError(f"{k} columns but {len(models)} models and {len(Ls)} partition sizes")
    dt = _dtype_of(values[0]) if k else LECO_U64
    if any(_dtype_of(v) != dt for v in values):
        raise ValueError("all columns of a batched encode must have the same value width")
    vals = (ctypes.c_void_p * max(k, 1))(*[_dev(v).value or 0 for v in values])
    ns = (ctypes.c_uint64 * max(k, 1))(*[v.numel() for v in values])
    ms = (ctypes.c_int * max(k, 1))(*[int(m) for m in models])
    ls = (ctypes.c_uint32 * max(k, 1))(*[int(x) for x in Ls])
    return k, dt, vals, ns, ms, ls


def leco_tune_batch_encode(values, models, Ls, stream=None) -> dict:
    """Time the batched encode's candidate shapes on these columns and keep the fastest (leco_batch.h)."""
    k, dt, vals, ns, ms, ls = _batch_args(values, models, Ls)
    cfg = EncodeConfig()
    _check(lib().leco_tune_batch_encode(vals, ns, ms, ls, k, dt, _stream(stream), ctypes.byref(cfg)),
           "leco_tune_batch_encode")
    return {"item_values": cfg.item_values, "fit_ctas": cfg.fit_ctas, "ms": cfg.ms}


def leco_batch_encode(values, models, Ls, stream=None) -> list:
    """Fixed-partition encode of several columns (CUDA tensors of one width) in one pass."""
    k, dt, vals, ns, ms, ls = _batch_args(values, models, Ls)
    out = (ctypes.c_void_p * max(k, 1))()
    _check(lib().leco_batch_encode(vals, ns, ms, ls, k, dt, _stream(stream), out), "leco_batch_encode")
    return [Column(ctypes.c_void_p(out[i])) for i in range(k)]


class BatchEncodePlan:
    """Owning handle of a leco_batch_encode_plan; keeps the input tensors its graph reads alive."""

    def __init__(self, handle, values):
        self._h = handle
        self._values = list(values)
        self.ncols = len(self._values)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("batch encode plan already freed")
        return self._h

    def free(self):
        if self._h:
            lib().leco_batch_encode_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def leco_batch_encode_plan_create(values, models, Ls, stream=None) -> BatchEncodePlan:
    """Prepare the batched encode of these columns as one CUDA graph (leco_batch.h)."""
    k, dt, vals, ns, ms, ls = _batch_args(values, models, Ls)
    h = ctypes.c_void_p()
    _check(lib().leco_batch_encode_plan_create(vals, ns, ms, ls, k, dt, _stream(stream), ctypes.byref(h)),
           "leco_batch_encode_plan_create")
    return BatchEncodePlan(h, values)


def leco_batch_encode_plan_run(plan: BatchEncodePlan, stream=None) -> None:
    _check(lib().leco_batch_encode_plan_run(plan.handle, _stream(stream)), "leco_batch_encode_plan_run")


def leco_batch_encode_plan_columns(plan: BatchEncodePlan, stream=None) -> list:
    out = (ctypes.c_void_p * max(plan.ncols, 1))()
    _check(lib().leco_batch_encode_plan_columns(plan.handle, _stream(stream), out), "leco_batch_encode_plan_columns")
    return [Column(ctypes.c_void_p(out[i])) for i in range(plan.ncols)]


def leco_batch_encode_plan_reserved_bytes(plan: BatchEncodePlan) -> int:
    return int(lib().leco_batch_encode_plan_reserved_bytes(plan.handle))


def leco_batch_encode_plan_free(plan: BatchEncodePlan) -> None:
    plan.free()
