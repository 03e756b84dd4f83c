"""The C-ABI library builds for sm_103a, loads, and exports every entry point its headers declare
(no GPU needed: nothing here launches a kernel)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(leco_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    import paper_2306_15374_gb300 as pkg

    return pkg.build()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("leco_encode", "leco_decode_all", "leco_random_access", "leco_filter_sum",
                     "leco_decode_range", "leco_serialize", "leco_deserialize", "leco_sync"):
        assert required in names
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        assert "torch" not in text and "at::" not in text and "c10" not in text


def test_library_exports_every_declared_symbol(built):
    import ctypes

    L = ctypes.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_resolves_entry_points(built):
    from paper_2306_15374_gb300 import leco

    names = set(leco.exported_symbols())
    assert {"leco_encode", "leco_decode_all", "leco_random_access", "leco_filter_sum"} <= names
    assert leco.leco_status_string(leco.LECO_ERR_CORRUPT) == "LECO_ERR_CORRUPT"
    assert leco.leco_version() >= 10000


def test_host_side_argument_errors(built):
    """Argument checks happen on the host, before any CUDA call."""
    import ctypes

    from paper_2306_15374_gb300 import leco

    L = leco.lib()
    h = ctypes.c_void_p()
    assert L.leco_encode(None, 10, 1, leco.fixed(16), 1, None, ctypes.byref(h)) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_encode(None, 0, 7, leco.fixed(16), 1, None, ctypes.byref(h)) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_encode(None, 0, 1, leco.fixed(16), 1, None, None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_decode_all(None, None, None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_deserialize(b"LECO", 4, None, ctypes.byref(h)) == leco.LECO_ERR_CORRUPT
    assert L.leco_deserialize(b"\0" * 64, 64, None, ctypes.byref(h)) == leco.LECO_ERR_CORRUPT
    assert L.leco_filter_sum(None, 0, 1, 0, None, None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_selftest_wait_timeout(0, None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_selftest_wait_timeout(2_000_000, None) == leco.LECO_ERR_INVALID_ARG
    L32, b64 = ctypes.c_uint32(0), ctypes.c_uint64(0)
    assert L.leco_search_partition_size(None, 0, 1, 1, 20000, 0.01, 0, None, ctypes.byref(L32), None,
                                        None) == leco.LECO_ERR_INVALID_ARG  # max_len above 16384
    assert L.leco_search_partition_size(None, 0, 1, 1, 100, 1.5, 0, None, ctypes.byref(L32), None,
                                        None) == leco.LECO_ERR_INVALID_ARG  # fraction above 1
    assert L.leco_search_partition_size(None, 0, 1, 1, 100, 0.01, 0, None, None, None, None) == leco.LECO_ERR_INVALID_ARG
    # models: 0 constant, 1 linear, 2 polynomial; anything else is refused
    assert L.leco_encode(None, 0, 1, leco.fixed(16), 3, None, ctypes.byref(h)) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_encode(None, 0, 1, leco.fixed(16), -1, None, ctypes.byref(h)) == leco.LECO_ERR_INVALID_ARG
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks below fail first
    assert L.leco_encode_with_starts(None, 0, 1, fake, 0, 3, None, ctypes.byref(h)) == leco.LECO_ERR_INVALID_ARG
    # the allocation-free encode takes constant and linear only; the batched encode all three models
    nw = ctypes.c_uint64(0)
    assert L.leco_encode_fixed_noalloc(fake, 10, 1, 16, leco.LECO_MODEL_POLY, fake, fake, 100, ctypes.byref(nw),
                                       None) == leco.LECO_ERR_INVALID_ARG
    vals = (ctypes.c_void_p * 1)(fake)
    ns, models, Ls = (ctypes.c_uint64 * 1)(10), (ctypes.c_int * 1)(3), (ctypes.c_uint32 * 1)(16)
    outs = (ctypes.c_void_p * 1)()
    assert L.leco_batch_encode(vals, ns, models, Ls, 1, 1, None, outs) == leco.LECO_ERR_INVALID_ARG
    # the graph-replayed batched encode: same argument checks, at least one column, NULL plans refused
    assert L.leco_batch_encode_plan_create(vals, ns, models, Ls, 1, 1, None, ctypes.byref(h)) == \
        leco.LECO_ERR_INVALID_ARG
    assert L.leco_batch_encode_plan_create(vals, ns, models, Ls, 0, 1, None, ctypes.byref(h)) == \
        leco.LECO_ERR_INVALID_ARG
    assert L.leco_batch_encode_plan_run(None, None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_batch_encode_plan_columns(None, None, outs) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_batch_encode_plan_reserved_bytes(None) == 0
    L.leco_batch_encode_plan_free(None)
    # variable partitioning takes the variable kinds (plain or seeded) and tau in [0, 1]
    m_out = ctypes.c_uint64(0)
    for pol in (leco.fixed(16), leco.auto(), leco.variable(1.5), leco.variable(-0.1, seeded=True)):
        assert L.leco_var_partition(fake, 10, 1, pol, 1, fake, ctypes.byref(m_out), None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_encode(fake, 10, 1, leco.variable(2.0, seeded=True), 1, None, ctypes.byref(h)) == \
        leco.LECO_ERR_INVALID_ARG
    # the execution-unit probe takes kinds 0..4 and an output pointer
    r = ctypes.c_double(0.0)
    assert L.leco_probe_throughput(5, ctypes.byref(r), None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_probe_throughput(-1, ctypes.byref(r), None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_probe_throughput(0, None, None) == leco.LECO_ERR_INVALID_ARG


def test_tuning_table_file_round_trip(built, tmp_path):
    """The tuning table's file form is host-only: load merges the entries that name a candidate
    the tuners can pick (2..8 stages with 4 or 8 consumer warps; 1024/2048/4096 values per pack
    item with 2..4 fit CTAs per SM) and skips the rest, save writes the whole table back as JSON.
    The keys used here (operation 7, dtype 99) name no scan or encode the library runs."""
    import json

    from paper_2306_15374_gb300 import leco

    L = leco.lib()
    src = tmp_path / "in.json"
    src.write_text(
        '{"scan_configs": [\n'
        '  {"op": 7, "dtype": 99, "width_bucket": 0, "stages": 3, "consumer_warps": 8},\n'
        '  {"op": 7, "dtype": 99, "width_bucket": 1, "stages": 9, "consumer_warps": 4},\n'
        '  {"op": 7, "dtype": 99, "width_bucket": 2, "stages": 2, "consumer_warps": 6},\n'
        '  {"op": 7, "dtype": 99, "width_bucket": 3, "stages": 8, "consumer_warps": 4}\n'
        '], "encode_configs": [\n'
        '  {"dtype": 99, "item_values": 2048, "fit_ctas": 3},\n'
        '  {"dtype": 98, "item_values": 3000, "fit_ctas": 3},\n'
        '  {"dtype": 97, "item_values": 1024, "fit_ctas": 5}\n'
        ']}\n')
    assert L.leco_tune_load(str(src).encode()) == leco.LECO_OK
    out = tmp_path / "out.json"
    assert L.leco_tune_save(str(out).encode()) == leco.LECO_OK
    table = json.loads(out.read_text())
    mine = {(e["op"], e["dtype"], e["width_bucket"]): (e["stages"], e["consumer_warps"])
            for e in table["scan_configs"] if e["dtype"] == 99}
    assert mine == {(7, 99, 0): (3, 8), (7, 99, 3): (8, 4)}
    enc = {e["dtype"]: (e["item_values"], e["fit_ctas"]) for e in table["encode_configs"] if e["dtype"] >= 97}
    assert enc == {99: (2048, 3)}
    # the saved file loads back to the same table
    assert L.leco_tune_load(str(out).encode()) == leco.LECO_OK
    again = tmp_path / "again.json"
    assert L.leco_tune_save(str(again).encode()) == leco.LECO_OK
    assert json.loads(again.read_text()) == table
    # a file that cannot be opened, or no path at all, is refused
    assert L.leco_tune_load(str(tmp_path / "missing.json").encode()) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_tune_load(None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_tune_save(None) == leco.LECO_ERR_INVALID_ARG
    assert L.leco_tune_save(str(tmp_path / "no" / "dir.json").encode()) == leco.LECO_ERR_INVALID_ARG


def test_binding_refuses_short_output_buffers(built):
    """The library cannot see a device buffer's size, so the binding checks every buffer a call
    writes before the call: a short one would otherwise be written past its end on the device.
    The column here is a stand-in whose size is set by hand; its handle is never passed on."""
    import ctypes

    import torch

    from paper_2306_15374_gb300 import leco

    col = leco.Column(ctypes.c_void_p(1))
    try:
        col._shape = (1000, 8)
        i64 = torch.int64
        with pytest.raises(ValueError, match="needs 8000"):
            leco.leco_decode_all(col, torch.empty(999, dtype=i64))
        with pytest.raises(ValueError, match="needs 800"):
            leco.leco_decode_range(col, 10, 100, torch.empty(99, dtype=i64))
        with pytest.raises(ValueError, match="8-byte"):
            leco.leco_random_access(col, torch.zeros(50, dtype=torch.int32), torch.empty(50, dtype=i64))
        with pytest.raises(ValueError, match="needs 400"):
            leco.leco_random_access(col, torch.zeros(50, dtype=i64), torch.empty(49, dtype=i64))
        with pytest.raises(ValueError, match="needs 24"):
            leco.leco_filter_sum(col, 0, 1, torch.empty(2, dtype=i64))
        with pytest.raises(ValueError, match="needs 808"):
            leco.leco_var_partition(torch.zeros(100, dtype=i64), torch.empty(100, dtype=i64), leco.variable(0.1))
        # buffers of the right size pass the checks and stop only at the device check (these are
        # host tensors); a 32-bit column needs 4 bytes per value
        for call in (lambda: leco.leco_decode_all(col, torch.empty(1000, dtype=i64)),
                     lambda: leco.leco_random_access(col, torch.zeros(50, dtype=i64), torch.empty(50, dtype=i64)),
                     lambda: leco.leco_filter_sum(col, 0, 1, torch.empty(3, dtype=i64))):
            with pytest.raises(ValueError, match="CUDA tensor"):
                call()
        col._shape = (1000, 4)
        with pytest.raises(ValueError, match="CUDA tensor"):
            leco.leco_decode_all(col, torch.empty(1000, dtype=torch.int32))
        with pytest.raises(ValueError, match="needs 4000"):
            leco.leco_decode_all(col, torch.empty(999, dtype=torch.int32))
        # batched decode: one output per column, each holding that column's values
        for fn in (leco.leco_batch_decode, leco.leco_batch_plan_create):
            with pytest.raises(ValueError, match="2 columns but 1 outputs"):
                fn([col, col], [torch.empty(1000, dtype=torch.int32)])
            with pytest.raises(ValueError, match="needs 4000"):
                fn([col, col], [torch.empty(999, dtype=torch.int32), torch.empty(1000, dtype=torch.int32)])
            with pytest.raises(ValueError, match="CUDA tensors"):
                fn([col], [torch.empty(1000, dtype=torch.int32)])
    finally:
        col._h = None  # the stand-in handle is not a column: nothing to free


def test_binding_checks_encode_arguments(built):
    """Batched encodes take one model and one partition size per column and device tensors only;
    given starts are 8-byte and hold m + 1 entries (the library reads that many)."""
    import torch

    from paper_2306_15374_gb300 import leco

    v = torch.zeros(100, dtype=torch.int64)
    for fn in (leco.leco_batch_encode, leco.leco_batch_encode_plan_create, leco.leco_tune_batch_encode):
        with pytest.raises(ValueError, match="1 columns but 2 models and 1 partition sizes"):
            fn([v], [1, 1], [16])
        with pytest.raises(ValueError, match="CUDA tensor"):
            fn([v], [1], [16])
    with pytest.raises(ValueError, match="8-byte"):
        leco.leco_encode_with_starts(v, torch.tensor([0, 100], dtype=torch.int32), 1)
    with pytest.raises(ValueError, match="needs m \\+ 1 = 3"):
        leco.leco_encode_with_starts(v, torch.tensor([0, 100], dtype=torch.int64), 2)


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment (the nearest one above it) names the section of the paper it
    follows, or says that the paper has no counterpart (library plumbing, batching, serving)."""
    missing = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        for m in re.finditer(r"\n(?:leco_status|void|uint64_t|uint32_t|const char\*)\s+(leco_[a-z0-9_]+)\s*\(", text):
            end = text.rfind("*/", 0, m.start())
            comment = text[text.rfind("/*", 0, end):end] if end >= 0 else ""
            if "§" not in comment and "counterpart" not in comment:
                missing.append(f"{os.path.basename(h)}:{m.group(1)}")
    assert not missing, missing
