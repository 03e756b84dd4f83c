"""Helpers for the GPU tests: host<->device copies of uint64 bit patterns, and a self-describing
blob built from oracle arrays (so the CUDA decoder can be tested on columns the oracle encoded).
The blob layout is restated here from include/leco.h's description, not shared with the library."""
import struct
import zlib

import numpy as np

LECO_MAGIC = 0x4F43454C
LECO_VERSION = 1


def to_dev(a: np.ndarray, dtype_bits: int = 64):
    import torch

    if dtype_bits == 32:
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def from_dev(t) -> np.ndarray:
    a = t.cpu().numpy()
    if a.dtype.itemsize == 4:
        return a.view(np.uint32).astype(np.uint64)
    return a.view(np.uint64)


def make_blob(records: np.ndarray, words: np.ndarray, n: int, L: int, dtype: int, kind: int,
              model: int, starts: np.ndarray | None = None, tau: float = 0.0) -> bytes:
    m = len(records)
    body = records.tobytes()
    if kind == 1:
        body += np.ascontiguousarray(starts, dtype=np.uint64).tobytes()
    body += np.ascontiguousarray(words, dtype=np.uint64).tobytes()
    b = (records["word3"].astype(np.uint64) >> np.uint64(48)) & np.uint64(0x7F)
    ends = np.append(records["start"][1:].astype(np.uint64), np.uint64(n)) if m else np.zeros(0, np.uint64)
    total_bits = int(((ends - records["start"].astype(np.uint64)) * b).sum()) if m else 0
    total_bits += 320 * int((records["word3"].astype(np.uint64) >> np.uint64(63)).sum()) if m else 0  # poly blocks
    header = struct.pack("<IIQQQBBBBIdQII", LECO_MAGIC, LECO_VERSION, n, m, len(words), dtype, kind,
                         model, 0, L if kind == 0 else 0, tau, total_bits, zlib.crc32(body), 0)
    assert len(header) == 64
    return header + body


def parse_blob(blob: bytes):
    (magic, ver, n, m, nwords, dtype, kind, model, _, L, tau, total_bits, crc, _) = struct.unpack(
        "<IIQQQBBBBIdQII", blob[:64])
    body = blob[64:]
    assert zlib.crc32(body) == crc
    import oracle

    rec = np.frombuffer(body[: 32 * m], dtype=oracle.RECORD_DTYPE).copy()
    p = 32 * m
    starts = None
    if kind == 1:
        starts = np.frombuffer(body[p: p + 8 * (m + 1)], dtype=np.uint64).copy()
        p += 8 * (m + 1)
    words = np.frombuffer(body[p: p + 8 * nwords], dtype=np.uint64).copy()
    return dict(n=n, m=m, nwords=nwords, dtype=dtype, kind=kind, model=model, L=L, tau=tau,
                total_bits=total_bits, records=rec, starts=starts, words=words)


def exact_sum(v: np.ndarray, lo: int, hi: int):
    """(count, sum) of lo <= v <= hi by direct summation in two 32-bit halves (exact)."""
    sel = v[(v >= np.uint64(lo)) & (v <= np.uint64(hi))]
    lo32 = (sel & np.uint64(0xFFFFFFFF)).sum(dtype=np.uint64)
    hi32 = (sel >> np.uint64(32)).sum(dtype=np.uint64)
    return int(sel.size), (int(hi32) << 32) + int(lo32)
