"""CPU oracle for format v1 (plain, slow, single-threaded C).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the GPU library and never imports it.

Every function states the decode as the paper defines it (absolute-offset
back-references into 16 KiB blocks, four streams per block behind an ANS
stage, a four-entry distance history, varint lengths, periodic overlap
semantics); ``oracle.c`` holds the byte layout and the arithmetic.  The C
source is compiled with gcc into ``liboracle.so`` beside this file on first
use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_lock = threading.Lock()
_lib = None

OK, E_ARG, E_CORRUPT, E_NOMEM = 0, -1, -2, -3
CMD, LEN, OFF, LIT = 0, 1, 2, 3
BLOCK = 16384


class OracleError(RuntimeError):
    def __init__(self, rc, what=""):
        super().__init__(f"oracle {what} failed with status {rc}")
        self.rc = rc


class EncParams(ctypes.Structure):
    _fields_ = [("no_rep", ctypes.c_int), ("min_match", ctypes.c_uint32), ("new_min", ctypes.c_uint32),
                ("max_lanes", ctypes.c_uint32), ("chain", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_uint64), ("n_tokens", ctypes.c_uint64), ("n_new", ctypes.c_uint64),
                ("n_rep", ctypes.c_uint64 * 4), ("n_litonly", ctypes.c_uint64),
                ("n_values", ctypes.c_uint64), ("n_multibyte_values", ctypes.c_uint64),
                ("n_match_bytes", ctypes.c_uint64), ("n_literal_bytes", ctypes.c_uint64),
                ("n_overlap_tokens", ctypes.c_uint64), ("n_external_tokens", ctypes.c_uint64),
                ("max_tokens_block", ctypes.c_uint64), ("hist_dependent", ctypes.c_uint64),
                ("runs", ctypes.c_uint64), ("run_len_sum", ctypes.c_uint64), ("median_run", ctypes.c_uint64),
                ("stream_raw", ctypes.c_uint64 * 4), ("stream_enc", ctypes.c_uint64 * 4)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if not isinstance(v, int) else v
        return d


def build(force: bool = False) -> str:
    """Compile liboracle.so beside the sources (idempotent)."""
    with _lock:
        newest = max(os.path.getmtime(s) for s in _SRCS)
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall", "-Wextra",
                                   "-Wno-unused-parameter", "-o", tmp, _SRCS[0]])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        c = ctypes
        L.orc_fnv1a64.argtypes = [c.c_void_p, c.c_uint64]
        L.orc_fnv1a64.restype = c.c_uint64
        L.orc_normalize.argtypes = [c.c_void_p, c.c_void_p]
        L.orc_normalize.restype = c.c_int
        L.orc_rans_encode.argtypes = [c.c_void_p, c.c_uint32, c.c_uint32, c.c_void_p, c.c_void_p, c.c_uint64]
        L.orc_rans_encode.restype = c.c_int64
        L.orc_rans_decode.argtypes = [c.c_void_p, c.c_uint64, c.c_uint32, c.c_uint32, c.c_void_p, c.c_void_p]
        L.orc_rans_decode.restype = c.c_int
        L.orc_enc_defaults.argtypes = [c.POINTER(EncParams)]
        L.orc_encode.argtypes = [c.c_void_p, c.c_uint64, c.POINTER(EncParams), c.POINTER(c.c_void_p),
                                 c.POINTER(c.c_uint64)]
        L.orc_encode.restype = c.c_int
        L.orc_free.argtypes = [c.c_void_p]
        L.orc_decode.argtypes = [c.c_void_p, c.c_uint64, c.c_void_p, c.c_uint64, c.c_int]
        L.orc_decode.restype = c.c_int
        L.orc_info.argtypes = [c.c_void_p, c.c_uint64, c.POINTER(c.c_uint64), c.POINTER(c.c_uint32),
                               c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]
        L.orc_info.restype = c.c_int
        L.orc_parse_block.argtypes = [c.c_void_p, c.c_uint64, c.c_uint32, c.c_uint64] + [c.c_void_p] * 6
        L.orc_parse_block.restype = c.c_int64
        L.orc_block_stream.argtypes = [c.c_void_p, c.c_uint64, c.c_uint32, c.c_int, c.c_void_p, c.c_uint64]
        L.orc_block_stream.restype = c.c_int64
        L.orc_block_levels.argtypes = [c.c_void_p, c.c_uint64, c.c_uint32, c.c_void_p, c.c_uint64]
        L.orc_block_levels.restype = c.c_int64
        L.orc_archive_stats.argtypes = [c.c_void_p, c.c_uint64, c.POINTER(Stats)]
        L.orc_archive_stats.restype = c.c_int
        _lib = L
    return _lib


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    a = np.ascontiguousarray(x, dtype=np.uint8)
    return a


def fnv1a64(data) -> int:
    a = _u8(data)
    return int(_load().orc_fnv1a64(a.ctypes.data, a.size))


def normalize(counts) -> np.ndarray:
    cnt = np.ascontiguousarray(counts, dtype=np.uint64)
    assert cnt.size == 256
    freq = np.zeros(256, dtype=np.uint16)
    rc = _load().orc_normalize(cnt.ctypes.data, freq.ctypes.data)
    if rc:
        raise OracleError(rc, "normalize")
    return freq


def rans_encode(sym, K: int, freq) -> bytes:
    s = _u8(sym)
    f = np.ascontiguousarray(freq, dtype=np.uint16)
    cap = 16 * ((4 * K + 15) // 16) + 2 * s.size + 16
    out = np.zeros(cap, dtype=np.uint8)
    n = _load().orc_rans_encode(s.ctypes.data, s.size, K, f.ctypes.data, out.ctypes.data, cap)
    if n < 0:
        raise OracleError(n, "rans_encode")
    return out[:n].tobytes()


def rans_decode(body, n: int, K: int, freq) -> np.ndarray:
    b = _u8(body)
    f = np.ascontiguousarray(freq, dtype=np.uint16)
    out = np.zeros(max(n, 1), dtype=np.uint8)
    rc = _load().orc_rans_decode(b.ctypes.data, b.size, n, K, f.ctypes.data, out.ctypes.data)
    if rc:
        raise OracleError(rc, "rans_decode")
    return out[:n]


def encode(data, no_rep: bool = False, min_match: int = 4, new_min: int = 8, max_lanes: int = 32,
           chain: int = 16) -> bytes:
    a = _u8(data)
    p = EncParams(int(no_rep), min_match, new_min, max_lanes, chain)
    ptr = ctypes.c_void_p()
    n = ctypes.c_uint64()
    L = _load()
    rc = L.orc_encode(a.ctypes.data if a.size else None, a.size, ctypes.byref(p), ctypes.byref(ptr),
                      ctypes.byref(n))
    if rc:
        raise OracleError(rc, "encode")
    try:
        return ctypes.string_at(ptr.value, n.value)
    finally:
        L.orc_free(ptr)


def info(arc) -> dict:
    a = _u8(arc)
    total = ctypes.c_uint64()
    nb, flags, mm = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = _load().orc_info(a.ctypes.data, a.size, ctypes.byref(total), ctypes.byref(nb), ctypes.byref(flags),
                          ctypes.byref(mm))
    if rc:
        raise OracleError(rc, "info")
    return {"total": total.value, "n_blocks": nb.value, "flags": flags.value, "min_match": mm.value}


def decode_status(arc, verify: bool = True):
    """Returns (status, bytes-or-None)."""
    a = _u8(arc)
    try:
        tot = info(a)["total"]
    except OracleError as e:
        return e.rc, None
    out = np.zeros(max(tot, 1), dtype=np.uint8)
    rc = _load().orc_decode(a.ctypes.data, a.size, out.ctypes.data, tot, int(verify))
    return rc, (out[:tot] if rc == 0 else None)


def decode(arc, verify: bool = True) -> np.ndarray:
    rc, out = decode_status(arc, verify)
    if rc:
        raise OracleError(rc, "decode")
    return out


def parse_block(arc, b: int) -> dict:
    a = _u8(arc)
    cap = 4 * BLOCK + 16
    cmd = np.zeros(cap, np.uint8)
    ll = np.zeros(cap, np.uint32)
    ml = np.zeros(cap, np.uint32)
    dst = np.zeros(cap, np.uint64)
    src = np.zeros(cap, np.uint64)
    lit = np.zeros(cap, np.uint32)
    n = _load().orc_parse_block(a.ctypes.data, a.size, b, cap, cmd.ctypes.data, ll.ctypes.data, ml.ctypes.data,
                                dst.ctypes.data, src.ctypes.data, lit.ctypes.data)
    if n < 0:
        raise OracleError(n, "parse_block")
    return {"cmd": cmd[:n], "ll": ll[:n], "ml": ml[:n], "dst": dst[:n], "src": src[:n], "lit": lit[:n]}


def block_stream(arc, b: int, which: int) -> np.ndarray:
    a = _u8(arc)
    cap = 4 * BLOCK + 16
    out = np.zeros(cap, np.uint8)
    n = _load().orc_block_stream(a.ctypes.data, a.size, b, which, out.ctypes.data, cap)
    if n < 0:
        raise OracleError(n, "block_stream")
    return out[:n]


def block_levels(arc, b: int) -> np.ndarray:
    """The level body of block b (archives whose flags have bit1 set)."""
    a = _u8(arc)
    cap = 4 * BLOCK + 16
    out = np.zeros(cap, np.uint8)
    n = _load().orc_block_levels(a.ctypes.data, a.size, b, out.ctypes.data, cap)
    if n < 0:
        raise OracleError(n, "block_levels")
    return out[:n]


def stats(arc) -> dict:
    a = _u8(arc)
    st = Stats()
    rc = _load().orc_archive_stats(a.ctypes.data, a.size, ctypes.byref(st))
    if rc:
        raise OracleError(rc, "stats")
    return st.as_dict()
