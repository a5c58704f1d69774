"""Thin ctypes binding of libaceapex.so (argument marshalling only).

Names follow the C ABI in include/aceapex.h.  Device buffers are passed as
raw device pointers (e.g. ``tensor.data_ptr()`` of a torch CUDA tensor) and
streams as ``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).
Every step of the decode runs in the library's CUDA kernels; there is no CPU
fallback: if the shared library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK, E_ARG, E_CORRUPT, E_NOMEM, E_CUDA, E_TIMEOUT, E_RANGE, E_BUSY = 0, -1, -2, -3, -4, -5, -6, -7
VARIANT_FAST, VARIANT_PLAIN, VARIANT_FUSED = 0, 1, 2
BLOCK_SIZE = 16384

EXPORTED = [
    "aceapex_status_string", "aceapex_last_error", "aceapex_ctx_create", "aceapex_ctx_destroy",
    "aceapex_ctx_set_params", "aceapex_encode", "aceapex_encode_ex", "aceapex_free", "aceapex_archive_open", "aceapex_archive_close",
    "aceapex_archive_get_info", "aceapex_decode_all", "aceapex_decode_all_async", "aceapex_sync",
    "aceapex_decode_host", "aceapex_archive_check", "aceapex_decode_noalloc", "aceapex_batch_create",
    "aceapex_batch_run_async", "aceapex_batch_wait", "aceapex_batch_run", "aceapex_batch_destroy",
    "aceapex_batch_decode", "aceapex_decode_range", "aceapex_archive_index", "aceapex_server_create",
    "aceapex_server_now_ns", "aceapex_server_submit_many", "aceapex_server_submit", "aceapex_server_poll",
    "aceapex_server_drain", "aceapex_server_get_stats", "aceapex_server_last_error", "aceapex_server_destroy",
    "aceapex_autotune", "aceapex_shard_range", "aceapex_archive_parse_stats",
]
BATCH_GRAPH = 1


class EncParams(ctypes.Structure):
    _fields_ = [("no_rep", ctypes.c_int), ("min_match", ctypes.c_uint32), ("max_lanes", ctypes.c_uint32),
                ("threads", ctypes.c_int), ("latest_source", ctypes.c_int),
                ("max_depth", ctypes.c_uint32), ("short_latest", ctypes.c_int), ("deps", ctypes.c_int),
                ("segment", ctypes.c_uint64), ("levels", ctypes.c_int)]


class DecParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("timeout_us", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("rans_ctas_per_sm", ctypes.c_uint32), ("queue_chunk", ctypes.c_uint32), ("wait_ns", ctypes.c_uint32),
                ("ignore_levels", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_ans", ctypes.c_double), ("ms_parse", ctypes.c_double),
                ("ms_copy", ctypes.c_double), ("blocks", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("pending_spans", ctypes.c_uint64), ("wait_polls", ctypes.c_uint64),
                ("pending_bytes", ctypes.c_uint64)]


class ArchiveInfo(ctypes.Structure):
    _fields_ = [("total_size", ctypes.c_uint64), ("n_blocks", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("min_match", ctypes.c_uint32), ("max_tokens", ctypes.c_uint32),
                ("archive_bytes", ctypes.c_uint64), ("tokens", ctypes.c_uint64)]


class EncStats(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_uint64), ("matches", ctypes.c_uint64),
                ("block_max_depth", ctypes.c_uint64 * 256), ("match_depth", ctypes.c_uint64 * 256),
                ("match_level", ctypes.c_uint64 * 256), ("level_bytes", ctypes.c_uint64 * 256)]

    def as_dict(self):
        return {"blocks": self.blocks, "matches": self.matches,
                "block_max_depth": list(self.block_max_depth), "match_depth": list(self.match_depth),
                "match_level": list(self.match_level), "level_bytes": list(self.level_bytes)}


class ParseStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64 * 4 if n == "rep_matches" else ctypes.c_uint64) for n in (
        "blocks", "tokens", "new_matches", "rep_matches", "lit_only", "values", "multibyte_values",
        "literal_bytes", "match_bytes", "overlap_matches", "external_matches", "max_tokens_block",
        "runs", "run_len_sum", "median_run", "max_run", "bad_blocks")]

    def as_dict(self):
        return {n: (list(getattr(self, n)) if n == "rep_matches" else getattr(self, n)) for n, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("arc", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("out_cap", ctypes.c_uint64),
                ("status", ctypes.c_int)]


class ServerParams(ctypes.Structure):
    _fields_ = [("cache_bytes", ctypes.c_uint64), ("max_tick_blocks", ctypes.c_uint32),
                ("max_tick_requests", ctypes.c_uint32), ("streams", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("closure_blocks", ctypes.c_uint32),
                ("decoded_blocks", ctypes.c_uint32), ("latency_us", ctypes.c_double), ("queue_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("completed", "failed", "refused", "bytes", "ticks", "blocks_decoded",
                                               "blocks_hit")] + \
               [(k, ctypes.c_double) for k in ("p50_us", "p99_us", "mean_us", "max_us", "closure_mean", "closure_p50",
                                               "closure_p99", "seconds", "gbs")] + \
               [(k, ctypes.c_uint64) for k in ("tick_overlaps", "tick_waits")] + \
               [(k, ctypes.c_double) for k in ("tick_host_ms", "walk_ms", "launch_ms")]


class TunePoint(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_uint32), ("rans_ctas_per_sm", ctypes.c_uint32),
                ("queue_chunk", ctypes.c_uint32), ("ms", ctypes.c_double)]


class AceapexError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"aceapex status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libaceapex.so (must have been built with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.SO
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -m paper_2608_10188_gb300.build)")
    L = ctypes.CDLL(path)
    c = ctypes
    vp, u64, u32 = c.c_void_p, c.c_uint64, c.c_uint32
    L.aceapex_status_string.argtypes = [c.c_int]
    L.aceapex_status_string.restype = c.c_char_p
    L.aceapex_last_error.argtypes = [vp]
    L.aceapex_last_error.restype = c.c_char_p
    L.aceapex_ctx_create.argtypes = [c.c_int, c.POINTER(DecParams), c.POINTER(vp)]
    L.aceapex_ctx_destroy.argtypes = [vp]
    L.aceapex_ctx_set_params.argtypes = [vp, c.POINTER(DecParams)]
    L.aceapex_encode.argtypes = [vp, u64, c.POINTER(EncParams), c.POINTER(vp), c.POINTER(u64)]
    L.aceapex_encode_ex.argtypes = [vp, u64, c.POINTER(EncParams), c.POINTER(vp), c.POINTER(u64), c.POINTER(EncStats)]
    L.aceapex_free.argtypes = [vp]
    L.aceapex_free.restype = None
    L.aceapex_archive_open.argtypes = [vp, vp, vp, u64, c.POINTER(vp)]
    L.aceapex_archive_close.argtypes = [vp]
    L.aceapex_archive_get_info.argtypes = [vp, c.POINTER(ArchiveInfo)]
    L.aceapex_archive_check.argtypes = [vp, u64, c.POINTER(ArchiveInfo)]
    L.aceapex_decode_noalloc.argtypes = [vp, u64, vp, u64, vp]
    L.aceapex_decode_all.argtypes = [vp, vp, vp, u64, vp, c.POINTER(Stats)]
    L.aceapex_decode_all_async.argtypes = [vp, vp, vp, u64, vp]
    L.aceapex_sync.argtypes = [vp, vp]
    L.aceapex_decode_host.argtypes = [vp, vp, vp, u64, vp, u64, vp, c.POINTER(Stats)]
    L.aceapex_batch_create.argtypes = [vp, c.POINTER(BatchItem), c.c_int, u32, c.POINTER(vp)]
    L.aceapex_batch_run_async.argtypes = [vp, vp]
    L.aceapex_batch_wait.argtypes = [vp, vp, c.POINTER(BatchItem), c.POINTER(Stats)]
    L.aceapex_batch_run.argtypes = [vp, vp, c.POINTER(BatchItem), c.POINTER(Stats)]
    L.aceapex_batch_destroy.argtypes = [vp]
    L.aceapex_decode_range.argtypes = [vp, vp, u64, u64, vp, vp, c.POINTER(Stats)]
    L.aceapex_archive_index.argtypes = [vp, vp]
    L.aceapex_archive_parse_stats.argtypes = [vp, vp, c.POINTER(ParseStats)]
    L.aceapex_server_create.argtypes = [vp, vp, c.POINTER(ServerParams), c.POINTER(vp)]
    L.aceapex_server_now_ns.argtypes = [vp]
    L.aceapex_server_now_ns.restype = c.c_int64
    L.aceapex_server_submit_many.argtypes = [vp, c.c_int, vp, vp, vp, vp, vp]
    L.aceapex_server_submit.argtypes = [vp, u64, u64, vp, c.c_int64, c.POINTER(u64)]
    L.aceapex_server_poll.argtypes = [vp, c.POINTER(Completion), c.c_int, c.c_int]
    L.aceapex_server_drain.argtypes = [vp, c.c_int]
    L.aceapex_server_get_stats.argtypes = [vp, c.c_int, c.POINTER(ServerStats)]
    L.aceapex_server_last_error.argtypes = [vp]
    L.aceapex_server_last_error.restype = c.c_char_p
    L.aceapex_server_destroy.argtypes = [vp]
    L.aceapex_shard_range.argtypes = [u64, c.c_int, c.c_int, c.POINTER(u64), c.POINTER(u64)]
    L.aceapex_autotune.argtypes = [vp, c.POINTER(BatchItem), c.c_int, c.c_int, c.POINTER(TunePoint), c.c_int,
                                   c.POINTER(c.c_int), c.POINTER(DecParams)]
    L.aceapex_batch_decode.argtypes = [vp, c.POINTER(BatchItem), c.c_int, vp, c.POINTER(Stats)]
    L.acx_debug_counters.argtypes = [vp, vp, u32]
    L.acx_debug_counters.restype = c.c_int
    for name in EXPORTED:
        if name not in ("aceapex_status_string", "aceapex_last_error", "aceapex_free", "aceapex_server_now_ns",
                        "aceapex_server_last_error"):
            getattr(L, name).restype = c.c_int
    _lib = L
    return L


def _check(rc, ctx=None, what=""):
    if rc != OK:
        L = load()
        msg = L.aceapex_last_error(ctx).decode() if ctx else L.aceapex_status_string(rc).decode()
        raise AceapexError(rc, f"{what}: {msg}")
    return rc


def encode(data, no_rep: bool = False, min_match: int = 4, max_lanes: int = 32, threads: int = 0,
           latest_source: bool = False, max_depth: int = 0, short_latest: bool = False, deps: bool = False,
           segment: int = 0, stats: dict = None, levels: bool = False) -> bytes:
    """aceapex_encode on host bytes (numpy uint8 array or bytes).  With a
    dict `stats`, aceapex_encode_ex fills it with the chain-depth statistics
    (see aceapex_enc_stats)."""
    import numpy as np
    L = load()
    a = np.ascontiguousarray(np.frombuffer(data, np.uint8) if isinstance(data, (bytes, bytearray)) else data,
                             dtype=np.uint8)
    p = EncParams(int(no_rep), min_match, max_lanes, threads, int(latest_source), max_depth, int(short_latest),
                  int(deps), segment, int(levels))
    ptr = ctypes.c_void_p()
    n = ctypes.c_uint64()
    st = EncStats()
    _check(L.aceapex_encode_ex(a.ctypes.data if a.size else None, a.size, ctypes.byref(p), ctypes.byref(ptr),
                               ctypes.byref(n), ctypes.byref(st) if stats is not None else None), None, "encode")
    if stats is not None:
        stats.update(st.as_dict())
    try:
        if n.value < (1 << 31):
            return ctypes.string_at(ptr.value, n.value)
        # ctypes.string_at takes a C int size: copy larger archives by memmove
        buf = bytearray(n.value)
        ctypes.memmove((ctypes.c_char * n.value).from_buffer(buf), ptr.value, n.value)
        return bytes(buf)
    finally:
        L.aceapex_free(ptr)


class Context:
    """aceapex_ctx on one CUDA device."""

    def __init__(self, device: int = 0, variant: int = VARIANT_FAST, timeout_us: int = 0, ctas_per_sm: int = 0,
                 rans_ctas_per_sm: int = 0, queue_chunk: int = 0, wait_ns: int = 0, ignore_levels: bool = False):
        L = load()
        self._L = L
        self.params = DecParams(variant, timeout_us, ctas_per_sm, rans_ctas_per_sm, queue_chunk, wait_ns,
                                int(ignore_levels))
        h = ctypes.c_void_p()
        _check(L.aceapex_ctx_create(device, ctypes.byref(self.params), ctypes.byref(h)), None, "ctx_create")
        self.h = h

    def set_params(self, variant: int = VARIANT_FAST, timeout_us: int = 0, ctas_per_sm: int = 0,
                   rans_ctas_per_sm: int = 0, queue_chunk: int = 0, wait_ns: int = 0, ignore_levels: bool = False):
        self.params = DecParams(variant, timeout_us, ctas_per_sm, rans_ctas_per_sm, queue_chunk, wait_ns,
                                int(ignore_levels))
        _check(self._L.aceapex_ctx_set_params(self.h, ctypes.byref(self.params)), self.h, "set_params")

    def close(self):
        if self.h:
            self._L.aceapex_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._L.aceapex_last_error(self.h).decode()

    def sync(self, stream: int = 0) -> int:
        return self._L.aceapex_sync(self.h, stream)

    def round_trace(self):
        """Diagnostics of the last whole decode on this context: the
        cross-block pass's rounds as (round, pieces in its list, start in µs
        after round 0 began); round 0 has no list."""
        import numpy as np
        cn = np.zeros(4096, np.uint32)
        if self._L.acx_debug_counters(self.h, cn.ctypes.data, cn.size) != 0:
            return None
        base, rows = 3800, []  # the trace words of the counter block
        t0 = int(cn[base + 1]) | (int(cn[base + 2]) << 32)
        for r in range(64):
            t = int(cn[base + 3 * r + 1]) | (int(cn[base + 3 * r + 2]) << 32)
            if t == 0 or t < t0:
                break
            rows.append((r, int(cn[base + 3 * r]), round((t - t0) / 1e3, 1)))
        return rows


class Archive:
    """aceapex_archive: a validated archive with its device decode plan."""

    def __init__(self, ctx: Context, d_arc: int, h_arc, arc_len: int):
        self.ctx = ctx
        h = ctypes.c_void_p()
        self._hbuf = h_arc
        hp = h_arc.ctypes.data if hasattr(h_arc, "ctypes") else ctypes.cast(ctypes.c_char_p(h_arc), ctypes.c_void_p).value
        _check(ctx._L.aceapex_archive_open(ctx.h, d_arc, hp, arc_len, ctypes.byref(h)), ctx.h, "archive_open")
        self.h = h
        info = ArchiveInfo()
        _check(ctx._L.aceapex_archive_get_info(self.h, ctypes.byref(info)), ctx.h, "archive_info")
        self.info = {k: getattr(info, k) for k, _ in ArchiveInfo._fields_}
        self._hbuf = None

    def build_index(self):
        """aceapex_archive_index: the match index for byte-level closures."""
        _check(self.ctx._L.aceapex_archive_index(self.ctx.h, self.h), self.ctx.h, "archive_index")

    def parse_stats(self) -> dict:
        """aceapex_archive_parse_stats: token, command and run counts of the
        device's parse-only pass (builds the match index if absent)."""
        st = ParseStats()
        _check(self.ctx._L.aceapex_archive_parse_stats(self.ctx.h, self.h, ctypes.byref(st)), self.ctx.h,
               "archive_parse_stats")
        return st.as_dict()

    @property
    def total(self) -> int:
        return self.info["total_size"]

    def close(self):
        if self.h:
            self.ctx._L.aceapex_archive_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def archive_check(h_arc) -> dict:
    """aceapex_archive_check: host-only structural validation; returns the info dict."""
    import numpy as np
    L = load()
    a = np.ascontiguousarray(np.frombuffer(h_arc, np.uint8) if isinstance(h_arc, (bytes, bytearray)) else h_arc,
                             dtype=np.uint8)
    info = ArchiveInfo()
    rc = L.aceapex_archive_check(a.ctypes.data, a.size, ctypes.byref(info))
    if rc != OK:
        raise AceapexError(rc, "archive_check")
    return {k: getattr(info, k) for k, _ in ArchiveInfo._fields_}


def decode_all(ctx: Context, arc: Archive, d_out: int, out_cap: int, stream: int = 0, stats: bool = False):
    """aceapex_decode_all: returns the status (and a Stats dict when stats=True)."""
    st = Stats() if stats else None
    rc = ctx._L.aceapex_decode_all(ctx.h, arc.h, d_out, out_cap, stream, ctypes.byref(st) if st else None)
    if stats:
        return rc, {k: getattr(st, k) for k, _ in Stats._fields_}
    return rc


def decode_range(ctx: Context, arc: Archive, start: int, length: int, d_out: int, stream: int = 0,
                 stats: bool = False):
    """aceapex_decode_range: bytes [start, start+length) into d_out; returns
    the status (and a Stats dict when stats=True)."""
    st = Stats() if stats else None
    rc = ctx._L.aceapex_decode_range(ctx.h, arc.h, start, length, d_out, stream, ctypes.byref(st) if st else None)
    if stats:
        return rc, {k: getattr(st, k) for k, _ in Stats._fields_}
    return rc


def decode_all_async(ctx: Context, arc: Archive, d_out: int, out_cap: int, stream: int = 0) -> int:
    return ctx._L.aceapex_decode_all_async(ctx.h, arc.h, d_out, out_cap, stream)


def decode_host(ctx: Context, arc, h_arc, h_out, stream: int = 0, stats: bool = False):
    """aceapex_decode_host: host archive (numpy uint8) -> host output (numpy uint8)."""
    st = Stats() if stats else None
    rc = ctx._L.aceapex_decode_host(ctx.h, arc.h if arc is not None else None, h_arc.ctypes.data, h_arc.size,
                                    h_out.ctypes.data, h_out.size, stream, ctypes.byref(st) if st else None)
    if stats:
        return rc, {k: getattr(st, k) for k, _ in Stats._fields_}
    return rc


def decode_noalloc(d_arc: int, arc_len: int, d_out: int, out_cap: int, stream: int = 0) -> int:
    """aceapex_decode_noalloc: decode a small archive (<= 64 blocks) that is
    already in device memory, using only the library's static scratch; for
    callers that must not allocate.  Returns the status."""
    return load().aceapex_decode_noalloc(d_arc, arc_len, d_out, out_cap, stream)


def _items(entries):
    arr = (BatchItem * max(len(entries), 1))()
    for i, (arc, d_out, out_cap) in enumerate(entries):
        arr[i].arc = arc.h.value if isinstance(arc.h, ctypes.c_void_p) else arc.h
        arr[i].d_out = d_out
        arr[i].out_cap = out_cap
        arr[i].status = 0
    return arr


class Batch:
    """aceapex_batch: a reusable decode of many archives by one set of
    launches (captured into a CUDA graph when graph=True).  entries: a list of
    (Archive, d_out, out_cap)."""

    def __init__(self, ctx: Context, entries, graph: bool = True):
        self.ctx = ctx
        self.n = len(entries)
        self._keep = [e[0] for e in entries]
        self._items = _items(entries)
        h = ctypes.c_void_p()
        _check(ctx._L.aceapex_batch_create(ctx.h, self._items, self.n, BATCH_GRAPH if graph else 0, ctypes.byref(h)),
               ctx.h, "batch_create")
        self.h = h

    def run_async(self, stream: int = 0) -> int:
        return self.ctx._L.aceapex_batch_run_async(self.h, stream)

    def wait(self, stream: int = 0, stats: bool = False):
        """Returns (status, per-item statuses[, stats dict])."""
        st = Stats() if stats else None
        rc = self.ctx._L.aceapex_batch_wait(self.h, stream, self._items, ctypes.byref(st) if st else None)
        per = [self._items[i].status for i in range(self.n)]
        if stats:
            return rc, per, {k: getattr(st, k) for k, _ in Stats._fields_}
        return rc, per

    def run(self, stream: int = 0, stats: bool = False):
        rc = self.run_async(stream)
        if rc != OK:
            return (rc, [rc] * self.n, None) if stats else (rc, [rc] * self.n)
        return self.wait(stream, stats)

    def close(self):
        if self.h:
            self.ctx._L.aceapex_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_decode(ctx: Context, entries, stream: int = 0, stats: bool = False):
    """aceapex_batch_decode (one-shot): returns (status, per-item statuses[, stats])."""
    items = _items(entries)
    st = Stats() if stats else None
    rc = ctx._L.aceapex_batch_decode(ctx.h, items, len(entries), stream, ctypes.byref(st) if st else None)
    per = [items[i].status for i in range(len(entries))]
    if stats:
        return rc, per, {k: getattr(st, k) for k, _ in Stats._fields_}
    return rc, per


class Server:
    """aceapex_server: continuous-batching region server over one opened
    archive with a bounded device cache of decoded blocks."""

    def __init__(self, ctx: Context, arc: Archive, cache_bytes: int = 0, max_tick_blocks: int = 0,
                 max_tick_requests: int = 0, streams: int = 0):
        self.ctx = ctx
        self.arc = arc
        self._L = ctx._L
        p = ServerParams(cache_bytes, max_tick_blocks, max_tick_requests, streams)
        h = ctypes.c_void_p()
        _check(self._L.aceapex_server_create(ctx.h, arc.h, ctypes.byref(p), ctypes.byref(h)), ctx.h, "server_create")
        self.h = h

    def now_ns(self) -> int:
        return self._L.aceapex_server_now_ns(self.h)

    def submit_many(self, starts, lens, d_outs, at_ns=None):
        """Queue regions (numpy arrays of uint64 starts/lengths, device
        pointers, optional int64 arrival times on the server clock); returns
        the request ids."""
        import numpy as np
        n = len(starts)
        st = np.ascontiguousarray(starts, dtype=np.uint64)
        ln = np.ascontiguousarray(lens, dtype=np.uint64)
        dp = np.ascontiguousarray(d_outs, dtype=np.uint64)
        at = None if at_ns is None else np.ascontiguousarray(at_ns, dtype=np.int64)
        ids = np.zeros(n, dtype=np.uint64)
        rc = self._L.aceapex_server_submit_many(self.h, n, st.ctypes.data, ln.ctypes.data, dp.ctypes.data,
                                                at.ctypes.data if at is not None else None, ids.ctypes.data)
        if rc != OK:
            raise AceapexError(rc, "server_submit")
        return ids

    def submit(self, start: int, length: int, d_out: int, at_ns: int = -1) -> int:
        i = ctypes.c_uint64()
        rc = self._L.aceapex_server_submit(self.h, start, length, d_out, at_ns, ctypes.byref(i))
        if rc != OK:
            raise AceapexError(rc, "server_submit")
        return i.value

    def poll(self, max_n: int = 4096, wait_ms: int = 0):
        buf = (Completion * max(max_n, 1))()
        n = self._L.aceapex_server_poll(self.h, buf, max_n, wait_ms)
        if n < 0:
            raise AceapexError(n, "server_poll")
        return [{k: getattr(buf[i], k) for k, _ in Completion._fields_} for i in range(n)]

    def drain(self, timeout_ms: int = 60000) -> int:
        return self._L.aceapex_server_drain(self.h, timeout_ms)

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(self._L.aceapex_server_get_stats(self.h, int(reset), ctypes.byref(st)), None, "server_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def last_error(self) -> str:
        return self._L.aceapex_server_last_error(self.h).decode()

    def close(self):
        if self.h:
            self._L.aceapex_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(ctx: Context, entries, reps: int = 3, max_points: int = 512):
    """aceapex_autotune over a list of (Archive, d_out, out_cap): returns
    (best params dict, measured points).  The context keeps the best params."""
    items = _items(entries)
    pts = (TunePoint * max_points)()
    npts = ctypes.c_int()
    best = DecParams()
    _check(ctx._L.aceapex_autotune(ctx.h, items, len(entries), reps, pts, max_points, ctypes.byref(npts),
                                   ctypes.byref(best)), ctx.h, "autotune")
    ctx.params = best
    b = {k: getattr(best, k) for k, _ in DecParams._fields_}
    return b, [{k: getattr(pts[i], k) for k, _ in TunePoint._fields_} for i in range(npts.value)]


def shard_range(total: int, n_ranks: int, rank: int):
    """aceapex_shard_range: (start, length) of this rank's block-aligned output range."""
    s, n = ctypes.c_uint64(), ctypes.c_uint64()
    rc = load().aceapex_shard_range(total, n_ranks, rank, ctypes.byref(s), ctypes.byref(n))
    if rc != OK:
        raise AceapexError(rc, "shard_range")
    return s.value, n.value
