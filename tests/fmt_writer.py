"""Test-side writer of format v1 archives with stored (not entropy-coded)
streams, from explicit token lists.  It restates the byte layout only (header,
tables, index, payload descriptors, 16-byte body alignment, LEB128 lengths,
offset byte planes); it performs no decoding, so archives it writes are an
independent input for pinning both the oracle and the GPU path.
"""
from __future__ import annotations

import struct

BLOCK = 16384


def leb128(v: int) -> bytes:
    out = bytearray()
    while v >= 0x80:
        out.append((v & 0x7F) | 0x80)
        v >>= 7
    out.append(v)
    return bytes(out)


def block_streams(tokens):
    """Raw (cmd, len, off, lit) streams of one block from its token list."""
    cmd = bytearray()
    lens = bytearray()
    lit = bytearray()
    srcs = []
    for t in tokens:
        cmd.append(t["cmd"])
        lens += leb128(len(t["lits"])) + leb128(t["ml"])
        lit += t["lits"]
        if t["cmd"] == 0:
            srcs.append(t["src"])
    off = bytearray()
    for p in range(5):
        for s in srcs:
            off.append((s >> (8 * p)) & 0xFF)
    return [bytes(cmd), bytes(lens), bytes(off), bytes(lit)]


def pad16(n: int) -> int:
    return (n + 15) & ~15


def build_archive(blocks, *, min_match=4, flags=0, expected=None, fnv=None, raw_streams=None,
                  raw_lens=None, total=None, tables=None, encoded=None, deps=None, levels=None):
    """blocks: list of token lists.  raw_streams: optional {block: [cmd, len,
    off, lit]} overriding the streams derived from tokens.  encoded: optional
    {(block, stream): (mode, K, body)} to place an entropy-coded body.
    expected: decoded bytes (for the per-block FNV via fnv).  deps: optional
    per-block lists of source-block ids (writes the dependency section).
    levels: optional per-block level bytes (one per token): sets flags bit1
    and writes each block's level body after its four stream bodies.
    Returns bytes."""
    nb = len(blocks)
    streams = [block_streams(t) for t in blocks]
    if raw_streams:
        for b, s in raw_streams.items():
            streams[b] = s
    if raw_lens is None:
        raw_lens = [sum(len(t["lits"]) + t["ml"] for t in toks) for toks in blocks]
    if total is None:
        total = sum(raw_lens)
    off_tables = 64
    off_index = 64 + 2048
    dep_ids, dep_pos = [], []
    if deps is not None:
        for lst in deps:
            dep_pos.append((len(dep_ids), len(lst)))
            dep_ids += list(lst)
        off_deps = pad16(off_index + 40 * nb)
        off_payload = pad16(off_deps + 4 * len(dep_ids))
    else:
        dep_pos = [(0, 0)] * nb
        off_deps = 0
        off_payload = pad16(off_index + 40 * nb)
    payload = bytearray()
    index = bytearray()
    for b in range(nb):
        base = len(payload)
        desc = bytearray()
        bodies = bytearray()
        for s in range(4):
            raw = streams[b][s]
            if encoded and (b, s) in encoded:
                mode, K, body = encoded[(b, s)]
                desc += struct.pack("<IIBBH", len(raw) if isinstance(raw, (bytes, bytearray)) else raw,
                                    len(body), mode, K, 0)
            else:
                body = raw
                desc += struct.pack("<IIBBH", len(raw), len(raw), 0, 0, 0)
            bodies += body + b"\0" * (pad16(len(body)) - len(body))
        if levels is not None:
            lv = bytes(levels[b])
            bodies += lv + b"\0" * (pad16(len(lv)) - len(lv))
        payload += desc + bodies
        n_tok = len(streams[b][0]) if isinstance(streams[b][0], (bytes, bytearray)) else streams[b][0]
        h = 0
        if fnv is not None and expected is not None:
            h = fnv(expected[b * BLOCK: b * BLOCK + raw_lens[b]])
        index += struct.pack("<QIIIIIIQ", off_payload + base, len(payload) - base, n_tok, raw_lens[b],
                             dep_pos[b][0], dep_pos[b][1], 0, h)
    hdr = bytearray(64)
    hdr[0:4] = b"ACX1"
    struct.pack_into("<HHIIQI", hdr, 4, 1, flags | (2 if levels is not None else 0), BLOCK, min_match, total, nb)
    struct.pack_into("<QQQQ", hdr, 32, off_tables, off_index, off_deps, off_payload)
    tab = bytearray(2048)
    if tables is not None:
        for s in range(4):
            for k in range(256):
                struct.pack_into("<H", tab, 512 * s + 2 * k, int(tables[s][k]))
    arc = bytes(hdr) + bytes(tab) + bytes(index)
    if deps is not None:
        arc += b"\0" * (off_deps - len(arc))
        arc += b"".join(struct.pack("<I", i) for i in dep_ids)
    arc += b"\0" * (off_payload - len(arc))
    return arc + bytes(payload)


def inflate_literal_stream(arc: bytes, extra: int = BLOCK) -> bytes:
    """The archive with the raw length of the first entropy-coded literal
    stream raised by `extra` bytes: every structural bound still holds (the
    descriptor's stream stays inside the payload), but the block claims more
    literals than it has bytes, which no valid block can."""
    a = bytearray(arc)
    nb = struct.unpack_from("<I", a, 24)[0]
    off_idx = struct.unpack_from("<Q", a, 40)[0]
    for b in range(nb):
        poff = struct.unpack_from("<Q", a, off_idx + 40 * b)[0]
        d = poff + 12 * 3  # the literal stream's descriptor
        if a[d + 8] == 1:  # rANS: its raw length is free of its encoded length
            struct.pack_into("<I", a, d, struct.unpack_from("<I", a, d)[0] + extra)
            return bytes(a)
    raise ValueError("no entropy-coded literal stream")
