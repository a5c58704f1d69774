"""Parse parity and fault isolation on the GPU.  (-m gpu)

* The device's parse-only pass (aceapex_archive_index: entropy stage without
  literals, then the token scans and the 4-entry history as a monoid scan)
  gives, for every match of every block, the destination, length and
  absolute source of the oracle's sequential parse.
* Self-overlapping matches of random period and length decode to their
  byte-serial definition (paper, Periods, Not Chains).
* A corrupt block fails only the requests that depend on it: range decodes
  and the region server refuse exactly the regions whose byte-level closure
  reaches it and decode every other region exactly.
"""
import ctypes
import struct

import numpy as np
import pytest

import oracle
import synth
from fmt_writer import build_archive

pytestmark = pytest.mark.gpu

BLOCK = 16384


@pytest.fixture(scope="module")
def acx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    acx.load()
    return acx


@pytest.fixture(scope="module")
def ctx(acx):
    c = acx.Context(0, timeout_us=2_000_000)
    yield c
    c.close()


def opened(acx, ctx, arc):
    import torch
    h = np.frombuffer(arc, np.uint8).copy()
    d = torch.from_numpy(h).to("cuda")
    A = acx.Archive(ctx, d.data_ptr(), h, h.size)
    A._keep = d
    return A


def device_index(acx, A, nb):
    L = acx.load()
    f = L.acx_debug_match_index
    f.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_uint64]
    f.restype = ctypes.c_int64
    cap = 4096 * nb + 64  # at most one match per four output bytes (min_match = 4)
    first = np.zeros(nb + 1, np.uint64)
    o, ml = np.zeros(cap, np.uint16), np.zeros(cap, np.uint16)
    src, bad = np.zeros(cap, np.uint64), np.zeros(nb, np.uint8)
    n = f(A.h, first.ctypes.data, o.ctypes.data, ml.ctypes.data, src.ctypes.data, bad.ctypes.data, cap)
    assert n >= 0
    return first, o[:n], ml[:n], src[:n], bad


@pytest.mark.parametrize("enc", ["lib-dna", "lib-dna-norep", "lib-text", "lib-text-k128", "oracle-dna"])
def test_parse_only_pass_equals_oracle_parse(acx, ctx, enc):
    if enc.startswith("lib-dna"):
        data = synth.dna((2 << 20) + 77, 41)
    else:
        data = synth.corpus("text" if "text" in enc else "dna", (2 << 20) + 77, 42)
    if enc == "oracle-dna":
        arc = oracle.encode(data)
    else:
        arc = acx.encode(data, no_rep="norep" in enc, max_lanes=128 if "k128" in enc else 32)
    nb = (data.size + BLOCK - 1) // BLOCK
    A = opened(acx, ctx, arc)
    A.build_index()
    first, o, ml, src, bad = device_index(acx, A, nb)
    assert not bad.any()
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        m = t["ml"] > 0
        k0, k1 = int(first[b]), int(first[b + 1])
        assert k1 - k0 == int(m.sum()), b
        assert np.array_equal(o[k0:k1].astype(np.int64), (t["dst"][m] - BLOCK * b).astype(np.int64)), b
        assert np.array_equal(ml[k0:k1].astype(np.int64), t["ml"][m].astype(np.int64)), b
        assert np.array_equal(src[k0:k1], t["src"][m]), b
    A.close()


@pytest.mark.parametrize("enc", ["lib-dna", "lib-dna-norep", "lib-text", "oracle-text"])
def test_parse_stats_equal_oracle_stats(acx, ctx, enc):
    """Command counts, repeat-code shares and the dependency-free runs (paper,
    The Last Sequential Element) of the device's parse equal the oracle's."""
    kind = "text" if "text" in enc else "dna"
    data = synth.corpus(kind, (3 << 20) + 901, 44)
    arc = oracle.encode(data) if enc.startswith("oracle") else acx.encode(data, no_rep="norep" in enc)
    A = opened(acx, ctx, arc)
    got = A.parse_stats()
    want = oracle.stats(arc)
    assert got["bad_blocks"] == 0
    pairs = [("blocks", "n_blocks"), ("tokens", "n_tokens"), ("new_matches", "n_new"), ("rep_matches", "n_rep"),
             ("lit_only", "n_litonly"), ("values", "n_values"), ("multibyte_values", "n_multibyte_values"),
             ("literal_bytes", "n_literal_bytes"), ("match_bytes", "n_match_bytes"),
             ("overlap_matches", "n_overlap_tokens"), ("external_matches", "n_external_tokens"),
             ("max_tokens_block", "max_tokens_block"), ("runs", "runs"), ("run_len_sum", "run_len_sum"),
             ("median_run", "median_run")]
    for g, w in pairs:
        assert got[g] == want[w], (g, got[g], want[w])
    assert sum(got["rep_matches"]) == want["hist_dependent"]
    if "norep" in enc:
        assert sum(got["rep_matches"]) == 0 and got["runs"] == got["blocks"]
    A.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_random_periodic_fills(acx, ctx, variant):
    """Random (distance, length) with distance in [1, 200] and length up to
    4096: the decode equals the byte-serial copy, also when a block holds
    many of them back to back and when a fill's source is in another block."""
    from gpu_util import gpu_decode
    rng = np.random.default_rng(9)
    blocks, expect = [], bytearray()
    for _ in range(6):
        toks, used = [], 0
        while True:
            d = int(rng.integers(1, 201))
            ml = int(rng.integers(4, 4097))
            if used + d + ml > BLOCK:
                break
            lits = bytes(rng.integers(0, 256, d, dtype=np.uint8))
            dst = len(expect) + d
            toks.append({"cmd": 0, "lits": lits, "ml": ml, "src": dst - d})
            expect += lits
            for j in range(ml):
                expect.append(expect[dst - d + j])
            used += d + ml
        # pad the block to exactly 16 KiB with a match reading the previous block
        rest = BLOCK - used
        if rest >= 4 and len(expect) > BLOCK:
            src = len(expect) - BLOCK
            toks.append({"cmd": 0, "lits": b"", "ml": rest, "src": src})
            for j in range(rest):
                expect.append(expect[src + j])
        else:
            lits = bytes(rng.integers(0, 256, rest, dtype=np.uint8))
            toks.append({"cmd": 5, "lits": lits, "ml": 0})
            expect += lits
        blocks.append(toks)
    arc = build_archive(blocks)
    assert oracle.decode(arc, verify=False).tobytes() == bytes(expect)
    rc, out = gpu_decode(ctx, arc, variant)
    assert rc == 0, ctx.last_error()
    assert out.tobytes() == bytes(expect)


def corrupt_block(arc, b):
    """Flip bytes in the middle of block b's command-stream body."""
    a = bytearray(arc)
    off_idx = struct.unpack_from("<Q", a, 40)[0]
    poff = struct.unpack_from("<Q", a, off_idx + 40 * b)[0]
    enc = struct.unpack_from("<I", a, poff + 4)[0]
    for j in range(max(1, enc // 2), min(enc, enc // 2 + 8)):
        a[poff + 48 + j] ^= 0xA7
    a[poff + 48] ^= 0x5B
    return bytes(a)


def test_corrupt_block_fails_only_its_dependents(acx, ctx):
    import torch
    data = synth.dna((3 << 20) + 500, 43)
    good = acx.encode(data)
    nb = (data.size + BLOCK - 1) // BLOCK
    X = 97
    bad = corrupt_block(good, X)
    assert oracle.decode_status(bad, verify=False)[0] == oracle.E_CORRUPT
    # which regions reach block X, from the good archive's parse
    from test_lib_cpu import _closure, _match_index
    idx = _match_index(good, nb)
    rng = np.random.default_rng(5)
    regions = [(X * BLOCK + 10, 100), (0, 50), (data.size - 40, 40)]
    regions += [(int(s), int(l)) for l in rng.integers(1, 60000, 40) for s in [rng.integers(0, data.size - l)]]
    reaches = [X in _closure(acx, good, idx, s, l) for s, l in regions]
    assert any(reaches) and not all(reaches)
    A = opened(acx, ctx, bad)
    A.build_index()  # the parse records the corrupt block and goes on
    assert device_index(acx, A, nb)[4][X] == 1
    stream = torch.cuda.current_stream().cuda_stream
    for (s, l), r in zip(regions, reaches):
        out = torch.zeros(l, dtype=torch.uint8, device="cuda")
        rc = acx.decode_range(ctx, A, s, l, out.data_ptr(), stream)
        if r:
            assert rc == -2, (s, l)
        else:
            assert rc == 0, (s, l, ctx.last_error())
            assert np.array_equal(out.cpu().numpy(), data[s:s + l])
    # the region server: the same split, in one burst sharing ticks
    srv = acx.Server(ctx, A, cache_bytes=512 * BLOCK)
    lens = np.array([l for _, l in regions], np.uint64)
    offs = np.concatenate([[0], np.cumsum(lens.astype(np.int64))])
    arena = torch.zeros(int(offs[-1]), dtype=torch.uint8, device="cuda")
    ids = srv.submit_many(np.array([s for s, _ in regions], np.uint64), lens,
                          (arena.data_ptr() + offs[:-1]).astype(np.uint64))
    assert srv.drain(30000) == 0
    by_id = {c["id"]: c["status"] for c in srv.poll(1000)}
    whole = arena.cpu().numpy()
    for k, ((s, l), r) in enumerate(zip(regions, reaches)):
        st = by_id[int(ids[k])]
        if r:
            assert st == -2, (s, l)
        else:
            assert st == 0, (s, l)
            assert np.array_equal(whole[offs[k]:offs[k] + l], data[s:s + l])
    srv.close()
    A.close()
