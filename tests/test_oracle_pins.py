"""Pins of the CPU oracle to facts outside itself: published vectors,
hand-worked examples, closed forms, brute force on tiny inputs and the
invariants the paper states.  (-m "not gpu")."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from fmt_writer import build_archive, leb128
from golden import worked_examples as W


# ---- FNV-1a 64 and the generator RNG -------------------------------------------------

@pytest.mark.parametrize("data,h", W.FNV1A64_VECTORS)
def test_fnv_published_vectors(data, h):
    assert oracle.fnv1a64(data) == h


def test_splitmix64_reference_sequence():
    assert [int(v) for v in synth.splitmix64(1234567, 3)] == W.SPLITMIX64_1234567


# ---- rANS --------------------------------------------------------------------------------

def _table(d):
    f = np.zeros(256, np.uint16)
    for k, v in d.items():
        f[k] = v
    return f


@pytest.mark.parametrize("ex", W.RANS_WORKED, ids=lambda e: e["name"])
def test_rans_worked_examples(ex):
    f = _table(ex["freq"])
    body = oracle.rans_encode(ex["symbols"], ex["K"], f)
    assert body.hex() == ex["body_hex"]
    dec = oracle.rans_decode(bytes.fromhex(ex["body_hex"]), len(ex["symbols"]), ex["K"], f)
    assert dec.tobytes() == ex["symbols"]


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16, 32, 64, 128])
def test_rans_roundtrip_lane_counts(K):
    rng = np.random.default_rng(K)
    for n in sorted({1, max(K - 1, 1), K, K + 1, 64 * K + 3, 5000}):
        counts = rng.integers(0, 50, 256).astype(np.uint64)
        counts[rng.integers(0, 256)] += 1
        f = oracle.normalize(counts)
        p = f / 4096.0
        sym = rng.choice(256, size=n, p=p).astype(np.uint8)
        body = oracle.rans_encode(sym, K, f)
        assert len(body) >= 16 * ((4 * K + 15) // 16)
        assert np.array_equal(oracle.rans_decode(body, n, K, f), sym)


def test_rans_single_symbol_table_emits_no_words():
    f = _table({7: 4096})
    sym = np.full(1000, 7, np.uint8)
    body = oracle.rans_encode(sym, 4, f)
    assert len(body) == 16  # 4 states, no words: x stays at L = 2^16
    assert all(int.from_bytes(body[4 * j:4 * j + 4], "little") == 65536 for j in range(4))
    assert np.array_equal(oracle.rans_decode(body, 1000, 4, f), sym)


def test_rans_size_matches_entropy_closed_form():
    """Coded size equals the ideal code length sum(-log2(f_s/4096)) up to the
    stored states (rANS is within a vanishing overhead of the table's
    entropy; a dropped or doubled renormalisation would break this)."""
    rng = np.random.default_rng(5)
    f = _table({65: 1500, 67: 1000, 71: 1000, 84: 590, 78: 6})
    p = f / 4096.0
    for K in (1, 32):
        sym = rng.choice(256, size=300_000, p=p).astype(np.uint8)
        ideal_bits = float(np.sum(-np.log2(p[sym])))
        body = oracle.rans_encode(sym, K, f)
        coded_bits = 8 * (len(body) - 16 * ((4 * K + 15) // 16))
        # the final states carry up to 16 useful bits each beyond the words
        assert ideal_bits - 16 * K - 16 <= coded_bits <= ideal_bits * 1.001 + 32
    # a uniform 4-symbol table costs exactly 2 bits per symbol
    fu = _table({65: 1024, 67: 1024, 71: 1024, 84: 1024})
    sym = rng.choice([65, 67, 71, 84], size=100_000).astype(np.uint8)
    body = oracle.rans_encode(sym, 1, fu)
    words = (len(body) - 16) // 2
    assert 16 * words + 17 <= 2 * 100_000 + 17 <= 16 * words + 32


def test_rans_corruption_detected():
    rng = np.random.default_rng(9)
    f = oracle.normalize(np.bincount(rng.integers(0, 4, 1000), minlength=256))
    sym = rng.integers(0, 4, 4000).astype(np.uint8)
    body = bytearray(oracle.rans_encode(sym, 8, f))
    # truncated words
    with pytest.raises(oracle.OracleError):
        oracle.rans_decode(bytes(body[:-2]), 4000, 8, f)
    # a state below L is invalid
    bad = bytearray(body)
    bad[0:4] = (100).to_bytes(4, "little")
    with pytest.raises(oracle.OracleError):
        oracle.rans_decode(bytes(bad), 4000, 8, f)


def test_normalize_properties():
    rng = np.random.default_rng(1)
    for _ in range(50):
        counts = np.zeros(256, np.uint64)
        k = rng.integers(1, 257)
        idx = rng.choice(256, k, replace=False)
        counts[idx] = rng.integers(1, 10 ** rng.integers(1, 7), k)
        f = oracle.normalize(counts)
        assert int(f.sum()) == 4096
        assert np.all((f > 0) == (counts > 0))
    assert int(oracle.normalize(np.zeros(256, np.uint64)).sum()) == 0


# ---- format: hand-built archives ----------------------------------------------------------

@pytest.mark.parametrize("ex", W.ARCHIVE_WORKED, ids=lambda e: e["name"])
def test_worked_archives(ex):
    arc = build_archive(ex["blocks"], expected=ex["expected"], fnv=oracle.fnv1a64)
    out = oracle.decode(arc, verify=True)
    assert out.tobytes() == ex["expected"]
    if "off_stream_block1_hex" in ex:
        assert oracle.block_stream(arc, 1, oracle.OFF).tobytes().hex() == ex["off_stream_block1_hex"]
        assert oracle.block_stream(arc, 0, oracle.LEN).tobytes().hex() == ex["len_stream_block0_hex"]


def test_worked_archive_parse_positions():
    ex = W.ARCHIVE_WORKED[1]
    arc = build_archive(ex["blocks"])
    t = oracle.parse_block(arc, 1)
    # hand-derived (see worked_examples): dst and src of the five matches
    assert list(t["dst"][:5]) == [16384, 16395, 16399, 16407, 16415]
    assert list(t["src"][:5]) == [300, 16380, 315, 16406, 331]
    assert list(t["lit"]) == [0, 0, 1, 1, 3, 3]


def test_overlap_equals_periodic_expansion_bruteforce():
    """Every (d, ML) with d <= 16, ML <= 64: the byte-serial decode equals the
    periodic fill out[dst+k] = out[src + (k mod d)] (paper, 'What Does:
    Periods, Not Chains')."""
    rng = np.random.default_rng(3)
    for d in range(1, 17):
        for ml in range(4, 65):
            lits = bytes(rng.integers(0, 256, d, dtype=np.uint8))
            toks = [{"cmd": 0, "lits": lits, "ml": ml, "src": 0}]
            expected = lits + bytes(lits[k % d] for k in range(ml))
            arc = build_archive([toks])
            assert oracle.decode(arc, verify=False).tobytes() == expected


def _corrupt_cases():
    ok = [{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 0}, {"cmd": 5, "lits": b"TT", "ml": 0}]
    yield "offset not before destination", [[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 4}]]
    yield "repeat distance beyond start", [[{"cmd": 1, "lits": b"", "ml": 4}]]
    yield "unknown command", [[{"cmd": 6, "lits": b"ACGT", "ml": 4, "src": 0}]]
    yield "lit-only not last", [[{"cmd": 5, "lits": b"AC", "ml": 0}, {"cmd": 0, "lits": b"GT", "ml": 4, "src": 0}]]
    yield "lit-only with match length", [[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 0},
                                          {"cmd": 5, "lits": b"TT", "ml": 3}]]
    yield "match shorter than min_match", [[{"cmd": 0, "lits": b"ACGT", "ml": 3, "src": 0}]]
    yield "valid control", [ok]


@pytest.mark.parametrize("name,blocks", list(_corrupt_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_corrupt_token_streams(name, blocks):
    arc = build_archive(blocks)
    rc, _ = oracle.decode_status(arc, verify=False)
    assert rc == (0 if name == "valid control" else oracle.E_CORRUPT)


def test_corrupt_varints_and_counts():
    toks = [{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 0}]
    cmd, lens, off, lit = [bytes([0]), leb128(4) + leb128(4), bytes(5), b"ACGT"]
    good = build_archive([toks], raw_streams={0: [cmd, lens, off, lit]})
    assert oracle.decode_status(good, verify=False)[0] == 0
    cases = {
        "4-byte varint": [cmd, b"\x84\x80\x80\x00" + leb128(4), off, lit],
        "trailing length byte": [cmd, lens + b"\x00", off, lit],
        "missing length": [cmd, lens[:1], off, lit],
        "offset stream not multiple of 5": [cmd, lens, bytes(6), lit],
        "extra offset": [cmd, lens, bytes(10), lit],
        "extra literal": [cmd, lens, off, lit + b"A"],
    }
    for name, streams in cases.items():
        arc = build_archive([toks], raw_streams={0: streams})
        assert oracle.decode_status(arc, verify=False)[0] == oracle.E_CORRUPT, name


# ---- round trips and invariants -------------------------------------------------------------

def test_exhaustive_tiny_roundtrips():
    for alphabet, maxlen in ((b"AC", 10), (b"ACGTN", 5)):
        for n in range(0, maxlen + 1):
            for tup in itertools.product(alphabet, repeat=n):
                data = bytes(tup)
                for nr in (False, True):
                    arc = oracle.encode(data, no_rep=nr)
                    assert oracle.decode(arc).tobytes() == data


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_corpus_roundtrip_and_invariants(kind, dna4m, text4m):
    data = dna4m if kind == "dna" else text4m
    data = data[: 1 << 20]
    arcs = {nr: oracle.encode(data, no_rep=nr) for nr in (False, True)}
    for nr, arc in arcs.items():
        assert np.array_equal(oracle.decode(arc), data)
        st = oracle.stats(arc)
        if nr:
            assert sum(st["n_rep"]) == 0
    # the history-free encoding keeps the same matches: same token boundaries
    # and sources, only the command codes and offset stream differ
    nb = oracle.info(arcs[False])["n_blocks"]
    for b in range(0, nb, 7):
        th, tf = oracle.parse_block(arcs[False], b), oracle.parse_block(arcs[True], b)
        for k in ("ll", "ml", "dst", "src", "lit"):
            assert np.array_equal(th[k], tf[k])
        assert np.all(tf["cmd"][tf["ml"] > 0] == 0)
        # every absolute offset precedes its destination
        m = th["ml"] > 0
        assert np.all(th["src"][m] < th["dst"][m])
        # positions: dst_i = B + sum_{j<i}(LL_j + ML_j) + LL_i
        B = b * oracle.BLOCK
        ends = B + np.cumsum(th["ll"].astype(np.int64) + th["ml"].astype(np.int64))
        starts = np.concatenate([[B], ends[:-1]])
        assert np.array_equal(th["dst"].astype(np.int64), starts + th["ll"])


def test_overlapping_tokens_are_periodic_in_corpus(dna4m):
    data = dna4m[: 1 << 19]
    arc = oracle.encode(data)
    out = oracle.decode(arc)
    seen = 0
    for b in range(oracle.info(arc)["n_blocks"]):
        t = oracle.parse_block(arc, b)
        for i in np.nonzero((t["ml"] > 0) & (t["dst"] - t["src"] < t["ml"]))[0]:
            dst, src, ml = int(t["dst"][i]), int(t["src"][i]), int(t["ml"][i])
            d = dst - src
            k = np.arange(ml)
            assert np.array_equal(out[dst + k], out[src + (k % d)])
            seen += 1
    assert seen > 50


def test_special_cases():
    rng = np.random.default_rng(11)
    # all-literal input: the literal stream is the input
    data = rng.integers(0, 256, 40000, dtype=np.uint8)
    arc = oracle.encode(data)
    assert oracle.stats(arc)["n_match_bytes"] == 0
    assert np.array_equal(np.concatenate([oracle.block_stream(arc, b, oracle.LIT) for b in range(3)]), data)
    # a single run of 'N': one literal, then a repeat match at distance 1
    data = b"N" * 1000
    arc = oracle.encode(data)
    t = oracle.parse_block(arc, 0)
    assert list(t["cmd"]) == [1] and int(t["ll"][0]) == 1 and int(t["ml"][0]) == 999
    assert int(t["dst"][0] - t["src"][0]) == 1
    assert oracle.decode(arc).tobytes() == data
    t2 = oracle.parse_block(oracle.encode(data, no_rep=True), 0)
    assert list(t2["cmd"]) == [0] and int(t2["src"][0]) == 0
    # the encoder is deterministic
    d = synth.dna(200_000, 7)
    assert oracle.encode(d) == oracle.encode(d)
    # empty input
    assert oracle.decode(oracle.encode(b"")).size == 0


def test_truncation_and_bit_flips_never_crash(dna4m):
    data = dna4m[: 100_000]
    arc = bytearray(oracle.encode(data))
    for cut in (10, 63, 2100, len(arc) // 2, len(arc) - 1):
        rc, _ = oracle.decode_status(bytes(arc[:cut]))
        assert rc == oracle.E_CORRUPT
    rng = np.random.default_rng(2)
    for _ in range(200):
        bad = bytearray(arc)
        pos = int(rng.integers(0, len(bad)))
        bad[pos] ^= 1 << int(rng.integers(0, 8))
        rc, out = oracle.decode_status(bytes(bad), verify=True)
        assert rc in (0, oracle.E_CORRUPT, oracle.E_ARG)
        if rc == 0:
            assert np.array_equal(out, data)


# ---- dependency lists -----------------------------------------------------------------

def _three_blocks(src, ml):
    """Blocks 0 and 1 are 16 KiB literal runs; block 2 (the short last block)
    holds one NEW match reading `ml` bytes from absolute position `src`."""
    rng = np.random.default_rng(21)
    b0 = bytes(rng.integers(0, 256, 16384, dtype=np.uint8))
    b1 = bytes(rng.integers(0, 256, 16384, dtype=np.uint8))
    blocks = [[{"cmd": 5, "lits": b0, "ml": 0}], [{"cmd": 5, "lits": b1, "ml": 0}],
              [{"cmd": 0, "lits": b"AB", "ml": ml, "src": src}]]
    full = b0 + b1 + b"AB"
    for j in range(ml):  # byte-serial definition of the copy
        full += bytes([full[src + j]])
    return blocks, full


@pytest.mark.parametrize("src,ml,need", [
    (100, 50, {0}),                 # reads block 0 only
    (16384 - 10, 50, {0, 1}),       # the read window straddles blocks 0 and 1
    (2 * 16384 - 4, 30, {1}),       # window runs into block 2 itself: only block 1 is listed
])
def test_dependency_lists_must_cover_every_block_read(src, ml, need):
    """Format v1 reading of the paper's block dependencies (Setup: a block is
    decodable once the blocks holding its sources exist): with a dependency
    section present, every other block a match reads must be listed in the
    reading block's list.  A list that covers the reads (or more) decodes to
    the byte-serial definition; a list that misses one is corrupt."""
    blocks, full = _three_blocks(src, ml)
    ok = build_archive(blocks, deps=[[], [], sorted(need)])
    assert oracle.decode(ok, verify=False).tobytes() == full
    over = build_archive(blocks, deps=[[], [0], [0, 1]])
    assert oracle.decode(over, verify=False).tobytes() == full
    for drop in need:
        short = build_archive(blocks, deps=[[], [], sorted(need - {drop})])
        assert oracle.decode_status(short, verify=False)[0] == oracle.E_CORRUPT
    # without a dependency section nothing is required
    assert oracle.decode(build_archive(blocks), verify=False).tobytes() == full


def test_self_overlap_reads_one_period_across_a_block_boundary():
    """A self-overlapping match reads one period (paper, Periods, Not Chains):
    at the start of block 1 with distance 6 it reads 4 bytes of block 0 and 2
    of its own block, so only block 0 must be listed."""
    rng = np.random.default_rng(3)
    b0 = bytes(rng.integers(0, 256, 16384, dtype=np.uint8))
    blocks = [[{"cmd": 5, "lits": b0, "ml": 0}], [{"cmd": 0, "lits": b"QR", "ml": 40, "src": 16384 - 4}]]
    full = bytearray(b0 + b"QR")
    for j in range(40):
        full.append(full[16384 - 4 + j])
    assert oracle.decode(build_archive(blocks, deps=[[], [0]]), verify=False).tobytes() == bytes(full)
    assert oracle.decode_status(build_archive(blocks, deps=[[], []]), verify=False)[0] == oracle.E_CORRUPT


def test_archive_statistics_of_a_hand_built_archive():
    """The oracle's archive statistics (the reference of the parse-statistics
    parity tests; paper, The Last Sequential Element) on a two-block archive
    whose every count is worked out by hand.  History starts [1,2,3,4]; NEW
    pushes its distance, REPk moves entry k to the front.

    Block 0 (16,384 B):
      t0 NEW  LL 4    ML 4    src 0     d 4    hist [4,1,2,3]
      t1 REP0 LL 0    ML 8              d 4    overlapping
      t2 NEW  LL 200  ML 5    src 0     d 216  hist [216,4,1,2]; LL takes 2 bytes
      t3 REP1 LL 0    ML 6              d 4    overlapping; hist [4,216,1,2]
      t4 NEW  LL 0    ML 300  src 10    d 217  overlapping; ML takes 2 bytes
      t5 LIT  LL 15857                         LL takes 2 bytes
      runs (non-repeat tokens before each repeat, then the tail): 1, 1, 2
    Block 1 (17 B):
      t0 NEW  LL 0    ML 10   src 100   (in block 0: external)
      t1 NEW  LL 2    ML 4    src 16384 d 12
      t2 LIT  LL 1
      runs: 3
    """
    lit = lambda n, c=b"a": (c * n)[:n]  # noqa: E731
    blk0 = [{"cmd": 0, "lits": b"ABCD", "ml": 4, "src": 0},
            {"cmd": 1, "lits": b"", "ml": 8},
            {"cmd": 0, "lits": lit(200), "ml": 5, "src": 0},
            {"cmd": 2, "lits": b"", "ml": 6},
            {"cmd": 0, "lits": b"", "ml": 300, "src": 10},
            {"cmd": 5, "lits": lit(15857, b"q"), "ml": 0}]
    blk1 = [{"cmd": 0, "lits": b"", "ml": 10, "src": 100},
            {"cmd": 0, "lits": b"xy", "ml": 4, "src": 16384},
            {"cmd": 5, "lits": b"z", "ml": 0}]
    arc = build_archive([blk0, blk1])
    st = oracle.stats(arc)
    want = {"n_blocks": 2, "n_tokens": 9, "n_new": 5, "n_rep": [1, 1, 0, 0], "n_litonly": 2, "n_values": 18,
            "n_multibyte_values": 3, "n_match_bytes": 337, "n_literal_bytes": 16064, "n_overlap_tokens": 3,
            "n_external_tokens": 1, "max_tokens_block": 6, "hist_dependent": 2, "runs": 4, "run_len_sum": 7,
            "median_run": 2}
    for k, v in want.items():
        assert st[k] == v, (k, st[k], v)
    assert oracle.decode(arc, verify=False).size == 16384 + 17


def test_level_bodies_are_hints_that_never_change_the_decode():
    """Format v1 flags bit1: each payload carries a stored level body (one
    byte per token) after its four stream bodies.  The levels are scheduling
    hints (paper, Depth Does Not Govern Latency: waves); an archive decodes
    to the same bytes with or without them, whatever their values, and a
    level body that leaves its payload is corrupt."""
    blk0 = [{"cmd": 0, "lits": b"ABCDEFGH", "ml": 8, "src": 0},
            {"cmd": 5, "lits": b"x" * (oracle.BLOCK - 16), "ml": 0}]
    blk1 = [{"cmd": 0, "lits": b"", "ml": 12, "src": 3},
            {"cmd": 1, "lits": b"yz", "ml": 5},
            {"cmd": 5, "lits": b"!", "ml": 0}]
    plain = build_archive([blk0, blk1])
    with_levels = build_archive([blk0, blk1], levels=[[0, 0], [1, 2, 0]])
    odd_levels = build_archive([blk0, blk1], levels=[[7, 255], [0, 0, 9]])
    want = oracle.decode(plain, verify=False)
    assert want.size == oracle.BLOCK + 20
    assert np.array_equal(oracle.decode(with_levels, verify=False), want)
    assert np.array_equal(oracle.decode(odd_levels, verify=False), want)
    assert oracle.block_levels(with_levels, 1).tolist() == [1, 2, 0]
    assert oracle.block_levels(odd_levels, 0).tolist() == [7, 255]
    with pytest.raises(oracle.OracleError):
        oracle.block_levels(plain, 0)
    # a level body cut short: the payload length no longer covers it
    bad = bytearray(with_levels)
    off_index = int.from_bytes(bad[40:48], "little")
    e = off_index + 40  # block 1's index entry
    plen = int.from_bytes(bad[e + 8:e + 12], "little")
    bad[e + 8:e + 12] = (plen - 16).to_bytes(4, "little")
    assert oracle.decode_status(bytes(bad), verify=False)[0] == oracle.E_CORRUPT
