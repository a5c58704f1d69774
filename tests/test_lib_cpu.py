"""Host-side checks of the product library (no GPU): the C ABI loads and
exports every function declared in include/aceapex.h, the library encoder's
archives decode bit-exactly in the oracle, and the host-side structural
validation agrees with the oracle on corrupt archives.  (-m "not gpu")"""
import os
import re

import numpy as np
import pytest

import oracle
import synth
from fmt_writer import build_archive

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def acx():
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    acx.load()
    return acx


def declared_functions():
    src = open(os.path.join(ROOT, "include", "aceapex.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aceapex_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(acx):
    import ctypes
    L = ctypes.CDLL(acx.build.SO)
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(acx.lib.EXPORTED)


@pytest.mark.parametrize("kind", ["dna", "text"])
@pytest.mark.parametrize("no_rep", [False, True])
@pytest.mark.parametrize("lanes", [1, 32, 128])
def test_library_encoder_decodes_in_oracle(acx, kind, no_rep, lanes):
    data = synth.corpus(kind, 300_000 + 1234, 5)
    arc = acx.encode(data, no_rep=no_rep, max_lanes=lanes)
    assert np.array_equal(oracle.decode(arc), data)
    st = oracle.stats(arc)
    if no_rep:
        assert sum(st["n_rep"]) == 0
    info = acx.archive_check(arc)
    assert info["total_size"] == len(data) and info["tokens"] == st["n_tokens"]


def test_library_encoder_edge_sizes(acx):
    rng = np.random.default_rng(0)
    for n in (0, 1, 15, 16, 17, 16383, 16384, 16385, 3 * 16384 + 7):
        data = rng.integers(0, 4, n, dtype=np.uint8) + 65
        for nr in (False, True):
            arc = acx.encode(data, no_rep=nr)
            assert np.array_equal(oracle.decode(arc), data)


def test_history_free_keeps_matches_and_costs_little(acx):
    """Paper, 'The Last Sequential Element': dropping the history keeps the
    matches.  Token boundaries are identical; a source may move to another
    position holding the same bytes (the encoder forwards explicit offsets to
    the root of a copy chain), so sources are compared by content."""
    data = synth.dna(2 << 20, 3)
    a0, a1 = acx.encode(data), acx.encode(data, no_rep=True)
    for b in range(0, 128, 9):
        t0, t1 = oracle.parse_block(a0, b), oracle.parse_block(a1, b)
        for k in ("ll", "ml", "dst"):
            assert np.array_equal(t0[k], t1[k])
        for s0, s1, ml in zip(t0["src"], t1["src"], t0["ml"]):
            assert np.array_equal(data[int(s0):int(s0) + int(ml)], data[int(s1):int(s1) + int(ml)])
    growth = (len(a1) - len(a0)) / len(a0)
    assert 0.0 < growth < 0.02
    assert oracle.stats(a0)["median_run"] < oracle.stats(a1)["median_run"]


def test_host_validation_rejects_structural_corruption(acx):
    data = synth.dna(100_000, 1)
    arc = bytearray(acx.encode(data))
    acx.archive_check(bytes(arc))
    for cut in (10, 63, 2100, len(arc) - 16):
        with pytest.raises(acx.AceapexError):
            acx.archive_check(bytes(arc[:cut]))
    bad = bytearray(arc)
    bad[0] ^= 1  # magic
    with pytest.raises(acx.AceapexError):
        acx.archive_check(bytes(bad))
    # a block that claims more literal bytes than it holds
    from fmt_writer import inflate_literal_stream
    big = inflate_literal_stream(bytes(arc))
    with pytest.raises(acx.AceapexError):
        acx.archive_check(big)
    assert oracle.decode_status(big, verify=False)[0] == oracle.E_CORRUPT
    # a hand-built archive with a token-level fault passes the structural
    # check (it is caught by the kernels) but not the oracle
    toks = [[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 4}]]
    a = build_archive(toks)
    acx.archive_check(a)
    assert oracle.decode_status(a, verify=False)[0] == oracle.E_CORRUPT


def read_deps(arc):
    """(off_deps, per-block dependency lists) from the header and index."""
    import struct
    nb = struct.unpack_from("<I", arc, 24)[0]
    off_idx, off_deps = struct.unpack_from("<QQ", arc, 40)
    lists = []
    for b in range(nb):
        dep_off, n_deps = struct.unpack_from("<II", arc, off_idx + 40 * b + 20)
        lists.append([struct.unpack_from("<I", arc, off_deps + 4 * (dep_off + k))[0] for k in range(n_deps)])
    return off_deps, lists


@pytest.mark.parametrize("kind", ["dna", "text"])
@pytest.mark.parametrize("no_rep", [False, True])
def test_library_dependency_lists_are_the_blocks_read(acx, kind, no_rep):
    """With deps=True each block lists exactly the earlier blocks its matches
    read (a self-overlapping match reads one period), as found by the oracle's
    own parse; without, the archive has no dependency section."""
    data = synth.corpus(kind, 700_000 + 77, 8)
    arc = acx.encode(data, no_rep=no_rep, deps=True)
    assert np.array_equal(oracle.decode(arc), data)
    off, lists = read_deps(arc)
    assert off != 0
    for b, got in enumerate(lists):
        t = oracle.parse_block(arc, b)
        want = set()
        for s, m, d in zip(t["src"].tolist(), t["ml"].tolist(), t["dst"].tolist()):
            if m == 0:
                continue
            e = s + min(m, d - s)
            want.update(a for a in range(s // 16384, (e - 1) // 16384 + 1) if a < b)
        assert got == sorted(want), b
    plain = acx.encode(data, no_rep=no_rep)
    assert read_deps(plain)[0] == 0
    assert len(plain) < len(arc)


def test_segmented_encode_keeps_sources_inside_segments(acx):
    """Segmented parallel parse: every match reads inside its own segment
    (checked on the oracle's parse), the archive decodes exactly, and the
    size stays close to the single-parse archive."""
    data = synth.dna((6 << 20) + 5000, 4)
    seg = 1 << 20
    arc = acx.encode(data, segment=seg, threads=4, deps=True)
    assert np.array_equal(oracle.decode(arc), data)
    nb = (len(data) + 16383) // 16384
    for b in range(0, nb, 7):
        t = oracle.parse_block(arc, b)
        for s, m, d in zip(t["src"].tolist(), t["ml"].tolist(), t["dst"].tolist()):
            if m:
                assert s // seg == d // seg
    whole = acx.encode(data)
    assert len(arc) < 1.02 * len(whole) + 64 * 1024
    with pytest.raises(acx.AceapexError):
        acx.encode(data, segment=1000)  # not a multiple of the block size


def _match_index(arc, nb):
    """The archive's matches block by block, from the oracle's parse."""
    first, o, ml, src = [0], [], [], []
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        for m, d, s in zip(t["ml"].tolist(), t["dst"].tolist(), t["src"].tolist()):
            if m:
                o.append(d - 16384 * b)
                ml.append(m)
                src.append(s)
        first.append(len(o))
    return (np.array(first, np.uint64), np.array(o, np.uint16), np.array(ml, np.uint16), np.array(src, np.uint64))


def _closure(acx, arc, idx, start, length):
    import ctypes
    L = acx.load()
    f = L.acx_debug_closure
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    f.argtypes = [vp, u64, vp, u64, vp, vp, vp, u64, u64, vp, vp, vp, u32, u32, vp]
    f.restype = ctypes.c_int
    first, o, ml, src = idx
    a = np.frombuffer(arc, np.uint8)
    cap = 1 << 16
    blocks, cnt, ivs = np.zeros(cap, np.uint32), np.zeros(cap, np.uint32), np.zeros(cap * 4, np.uint32)
    n = np.zeros(1, np.uint32)
    rc = f(a.ctypes.data, a.size, first.ctypes.data, o.size, o.ctypes.data, ml.ctypes.data, src.ctypes.data,
           start, length, blocks.ctypes.data, cnt.ctypes.data, ivs.ctypes.data, cap, cap * 4, n.ctypes.data)
    assert rc == 0
    out, k = {}, 0
    for i in range(int(n[0])):
        out[int(blocks[i])] = [(int(v) & 0xffff, int(v) >> 16) for v in ivs[k:k + int(cnt[i])]]
        k += int(cnt[i])
    return out


@pytest.mark.parametrize("kind,no_rep", [("dna", False), ("dna", True), ("text", False)])
def test_byte_level_closure_is_sufficient(acx, kind, no_rep):
    """The byte-level closure walk (Random Access at Scale): decoding only the
    closure's blocks, and in them only the matches touching their wanted
    bytes (byte-serially, in output order, everything else left at zero),
    reproduces the requested region exactly; the wanted bytes cover the
    region and every wanted match lies inside them."""
    data = synth.corpus(kind, (1 << 20) + 333, 21)
    arc = acx.encode(data, no_rep=no_rep)
    nb = (data.size + 16383) // 16384
    idx = _match_index(arc, nb)
    toks = [oracle.parse_block(arc, b) for b in range(nb)]
    lits = [oracle.block_stream(arc, b, 3) for b in range(nb)]
    rng = np.random.default_rng(3)
    regions = [(0, 1), (data.size - 1, 1), (16380, 10)]
    regions += [(int(s), int(l)) for l in rng.integers(1, 40000, 12)
                for s in [rng.integers(0, data.size - l)]]
    for start, length in regions:
        need = _closure(acx, arc, idx, start, length)
        # the region's bytes are wanted
        for p in range(start // 16384, (start + length - 1) // 16384 + 1):
            s0, e0 = max(start, 16384 * p) - 16384 * p, min(start + length, 16384 * (p + 1)) - 16384 * p
            assert any(s <= s0 and e0 <= e for s, e in need[p]), (start, length, p)
        out = np.zeros(data.size, np.uint8)
        for b in sorted(need):
            t, lit, B = toks[b], lits[b], 16384 * b
            ivs = need[b]
            for ll, m, d, s, li in zip(t["ll"].tolist(), t["ml"].tolist(), t["dst"].tolist(), t["src"].tolist(),
                                       t["lit"].tolist()):
                out[d - ll:d] = lit[li:li + ll]
                if m and any(s0 < d - B + m and d - B < e0 for s0, e0 in ivs):
                    assert any(s0 <= d - B and d - B + m <= e0 for s0, e0 in ivs)  # the whole match is wanted
                    for j in range(m):
                        out[d + j] = out[s + j]
        assert np.array_equal(out[start:start + length], data[start:start + length]), (start, length)


BLOCK = 16384
PARSE_STAT_PAIRS = [("blocks", "n_blocks"), ("tokens", "n_tokens"), ("new_matches", "n_new"),
                    ("rep_matches", "n_rep"), ("lit_only", "n_litonly"), ("values", "n_values"),
                    ("multibyte_values", "n_multibyte_values"), ("literal_bytes", "n_literal_bytes"),
                    ("match_bytes", "n_match_bytes"), ("overlap_matches", "n_overlap_tokens"),
                    ("external_matches", "n_external_tokens"), ("max_tokens_block", "max_tokens_block"),
                    ("runs", "runs"), ("run_len_sum", "run_len_sum"), ("median_run", "median_run")]


@pytest.mark.parametrize("kind,no_rep", [("dna", False), ("dna", True), ("text", False)])
def test_parse_stats_counting_equals_oracle_counts(acx, kind, no_rep):
    """The host counting behind aceapex_archive_parse_stats (paper, The Last
    Sequential Element: repeat-coded share and dependency-free runs), fed the
    token records the parse-only pass would write, built here from the
    oracle's parse, gives the oracle's own counts."""
    import ctypes
    data = synth.corpus(kind, (1 << 20) + 333, 7)
    arc = acx.encode(data, no_rep=no_rep)
    nb = (data.size + BLOCK - 1) // BLOCK
    recs, ntok = [], np.zeros(nb, np.uint32)
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        ntok[b] = t["cmd"].size
        r = np.zeros((t["cmd"].size, 4), np.uint32)
        src = t["src"].astype(np.uint64)
        r[:, 0] = (src & np.uint64(0xffffffff)).astype(np.uint32)
        r[:, 1] = ((src >> np.uint64(32)) & np.uint64(0xff)).astype(np.uint32)
        r[:, 2] = (t["dst"].astype(np.int64) - b * BLOCK).astype(np.uint32) | (t["ml"].astype(np.uint32) << 16)
        r[:, 3] = t["cmd"]
        recs.append(r)
    recs = np.ascontiguousarray(np.concatenate(recs))
    f = acx.load().acx_debug_parse_stats
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = acx.lib.ParseStats()
    assert f(recs.ctypes.data, ntok.ctypes.data, nb, ctypes.byref(st)) == 0
    got, want = st.as_dict(), oracle.stats(arc)
    for g, w in PARSE_STAT_PAIRS:
        assert got[g] == want[w], (g, got[g], want[w])
    assert sum(got["rep_matches"]) == want["hist_dependent"]
    if no_rep:
        # no repeat codes: one run per block, the block's token count
        assert got["runs"] == nb and got["median_run"] == int(np.sort(ntok)[nb // 2])


@pytest.mark.parametrize("kind,max_depth", [("dna", 0), ("dna", 0xFFFFFFFF), ("text", 0), ("text", 4)])
def test_encoder_depth_statistics_follow_the_archive(acx, kind, max_depth):
    """aceapex_encode_ex's chain-depth histograms (paper, Depth Does Not
    Govern Latency) equal the depths recomputed from the archive alone: each
    match, in output order, gets 1 + the deepest byte of the source window it
    reads (one period of a self-overlapping match), literals depth 0.  With a
    cap, no match is deeper than the cap."""
    data = synth.corpus(kind, (1 << 20) + 4321, 11)
    st = {}
    arc = acx.encode(data, max_depth=max_depth, stats=st)
    nb = (data.size + BLOCK - 1) // BLOCK
    D = np.zeros(data.size, np.int64)
    match_hist = np.zeros(256, np.int64)
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        for dst, src, ml in zip(t["dst"].tolist(), t["src"].tolist(), t["ml"].tolist()):
            if not ml:
                continue
            w = min(dst - src, ml)
            dep = min(1 + int(D[src:src + w].max()), 255)
            D[dst:dst + ml] = dep
            match_hist[dep] += 1
    blk = np.array([D[b * BLOCK:(b + 1) * BLOCK].max() for b in range(nb)])
    assert st["blocks"] == nb and st["matches"] == int(match_hist.sum())
    assert st["match_depth"] == match_hist.tolist()
    assert st["block_max_depth"] == np.bincount(blk, minlength=256).tolist()
    cap = 16 if max_depth == 0 else max_depth
    if cap < 255:
        assert max(d for d in range(256) if st["match_depth"][d]) <= cap


@pytest.mark.parametrize("kind,max_depth", [("dna", 0), ("text", 0), ("text", 4)])
def test_encoder_level_statistics_follow_the_archive(acx, kind, max_depth):
    """The cross-block levels of aceapex_encode_ex, recomputed from the
    archive alone: in output order, a match whose source window lies in its
    own block and holds only level-0 bytes gets level 0 (the local pass
    finishes it); any other match gets 1 + the highest level in its window."""
    data = synth.corpus(kind, (1 << 20) + 999, 12)
    st = {}
    arc = acx.encode(data, max_depth=max_depth, stats=st)
    nb = (data.size + BLOCK - 1) // BLOCK
    lv = np.zeros(data.size, np.int64)
    count, nbytes = np.zeros(256, np.int64), np.zeros(256, np.int64)
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        for dst, src, ml in zip(t["dst"].tolist(), t["src"].tolist(), t["ml"].tolist()):
            if not ml:
                continue
            mx = int(lv[src:src + min(dst - src, ml)].max())
            level = 0 if (src >= b * BLOCK and mx == 0) else min(mx + 1, 255)
            lv[dst:dst + ml] = level
            count[level] += 1
            nbytes[level] += ml
    assert st["match_level"] == count.tolist()
    assert st["level_bytes"] == nbytes.tolist()
    # a match's level never exceeds its chain depth
    assert max(l for l in range(256) if count[l]) <= max(d for d in range(256) if st["match_depth"][d])


@pytest.mark.parametrize("kind,no_rep", [("dna", False), ("text", False), ("text", True)])
def test_encoder_level_bodies(acx, kind, no_rep):
    """aceapex_enc_params.levels: the archive carries, per token, the level
    recomputed from its own parse (a match whose source window lies in its
    own block and holds only level-0 bytes: 0; any other: 1 + the highest
    level in the window; a closing literal-only token: 0).  The four streams
    are those of the archive without levels, so both decode alike."""
    data = synth.corpus(kind, (1 << 20) + 555, 13)
    arc = acx.encode(data, no_rep=no_rep, levels=True)
    arc0 = acx.encode(data, no_rep=no_rep)
    assert np.array_equal(oracle.decode(arc), data)
    acx.archive_check(arc)
    nb = (data.size + BLOCK - 1) // BLOCK
    lv = np.zeros(data.size, np.int64)
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        want = []
        for cmd, dst, src, ml in zip(t["cmd"].tolist(), t["dst"].tolist(), t["src"].tolist(), t["ml"].tolist()):
            if cmd == 5:
                want.append(0)
                continue
            mx = int(lv[src:src + min(dst - src, ml)].max())
            level = 0 if (src >= b * BLOCK and mx == 0) else min(mx + 1, 255)
            lv[dst:dst + ml] = level
            want.append(level)
        assert oracle.block_levels(arc, b).tolist() == want, b
        for s in range(4):
            assert np.array_equal(oracle.block_stream(arc, b, s), oracle.block_stream(arc0, b, s))


def test_host_checks_accept_level_bodies_and_reject_short_ones(acx):
    from fmt_writer import build_archive as build
    blk0 = [{"cmd": 0, "lits": b"ABCDEFGH", "ml": 8, "src": 0},
            {"cmd": 5, "lits": b"x" * (BLOCK - 16), "ml": 0}]
    blk1 = [{"cmd": 0, "lits": b"", "ml": 12, "src": 3}, {"cmd": 5, "lits": b"!", "ml": 0}]
    good = build([blk0, blk1], levels=[[0, 0], [1, 0]])
    assert acx.archive_check(good)["n_blocks"] == 2
    bad = bytearray(good)
    e = int.from_bytes(bad[40:48], "little") + 40
    plen = int.from_bytes(bad[e + 8:e + 12], "little")
    bad[e + 8:e + 12] = (plen - 16).to_bytes(4, "little")
    with pytest.raises(acx.AceapexError):
        acx.archive_check(bytes(bad))


def _levels_from_parse(arc, nb, size):
    lv = np.zeros(max(size, 1), np.int64)
    out = []
    for b in range(nb):
        t = oracle.parse_block(arc, b)
        want = []
        for cmd, dst, src, ml in zip(t["cmd"].tolist(), t["dst"].tolist(), t["src"].tolist(), t["ml"].tolist()):
            if cmd == 5:
                want.append(0)
                continue
            mx = int(lv[src:src + min(dst - src, ml)].max())
            level = 0 if (src >= b * BLOCK and mx == 0) else min(mx + 1, 255)
            lv[dst:dst + ml] = level
            want.append(level)
        out.append(want)
    return out


def test_randomized_encoder_options_round_trip(acx):
    """Random inputs (random bytes, long repeats, DNA, text, their mixtures;
    0 to 200 KB) under random encoder options: each archive passes the
    library's host checks, decodes to its input in the oracle, and when it
    carries levels they are the levels of its own parse."""
    rng = np.random.default_rng(2024)
    for it in range(150):
        n = int(rng.choice([0, 1, 17, 4095, 16384, 16385, int(rng.integers(1, 200_000))]))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            data = rng.integers(0, 256, n, dtype=np.uint8)
        elif kind == 1:
            unit = rng.integers(0, 256, int(rng.integers(1, 40)), dtype=np.uint8)
            data = np.resize(unit, n).astype(np.uint8)
        elif kind == 2:
            data = synth.dna(n, int(rng.integers(0, 1000))) if n else np.zeros(0, np.uint8)
        else:
            data = synth.text(n, int(rng.integers(0, 1000))) if n else np.zeros(0, np.uint8)
        opts = {"no_rep": bool(rng.integers(0, 2)), "levels": bool(rng.integers(0, 2)),
                "max_depth": int(rng.choice([0, 1, 2, 5, 0xFFFFFFFF])),
                "max_lanes": int(rng.choice([1, 4, 32, 128])), "deps": bool(rng.integers(0, 2)),
                "segment": int(rng.choice([0, 16384, 65536]))}
        arc = acx.encode(data, **opts)
        acx.archive_check(arc)
        assert np.array_equal(oracle.decode(arc), data), (it, n, kind, opts)
        if opts["levels"] and n:
            nb = (n + BLOCK - 1) // BLOCK
            want = _levels_from_parse(arc, nb, n)
            for b in range(nb):
                assert oracle.block_levels(arc, b).tolist() == want[b], (it, b, opts)


def _lanes_for(rn, per_lane, cap=32):
    k = 1
    while 2 * k <= cap and per_lane * 2 * k <= rn:
        k *= 2
    return k


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_encoder_lane_counts_follow_the_stream_lengths(acx, kind):
    """rANS lanes per stream: the most (a power of two up to the cap) that
    leave 64 symbols a lane; the three short streams take 16 symbols a lane
    when their lanes then fit one warp together.  Read back from the block
    descriptors of the archive."""
    import struct
    data = synth.corpus(kind, (2 << 20) + 77, 23)
    arc = acx.encode(data)
    nb = struct.unpack_from("<I", arc, 24)[0]
    off_idx = struct.unpack_from("<Q", arc, 40)[0]
    packed = 0
    for b in range(nb):
        poff = struct.unpack_from("<Q", arc, off_idx + 40 * b)[0]
        desc = [struct.unpack_from("<IIBB", arc, poff + 12 * s) for s in range(4)]
        raw = [d[0] for d in desc]
        want = [_lanes_for(r, 64) for r in raw]
        short = [_lanes_for(r, 16) for r in raw[:3]]
        if sum(short) <= 32:
            want[:3] = short
            packed += 1
        for s, (sraw, enc, mode, K) in enumerate(desc):
            if mode == 1:
                assert K == want[s], (b, s, sraw, K, want[s])
    # the genome's blocks all take the packed rule; the text's short streams are too long
    assert packed == nb if kind == "dna" else packed < nb
    assert oracle.decode_status(arc, verify=False)[0] == 0
