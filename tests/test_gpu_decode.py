"""Parity of the CUDA decode path (through the C ABI) with the CPU oracle.
The bar is bit-exact output.  (-m gpu)"""
import numpy as np
import pytest

import oracle
import synth
from fmt_writer import build_archive
from golden import worked_examples as W

BLOCK = 16384

pytestmark = pytest.mark.gpu

FAST, PLAIN = 0, 1


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


def dec(ctx, arc, variant=FAST):
    from gpu_util import gpu_decode
    return gpu_decode(ctx, arc, variant)


@pytest.mark.parametrize("variant", [FAST, PLAIN])
@pytest.mark.parametrize("ex", W.ARCHIVE_WORKED, ids=lambda e: e["name"])
def test_worked_archives(ctx, ex, variant):
    arc = build_archive(ex["blocks"], expected=ex["expected"], fnv=oracle.fnv1a64)
    rc, out = dec(ctx, arc, variant)
    assert rc == 0, ctx.last_error()
    assert out.tobytes() == ex["expected"]


@pytest.mark.parametrize("variant", [FAST, PLAIN])
def test_periodic_overlap_all_small_periods(ctx, variant):
    rng = np.random.default_rng(4)
    for d in (1, 2, 3, 5, 7, 12, 16, 33):
        for ml in (4, 5, 31, 32, 33, 64, 200):
            lits = bytes(rng.integers(0, 256, d, dtype=np.uint8))
            arc = build_archive([[{"cmd": 0, "lits": lits, "ml": ml, "src": 0}]])
            rc, out = dec(ctx, arc, variant)
            assert rc == 0
            assert out.tobytes() == lits + bytes(lits[k % d] for k in range(ml))


@pytest.mark.parametrize("variant", [FAST, PLAIN])
@pytest.mark.parametrize("no_rep", [False, True])
@pytest.mark.parametrize("kind", ["dna", "text"])
def test_oracle_encoded_small_config(ctx, dna4m, text4m, kind, no_rep, variant):
    data = dna4m if kind == "dna" else text4m
    arc = oracle.encode(data, no_rep=no_rep)
    rc, out = dec(ctx, arc, variant)
    assert rc == 0, ctx.last_error()
    assert np.array_equal(out, oracle.decode(arc))
    assert np.array_equal(out, data)


@pytest.mark.parametrize("lanes", [1, 8, 32, 64, 128])
@pytest.mark.parametrize("no_rep", [False, True])
@pytest.mark.parametrize("kind", ["dna", "text"])
def test_library_encoded_small_config(acx, ctx, dna4m, text4m, kind, no_rep, lanes):
    data = (dna4m if kind == "dna" else text4m)[: (1 << 20) + 12345]
    arc = acx.encode(data, no_rep=no_rep, max_lanes=lanes)
    rc, out = dec(ctx, arc, FAST)
    assert rc == 0, ctx.last_error()
    assert np.array_equal(out, oracle.decode(arc))


@pytest.mark.parametrize("no_rep", [False, True])
@pytest.mark.parametrize("kind", ["dna", "text"])
def test_fused_variant_matches_oracle(acx, dna4m, text4m, kind, no_rep):
    """The fused comparison variant (entropy warps and local groups in one
    kernel) decodes bit-exact against the oracle, with and without lists."""
    from gpu_util import gpu_decode
    data = (dna4m if kind == "dna" else text4m)[: (1 << 20) + 4567]
    ctx = acx.Context(0, variant=acx.lib.VARIANT_FUSED, timeout_us=2_000_000)
    try:
        for arc in (acx.encode(data, no_rep=no_rep), acx.encode(data, no_rep=no_rep, deps=True)):
            rc, out = gpu_decode(ctx, arc, acx.lib.VARIANT_FUSED)
            assert rc == 0, ctx.last_error()
            assert np.array_equal(out, oracle.decode(arc))
    finally:
        ctx.close()


@pytest.mark.parametrize("variant", [FAST, PLAIN])
@pytest.mark.parametrize("kind", ["dna", "text"])
def test_level_bodies_do_not_change_the_decode(acx, ctx, dna4m, text4m, kind, variant):
    """Archives that carry level bodies (flags bit1, one scheduling hint per
    token) decode bit-exact, like the same archive without them."""
    data = (dna4m if kind == "dna" else text4m)[: (1 << 20) + 777]
    arc = acx.encode(data, levels=True)
    want = oracle.decode(arc)
    assert np.array_equal(want, data)
    rc, out = dec(ctx, arc, variant)
    assert rc == 0, ctx.last_error()
    assert np.array_equal(out, want)


def _rewrite_levels(arc, f):
    """The archive with every block's level body replaced by f(levels, block)
    (the level bytes are scheduling hints: the decoded bytes must not change)."""
    import struct
    a = bytearray(arc)
    nb = struct.unpack_from("<I", a, 24)[0]
    off_idx = struct.unpack_from("<Q", a, 40)[0]
    for b in range(nb):
        poff, plen, ntok = struct.unpack_from("<QII", a, off_idx + 40 * b)
        off = 48
        for s_ in range(4):
            enc = struct.unpack_from("<I", a, poff + 12 * s_ + 4)[0]
            off = (off + enc + 15) & ~15
        lv = np.frombuffer(bytes(a[poff + off:poff + off + ntok]), np.uint8)
        a[poff + off:poff + off + ntok] = np.asarray(f(lv, b), np.uint8).tobytes()
    return bytes(a)


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_level_rounds_with_true_and_wrong_hints(acx, dna4m, text4m, kind):
    """Level-ordered cross-block pass (paper, Depth Does Not Govern Latency:
    the waves): pieces are handed out level by level; with hints that are too
    low, zero, too high or random the pieces that are not ready in time go to
    the work lists and the decode is still the oracle's, byte for byte."""
    from gpu_util import gpu_decode
    # 8 MiB: with one local CTA per SM every CTA takes several blocks, so the
    # next block's streams are staged while a block still sorts its pieces
    data = synth.corpus(kind, (8 << 20) + 999, 12)
    arc = acx.encode(data, levels=True, max_depth=0xFFFFFFFF)
    rng = np.random.default_rng(3)
    hints = {"true": lambda lv, b: lv, "lowered": lambda lv, b: np.maximum(lv.astype(int) - 1, 0),
             "zero": lambda lv, b: np.zeros_like(lv), "raised": lambda lv, b: np.minimum(lv.astype(int) + 3, 255),
             "random": lambda lv, b: rng.integers(0, 8, lv.size), "inverted": lambda lv, b: lv.max(initial=0) - lv}
    # an explicit round-0 wait: level order whatever the pieces per lane
    ctx = acx.Context(0, timeout_us=2_000_000, ctas_per_sm=1, wait_ns=20_000)
    try:
        for name, f in hints.items():
            a2 = _rewrite_levels(arc, f)
            want = oracle.decode(a2)
            assert np.array_equal(want, data), name
            rc, out = gpu_decode(ctx, a2)
            assert rc == 0, (name, ctx.last_error())
            assert np.array_equal(out, want), name
        # true hints, pieces waiting without limit: in level order the lowest
        # unfinished piece always has final sources, so the first round
        # finishes every piece (scrambled levels could stall here instead)
        strict = acx.Context(0, timeout_us=500_000, ctas_per_sm=1, wait_ns=0xFFFFFFFF)
        try:
            rc, out, st = gpu_decode(strict, arc, stats=True)
            assert rc == 0, strict.last_error()
            assert np.array_equal(out, data)
            assert st["pending_spans"] > 0 and st["wait_polls"] == 0, st
        finally:
            strict.close()
        # the level bodies ignored: the round-0 hand-out
        ctx.set_params(ignore_levels=True, timeout_us=2_000_000, ctas_per_sm=1)
        rc, out = gpu_decode(ctx, arc)
        assert rc == 0 and np.array_equal(out, data)
    finally:
        ctx.close()



@pytest.mark.parametrize("variant", [FAST, PLAIN])
def test_edge_sizes_and_ragged_tail(acx, ctx, variant):
    from gpu_util import gpu_decode
    rng = np.random.default_rng(7)
    for n in (1, 15, 16, 17, 100, 16383, 16384, 16385, 5 * 16384 + 999):
        data = synth.dna(n, 11) if n > 64 else (rng.integers(0, 4, n, dtype=np.uint8) + 65)
        for arc in (oracle.encode(data), acx.encode(data, no_rep=True)):
            rc, out, tail = gpu_decode(ctx, arc, variant, out_pad=64)
            assert rc == 0, ctx.last_error()
            assert np.array_equal(out, data)
            assert np.all(tail == 0xA5)  # nothing written past the output


def test_all_literal_and_long_runs(acx, ctx):
    rng = np.random.default_rng(1)
    data = rng.integers(0, 256, 200_000, dtype=np.uint8)
    for arc in (oracle.encode(data), acx.encode(data)):
        rc, out = dec(ctx, arc)
        assert rc == 0 and np.array_equal(out, data)
    data = np.frombuffer(b"N" * 100_000 + b"ACGT" * 30_000, dtype=np.uint8)
    for arc in (oracle.encode(data), acx.encode(data), acx.encode(data, no_rep=True)):
        rc, out = dec(ctx, arc)
        assert rc == 0 and np.array_equal(out, data)


def _corrupt_archives():
    yield "offset not before destination", build_archive([[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 4}]])
    yield "repeat distance beyond start", build_archive([[{"cmd": 1, "lits": b"", "ml": 4}]])
    yield "unknown command", build_archive([[{"cmd": 6, "lits": b"ACGT", "ml": 4, "src": 0}]])
    yield "lit-only not last", build_archive([[{"cmd": 5, "lits": b"AC", "ml": 0},
                                               {"cmd": 0, "lits": b"GT", "ml": 4, "src": 0}]])
    yield "short match", build_archive([[{"cmd": 0, "lits": b"ACGT", "ml": 3, "src": 0}]])
    from fmt_writer import leb128
    toks = [[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 0}]]
    yield "4-byte varint", build_archive(toks, raw_streams={0: [bytes([0]), b"\x84\x80\x80\x00" + leb128(4),
                                                                bytes(5), b"ACGT"]})
    yield "trailing length byte", build_archive(toks, raw_streams={0: [bytes([0]), leb128(4) + leb128(4) + b"\x00",
                                                                       bytes(5), b"ACGT"]})


@pytest.mark.parametrize("variant", [FAST, PLAIN])
@pytest.mark.parametrize("name,arc", list(_corrupt_archives()), ids=lambda x: x if isinstance(x, str) else "")
def test_corrupt_token_streams_are_reported(ctx, name, arc, variant):
    assert oracle.decode_status(arc, verify=False)[0] == oracle.E_CORRUPT
    rc, _ = dec(ctx, arc, variant)
    assert rc == -2, (name, rc, ctx.last_error())
    # the context stays usable after an error
    good = build_archive([W.ARCHIVE_WORKED[0]["blocks"][0]])
    rc, out = dec(ctx, good, variant)
    assert rc == 0 and out.tobytes() == W.ARCHIVE_WORKED[0]["expected"]


def test_corrupt_rans_payload_is_reported(acx, ctx, dna4m):
    data = dna4m[:200_000]
    arc = bytearray(acx.encode(data))
    info = oracle.info(bytes(arc))
    rng = np.random.default_rng(5)
    seen_corrupt = 0
    for _ in range(12):
        bad = bytearray(arc)
        # flip a byte inside the payload section (after header/tables/index)
        lo = 64 + 2048 + 40 * info["n_blocks"] + 64
        pos = int(rng.integers(lo, len(bad)))
        bad[pos] ^= 0x5A
        rc_o, ref = oracle.decode_status(bytes(bad), verify=False)
        try:
            rc, out = dec(ctx, bytes(bad))
        except Exception as e:  # structural rejection at open
            assert getattr(e, "status", None) == -2
            continue
        if rc_o == 0:
            assert rc == 0 and np.array_equal(out, ref)
        else:
            assert rc in (-2, 0)
            seen_corrupt += rc == -2
    assert seen_corrupt >= 1


@pytest.mark.slow
def test_full_size_genome_matches_oracle(acx, ctx):
    """The benchmark's workload at its full size (253,935,557 B genome,
    history-bound encoding, fast decoder): every byte equals the oracle's
    decode and the generator's input."""
    data = synth.dna(synth.GENOME_CHR1_SIZE, 0)
    arc = acx.encode(data)
    rc, out = dec(ctx, arc, FAST)
    assert rc == 0, ctx.last_error()
    assert np.array_equal(out, data)
    ref = oracle.decode(arc)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_cross_block_policies_depths_and_launch_shapes(acx, dna4m, text4m, kind):
    """The cross-block pass under every round-0 policy (wait without limit,
    defer at once, the automatic choice), on archives with deep uncapped
    chains, a cap of 1, and independent segments, and the decode under
    small launch shapes: every combination decodes bit-exact."""
    from gpu_util import gpu_decode
    data = (dna4m if kind == "dna" else text4m)[: (2 << 20) + 4321]
    archives = {"no cap": acx.encode(data, max_depth=0xFFFFFFFF), "cap 1": acx.encode(data, max_depth=1),
                "segments": acx.encode(data, segment=1 << 18), "levels": acx.encode(data, levels=True)}
    want = {name: oracle.decode(arc) for name, arc in archives.items()}
    for name in archives:
        assert np.array_equal(want[name], data), name
    shapes = [dict(wait_ns=0xFFFFFFFF), dict(wait_ns=1), dict(wait_ns=0),
              dict(ctas_per_sm=1, rans_ctas_per_sm=1, queue_chunk=4)]
    for shape in shapes:
        ctx = acx.Context(0, timeout_us=2_000_000, **shape)
        try:
            for name, arc in archives.items():
                rc, out = gpu_decode(ctx, arc)  # the context's own parameters (fast decoder)
                assert rc == 0, (name, shape, ctx.last_error())
                assert np.array_equal(out, want[name]), (name, shape)
        finally:
            ctx.close()


def _local_pieces(arc, n_blocks):
    """Pending pieces left by a local pass that resolves every in-block match
    it can: per block (from the oracle's parse), the matches whose source
    precedes the block are pending; an in-block match is resolved once every
    byte of its source window [src, src + min(distance, length)) is final
    (a literal, or a byte of a resolved match), repeated to a fixed point;
    the rest leave ceil(length / 32) pieces each."""
    total = 0
    for b in range(n_blocks):
        t = oracle.parse_block(arc, b)
        B = b * BLOCK
        ml, dst, src = t["ml"].astype(np.int64), t["dst"].astype(np.int64), t["src"].astype(np.int64)
        final = np.ones(BLOCK, bool)
        todo = []
        for k in range(len(ml)):
            if ml[k] == 0:
                continue
            o = dst[k] - B
            final[o:o + ml[k]] = False
            if src[k] < B:
                total += (ml[k] + 31) // 32
            else:
                todo.append(k)
        while todo:
            rest = []
            for k in todo:
                so, d = src[k] - B, dst[k] - src[k]
                if final[so:so + min(d, ml[k])].all():
                    o = dst[k] - B
                    final[o:o + ml[k]] = True
                else:
                    rest.append(k)
            if len(rest) == len(todo):
                break
            todo = rest
        total += sum((ml[k] + 31) // 32 for k in todo)
    return total


@pytest.mark.parametrize("kind", ["dna", "text"])
def test_local_pass_resolves_every_in_block_chain(acx, ctx, kind):
    """The local pass finishes every in-block match whose chain of sources
    stays in the block (periodic fills in rounds, "What Does: Periods, Not
    Chains"); only the rest reach the cross-block pass.  The pending-piece
    count of the decode equals the count from the oracle's parse, on every
    run (the rounds must not end early)."""
    from gpu_util import gpu_decode
    data = synth.corpus(kind, (2 << 20) + 333, 17)
    arc = acx.encode(data)
    nb = (data.size + BLOCK - 1) // BLOCK
    want = _local_pieces(arc, nb)
    assert want > 0
    for _ in range(3):
        rc, out, st = gpu_decode(ctx, arc, stats=True)
        assert rc == 0 and np.array_equal(out, data)
        assert st["pending_spans"] == want, (st["pending_spans"], want)
