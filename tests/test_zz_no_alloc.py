"""The allocation-free entry point (aceapex_decode_noalloc).  (-m gpu)

It serves callers that may not allocate device memory while they decode:
processes whose device memory was handed to a framework's pool at start-up,
and latency-bound paths where an allocation can stall or fail.  All of its
scratch is one static device array, so its output must equal the CPU oracle's
and the regular entry point's (aceapex_decode_all) byte for byte on two calls
in a row, although the second call finds the first call's leftovers in that
array.  It must also agree with the regular entry point on which archives are
corrupt, since it plans the archive on the device with its own checks.  The
call synchronises its stream, so it is not meant for graph capture.  The file
is collected last so that a failure here cannot stop the rest of the GPU
suite.
"""
import struct

import numpy as np
import pytest

import oracle
import synth
from fmt_writer import inflate_literal_stream

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


def _regular(acx, ctx, arc_h, d_arc, cap):
    """Status and output of the regular path (archive_open + decode_all)."""
    import torch
    try:
        A = acx.Archive(ctx, d_arc.data_ptr(), arc_h, arc_h.size)
    except acx.AceapexError as e:
        return e.status, None
    out = torch.zeros(max(cap, 1), dtype=torch.uint8, device="cuda")
    rc = acx.decode_all(ctx, A, out.data_ptr(), cap, torch.cuda.current_stream().cuda_stream)
    total = A.total
    A.close()
    return rc, (out[:total].cpu().numpy() if rc == 0 else None)


def _noalloc(acx, arc_h, d_arc, cap, fill=0x5A):
    import torch
    out = torch.full((max(cap, 1),), fill, dtype=torch.uint8, device="cuda")
    rc = acx.lib.decode_noalloc(d_arc.data_ptr(), arc_h.size, out.data_ptr(), cap,
                                torch.cuda.current_stream().cuda_stream)
    return rc, out.cpu().numpy()


@pytest.mark.parametrize("kind,no_rep,levels,deps", [("dna", False, False, False), ("text", False, False, False),
                                                     ("dna", True, False, False), ("text", False, True, False),
                                                     ("dna", False, False, True)])
def test_noalloc_matches_oracle_and_decode_all_twice(acx, kind, no_rep, levels, deps):
    import torch
    data = synth.corpus(kind, (1 << 20) - 777, 21)  # 64 blocks, ragged last block
    arc = acx.encode(data, no_rep=no_rep, levels=levels, deps=deps)
    want = oracle.decode(arc)
    assert np.array_equal(want, data)
    arc_h = np.frombuffer(arc, dtype=np.uint8).copy()
    d_arc = torch.from_numpy(arc_h).cuda()
    ctx = acx.Context(0)
    rc, ref = _regular(acx, ctx, arc_h, d_arc, data.size)
    assert rc == 0, ctx.last_error()
    assert np.array_equal(ref, want)
    for fill in (0x5A, 0xC3):
        rc, out = _noalloc(acx, arc_h, d_arc, data.size, fill)
        assert rc == 0
        assert np.array_equal(out[:data.size], want)
    ctx.close()


def test_noalloc_rejects_archives_beyond_its_limit(acx):
    import torch
    data = synth.dna(65 * BLOCK, 3)  # 65 blocks: one more than the static scratch holds
    arc_h = np.frombuffer(acx.encode(data), dtype=np.uint8).copy()
    d_arc = torch.from_numpy(arc_h).cuda()
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    rc = acx.lib.decode_noalloc(d_arc.data_ptr(), arc_h.size, out.data_ptr(), data.size,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == acx.lib.E_ARG
    # a too-small output buffer is refused too
    small = synth.dna(4096, 4)
    sh = np.frombuffer(acx.encode(small), dtype=np.uint8).copy()
    ds = torch.from_numpy(sh).cuda()
    rc = acx.lib.decode_noalloc(ds.data_ptr(), sh.size, out.data_ptr(), 100,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == acx.lib.E_ARG


def _corruptions(acx):
    """(name, archive bytes, decoded size) of archives that the oracle finds corrupt."""
    data = synth.dna(40 * BLOCK + 123, 8)
    good = bytearray(acx.encode(data))
    off_tab, off_idx = struct.unpack_from("<QQ", good, 32)
    nb = struct.unpack_from("<I", good, 24)[0]
    out = []
    a = bytearray(good)
    a[0] ^= 1
    out.append(("bad magic", a))
    a = bytearray(good)
    for s in range(4):  # a table that sums to 4096 gains one count
        t = struct.unpack_from("<256H", good, off_tab + 512 * s)
        if sum(t) == 4096:
            k = int(np.argmax(t))
            struct.pack_into("<H", a, off_tab + 512 * s + 2 * k, t[k] + 1)
            break
    out.append(("table sum", a))
    a = bytearray(good)
    poff = struct.unpack_from("<Q", good, off_idx + 40 * 5)[0]
    struct.pack_into("<Q", a, off_idx + 40 * 5, poff + 1)
    out.append(("misaligned payload", a))
    out.append(("truncated index", bytearray(good[:off_idx + 40 * (nb // 2) + 7])))
    a = bytearray(good)
    struct.pack_into("<H", a, 6, struct.unpack_from("<H", good, 6)[0] | 2)  # level bodies that are not there
    out.append(("level body out of bounds", a))
    a = bytearray(good)
    poff, _plen, ntok = struct.unpack_from("<QII", good, off_idx + 40 * 9)
    enc = struct.unpack_from("<I", good, poff + 4)[0]
    for j in range(max(1, enc // 2), min(enc, enc // 2 + 8)):  # scramble block 9's command stream
        a[poff + 48 + j] ^= 0xA7
    out.append(("command stream", a))
    out.append(("literal stream longer than the block", bytearray(inflate_literal_stream(bytes(good)))))
    # an archive with dependency lists, one of which misses a block that its matches read
    dl = bytearray(acx.encode(data, deps=True))
    idx2 = struct.unpack_from("<Q", dl, 40)[0]
    for b in range(nb):
        if struct.unpack_from("<I", dl, idx2 + 40 * b + 24)[0] == 0:
            continue
        a = bytearray(dl)
        struct.pack_into("<I", a, idx2 + 40 * b + 24, 0)
        if oracle.decode_status(bytes(a), verify=False)[0] == oracle.E_CORRUPT:
            out.append(("dependency list", a))
            break
    else:
        raise AssertionError("no block with a needed dependency list")
    return [(n, bytes(a), data.size) for n, a in out]


def test_noalloc_agrees_with_decode_all_on_corrupt_archives(acx):
    import torch
    ctx = acx.Context(0)
    names = []
    for name, arc, size in _corruptions(acx):
        assert oracle.decode_status(arc, verify=False)[0] == oracle.E_CORRUPT, name
        arc_h = np.frombuffer(arc, dtype=np.uint8).copy()
        d_arc = torch.from_numpy(arc_h).cuda()
        want, _ = _regular(acx, ctx, arc_h, d_arc, size)
        got, _ = _noalloc(acx, arc_h, d_arc, size)
        assert want == acx.lib.E_CORRUPT, (name, want)
        assert got == want, (name, got, want)
        names.append(name)
    assert len(names) == 8
    # a good archive still decodes after the corrupt ones
    data = synth.dna(20 * BLOCK, 9)
    arc_h = np.frombuffer(acx.encode(data), dtype=np.uint8).copy()
    rc, out = _noalloc(acx, arc_h, torch.from_numpy(arc_h).cuda(), data.size)
    assert rc == 0 and np.array_equal(out[:data.size], data)
    ctx.close()
