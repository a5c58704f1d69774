"""Range decodes (aceapex_decode_range) against the oracle: any region of an
archive, decoded through its block-dependency closure only, equals the same
bytes of the oracle's full decode; the closure is exactly the blocks reachable
through the archive's dependency lists; a list that misses a block read is
reported corrupt.  (-m gpu)"""
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


def closure_size(arc, b0, b1):
    """Blocks reachable from [b0, b1] through the dependency lists (read from
    the archive bytes), or b1 + 1 without lists."""
    import struct
    nb = struct.unpack_from("<I", arc, 24)[0]
    off_idx, off_deps = struct.unpack_from("<QQ", arc, 40)
    if off_deps == 0:
        return b1 + 1
    seen, todo = set(range(b0, b1 + 1)), list(range(b0, b1 + 1))
    while todo:
        b = todo.pop()
        dep_off, n_deps = struct.unpack_from("<II", arc, off_idx + 40 * b + 20)
        for k in range(n_deps):
            d = struct.unpack_from("<I", arc, off_deps + 4 * (dep_off + k))[0]
            if d not in seen:
                seen.add(d)
                todo.append(d)
    assert max(seen) < nb
    return len(seen)


class Opened:
    def __init__(self, acx, ctx, arc):
        import torch
        self.torch = torch
        h = np.frombuffer(arc, np.uint8).copy()
        self.d = torch.from_numpy(h).to("cuda")
        self.A = acx.Archive(ctx, self.d.data_ptr(), h, h.size)

    def close(self):
        self.A.close()


def ranges(total, seed, n=24):
    """Edge regions plus lognormal-length regions at uniform starts."""
    rng = np.random.default_rng(seed)
    out = [(0, 1), (0, total), (total - 1, 1), (BLOCK - 3, 7), (BLOCK, BLOCK), (total // 2, 1),
           ((total // BLOCK) * BLOCK, total - (total // BLOCK) * BLOCK)]
    for _ in range(n):
        ln = int(np.clip(rng.lognormal(np.log(16384), 1.0), 1, 1 << 20))
        ln = min(ln, total)
        st = int(rng.integers(0, total - ln + 1))
        out.append((st, ln))
    return [(s, l) for s, l in out if l > 0]


@pytest.mark.parametrize("kind,no_rep", [("dna", False), ("dna", True), ("text", False)])
def test_byte_level_closure_ranges_match_oracle(acx, ctx, kind, no_rep):
    """With a match index the range decode follows byte-level chains only:
    every region still equals the oracle's bytes, never touches more blocks
    than its block-level closure, and on the genome far fewer (on Zipf text,
    whose words are copied from anywhere in the short window, the two are
    close)."""
    data = synth.corpus(kind, (6 << 20) + 999, 13)
    arc = acx.encode(data, no_rep=no_rep, deps=True)
    ref = oracle.decode(arc)
    op = Opened(acx, ctx, arc)
    op.A.build_index()
    torch = op.torch
    stream = torch.cuda.current_stream().cuda_stream
    touched, block_level = [], []
    for s, ln in ranges(len(data), 9, n=40):
        out = torch.full((ln + 32,), 0x5A, dtype=torch.uint8, device="cuda")
        rc, st = acx.decode_range(ctx, op.A, s, ln, out.data_ptr(), stream, stats=True)
        assert rc == 0, (s, ln, ctx.last_error())
        o = out.cpu().numpy()
        assert np.array_equal(o[:ln], ref[s:s + ln]), (s, ln)
        assert np.all(o[ln:] == 0x5A)
        if ln <= 32768 and s > len(data) // 2:
            touched.append(st["blocks"])
            block_level.append(closure_size(arc, s // BLOCK, (s + ln - 1) // BLOCK))
    assert touched and all(t <= b for t, b in zip(touched, block_level))
    if kind == "dna":  # copies of a few bytes each: chains stay narrow
        assert np.mean(touched) < 0.5 * np.mean(block_level), (touched, block_level)
    op.close()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("deps", [True, False])
@pytest.mark.parametrize("kind,no_rep", [("dna", False), ("dna", True), ("text", False)])
def test_ranges_match_oracle(acx, ctx, kind, no_rep, deps, variant):
    data = synth.corpus(kind, (3 << 20) + 4321, 12)
    arc = acx.encode(data, no_rep=no_rep, deps=deps)
    ref = oracle.decode(arc)
    assert np.array_equal(ref, data)
    ctx.set_params(variant=variant, timeout_us=2_000_000)
    try:
        op = Opened(acx, ctx, arc)
        torch = op.torch
        stream = torch.cuda.current_stream().cuda_stream
        for s, ln in ranges(len(data), 5):
            out = torch.full((ln + 32,), 0x5A, dtype=torch.uint8, device="cuda")
            rc, st = acx.decode_range(ctx, op.A, s, ln, out.data_ptr(), stream, stats=True)
            assert rc == 0, (s, ln, ctx.last_error())
            o = out.cpu().numpy()
            assert np.array_equal(o[:ln], ref[s:s + ln]), (s, ln)
            assert np.all(o[ln:] == 0x5A)
            assert st["blocks"] == closure_size(arc, s // BLOCK, (s + ln - 1) // BLOCK)
            assert st["bytes"] == ln
        op.close()
    finally:
        ctx.set_params(variant=0, timeout_us=2_000_000)


def test_range_errors_and_empty(acx, ctx):
    data = synth.dna(100_000, 3)
    op = Opened(acx, ctx, acx.encode(data, deps=True))
    torch = op.torch
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    assert acx.decode_range(ctx, op.A, 0, 0, out.data_ptr()) == 0
    assert acx.decode_range(ctx, op.A, len(data), 0, out.data_ptr()) == 0
    assert acx.decode_range(ctx, op.A, len(data) - 10, 11, out.data_ptr()) == -6
    assert acx.decode_range(ctx, op.A, len(data) + 1, 1, out.data_ptr()) == -6
    # the context still decodes after the refusals
    assert acx.decode_range(ctx, op.A, 5, 40, out.data_ptr()) == 0
    assert out[:40].cpu().numpy().tobytes() == data[5:45].tobytes()
    op.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_incomplete_dependency_list_is_corrupt(acx, ctx, variant):
    """The oracle's rule for dependency lists: a match reading a block its list
    misses makes the archive corrupt; the range decode, which reads only the
    listed closure, and the full decode both report it (and a covering list
    decodes exactly)."""
    rng = np.random.default_rng(21)
    b0 = bytes(rng.integers(0, 256, BLOCK, dtype=np.uint8))
    b1 = bytes(rng.integers(0, 256, BLOCK, dtype=np.uint8))
    blocks = [[{"cmd": 5, "lits": b0, "ml": 0}], [{"cmd": 5, "lits": b1, "ml": 0}],
              [{"cmd": 0, "lits": b"AB", "ml": 50, "src": BLOCK - 10}]]
    good = build_archive(blocks, deps=[[], [], [0, 1]])
    bad = build_archive(blocks, deps=[[], [], [1]])
    ref = oracle.decode(good, verify=False)
    assert oracle.decode_status(bad, verify=False)[0] == oracle.E_CORRUPT
    ctx.set_params(variant=variant, timeout_us=2_000_000)
    try:
        import torch
        out = torch.zeros(BLOCK, dtype=torch.uint8, device="cuda")
        for arc, want in ((good, 0), (bad, -2)):
            op = Opened(acx, ctx, arc)
            rc = acx.decode_range(ctx, op.A, 2 * BLOCK, 52, out.data_ptr())
            assert rc == want, ctx.last_error()
            if want == 0:
                assert np.array_equal(out[:52].cpu().numpy(), ref[2 * BLOCK:])
            op.close()
        from gpu_util import gpu_decode
        assert gpu_decode(ctx, bad, variant)[0] == -2
        assert gpu_decode(ctx, good, variant)[0] == 0
    finally:
        ctx.set_params(variant=0, timeout_us=2_000_000)
