"""The region server (aceapex_server_*) against the oracle: every request's
bytes equal the oracle's decode of that region, whether the request runs
alone or mixed into ticks with many others (continuous batching), with a
cache small enough to force evictions and re-decodes; admission refuses what
can never fit.  (-m gpu)"""
import numpy as np
import pytest

import oracle
import synth

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


@pytest.fixture(scope="module", params=[("dna", False), ("text", True)], ids=["dna-history", "text-nohist"])
def served(request, acx, ctx):
    import torch
    kind, no_rep = request.param
    data = synth.corpus(kind, (8 << 20) + 12345, 31)
    arc = acx.encode(data, no_rep=no_rep)
    ref = oracle.decode(arc)
    assert np.array_equal(ref, data)
    h = np.frombuffer(arc, np.uint8).copy()
    d = torch.from_numpy(h).to("cuda")
    A = acx.Archive(ctx, d.data_ptr(), h, h.size)
    # caches below the archive size, so evictions happen; text closures are
    # wide (Zipf words are copied from anywhere), so text gets more slots
    cache_blocks = 192 if kind == "dna" else 500
    yield ref, A, cache_blocks
    A.close()
    del d


def workload(total, n, seed):
    """Request regions: lengths lognormal (median 16 KiB, sigma 1) clipped to
    [1 B, 256 KiB], starts uniform, plus edge regions."""
    rng = np.random.default_rng(seed)
    lens = np.clip(rng.lognormal(np.log(16384), 1.0, n), 1, 256 << 10).astype(np.int64)
    starts = np.array([rng.integers(0, total - l + 1) for l in lens], dtype=np.int64)
    edge = [(0, 1), (total - 1, 1), (BLOCK - 5, 10), (0, 3 * BLOCK + 7), (total - BLOCK - 3, BLOCK + 3)]
    starts = np.concatenate([starts, [s for s, _ in edge]])
    lens = np.concatenate([lens, [l for _, l in edge]])
    return starts.astype(np.uint64), lens.astype(np.uint64)


class Arena:
    def __init__(self, lens):
        import torch
        self.off = np.concatenate([[0], np.cumsum(lens.astype(np.int64) + 64)])
        self.buf = torch.full((int(self.off[-1]),), 0xA5, dtype=torch.uint8, device="cuda")
        self.lens = lens

    def ptrs(self):
        return (self.buf.data_ptr() + self.off[:-1]).astype(np.uint64)

    def get(self, i):
        o = int(self.off[i])
        return self.buf[o:o + int(self.lens[i]) + 64].cpu().numpy()


def check_all(ref, starts, lens, arena):
    whole = arena.buf.cpu().numpy()
    for i in range(len(starts)):
        o, s, l = int(arena.off[i]), int(starts[i]), int(lens[i])
        assert np.array_equal(whole[o:o + l], ref[s:s + l]), (i, s, l)
        assert np.all(whole[o + l:o + l + 64] == 0xA5), i
    return whole


def test_alone_and_mixed_give_the_oracle_bytes(acx, ctx, served):
    """Each request alone (one tick each, drained before the next), then the
    same requests all at once, then with staggered open-loop arrivals: every
    result equals the oracle's bytes, so a request's result does not depend
    on what shares its tick or what the cache holds."""
    ref, A, cache_blocks = served
    starts, lens = workload(len(ref), 120, 7)
    alone = Arena(lens)
    srv = acx.Server(ctx, A, cache_bytes=cache_blocks * BLOCK)
    ptrs = alone.ptrs()
    for i in range(len(starts)):
        srv.submit(int(starts[i]), int(lens[i]), int(ptrs[i]))
        assert srv.drain(30000) == 0, srv.last_error()
    got = srv.poll(100000)
    assert len(got) == len(starts) and all(c["status"] == 0 for c in got)
    st_alone = srv.stats()
    assert st_alone["completed"] == len(starts) and st_alone["ticks"] == len(starts)
    assert st_alone["blocks_decoded"] > cache_blocks  # blocks were evicted and decoded again
    whole_alone = check_all(ref, starts, lens, alone)
    srv.close()

    burst = Arena(lens)
    srv = acx.Server(ctx, A, cache_bytes=cache_blocks * BLOCK)
    srv.submit_many(starts, lens, burst.ptrs())
    assert srv.drain(60000) == 0, srv.last_error()
    got = srv.poll(100000)
    assert all(c["status"] == 0 for c in got), [c for c in got if c["status"]][:3]
    st = srv.stats()
    assert st["ticks"] < len(starts)  # requests shared ticks
    whole_burst = check_all(ref, starts, lens, burst)
    assert np.array_equal(whole_alone, whole_burst)

    # staggered arrivals on the same (now warm) server: hits and re-decodes mix
    stag = Arena(lens)
    t0 = srv.now_ns() + 2_000_000
    at = t0 + np.arange(len(starts), dtype=np.int64) * 30_000
    srv.submit_many(starts, lens, stag.ptrs(), at)
    assert srv.drain(60000) == 0, srv.last_error()
    got = srv.poll(100000)
    assert len(got) == len(starts) and all(c["status"] == 0 for c in got)
    assert all(c["latency_us"] > 0 for c in got)
    st2 = srv.stats()
    assert st2["blocks_hit"] > 0 and st2["p50_us"] <= st2["p99_us"]
    check_all(ref, starts, lens, stag)
    srv.close()


def test_admission_refuses_what_can_never_fit(acx, ctx, served):
    ref, A, _ = served
    import torch
    srv = acx.Server(ctx, A, cache_bytes=4 * BLOCK)  # four slots
    out = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    big = srv.submit(0, 1 << 20, out.data_ptr())       # 64 blocks: can never fit
    small = srv.submit(100, 50, out.data_ptr() + (1 << 19))
    assert srv.drain(30000) == 0
    by_id = {c["id"]: c for c in srv.poll(10)}
    assert by_id[big]["status"] == -7
    assert by_id[small]["status"] == 0
    assert np.array_equal(out[(1 << 19):(1 << 19) + 50].cpu().numpy(), ref[100:150])
    with pytest.raises(acx.AceapexError):
        srv.submit(len(ref) - 5, 10, out.data_ptr())
    srv.close()


@pytest.fixture(scope="module")
def segmented(acx, ctx):
    """An 8 MiB genome encoded in 1 MiB segments (every source inside its
    segment), so that requests in different segments have disjoint closures."""
    import torch
    data = synth.dna((8 << 20) + 777, 41)
    arc = acx.encode(data, segment=1 << 20)
    ref = oracle.decode(arc)
    assert np.array_equal(ref, data)
    h = np.frombuffer(arc, np.uint8).copy()
    d = torch.from_numpy(h).to("cuda")
    A = acx.Archive(ctx, d.data_ptr(), h, h.size)
    yield ref, A
    A.close()
    del d


def _one_per_tick(acx, ctx, A, ref, starts, lens, streams, cache_blocks):
    arena = Arena(lens)
    srv = acx.Server(ctx, A, cache_bytes=cache_blocks * BLOCK, max_tick_requests=1, streams=streams)
    srv.submit_many(starts, lens, arena.ptrs())
    assert srv.drain(60000) == 0, srv.last_error()
    got = srv.poll(100000)
    assert len(got) == len(starts) and all(c["status"] == 0 for c in got)
    st = srv.stats()
    srv.close()
    check_all(ref, starts, lens, arena)
    return st


def test_ticks_on_two_lanes_overlap_on_the_device(acx, ctx, segmented):
    """A burst of one-request ticks that alternate between segments: ticks
    on the two lanes have disjoint closures, so they run side by side (their
    device intervals overlap) and none waits for another; every request
    equals the oracle's bytes.  One lane never overlaps two ticks."""
    ref, A = segmented
    rng = np.random.default_rng(5)
    seg = 1 << 20
    n = 48
    starts = np.array([(i % 8) * seg + rng.integers(0, seg - 40000) for i in range(n)], dtype=np.uint64)
    lens = rng.integers(4096, 32768, n).astype(np.uint64)
    st2 = _one_per_tick(acx, ctx, A, ref, starts, lens, 2, 600)
    assert st2["ticks"] == n
    assert st2["tick_overlaps"] > 0, st2
    st1 = _one_per_tick(acx, ctx, A, ref, starts, lens, 1, 600)
    assert st1["tick_overlaps"] == 0 and st1["tick_waits"] == 0, st1


def test_ticks_that_share_blocks_are_ordered(acx, ctx, segmented):
    """One-request ticks on four lanes over one segment, with a cache small
    enough to evict and decode blocks again: ticks that read blocks another
    unfinished tick decodes (or decode blocks it reads) wait for it, and
    every request still equals the oracle's bytes."""
    ref, A = segmented
    rng = np.random.default_rng(6)
    seg = 1 << 20
    n = 64
    starts = (3 * seg + rng.integers(0, seg - 40000, n)).astype(np.uint64)
    lens = rng.integers(1, 40000, n).astype(np.uint64)
    st = _one_per_tick(acx, ctx, A, ref, starts, lens, 4, 96)
    assert st["ticks"] == n and st["tick_waits"] > 0, st
