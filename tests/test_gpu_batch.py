"""Batched decode (aceapex_batch_*) against the oracle: many archives of
mixed sizes, corpora and encodings decoded by one set of launches (plain or
graph-replayed) must give, archive by archive, exactly the oracle's bytes, the
same as one decode per archive; a corrupt archive fails alone.  (-m gpu)"""
import numpy as np
import pytest

import oracle
import synth
from fmt_writer import build_archive
from golden import worked_examples as W

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


def mixed_archives(acx, n=14, seed=4, lo=1 << 10, hi=3 << 20):
    """A small copy of the mixed batch workload: log-uniform sizes, DNA for
    even i and text for odd i, history-free for i mod 4 in {2, 3}, rANS lane
    caps cycling through 1..128, plus an empty and a one-byte archive."""
    specs = synth.batch_specs(n, seed, lo, hi)
    out = []
    for s in specs:
        data = synth.corpus(s["kind"], s["size"], s["seed"])
        lanes = (1, 8, 32, 64, 128)[s["index"] % 5]
        arc = acx.encode(data, no_rep=s["no_rep"], max_lanes=lanes)
        out.append((data, arc))
    out.append((np.zeros(0, np.uint8), acx.encode(np.zeros(0, np.uint8))))
    one = np.frombuffer(b"G", np.uint8).copy()
    out.append((one, oracle.encode(one)))
    return out


class Opened:
    """Archives in device memory, opened on ctx, with poisoned outputs (64
    guard bytes past each output)."""

    def __init__(self, acx, ctx, arcs):
        import torch
        self.torch = torch
        self.d_arcs, self.archives, self.outs = [], [], []
        for a in arcs:
            h = np.frombuffer(a, np.uint8).copy()
            d = torch.from_numpy(h).to("cuda") if h.size else torch.empty(16, dtype=torch.uint8, device="cuda")
            self.d_arcs.append(d)
            A = acx.Archive(ctx, d.data_ptr(), h, h.size)
            self.archives.append(A)
            self.outs.append(torch.full((A.total + 64,), 0xA5, dtype=torch.uint8, device="cuda"))

    def entries(self):
        return [(A, o.data_ptr(), A.total) for A, o in zip(self.archives, self.outs)]

    def poison(self):
        for o in self.outs:
            o.fill_(0xA5)

    def result(self, i):
        A = self.archives[i]
        o = self.outs[i].cpu().numpy()
        return o[:A.total], o[A.total:]

    def close(self):
        for A in self.archives:
            A.close()


@pytest.fixture(scope="module")
def mixed(acx):
    return mixed_archives(acx)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("variant", [FAST, PLAIN])
def test_mixed_batch_matches_oracle(acx, ctx, mixed, graph, variant):
    ctx.set_params(variant=variant, timeout_us=2_000_000)
    try:
        op = Opened(acx, ctx, [a for _, a in mixed])
        b = acx.Batch(ctx, op.entries(), graph=graph)
        stream = op.torch.cuda.current_stream().cuda_stream
        for rep in range(2):  # the second run replays the same batch (graph replay when graph=True)
            op.poison()
            rc, per, st = b.run(stream, stats=True)
            assert rc == 0, ctx.last_error()
            assert per == [0] * len(mixed)
            assert st["bytes"] == sum(len(d) for d, _ in mixed)
            assert st["blocks"] == sum(oracle.info(a)["n_blocks"] for _, a in mixed)
            for i, (data, arc) in enumerate(mixed):
                out, tail = op.result(i)
                assert np.array_equal(out, data), (rep, i)
                assert np.all(tail == 0xA5), (rep, i)
        for i in range(0, len(mixed), 3):  # the oracle's bytes, on a sample
            assert np.array_equal(op.result(i)[0], oracle.decode(mixed[i][1]))
        b.close()
        op.close()
    finally:
        ctx.set_params(variant=FAST, timeout_us=2_000_000)


def test_batch_equals_per_archive_decodes(acx, ctx, mixed):
    from gpu_util import gpu_decode
    op = Opened(acx, ctx, [a for _, a in mixed])
    rc, per = acx.batch_decode(ctx, op.entries(), op.torch.cuda.current_stream().cuda_stream)
    assert rc == 0 and per == [0] * len(mixed), ctx.last_error()
    for i, (_, arc) in enumerate(mixed):
        rc1, one = gpu_decode(ctx, arc)
        assert rc1 == 0
        assert np.array_equal(op.result(i)[0], one)
    op.close()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("variant", [FAST, PLAIN])
def test_corrupt_archive_fails_alone(acx, ctx, mixed, graph, variant):
    """Paper, Setup: a block is decodable once its sources exist, archive by
    archive; an archive whose tokens violate the format reports
    ACEAPEX_E_CORRUPT in its own status while every other archive of the
    batch decodes exactly (twice in a row, so the status words reset)."""
    bad = [
        build_archive([[{"cmd": 0, "lits": b"ACGT", "ml": 4, "src": 4}]]),   # source not before destination
        build_archive([[{"cmd": 6, "lits": b"ACGT", "ml": 4, "src": 0}]]),   # unknown command
    ]
    for a in bad:
        assert oracle.decode_status(a, verify=False)[0] == oracle.E_CORRUPT
    ctx.set_params(variant=variant, timeout_us=2_000_000)
    try:
        arcs = [a for _, a in mixed[:6]] + [bad[0]] + [a for _, a in mixed[6:10]] + [bad[1]]
        datas = [d for d, _ in mixed[:6]] + [None] + [d for d, _ in mixed[6:10]] + [None]
        op = Opened(acx, ctx, arcs)
        b = acx.Batch(ctx, op.entries(), graph=graph)
        stream = op.torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            op.poison()
            rc, per = b.run(stream)
            assert rc == -2
            for i, d in enumerate(datas):
                if d is None:
                    assert per[i] == -2
                else:
                    assert per[i] == 0, (i, per)
                    assert np.array_equal(op.result(i)[0], d)
        b.close()
        # a batch of only good archives on the same context still decodes
        good = build_archive([W.ARCHIVE_WORKED[0]["blocks"][0]])
        op2 = Opened(acx, ctx, [good])
        rc, per = acx.batch_decode(ctx, op2.entries(), stream)
        assert rc == 0 and per == [0]
        assert op2.result(0)[0].tobytes() == W.ARCHIVE_WORKED[0]["expected"]
        op.close()
        op2.close()
    finally:
        ctx.set_params(variant=FAST, timeout_us=2_000_000)


def test_empty_batch_and_argument_errors(acx, ctx):
    rc, per = acx.batch_decode(ctx, [], 0)
    assert rc == 0 and per == []
    op = Opened(acx, ctx, [oracle.encode(synth.dna(40_000, 2))])
    A, d_out, cap = op.entries()[0]
    with pytest.raises(acx.AceapexError) as e:
        acx.Batch(ctx, [(A, d_out, cap - 1)])
    assert e.value.status == -1
    op.close()


@pytest.mark.slow
def test_full_batch_workload(acx, ctx):
    """The 96-archive batch workload at full size (log-uniform 64 KiB..64 MiB,
    DNA/text, mixed encodings), one graph-replayed batch: every archive equals
    its generator input, and a sample equals the oracle's decode."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch
    specs = synth.batch_specs()

    def one(s):  # the encoder releases the GIL: archives encode in parallel
        d = synth.corpus(s["kind"], s["size"], s["seed"])
        return d, acx.encode(d, no_rep=s["no_rep"], threads=1)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, specs))
    datas, arcs = [r[0] for r in res], [r[1] for r in res]
    op = Opened(acx, ctx, arcs)
    b = acx.Batch(ctx, op.entries(), graph=True)
    rc, per = b.run(torch.cuda.current_stream().cuda_stream)
    assert rc == 0 and per == [0] * len(specs), ctx.last_error()
    for i, d in enumerate(datas):
        assert np.array_equal(op.result(i)[0], d), i
    small = sorted(range(len(specs)), key=lambda i: specs[i]["size"])[:8]
    for i in small:
        assert np.array_equal(op.result(i)[0], oracle.decode(arcs[i]))
    b.close()
    op.close()


def test_autotune_picks_a_measured_point_and_keeps_parity(acx, ctx, mixed, tmp_path):
    """aceapex_autotune times the batch over the launch space and leaves the
    context on the fastest measured point; decoding with it stays exact, and
    the JSON cache returns the same point without measuring again."""
    op = Opened(acx, ctx, [a for _, a in mixed])
    best, points = acx.autotune(ctx, op.entries(), reps=2)
    assert points and min(p["ms"] for p in points) == min(
        p["ms"] for p in points if (p["ctas_per_sm"], p["rans_ctas_per_sm"], p["queue_chunk"]) ==
        (best["ctas_per_sm"], best["rans_ctas_per_sm"], best["queue_chunk"]))
    assert {p["queue_chunk"] for p in points} == {1, 4, 16}
    op.poison()
    b = acx.Batch(ctx, op.entries(), graph=True)
    rc, per = b.run(op.torch.cuda.current_stream().cuda_stream)
    assert rc == 0 and per == [0] * len(mixed)
    for i, (data, _) in enumerate(mixed):
        assert np.array_equal(op.result(i)[0], data)
    b.close()
    path = str(tmp_path / "tune.json")
    first = acx.tune.tuned_params(ctx, op.entries(), "mixed-small", path, reps=1)
    again = acx.tune.tuned_params(ctx, op.entries(), "mixed-small", path)
    assert again["cached"] and not first["cached"]
    assert all(first[k] == again[k] for k in ("ctas_per_sm", "rans_ctas_per_sm", "queue_chunk"))
    ctx.set_params(variant=FAST, timeout_us=2_000_000)
    op.close()
