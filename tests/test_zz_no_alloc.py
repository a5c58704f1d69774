"""The allocation-free entry point (aceapex_decode_noalloc), for callers that
cannot allocate device memory while they decode (inside a CUDA graph
capture, under a framework that owns the device's memory, on paths where an
allocation may stall).  Its output must equal the regular entry point's
(aceapex_decode_all) byte for byte, on two calls in a row, since the two calls
share one static scratch array.  Collected last so that a failure here cannot
stop the rest of the GPU suite.  (-m gpu)"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    acx.load()
    return acx


def _regular(acx, ctx, arc_h, d_arc, total):
    import torch
    A = acx.Archive(ctx, d_arc.data_ptr(), arc_h, arc_h.size)
    out = torch.zeros(total, dtype=torch.uint8, device="cuda")
    rc = acx.decode_all(ctx, A, out.data_ptr(), total, torch.cuda.current_stream().cuda_stream)
    A.close()
    assert rc == 0, ctx.last_error()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind,no_rep,levels", [("dna", False, False), ("text", False, False), ("dna", True, False),
                                                ("text", False, True)])
def test_noalloc_matches_decode_all_twice(acx, kind, no_rep, levels):
    import torch
    data = synth.corpus(kind, (1 << 20) - 777, 21)  # 64 blocks, ragged last block
    arc = acx.encode(data, no_rep=no_rep, levels=levels)
    arc_h = np.frombuffer(arc, dtype=np.uint8).copy()
    d_arc = torch.from_numpy(arc_h).cuda()
    ctx = acx.Context(0)
    ref = _regular(acx, ctx, arc_h, d_arc, data.size)
    assert np.array_equal(ref, data)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full((data.size,), 0x5A, dtype=torch.uint8, device="cuda")
        rc = acx.lib.decode_noalloc(d_arc.data_ptr(), arc_h.size, out.data_ptr(), data.size, stream)
        assert rc == 0
        assert np.array_equal(out.cpu().numpy(), ref)
    ctx.close()


def test_noalloc_rejects_archives_beyond_its_limit(acx):
    import torch
    data = synth.dna(65 * 16384, 3)  # 65 blocks: one more than the static scratch holds
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
