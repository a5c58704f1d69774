"""End-to-end decode from host memory (aceapex_decode_host), a pipeline over
chunks of blocks (512, 1536, then 4096 each): uploads, chunk decodes and
downloads on three streams.  Archives of one chunk, several chunks and a
ragged last chunk decode to the oracle's bytes, with and without
level-ordered cross-block passes, history and history-free, on an opened
archive and on a temporary one.  (-m gpu)"""
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


@pytest.mark.parametrize("kind,size,kw", [
    ("dna", 6144 * BLOCK + 5 * BLOCK + 123, {}),                      # 4 chunks, ragged last one
    ("text", 2048 * BLOCK + 77, {"levels": True}),                    # 3 chunks, level order
    ("dna", 512 * BLOCK, {"no_rep": True}),                           # exactly one chunk
    ("text", 100_000, {"no_rep": True, "levels": True}),              # less than a chunk
])
def test_host_pipeline_matches_oracle(acx, kind, size, kw):
    import torch
    data = synth.corpus(kind, size, 61)
    arc = acx.encode(data, **kw)
    want = oracle.decode(arc)
    assert np.array_equal(want, data)
    t_arc = torch.from_numpy(np.frombuffer(arc, np.uint8).copy()).pin_memory()
    t_out = torch.full((size,), 0x3C, dtype=torch.uint8).pin_memory()
    h_arc, h_out = t_arc.numpy(), t_out.numpy()
    # a level-ordered cross-block pass whatever the pieces per lane (explicit wait)
    ctx = acx.Context(0, wait_ns=20_000 if kw.get("levels") else 0)
    try:
        d_arc = torch.from_numpy(h_arc.copy()).cuda()
        A = acx.Archive(ctx, d_arc.data_ptr(), h_arc, h_arc.size)
        stream = torch.cuda.current_stream().cuda_stream
        for rep in range(2):
            h_out[:] = 0x3C
            rc = acx.decode_host(ctx, A if rep == 0 else None, h_arc, h_out, stream)
            assert rc == 0, ctx.last_error()
            assert np.array_equal(h_out, want), rep
        A.close()
    finally:
        ctx.close()
