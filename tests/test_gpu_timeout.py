"""A device-side dependency wait that runs out.  (-m gpu)

Every wait of the cross-block pass on other work (a piece on its sources, a
CTA on the grid barrier) is bounded by the context's timeout_us; when the
limit passes, the kernel records ACEAPEX_E_TIMEOUT and returns, and the
context stays usable.  The test makes the wait run out without any fault:
level hints that hand the last blocks' pieces out first, with pieces waiting
without a limit of their own, leave every lane of the pass holding a piece
whose sources are pieces of earlier blocks that are only handed out later.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_decode import _rewrite_levels

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


def test_dependency_wait_runs_out_then_the_context_decodes(acx):
    from gpu_util import gpu_decode
    data = synth.text((8 << 20) + 5, 33)
    nb = (data.size + BLOCK - 1) // BLOCK
    arc = acx.encode(data, levels=True, max_depth=0xFFFFFFFF)
    backwards = _rewrite_levels(arc, lambda lv, b: np.full(lv.size, max(1, 255 - (255 * b) // nb), np.uint8))
    want = oracle.decode(backwards)
    assert np.array_equal(want, data)
    ctx = acx.Context(0, timeout_us=20_000, wait_ns=0xFFFFFFFF)
    try:
        rc, out = gpu_decode(ctx, backwards)
        assert rc == acx.lib.E_TIMEOUT, (rc, ctx.last_error())
        assert "timed out" in ctx.last_error()
        # the same context, default limits: the misleading hints cost time only
        ctx.set_params(timeout_us=2_000_000)
        rc, out = gpu_decode(ctx, backwards)
        assert rc == 0, ctx.last_error()
        assert np.array_equal(out, want)
        rc, out = gpu_decode(ctx, arc)
        assert rc == 0 and np.array_equal(out, data)
    finally:
        ctx.close()
