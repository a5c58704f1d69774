"""Helpers for GPU tests: run the C-ABI decode on device buffers allocated
with torch, and return host bytes."""
from __future__ import annotations

import numpy as np


def torch_cuda():
    import torch
    return torch


def to_dev(arr: np.ndarray):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(arr)).to("cuda")
    return t


def gpu_decode(ctx, arc_bytes: bytes, variant: int | None = None, out_pad: int = 0, stats: bool = False):
    """Open the archive on the device, decode it with aceapex_decode_all and
    return (status, output numpy array or None[, stats])."""
    import paper_2608_10188_gb300 as acx
    torch = torch_cuda()
    if variant is not None:
        ctx.set_params(variant=variant, timeout_us=ctx.params.timeout_us)
    h = np.frombuffer(arc_bytes, dtype=np.uint8).copy()
    d_arc = to_dev(h) if h.size else torch.empty(16, dtype=torch.uint8, device="cuda")
    arc = acx.Archive(ctx, d_arc.data_ptr(), h, h.size)
    total = arc.total
    out = torch.full((max(total + out_pad, 1),), 0xA5, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    r = acx.decode_all(ctx, arc, out.data_ptr(), out.numel(), stream, stats=stats)
    rc, st = (r if stats else (r, None))
    torch.cuda.synchronize()
    res = out[:total].cpu().numpy() if rc == 0 else None
    tail = out[total:].cpu().numpy() if out_pad else None
    arc.close()
    del d_arc
    if stats:
        return rc, res, st
    if out_pad:
        return rc, res, tail
    return rc, res
