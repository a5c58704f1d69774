"""Autotuned decoder parameters with a JSON cache (argument marshalling and
bookkeeping only; the search itself is aceapex_autotune in the library).

The cache file maps "<device name>|<workload key>" to the best point of the
launch space (CTAs per SM of the local pass and the entropy stage, blocks per
queue ticket) and the measured points, so a workload class is tuned once per
device type.
"""
from __future__ import annotations

import json
import os

from . import lib


def _device_name(device: int) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:  # no torch or no device query: one shared entry
        return "cuda"


def tuned_params(ctx: lib.Context, entries, key: str, cache_path: str | None = None, reps: int = 3,
                 device: int = 0) -> dict:
    """Decoder parameters for `entries` (a list of (Archive, d_out, out_cap)),
    from the cache when `key` was tuned on this device type before, else by
    aceapex_autotune (whose result is stored).  Applies them to ctx."""
    ck = f"{_device_name(device)}|{key}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if ck in cache:
        b = cache[ck]["best"]
        ctx.set_params(variant=ctx.params.variant, timeout_us=ctx.params.timeout_us,
                       ctas_per_sm=b["ctas_per_sm"], rans_ctas_per_sm=b["rans_ctas_per_sm"],
                       queue_chunk=b["queue_chunk"])
        return dict(b, cached=True)
    best, points = lib.autotune(ctx, entries, reps=reps)
    rec = {"best": {k: best[k] for k in ("ctas_per_sm", "rans_ctas_per_sm", "queue_chunk")}, "points": points}
    if cache_path:
        cache[ck] = rec
        tmp = cache_path + f".{os.getpid()}"
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(rec["best"], cached=False, points=len(points))
