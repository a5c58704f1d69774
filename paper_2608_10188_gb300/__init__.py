"""GB300 (sm_103a) decoder for the blockwise absolute-offset LZ77 format of
"What Actually Serializes GPU LZ77 Decode" (format v1).

The compute path is the CUDA library ``libaceapex.so`` (built in-tree by
``paper_2608_10188_gb300.build``); ``lib`` is its ctypes binding.  PyTorch is
only used by callers for device memory and streams.
"""
from . import build, lib, tune  # noqa: F401
from .lib import (Archive, Batch, Context, Server, autotune, AceapexError, archive_check, batch_decode, decode_all,  # noqa: F401
                  decode_all_async, decode_host, decode_range, encode, load, shard_range)
