"""Seeded synthetic corpora (DNA-like genome, Zipf text) for tests and benchmarks.

The generators hold none of the codec's arithmetic; they only produce the
input bytes that both the CPU oracle and the GPU library consume.  The C
source (``synth.c``) is compiled into ``libsynth.so`` beside this file on
first use (gcc, no architecture-specific flags, so it gives identical bytes on
x86_64 and aarch64).

Workload recipes (stand-ins for the paper's chr1 / text corpora, which are
not available):

* ``dna(n, seed)``: uniform {A,C,G,T} with 0.5% 'N' runs (length 10-1000),
  24% of positions in copies of earlier spans (lognormal length, median 7 B,
  clipped to [4, 4096], distance log-uniform, 1% point mutations) and 6% in
  tandem repeats (period 1-12, length 20-200).
* ``text(n, seed)``: Zipf(s=1.1) over a 50,000-word vocabulary of 2-12
  lowercase letters, sentences of 5-25 words ending in ". ", 5% of sentences
  repeated verbatim.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lock = threading.Lock()
_lib = None

GENOME_CHR1_SIZE = 253_935_557
BLOCK_SIZE = 16384


class DnaStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "n_bytes_random", "n_bytes_nrun", "n_bytes_copy", "n_bytes_tandem",
        "n_copies", "n_tandems", "n_nruns", "n_mutations")]


class TextStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("n_sentences", "n_repeated", "n_words")]


def build(force: bool = False) -> str:
    """Compile libsynth.so beside the source (idempotent)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.synth_dna.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.POINTER(DnaStats)]
        lib.synth_dna.restype = ctypes.c_int
        lib.synth_text.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_double, ctypes.c_double, ctypes.POINTER(TextStats)]
        lib.synth_text.restype = ctypes.c_int
        for name in ("synth_splitmix64", "synth_xoshiro256ss"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64]
            f.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _out(n: int, out):
    if out is None:
        return np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
    return out


def dna(n: int, seed: int = 0, n_frac: float = 0.005, copy_frac: float = 0.24,
        tandem_frac: float = 0.06, out=None, stats: bool = False):
    """DNA-like genome of n bytes (numpy uint8)."""
    buf = _out(n, out)
    st = DnaStats()
    rc = _load().synth_dna(buf.ctypes.data, n, seed, n_frac, copy_frac, tandem_frac, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"synth_dna failed ({rc})")
    return (buf[:n], st) if stats else buf[:n]


def text(n: int, seed: int = 0, n_vocab: int = 50_000, zipf_s: float = 1.1, p_repeat: float = 0.05,
         out=None, stats: bool = False):
    """Zipf text of n bytes (numpy uint8)."""
    buf = _out(n, out)
    st = TextStats()
    rc = _load().synth_text(buf.ctypes.data, n, seed, n_vocab, zipf_s, p_repeat, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"synth_text failed ({rc})")
    return (buf[:n], st) if stats else buf[:n]


def splitmix64(seed: int, n: int) -> np.ndarray:
    a = np.empty(n, dtype=np.uint64)
    _load().synth_splitmix64(seed, a.ctypes.data, n)
    return a


def xoshiro256ss(seed: int, n: int) -> np.ndarray:
    a = np.empty(n, dtype=np.uint64)
    _load().synth_xoshiro256ss(seed, a.ctypes.data, n)
    return a


def batch_specs(n_archives: int = 96, seed: int = 4, lo: int = 64 << 10, hi: int = 64 << 20):
    """The mixed batch workload: archive sizes log-uniform in [lo, hi] drawn
    from ``seed``; archive i uses seed 1000+i, DNA for even i and text for odd
    i, history-free encoding for i mod 4 in {2, 3}.  Returns a list of dicts."""
    raw = splitmix64(seed, n_archives)
    specs = []
    for i in range(n_archives):
        u = float(int(raw[i]) >> 11) / float(1 << 53)
        size = int(round(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)))
        specs.append({"index": i, "size": size, "seed": 1000 + i,
                      "kind": "dna" if i % 2 == 0 else "text", "no_rep": (i % 4) in (2, 3)})
    return specs


def corpus(kind: str, n: int, seed: int):
    if kind == "dna":
        return dna(n, seed)
    if kind == "text":
        return text(n, seed)
    raise ValueError(kind)
