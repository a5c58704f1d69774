"""bench.py's host arithmetic, on the CPU: the stream byte counts it reads
from an archive (against the oracle's own stream dumps) and the roofline
fields of the bench line (the algorithmic bytes of one decode are the archive
read plus the output written; `achieved` divides them by the dominant
kernel's time; `frac` by the measured copy peak)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import sys
    sys.path.insert(0, ROOT)
    import bench as b
    return b


@pytest.fixture(scope="module")
def arc():
    import paper_2608_10188_gb300 as acx
    acx.build.build()
    data = synth.dna(3 * 16384 + 555, 4)
    return data, acx.encode(data)


def test_stream_bytes_match_the_oracles_streams(bench, arc):
    import struct
    data, a = arc
    sb = bench.stream_bytes(a)
    nb = struct.unpack_from("<I", a, 24)[0]
    decoded = sum(oracle.block_stream(a, b, s).size for b in range(nb) for s in range(4))
    assert sb["decoded"] == decoded
    off_idx = struct.unpack_from("<Q", a, 40)[0]
    assert sb["payload"] == sum(struct.unpack_from("<QI", a, off_idx + 40 * b)[1] for b in range(nb))
    assert 0 < sb["payload"] < len(a)


def test_roofline_fields(bench, arc):
    data, a = arc
    sb = bench.stream_bytes(a)
    stage = {"ans": 0.02, "local": 0.05, "cross": 0.01}
    st = {"pending_bytes": 1000, "pending_spans": 40}
    roof, path = bench.rooflines(stage, sb, data.size, len(a), st, 4, "fast", 0.08, wname="")
    peak, kind = bench.measured_peaks()
    want_bytes = len(a) + data.size
    assert roof["algorithmic_bytes"] == want_bytes
    assert roof["kernel"] == "k_local" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    achieved = want_bytes / (0.05 / 1e3) / 1e9
    assert roof["achieved"] == pytest.approx(achieved, abs=0.05)  # (reported to 0.1 GB/s)
    assert roof["frac"] == pytest.approx(achieved / peak, abs=1e-4)
    assert roof["peak"] == peak and roof["peak_kind"].startswith(kind)
    k = roof["kernels"]
    assert k["k_rans"]["design_bytes"] == sb["payload"] + sb["decoded"]
    assert k["k_local"]["design_bytes"] == sb["decoded"] + data.size
    assert k["k_external"]["design_bytes"] == 2 * 1000 + 16 * 40 + 4 * 4
    # counters captured on other sources or another workload are not reported
    assert roof["traffic"] is None and all(v["traffic"] is None for v in k.values())
    assert path["bytes"] == want_bytes
    assert path["achieved"] == pytest.approx(want_bytes / (0.08 / 1e3) / 1e9, abs=0.05)
    # the fused variant is one kernel for the entropy stage and the local pass
    roof_f, _ = bench.rooflines(stage, sb, data.size, len(a), st, 4, "fused", 0.08)
    assert set(roof_f["kernels"]) == {"k_fused", "k_external"}
    assert roof_f["kernels"]["k_fused"]["design_bytes"] == sb["payload"] + data.size


def test_captured_counters_are_keyed_to_the_sources(bench):
    key = bench.kernel_source_key()
    assert len(key) == 16 and int(key, 16) >= 0
    for (src, wname, kern), v in bench.CAPTURED_DRAM.items():
        assert len(src) == 16 and wname and kern in ("k_rans", "k_local", "k_external") and v > 0
    for (src, wname), v in bench.CAPTURED_RANS_INSTR_PER_SYMBOL.items():
        assert 0 < v < 4


def test_measured_peak_is_read_from_the_peaks_file(bench):
    peak, kind = bench.measured_peaks()
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        assert kind == "measured" and peak == float(json.load(open(p))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0
