"""The host code under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

The library's host side parses untrusted archives (the plan builder behind
archive_open and archive_check, the byte-level closure walk, the parse
statistics) and its encoder writes them; the oracle parses them too.
tests/sanitize/san_driver.cpp runs all of them, built with
-fsanitize=address,undefined (no recovery), on archives from both encoders and
on truncations and bit flips of each.  Any sanitizer report or failed check
makes the driver exit non-zero.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_10188_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
SAN = ["-g", "-O1", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]


def test_host_code_is_clean_under_asan_and_ubsan(tmp_path):
    if not shutil.which("g++") or not os.path.exists(os.path.join(CUDA, "lib64", "libcudart_static.a")):
        pytest.skip("needs g++ and the CUDA runtime's static library")
    d = str(tmp_path)
    run = lambda cmd: subprocess.run(cmd, cwd=d, check=True, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    run(["gcc", "-c", *SAN, "-std=c11", os.path.join(ROOT, "oracle", "oracle.c"), "-o", "oracle.o"])
    run(["gcc", "-c", *SAN, "-std=c11", "-ffp-contract=off", os.path.join(ROOT, "synth", "synth.c"), "-o", "synth.o"])
    # the host sources that parse or write archives; the driver never calls
    # into the device code, which --gc-sections leaves out
    srcs = [os.path.join(CSRC, f) for f in ("plan.cpp", "encode.cpp", "closure.cpp", "api.cpp")]
    run(["g++", *SAN, "-std=c++17", "-ffunction-sections", "-fdata-sections", "-I", CSRC,
         "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "sanitize", "san_driver.cpp"), *srcs,
         "oracle.o", "synth.o", "-Wl,--gc-sections", "-L", os.path.join(CUDA, "lib64"), "-lcudart_static", "-ldl",
         "-lpthread", "-lrt", "-o", "san_driver"])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([os.path.join(d, "san_driver"), "40"], cwd=d, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, timeout=600)
    out = r.stdout.decode(errors="replace")
    assert r.returncode == 0, out[-4000:]
    assert "0 failures" in out and "ERROR: AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
