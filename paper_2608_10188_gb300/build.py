"""Build libaceapex.so in-tree: the CUDA kernels for sm_103a (nvcc) and the
host library (C++), linked into one shared library beside this file.

Run ``python -m paper_2608_10188_gb300.build`` or call ``build()``.
Translation units compile in parallel; nothing is architecture-specific on
the host side, so the same command builds on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libaceapex.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaceapex.so")


def sources():
    return [os.path.join(CSRC, f) for f in ("rans.cu", "assemble.cu", "fused.cu", "plain.cu", "noalloc.cu", "gather.cu", "api.cpp",
                                          "batch.cpp", "subset.cpp", "closure.cpp", "serve.cpp", "plan.cpp",
                                          "encode.cpp")]


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in ("internal.h", "plan.h", "common.cuh", "launch.h", "host.h", "rans_dev.cuh", "local_dev.cuh")] + [
        os.path.join(os.path.dirname(HERE), "include", "aceapex.h")]


def up_to_date() -> bool:
    if not os.path.exists(SO):
        return False
    t = os.path.getmtime(SO)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return SO
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC]
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, ARCH, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3", *common, "-c", src, "-o", obj]
        else:
            cmd = [nvcc, *common, "-Xcompiler", "-pthread", "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("libaceapex build failed:\n" + msg)
    tmp = SO + f".tmp{os.getpid()}"
    link = [nvcc, ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libaceapex link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
