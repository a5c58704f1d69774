"""The Python binding's ctypes structures against the C header: a small C
program built with the header prints every struct's size and every field's
offset, and the binding's structures must agree field for field (a field
appended to a header struct and not to the binding, or the reverse, fails
here rather than as garbled values at run time)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# binding class -> header type
PAIRS = {
    "EncParams": "aceapex_enc_params",
    "DecParams": "aceapex_dec_params",
    "Stats": "aceapex_stats",
    "ArchiveInfo": "aceapex_archive_info",
    "EncStats": "aceapex_enc_stats",
    "ParseStats": "aceapex_parse_stats",
    "BatchItem": "aceapex_batch_item",
    "ServerParams": "aceapex_server_params",
    "Completion": "aceapex_completion",
    "ServerStats": "aceapex_server_stats",
    "TunePoint": "aceapex_tune_point",
}


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_2608_10188_gb300 import lib
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aceapex.h"', "int main(void) {"]
    for cls, ctype in PAIRS.items():
        lines.append(f'  printf("{cls} size %zu\\n", sizeof({ctype}));')
        for name, _ in getattr(lib, cls)._fields_:
            lines.append(f'  printf("{cls} {name} %zu\\n", offsetof({ctype}, {name}));')
    lines += ["  return 0;", "}"]
    src = d / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "abi"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, stdout=subprocess.PIPE, text=True).stdout
    got = {}
    for ln in out.splitlines():
        cls, name, val = ln.split()
        got[(cls, name)] = int(val)
    return lib, got


@pytest.mark.parametrize("cls", sorted(PAIRS))
def test_binding_structs_match_the_header(layout, cls):
    lib, got = layout
    st = getattr(lib, cls)
    import ctypes
    assert ctypes.sizeof(st) == got[(cls, "size")], cls
    for name, _ in st._fields_:
        assert getattr(st, name).offset == got[(cls, name)], (cls, name)
