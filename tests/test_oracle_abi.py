"""The oracle's ctypes mirrors (oracle/__init__.py) have the C layout of oracle/ivs_oracle.h:
the compiler's size and field offsets for orc_system, orc_options and orc_stats."""

import os
import shutil
import subprocess

import ctypes as C
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_structs_match_the_header(tmp_path):
    import oracle
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("orc_system", oracle._Sys), ("orc_options", oracle._Opt), ("orc_stats", oracle._Stats)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ivs_oracle.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        sname, field, val = ln.split()
        got[(sname, field)] = int(val)
    for cname, cls in pairs:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
