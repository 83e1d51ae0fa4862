"""The C-ABI library builds, loads and exports every entry point include/ivsolve.h
declares; host-only calls behave; without a GPU the solver fails loudly (no CPU
fallback exists).  Runs on CPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ivsolve.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ivs_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1802_00330_gb300 import build, _binding
    build.build()
    return _binding.load()


def test_exports_every_declared_symbol(lib):
    from paper_1802_00330_gb300 import _binding
    names = header_functions()
    assert len(names) >= 15
    raw = C.CDLL(_binding.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
    assert names == set(_binding.SIGNATURES), names ^ set(_binding.SIGNATURES)


def test_host_only_calls(lib):
    from paper_1802_00330_gb300 import _binding as B
    o = B.ivs_options()
    lib.ivs_options_default(C.byref(o))
    assert o.tol == 1e-6 and o.hs_enable == 1 and o.prefilter_fp32 == 1 and o.max_depth == 200
    assert lib.ivs_status_str(0) == b"ok"
    assert b"budget" in lib.ivs_status_str(3)
    s = synth.config_n6()
    ref = B._SysRef(s)
    nb = lib.ivs_workspace_bytes(1, C.byref(ref.c), 1 << 20, 1 << 20, 1 << 16)
    assert nb > (1 << 20) * 8 * 3 * 6


def _call_solve(lib, s, lo, hi, **kw):
    from paper_1802_00330_gb300 import _binding as B
    ref = B._SysRef(s)
    o = B.make_options(**{"tol": s.tol, **kw})
    res = C.c_void_p()
    rc = lib.ivs_solve(C.byref(ref.c), B._ptr(np.ascontiguousarray(lo, float)),
                       B._ptr(np.ascontiguousarray(hi, float)), C.byref(o), C.byref(res))
    if res:
        lib.ivs_result_free(res)
    return rc


def test_validation_before_any_device_work(lib):
    """Invalid inputs are rejected on the host with IVS_ERR_INVALID (no GPU needed)."""
    s = synth.config_n2()
    assert _call_solve(lib, s, [1.0, 0.0], [0.0, 1.0]) == 1             # lo > hi
    assert _call_solve(lib, s, [np.nan, 0.0], [1.0, 1.0]) == 1          # non-finite
    assert _call_solve(lib, s, s.box_lo, s.box_hi, tol=-1.0) == 1
    s3 = synth.parse_system(["x1 + x2 + x3"], 3)
    assert _call_solve(lib, s3, s3.box_lo, s3.box_hi, hs_enable=True) == 1   # m != n with HS
    big = synth.parse_system(["x1^16 - 1"], 1)
    assert _call_solve(lib, big, [-1.0], [1.0]) == 1                     # exponent > 15


def test_no_gpu_fails_loudly(lib):
    """On a machine without a GPU a valid solve returns IVS_ERR_CUDA: there is no CPU
    path to fall back to."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    s = synth.config_n2()
    assert _call_solve(lib, s, s.box_lo, s.box_hi) == 5
    assert b"cuda" in lib.ivs_last_error().lower() or len(lib.ivs_last_error()) > 0


def test_server_without_gpu_fails_loudly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from paper_1802_00330_gb300 import _binding as B
    with pytest.raises(B.IvsError) as e:
        B.Server(workspace_bytes=1 << 26, max_slots=4)
    assert e.value.status == 5


STRUCTS = ["ivs_system", "ivs_options", "ivs_stats", "ivs_plan_cfg", "ivs_server_cfg", "ivs_server_stats",
           "ivs_kernel_time"]


def header_struct_fields(name):
    """Field names of `typedef struct name { ... } name;` in declaration order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef\s+struct\s+" + name + r"\s*\{(.*?)\}\s*" + name + r"\s*;", text, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        mm = re.match(r"((?:const\s+)?(?:unsigned\s+)?[A-Za-z_]\w*(?:\s+const)?)\s+(.*)$", decl, flags=re.S)
        for d in mm.group(2).split(","):
            fields.append(re.sub(r"\[.*\]", "", d).replace("*", "").strip())
    return fields


def test_binding_structs_have_the_header_fields():
    from paper_1802_00330_gb300 import _binding as B
    for name in STRUCTS:
        assert [f for f, _ in getattr(B, name)._fields_] == header_struct_fields(name), name


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field offsets
    (a field added on one side only would shift everything after it)."""
    import shutil
    import subprocess
    from paper_1802_00330_gb300 import _binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ivsolve.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(B, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            sname, field, val = ln.split()
            got[(sname, field)] = int(val)
    for name in STRUCTS:
        cls = getattr(B, name)
        assert got[(name, "size")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
