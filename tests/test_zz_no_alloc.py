"""ivs_solve_noalloc: the allocation-free solve, for callers that cannot call cudaMalloc
(code running under stream capture, pool-managed processes, allocation-free loops).

Called through the C ABI, it must return exactly what ivs_solve returns (the same sorted
boxes, flags and processed-box count), twice in a row (the fixed scratch keeps the last
call's contents, so the second call checks that everything that must start at zero is
cleared), and it must reject systems too large for its fixed buffers with a clear error.
This file is collected last so that a failure here comes after every other test ran.
"""

import ctypes as C

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


def noalloc(B, s, out_cap=1 << 14, **opts):
    lib = B.load()
    ref = B._SysRef(s)
    o = B.make_options(**{"tol": s.tol, **opts})
    n = int(s.n_vars)
    lo = np.zeros((out_cap, n))
    hi = np.zeros((out_cap, n))
    fl = np.zeros(out_cap, np.int32)
    cnt = C.c_int64(-1)
    st = B.ivs_stats()
    msg = C.create_string_buffer(256)
    rc = lib.ivs_solve_noalloc(C.byref(ref.c), B._ptr(ref.lo), B._ptr(ref.hi), C.byref(o), None,
                               B._ptr(lo), B._ptr(hi), B._ptr(fl), out_cap, C.byref(cnt), C.byref(st),
                               msg, 256)
    k = cnt.value
    return rc, lo[:k], hi[:k], fl[:k], {f: getattr(st, f) for f, _ in B.ivs_stats._fields_}, msg.value.decode()


def test_noalloc_matches_ivs_solve_twice(B):
    systems = [synth.config_n2()] + synth.config_batched(count=3, seed=2024, n_range=(3, 5)) + [synth.config_n6()]
    for s in systems:
        ref = B.solve(s)
        for _ in range(2):
            rc, lo, hi, fl, st, msg = noalloc(B, s)
            assert rc == ref["status"], msg
            assert np.array_equal(lo, ref["lo"]) and np.array_equal(hi, ref["hi"])
            assert np.array_equal(fl, ref["flags"])
            assert st["boxes"] == ref["stats"]["boxes"]
            assert st["accepted"] == ref["stats"]["accepted"]


def test_noalloc_rejects_oversized_system(B):
    s = synth.parse_system([f"x{j + 1}^2 - 1" for j in range(13)], 13, box=(-2, 2))
    rc, *_, msg = noalloc(B, s)
    assert rc == 1 and "n_vars" in msg


def test_noalloc_krawczyk_matches_ivs_solve(B):
    for s in [synth.config_n2()] + synth.config_batched(count=2, seed=2025, n_range=(3, 5)):
        ref = B.solve(s, krawczyk=True)
        rc, lo, hi, fl, st, msg = noalloc(B, s, krawczyk=True)
        assert rc == ref["status"], msg
        assert np.array_equal(lo, ref["lo"]) and np.array_equal(hi, ref["hi"])
        assert st["boxes"] == ref["stats"]["boxes"] and st["hs_applied"] == ref["stats"]["hs_applied"]
