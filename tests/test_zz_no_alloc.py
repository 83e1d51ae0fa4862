"""ivs_solve_noalloc: the allocation-free solve, for callers that cannot call cudaMalloc
(processes whose device memory belongs to a pool they must not bypass, plug-ins running
inside a runtime that forbids allocation, real-time loops that cannot afford cudaMalloc's
implicit synchronisation).

Called through the C ABI, it must return exactly what ivs_solve returns (the same sorted
boxes, flags and processed-box count), twice in a row (the fixed scratch keeps the last
call's contents, so the second call checks that everything that must start at zero is
cleared), and it must reject systems too large for its fixed buffers with a clear error.
After its first call on a device it must leave the device's free memory unchanged.
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


def test_noalloc_leaves_device_memory_unchanged(B):
    """The defining property: after a first call (which looks up the scratch address),
    a solve changes the device's free memory by nothing."""
    import torch
    s = synth.config_n6()
    rc, *_ = noalloc(B, s)
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        rc, lo, *_ = noalloc(B, s)
        assert rc == 0 and len(lo) > 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_budget_when_the_output_is_too_small(B):
    """Two roots, room for one box: IVS_ERR_BUDGET with one of ivs_solve's boxes."""
    s = synth.config_n2()
    ref = B.solve(s)
    rc, lo, hi, fl, st, msg = noalloc(B, s, out_cap=1)
    assert rc == 3 and len(lo) == 1
    assert any(np.array_equal(lo[0], a) and np.array_equal(hi[0], b) for a, b in zip(ref["lo"], ref["hi"]))
    assert st["accepted"] == ref["stats"]["accepted"] == 2


def _many_terms_system(n=12, terms_per_eq=180):
    """n equations of `terms_per_eq` monomials of degree <= 3: more terms than the fixed
    table holds (2048)."""
    rng = np.random.default_rng(5)
    mons = synth.monomials(n, 3)
    exps, offs = [], [0]
    for _ in range(n):
        idx = rng.choice(len(mons), size=terms_per_eq, replace=False)
        exps += [mons[q] for q in sorted(idx)]
        offs.append(len(exps))
    coef = rng.integers(1, 5, size=len(exps)).astype(np.float64)
    return synth.PolySystem(n_vars=n, n_eqs=n, eq_offsets=np.array(offs, np.int32), coef_lo=coef,
                            coef_hi=coef.copy(), exps=np.array(exps, np.uint8), box_lo=np.full(n, -1.0),
                            box_hi=np.full(n, 1.0), tol=1e-3)


def test_noalloc_rejects_an_oversized_term_table(B):
    rc, *_, msg = noalloc(B, _many_terms_system())
    assert rc == 1 and "term table" in msg


def test_noalloc_error_text_without_a_buffer(B):
    """With errbuf = NULL the message is still kept as ivs_last_error()."""
    lib = B.load()
    s = synth.parse_system([f"x{j + 1}^2 - 1" for j in range(13)], 13, box=(-2, 2))
    ref = B._SysRef(s)
    o = B.make_options(tol=s.tol)
    lo = np.zeros((4, 13))
    hi = np.zeros((4, 13))
    cnt = C.c_int64(-1)
    rc = lib.ivs_solve_noalloc(C.byref(ref.c), B._ptr(ref.lo), B._ptr(ref.hi), C.byref(o), None,
                               B._ptr(lo), B._ptr(hi), None, 4, C.byref(cnt), None, None, 0)
    assert rc == 1 and cnt.value == 0
    assert "n_vars" in lib.ivs_last_error().decode()
