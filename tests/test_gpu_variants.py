"""The two split variants on the GPU against the oracle, bit for bit with every counter:
widest-coordinate bisection (split_mode = 1, two children per box instead of Algorithm
2's 2^n) and the two-box split at an extended-division gap (gap_split = 1, Section 2.3
after eq 22) -- alone, together, with the FP32 stage on and off, with Krawczyk's
operator, with several sweeps per visit, on the small planted systems and on the n = 7..15
subtrees of the large-n parity cases, mixed in one plan, served, and through the
allocation-free entry point.
"""

import ctypes as C
import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

import test_gpu_parity_large as L

pytestmark = pytest.mark.gpu

SMALL = synth.config_batched(count=12, seed=777, n_range=(2, 5))
VARIANTS = {"bisect": {"split_mode": 1}, "gap": {"gap_split": True}, "both": {"split_mode": 1, "gap_split": True}}
EXTRA = {"kr": {"krawczyk": True}, "iters3": {"hs_iters": 3}, "nohs": {"hs_enable": False}}
LARGE = ["sub_n7", "sub_n8", "sub_n9", "sub_n10_config", "sub_n10", "sub_n11", "sub_n12", "sub_n13", "sub_n15"]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


def _small_jobs():
    jobs = []
    for k, s in enumerate(SMALL):
        for v, kw in VARIANTS.items():
            jobs.append((("small", k, v, ""), s, dict(tol=1e-4, **kw)))
            for e, ekw in EXTRA.items():
                if v == "gap" or (v == "bisect" and e != "iters3"):
                    jobs.append((("small", k, v, e), s, dict(tol=1e-4, **kw, **ekw)))
    for c in LARGE:
        s, lo, hi, rd, md = L.CASES[c]
        jobs.append((("large", c, "bisect", ""), s, dict(box_lo=lo, box_hi=hi, root_depth=rd, max_depth=md,
                                                         split_mode=1)))
    s, lo, hi, rd, md = L.CASES["sub_n7"]
    jobs.append((("large", "sub_n7", "gap", ""), s, dict(box_lo=lo, box_hi=hi, root_depth=rd, max_depth=md,
                                                        gap_split=True)))
    one = synth.parse_system(["x1^2 - 1"], 1, box=(-2, 3), tol=1e-10)
    jobs.append((("one", 0, "gap", ""), one, dict(gap_split=True)))
    jobs.append((("one", 0, "both", ""), one, dict(gap_split=True, split_mode=1)))
    return jobs


JOBS = _small_jobs()


@pytest.fixture(scope="module")
def expected(orc):
    def one(job):
        key, s, kw = job
        okw = dict(kw)
        okw["centred"] = okw.pop("centred_form", False)
        return key, orc.solve(s, **okw)
    with ThreadPoolExecutor(max_workers=16) as ex:
        return dict(ex.map(one, JOBS))


def assert_same(g, o):
    L.assert_same(g, o)
    assert g["stats"]["gap_splits"] == o["stats"]["gap_splits"]


def _gpu_kw(kw):
    g = dict(kw)
    g["max_results"] = 1 << 16
    return g


def test_variants_are_exercised(expected):
    gaps = sum(o["stats"]["gap_splits"] for k, o in expected.items() if k[2] in ("gap", "both"))
    assert gaps > 1000
    assert expected[("one", 0, "gap", "")]["stats"]["gap_splits"] >= 1
    assert all(o["stats"]["hs_empty"] > 0 for k, o in expected.items() if k[0] == "large" and k[2] == "bisect"
               and k[1] not in ("sub_n13",))


@pytest.mark.parametrize("pre", [1, 0])
def test_variants_bit_exact(gpu, expected, pre):
    for key, s, kw in JOBS:
        g = gpu.solve(s, prefilter_fp32=pre, **_gpu_kw(kw))
        try:
            assert_same(g, expected[key])
        except AssertionError as e:
            raise AssertionError(f"{key}: {e}") from e


def test_variants_mixed_in_one_plan(gpu, expected):
    """Systems with different split rules in one plan: the sweeps hold parents with 2,
    4..32 and 2^n children at once."""
    jobs = [j for j in JOBS if j[0][0] == "small" and j[0][3] == ""]
    jobs += [j for j in JOBS if j[0][0] == "large"]
    systems, opts = [], []
    for key, s, kw in jobs:
        kw = dict(kw)
        lo, hi = kw.pop("box_lo", s.box_lo), kw.pop("box_hi", s.box_hi)
        systems.append(dataclasses.replace(s, box_lo=np.array(lo), box_hi=np.array(hi)))
        opts.append(gpu.make_options(**{"tol": s.tol, "max_results": 1 << 16, **kw}))
    # and the same systems with the default split, so both fan-outs share the sweeps
    for key, s, kw in jobs[:12]:
        systems.append(s)
        opts.append(gpu.make_options(tol=1e-4, max_results=1 << 16))
    plan = gpu.Plan(systems, opts=opts)
    try:
        plan.run()
        for k, (key, _, _) in enumerate(jobs):
            assert_same(plan.result(k), expected[key])
        import oracle
        for k in range(len(jobs), len(systems)):
            assert_same(plan.result(k), oracle.solve(systems[k], tol=1e-4))
    finally:
        plan.close()


def test_variants_served(gpu, expected):
    import time
    jobs = [j for j in JOBS if j[0][0] in ("small", "one") and j[0][3] in ("", "kr")]
    sv = gpu.Server(workspace_bytes=2 << 30, max_slots=64, wave_children=1 << 20, max_vars=8)
    try:
        tickets = []
        for key, s, kw in jobs:
            tickets.append((key, sv.submit(s, **_gpu_kw(kw))))
        deadline = time.time() + 300
        for key, t in tickets:
            r = sv.wait(t, timeout_s=max(1.0, deadline - time.time()))
            assert r is not None, key
            assert_same(r, expected[key])
    finally:
        sv.close()


def test_variants_without_allocation(gpu, expected):
    lib = gpu.load()
    for key, s, kw in JOBS:
        if key[0] != "small" or key[1] > 3 or key[3] not in ("", "kr"):
            continue
        ref = gpu._SysRef(s)
        o = gpu.make_options(**kw)
        cap = 1 << 14
        lo, hi = np.zeros((cap, s.n_vars)), np.zeros((cap, s.n_vars))
        fl = np.zeros(cap, np.int32)
        cnt = C.c_int64()
        st = gpu.ivs_stats()
        rc = lib.ivs_solve_noalloc(C.byref(ref.c), gpu._ptr(ref.lo), gpu._ptr(ref.hi), C.byref(o), None,
                                   gpu._ptr(lo), gpu._ptr(hi), gpu._ptr(fl), cap, C.byref(cnt), C.byref(st), None, 0)
        e = expected[key]
        k = cnt.value
        assert rc == e["status"], key
        assert np.array_equal(lo[:k], e["lo"]) and np.array_equal(hi[:k], e["hi"]), key
        assert st.boxes == e["stats"]["boxes"] and st.gap_splits == e["stats"]["gap_splits"], key
