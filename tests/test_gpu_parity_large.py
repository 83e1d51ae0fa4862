"""GPU path against the serial oracle for n = 7..15: the sizes of the batched (n <= 8),
served (n <= 12) and n=10 configurations, and the largest kernels the library builds.

A full solve of these systems is far beyond the serial oracle (10^8-10^10 boxes), so the
cases are exact parts of the real solves, each of which the oracle finishes in seconds:

* subtrees: the cell of the solve's own dyadic tree that holds the planted root at level
  L (the initial box split L times), solved to the system's tolerance with
  root_depth = L -- every box of it is a box of the full solve, processed the same way
  (Algorithm 1-3); near the root the Hansen-Sengupta sweeps empty or contract hundreds
  to thousands of boxes;
* depth cuts: the full initial box to max_depth = 1 (the first 2^n children, all with a
  Hansen-Sengupta sweep at full width).

Each is compared bit for bit (sorted boxes, flags, depths) with every counter, for the
Gauss-Seidel sweep (eq 21-22) and Krawczyk's operator (eq 15-16), with and without the
FP32 stage; then all of them in one plan (wide sweeps: the independent kernel form and
several dimensions per sweep) and all of them served together in one server.
"""

import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


def root_cell(s, level):
    """(lo, hi) of the level-`level` cell of the solve's tree that holds the planted root
    (the initial box split `level` times at its midpoints; dyadic, so exact)."""
    r = np.array([float(v) for v in s.roots[0]])
    w = (s.box_hi - s.box_lo) / 2.0 ** level
    k = np.minimum(np.floor((r - s.box_lo) / w), 2 ** level - 1)
    lo = s.box_lo + k * w
    return lo, lo + w


def _served(seed, n_range, index):
    return synth.config_served(duration_s=0.05, rate=2000.0, seed=seed, n_range=n_range)[1][index]


def _cases():
    """name -> (system, initial box lo, hi, root depth, max depth)."""
    served = synth.config_served(duration_s=0.02, rate=2000.0)[1]
    by_name = {s.name: s for s in served}
    big = synth.config_served(duration_s=0.01, rate=2000.0, seed=77, n_range=(13, 16))[1]
    big = {s.name: s for s in big}
    batched = synth.config_batched(count=4, seed=2026, n_range=(7, 8))
    sub = [("n7", by_name["served_14_n7"], 5), ("n8", batched[0], 4), ("n8b", batched[3], 4),
           ("n9", by_name["served_6_n9"], 5), ("n10_config", synth.config_n10(), 6),
           ("n10", by_name["served_0_n10"], 6), ("n11", by_name["served_1_n11"], 7),
           ("n12", by_name["served_10_n12"], 7), ("n13", big["served_0_n13"], 8),
           ("n15", big["served_1_n15"], 8)]
    out = {}
    for name, s, level in sub:
        lo, hi = root_cell(s, level)
        out["sub_" + name] = (s, lo, hi, level, 200)
    for name, s in (("n10_config", synth.config_n10()), ("n11", by_name["served_1_n11"]),
                    ("n12", by_name["served_10_n12"])):
        out["cut_" + name] = (s, s.box_lo, s.box_hi, 0, 1)
    return out


CASES = _cases()
METHODS = {"gs": {}, "kr": {"krawczyk": True}}
_ORACLE = {}


def _oracle_kw(case, method):
    s, lo, hi, rd, md = CASES[case]
    return dict(box_lo=lo, box_hi=hi, root_depth=rd, max_depth=md, **METHODS[method])


@pytest.fixture(scope="module")
def expected(orc):
    """Oracle results of every case and method, computed once (threads: the oracle's
    ctypes calls release the interpreter lock and each thread keeps its own rounding
    mode)."""
    keys = [(c, m) for c in CASES for m in METHODS]
    keys += [("sub_n10_config", "iters4"), ("sub_n10_config", "centred")]

    def one(key):
        c, m = key
        s = CASES[c][0]
        if m == "iters4":
            return orc.solve(s, **_oracle_kw(c, "gs"), hs_iters=4)
        if m == "centred":
            return orc.solve(s, **_oracle_kw(c, "gs"), centred=True)
        return orc.solve(s, **_oracle_kw(c, m))

    with ThreadPoolExecutor(max_workers=16) as ex:
        for k, r in zip(keys, ex.map(one, keys)):
            _ORACLE[k] = r
    return _ORACLE


def assert_same(g, o):
    assert g["status"] == o["status"]
    assert g["lo"].shape == o["lo"].shape, (g["lo"].shape, o["lo"].shape)
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    assert np.array_equal(g["flags"], o["flags"]) and np.array_equal(g["depth"], o["depth"])
    gs, os_ = g["stats"], o["stats"]
    assert gs["boxes"] == os_["boxes"]
    assert gs["excluded_prefilter"] + gs["excluded_eval"] == os_["excluded_eval"]
    for k in ("hs_applied", "hs_empty", "hs_contracted", "hs_singular", "accepted", "unsplittable", "split",
              "excluded_centred", "max_depth_seen"):
        assert gs[k] == os_[k], k
    assert np.array_equal(gs["depth_boxes"], os_["depth_boxes"])
    assert np.array_equal(gs["depth_kept"], os_["depth_kept"])


def _gpu_kw(case, method, **extra):
    s, lo, hi, rd, md = CASES[case]
    kw = dict(box_lo=lo, box_hi=hi, root_depth=rd, max_depth=md, max_results=1 << 16)
    kw.update({"krawczyk": 1} if method == "kr" else {})
    kw.update(extra)
    return kw


def test_cases_exercise_the_contraction(expected):
    """Every subtree case has sweeps that empty boxes and sweeps that contract them, and
    the sizes cover n = 7..13 and 15."""
    for c in CASES:
        st = expected[(c, "gs")]["stats"]
        assert st["hs_applied"] > 0, c
        if c.startswith("sub_"):
            assert st["hs_empty"] > 0 and st["hs_contracted"] > 0, c
    assert {CASES[c][0].n_vars for c in CASES} >= set(range(7, 14)) | {15}


@pytest.mark.parametrize("pre", [1, 0])
@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("case", list(CASES))
def test_large_n_bit_exact(gpu, expected, case, method, pre):
    s = CASES[case][0]
    g = gpu.solve(s, prefilter_fp32=pre, **_gpu_kw(case, method))
    assert_same(g, expected[(case, method)])


def test_n10_config_iterated_sweeps_and_centred_form(gpu, expected):
    s = CASES["sub_n10_config"][0]
    assert_same(gpu.solve(s, hs_iters=4, **_gpu_kw("sub_n10_config", "gs")), expected[("sub_n10_config", "iters4")])
    assert_same(gpu.solve(s, centred_form=True, **_gpu_kw("sub_n10_config", "gs")),
                expected[("sub_n10_config", "centred")])


def _case_system(case):
    """The case's system with its initial box (plans and servers take the box from it)."""
    s, lo, hi, _, _ = CASES[case]
    return dataclasses.replace(s, box_lo=np.array(lo), box_hi=np.array(hi))


def test_all_sizes_in_one_plan(gpu, expected):
    """Every case in one plan, odd ones with Krawczyk's operator: the sweeps hold several
    dimensions and enough boxes for the independent kernel form."""
    names = list(CASES)
    systems = [_case_system(c) for c in names]
    opts = []
    for k, c in enumerate(names):
        _, _, _, rd, md = CASES[c]
        opts.append(gpu.make_options(tol=systems[k].tol, root_depth=rd, max_depth=md, max_results=1 << 16,
                                     krawczyk=(k % 2 == 1)))
    plan = gpu.Plan(systems, opts=opts)
    try:
        plan.run()
        for k, c in enumerate(names):
            assert_same(plan.result(k), expected[(c, "kr" if k % 2 == 1 else "gs")])
    finally:
        plan.close()


def test_served_mix_of_large_n(gpu, expected):
    """Every case submitted to one server (n = 7..15 in flight together, each in its own
    queue region), Gauss-Seidel and Krawczyk requests interleaved: each result equals the
    oracle's."""
    import time
    names = list(CASES)
    sv = gpu.Server(workspace_bytes=8 << 30, max_slots=64, wave_children=1 << 22, max_vars=16)
    try:
        tickets = []
        for k, c in enumerate(names):
            for m in METHODS:
                _, _, _, rd, md = CASES[c]
                kw = dict(root_depth=rd, max_depth=md, max_results=1 << 16, **METHODS[m])
                tickets.append(((c, m), sv.submit(_case_system(c), **kw)))
        deadline = time.time() + 300
        for key, t in tickets:
            r = sv.wait(t, timeout_s=max(1.0, deadline - time.time()))
            assert r is not None, ("server did not finish", key, sv.stats())
            assert_same(r, expected[key])
        st = sv.stats()
        assert st["last_error"] == "", st["last_error"]
    finally:
        sv.close()
