"""Root isolation and Algorithm 5 backtracking on the GPU (ivs_clusters_gpu,
ivs_backtrack_gpu, ivs_plan_clusters, ivs_plan_backtrack) against the oracle's
orc_clusters / orc_backtrack on the same box sets, element by element, and the paper's
isolated-root counts from a plan's device-resident result (Section 3.4, Algorithm 5;
Section 4: noon9 19 roots, Table 6; kinema 8 roots, Table 8).
"""

import random

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

from test_oracle_clusters import random_boxes

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


@pytest.mark.parametrize("n,k,seed", [(1, 40, 11), (2, 200, 12), (3, 300, 13), (6, 150, 14), (9, 100, 15),
                                      (4, 3000, 16)])
def test_clusters_gpu_equal_oracle(gpu, orc, n, k, seed):
    lo, hi = random_boxes(random.Random(seed), n, k)
    c, labels, hl, hh = gpu.clusters_gpu(lo, hi)
    oc, olabels = orc.clusters(lo, hi)
    assert c == oc and np.array_equal(labels, olabels)
    for q in range(c):
        m = labels == q
        assert np.array_equal(hl[q], lo[m].min(axis=0)) and np.array_equal(hh[q], hi[m].max(axis=0))


@pytest.mark.parametrize("level", [0, 1, 3, 6, 10, 20])
def test_backtrack_gpu_equals_oracle(gpu, orc, level):
    """Random boxes of 0 to ~3 cells per coordinate at the level, anywhere in the box."""
    rng = random.Random(200 + level)
    d_lo, d_hi = np.array([-4.0, -1.0, 0.0, -32.0]), np.array([4.0, 1.0, 2.0, 32.0])
    cw = (d_hi - d_lo) / 2 ** level
    lo = np.array([[rng.uniform(a, b) for a, b in zip(d_lo, d_hi)] for _ in range(2000)])
    hi = lo + np.array([[rng.choice([0.0, 0.01, 0.5, 2.5]) * cw[j] for j in range(4)] for _ in range(2000)])
    assert gpu.backtrack_gpu(lo, hi, d_lo, d_hi, level, groups=True) == orc.backtrack(lo, hi, d_lo, d_hi, level,
                                                                                      groups=True)


def test_on_solver_output(gpu, orc):
    """The oracle's result boxes of small planted systems (boxes on split planes around
    each root): same clusters, cells and groups as the oracle."""
    checked = 0
    for s in synth.config_batched(count=10, seed=321, n_range=(2, 5)):
        r = orc.solve(s, max_boxes=200_000)
        if r["status"] != 0 or len(r["lo"]) == 0:
            continue
        c, labels, _, _ = gpu.clusters_gpu(r["lo"], r["hi"])
        oc, olabels = orc.clusters(r["lo"], r["hi"])
        assert c == oc and np.array_equal(labels, olabels)
        for level in (2, 5, 9, 14):
            if s.n_vars * level > 127:
                continue
            assert gpu.backtrack_gpu(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True) == \
                orc.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True)
        checked += 1
    assert checked >= 5


def test_plan_level_matches_host(gpu, orc):
    """From a plan's device-resident results (no host copy), the same counts as the
    oracle's functions on the host-sorted result boxes."""
    systems = synth.config_batched(count=12, seed=4040, n_range=(2, 5))
    plan = gpu.Plan(systems, opts={"tol": 1e-4})
    try:
        plan.run()
        for k, s in enumerate(systems):
            r = plan.result(k)
            assert plan.clusters(k) == orc.clusters(r["lo"], r["hi"])[0]
            for level in (3, 8, 13):
                if s.n_vars * level > 127:
                    continue
                assert plan.backtrack(k, level) == orc.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level,
                                                                 groups=True)
    finally:
        plan.close()


def _root_like_boxes(rng, n, k, roots=40):
    """k tiny boxes scattered around `roots` points in [-8, 8]^n (the shape of a solve's
    output: many small boxes per isolated root)."""
    centres = rng.uniform(-7.0, 7.0, size=(roots, n))
    which = rng.integers(0, roots, size=k)
    w = 2.0 ** rng.integers(-12, -7, size=(k, n))
    lo = centres[which] + rng.uniform(-0.02, 0.02, size=(k, n))
    return lo, lo + w


def test_large_sets_match_host(gpu):
    """Many boxes (beyond the quadratic oracle): the GPU equals the host library."""
    rng = np.random.default_rng(77)
    for n, k in ((3, 200_000), (6, 100_000), (9, 50_000)):
        lo, hi = _root_like_boxes(rng, n, k)
        c, labels, hl, hh = gpu.clusters_gpu(lo, hi)
        hc, hlabels, hhl, hhh = gpu.clusters(lo, hi)
        assert c == hc and np.array_equal(labels, hlabels)
        assert np.array_equal(hl, hhl) and np.array_equal(hh, hhh)
        d_lo, d_hi = np.full(n, -8.0), np.full(n, 8.0)
        for level in ((6, 10) if n < 9 else (6,)):   # the host groups n = 9 at level 10 in minutes
            assert gpu.backtrack_gpu(lo, hi, d_lo, d_hi, level, groups=True) == \
                gpu.backtrack(lo, hi, d_lo, d_hi, level, groups=True)


def test_edge_cases(gpu):
    assert gpu.clusters_gpu(np.zeros((0, 3)), np.zeros((0, 3)))[0] == 0
    assert gpu.backtrack_gpu(np.zeros((0, 2)), np.zeros((0, 2)), [0.0, 0.0], [1.0, 1.0], 5, groups=True) == (0, 0)
    one = np.array([[0.25, 0.5]])
    assert gpu.backtrack_gpu(one, one, [0.0, 0.0], [1.0, 1.0], 2, groups=True) == \
        gpu.backtrack(one, one, [0.0, 0.0], [1.0, 1.0], 2, groups=True)
    with pytest.raises(gpu.IvsError):   # n_vars * level above 127
        gpu.backtrack_gpu(np.zeros((1, 9)), np.ones((1, 9)), np.zeros(9), np.ones(9), 15)
    with pytest.raises(gpu.IvsError):   # more cells than allowed
        gpu.backtrack_gpu(np.zeros((1, 3)), np.ones((1, 3)), np.zeros(3), np.ones(3), 10, max_cells=1000)


@pytest.mark.parametrize("name,roots,widths", [("noon9", 19, (8, 7)), ("kinema", 8, (11, 10))])
def test_paper_root_counts_on_the_device(gpu, orc, name, roots, widths):
    """The paper's printed systems solved with HS from the first round; backtracked and
    merged on the device from the plan's result: exactly the paper's isolated real
    roots (noon9 19 at widths 0.0625 and 0.125; kinema 8 at 0.03125 and 0.0625), and the
    oracle's backtracking of the same boxes agrees."""
    s = synth.load_fixture(f"tests/golden/{name}.txt")
    plan = gpu.Plan([s], opts={"tol": 1e-3})
    try:
        plan.run()
        r = plan.result(0)
        assert r["status"] == 0
        for level in widths:
            cells, groups = plan.backtrack(0, level)
            assert groups == roots, (level, cells, groups)
            assert orc.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True) == (cells, groups)
        if name == "kinema":
            assert plan.clusters(0) == roots
    finally:
        plan.close()
