"""Root isolation and backtracking through the C ABI (host code of libivsolve.so; no GPU
needed) against the oracle on the same box sets, element by element; on the GPU, the
isolated-root counts of the paper's systems.

Paper: Section 3.4 and Algorithm 5; Section 4 (noon9: 19 real roots, Table 6; kinema:
8 real roots, Table 8).
"""

import random

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

from test_oracle_clusters import random_boxes


@pytest.fixture(scope="module")
def lib():
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


@pytest.mark.parametrize("n,k,seed", [(1, 40, 11), (2, 200, 12), (3, 300, 13), (6, 150, 14), (9, 100, 15)])
def test_clusters_equal_oracle(lib, orc, n, k, seed):
    lo, hi = random_boxes(random.Random(seed), n, k)
    c, labels, hl, hh = lib.clusters(lo, hi)
    oc, olabels = orc.clusters(lo, hi)
    assert c == oc and np.array_equal(labels, olabels)
    for q in range(c):
        m = labels == q
        assert np.array_equal(hl[q], lo[m].min(axis=0)) and np.array_equal(hh[q], hi[m].max(axis=0))


@pytest.mark.parametrize("level", [0, 1, 3, 6, 10])
def test_backtrack_equals_oracle(lib, orc, level):
    """Random boxes of 0 to ~3 cells per coordinate at the level, anywhere in the box."""
    rng = random.Random(200 + level)
    d_lo, d_hi = np.array([-4.0, -1.0, 0.0, -32.0]), np.array([4.0, 1.0, 2.0, 32.0])
    cw = (d_hi - d_lo) / 2 ** level
    lo = np.array([[rng.uniform(a, b) for a, b in zip(d_lo, d_hi)] for _ in range(300)])
    hi = lo + np.array([[rng.choice([0.0, 0.01, 0.5, 2.5]) * cw[j] for j in range(4)] for _ in range(300)])
    assert lib.backtrack(lo, hi, d_lo, d_hi, level, groups=True) == orc.backtrack(lo, hi, d_lo, d_hi, level,
                                                                                  groups=True)


def test_on_solver_output(lib, orc):
    """The oracle's result boxes of small planted systems: same clusters, same cells."""
    for s in synth.config_batched(count=6, seed=321, n_range=(2, 4)):
        r = orc.solve(s, max_boxes=200_000)
        if r["status"] != 0 or len(r["lo"]) == 0:
            continue
        c, labels, _, _ = lib.clusters(r["lo"], r["hi"])
        oc, olabels = orc.clusters(r["lo"], r["hi"])
        assert c == oc and np.array_equal(labels, olabels)
        for level in (2, 5, 9):
            assert lib.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True) == \
                orc.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True)


def test_empty_and_invalid(lib):
    assert lib.clusters(np.zeros((0, 3)), np.zeros((0, 3)))[0] == 0
    with pytest.raises(lib.IvsError):
        lib.backtrack(np.zeros((1, 2)), np.ones((1, 2)), [0.0, 0.0], [0.0, 1.0], 3)   # empty initial box


@pytest.mark.gpu
@pytest.mark.parametrize("name,roots,widths", [("noon9", 19, (8, 7)), ("kinema", 8, (11, 10))])
def test_paper_root_counts(lib, orc, name, roots, widths):
    """The paper's printed systems solved on the GPU with HS from the first round, then
    backtracked (Algorithm 5) to the widths the paper reports and merged: exactly the
    paper's number of isolated real roots at both widths (Section 4: noon9 19 roots at
    width 0.0625 and 0.125, Table 6; kinema 8 roots at width 0.03125 and 0.0625, Table 8),
    the same as the oracle's backtracking of the same boxes."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = synth.load_fixture(f"tests/golden/{name}.txt")
    r = lib.solve(s, tol=1e-3)
    assert r["status"] == 0
    for level in widths:
        cells, groups = lib.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True)
        assert groups == roots, (level, cells, groups)
        assert orc.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True) == (cells, groups)
    if name == "kinema":
        # kinema's roots are also separated as touching components of the boxes themselves
        assert lib.clusters(r["lo"], r["hi"])[0] == roots
