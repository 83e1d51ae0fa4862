"""Pins of the oracle's root isolation (connected components of touching boxes) and of
its backtracking (Algorithm 5 read on the dyadic grid of the initial box).

Paper: Section 3.4 (backtracking merges the tiny configurations of the last round into
bigger ones; the isolated roots are counted after merging), Algorithm 5, Tables 3, 6, 8.
"""

import itertools
import random
from fractions import Fraction as Q

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth


def brute_components(lo, hi):
    """Plain pairwise union-find; clusters numbered by their first box."""
    k = len(lo)
    comp = list(range(k))

    def find(a):
        while comp[a] != a:
            a = comp[a]
        return a

    for i in range(k):
        for j in range(i + 1, k):
            if all(lo[i][d] <= hi[j][d] and lo[j][d] <= hi[i][d] for d in range(len(lo[i]))):
                a, b = find(i), find(j)
                if a != b:
                    comp[max(a, b)] = min(a, b)
    labels, names = [], {}
    for i in range(k):
        r = find(i)
        names.setdefault(r, len(names))
        labels.append(names[r])
    return len(names), labels


def random_boxes(rng, n, k, spread=8, size=(0.1, 1.5)):
    lo, hi = [], []
    for _ in range(k):
        c = [rng.randint(0, spread) * 0.5 for _ in range(n)]
        w = [rng.choice([0.0, 0.25, 0.5, 1.0, size[1]]) for _ in range(n)]
        lo.append([c[d] for d in range(n)])
        hi.append([c[d] + w[d] for d in range(n)])
    return np.array(lo), np.array(hi)


@pytest.mark.parametrize("n,k,seed", [(1, 30, 1), (2, 60, 2), (3, 80, 3), (5, 60, 4)])
def test_components_equal_brute_force(orc, n, k, seed):
    rng = random.Random(seed)
    lo, hi = random_boxes(rng, n, k)
    nc, labels = orc.clusters(lo, hi)
    bnc, blabels = brute_components(lo.tolist(), hi.tolist())
    assert nc == bnc and labels.tolist() == blabels


def test_orthant_boxes_around_a_grid_point_are_one_cluster(orc):
    """2^n boxes meeting only at a corner touch there: one cluster (as the boxes around a
    root on a split point do); shifted by a gap they are 2^n clusters."""
    n = 4
    lo, hi = [], []
    for c in itertools.product((0, 1), repeat=n):
        lo.append([(-1e-3 if b == 0 else 0.0) for b in c])
        hi.append([(0.0 if b == 0 else 1e-3) for b in c])
    assert orc.clusters(np.array(lo), np.array(hi))[0] == 1
    lo2 = np.array(lo) + np.array([[2e-3 * b for b in c] for c in itertools.product((0, 1), repeat=n)])
    hi2 = np.array(hi) + np.array([[2e-3 * b for b in c] for c in itertools.product((0, 1), repeat=n)])
    assert orc.clusters(lo2, hi2)[0] == 2 ** n


def test_n2_has_two_roots(orc):
    s = synth.config_n2()
    r = orc.solve(s)
    nc, labels = orc.clusters(r["lo"], r["hi"])
    assert nc == 2
    for k in range(2):
        mine = r["lo"][labels == k]
        assert np.all(np.sign(mine[:, 0]) == np.sign(mine[0, 0]))   # one cluster per sign of x


def exact_cells(lo, hi, d_lo, d_hi, level):
    """Exact rational version of the backtracking map for dyadic data."""
    side = 2 ** level
    cells = set()
    for bl, bh in zip(lo, hi):
        ranges = []
        for j in range(len(bl)):
            w = (Q(d_hi[j]) - Q(d_lo[j])) / side
            tl, th = (Q(bl[j]) - Q(d_lo[j])) / w, (Q(bh[j]) - Q(d_lo[j])) / w
            a, b = tl.numerator // tl.denominator, -((-th.numerator) // th.denominator) - 1
            x, y = min(a, b), max(a, b)
            x, y = max(x, 0), min(y, side - 1)
            if y < x:
                y = x
            if x > side - 1:
                x = y = side - 1
            ranges.append(range(x, y + 1))
        cells.update(itertools.product(*ranges))
    return len(cells)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_backtrack_equals_exact_on_dyadic_boxes(orc, level):
    rng = random.Random(100 + level)
    d_lo, d_hi = np.array([-4.0, -2.0, 0.0]), np.array([4.0, 2.0, 8.0])
    lo, hi = [], []
    for _ in range(50):
        l = [rng.randint(-32, 31) / 8.0, rng.randint(-16, 15) / 8.0, rng.randint(0, 63) / 8.0]
        w = [rng.choice([0, 1, 2, 4]) / 8.0 for _ in range(3)]
        lo.append(l)
        hi.append([l[0] + w[0], l[1] + w[1], l[2] + w[2]])
    lo, hi = np.array(lo), np.array(hi)
    assert orc.backtrack(lo, hi, d_lo, d_hi, level) == exact_cells(lo, hi, d_lo, d_hi, level)


def test_backtrack_of_grid_boxes_is_their_ancestors(orc):
    """Boxes that are cells of level 6 map at level L to their ancestor cells (index >> (6-L))."""
    rng = random.Random(9)
    d_lo, d_hi = np.array([-2.0, -2.0]), np.array([2.0, 2.0])
    idx = {(rng.randint(0, 63), rng.randint(0, 63)) for _ in range(40)}
    w = 4.0 / 64
    lo = np.array([[-2.0 + i * w, -2.0 + j * w] for i, j in idx])
    hi = lo + w
    for level in range(0, 7):
        want = len({(i >> (6 - level), j >> (6 - level)) for i, j in idx})
        assert orc.backtrack(lo, hi, d_lo, d_hi, level) == want
