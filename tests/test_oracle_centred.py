"""Pins of the oracle's centred (mean-value) form and of the solver with it as a second
exclusion test.

Paper: Section 2.3 eq 13 expands f about the midpoint, f(y) = f(x) + J(xi)(y - x) with
xi in X, so f_i(X) lies in F_c,i(X) = f_i(x) + sum_j J_ij(X)(X_j - x_j).
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth


def _exact_f(s, pt):
    out = []
    for i in range(s.n_eqs):
        acc = Q(0)
        for t in s.terms_of(i):
            m = Q(float(s.coef_lo[t]))
            for j in range(s.n_vars):
                m *= pt[j] ** int(s.exps[t, j])
            acc += m
        out.append(acc)
    return out


def _rand_box(rng, n, lo=-4.0, hi=4.0):
    blo, bhi = [], []
    for _ in range(n):
        w = math.exp(rng.uniform(math.log(1e-4), math.log(3.0)))
        c = rng.uniform(lo + w / 2, hi - w / 2)
        blo.append(c - w / 2)
        bhi.append(c + w / 2)
    return np.array(blo), np.array(bhi)


def test_square_closed_form(orc):
    """x^2 on [1, 3]: mid 2, f(2) = 4, J = [2, 6], X - 2 = [-1, 1]: F_c = [-2, 10]
    exactly (every step is exact in doubles)."""
    s = synth.parse_system(["x1^2"], 1)
    lo, hi = orc.centred(s, [1.0], [3.0])
    assert (lo[0], hi[0]) == (-2.0, 10.0)


def test_linear_is_tight(orc):
    """For f = a.x + c with dyadic data the centred form is the exact range (every
    operation exact), and equals the natural form."""
    s = synth.parse_system(["3*x1 - 2*x2 + 0.5*x3 - 1", "x1 + x2 + x3", "-x1 + 4*x3 + 2"], 3)
    lo = np.array([-1.0, 0.25, 2.0])
    hi = np.array([0.5, 1.75, 2.5])
    cl, ch = orc.centred(s, lo, hi)
    nl, nh = orc.eval_box(s, lo, hi)
    for i in range(3):
        vals = []
        for c in range(8):
            pt = [Q(float(hi[j] if (c >> j) & 1 else lo[j])) for j in range(3)]
            vals.append(_exact_f(s, pt)[i])
        assert Q(float(cl[i])) == min(vals) and Q(float(ch[i])) == max(vals), i
        assert cl[i] == nl[i] and ch[i] == nh[i]


@pytest.mark.parametrize("which", ["n6", "n10"])
def test_contains_exact_values(orc, which):
    """Every exact value f_i(p), p in X (corners and random points), lies in F_c,i(X)."""
    s = synth.config_n6() if which == "n6" else synth.config_n10()
    rng = random.Random(2024)
    for _ in range(40):
        lo, hi = _rand_box(rng, s.n_vars, float(s.box_lo[0]), float(s.box_hi[0]))
        cl, ch = orc.centred(s, lo, hi)
        pts = [[Q(float(lo[j])) for j in range(s.n_vars)], [Q(float(hi[j])) for j in range(s.n_vars)]]
        pts += [[Q(rng.uniform(float(lo[j]), float(hi[j]))) for j in range(s.n_vars)] for _ in range(6)]
        for pt in pts:
            v = _exact_f(s, pt)
            for i in range(s.n_eqs):
                assert Q(float(cl[i])) <= v[i] <= Q(float(ch[i])), (i, float(v[i]), cl[i], ch[i])


def test_tighter_than_natural_on_small_boxes(orc):
    """On narrow boxes the centred form's width shrinks quadratically faster than the
    natural form's overestimate: for the n=6 system on boxes of width 1e-3 it is the
    narrower of the two for most equations."""
    s = synth.config_n6()
    rng = random.Random(7)
    better = total = 0
    for _ in range(30):
        c = [rng.uniform(-3, 3) for _ in range(6)]
        lo = np.array(c) - 5e-4
        hi = np.array(c) + 5e-4
        cl, ch = orc.centred(s, lo, hi)
        nl, nh = orc.eval_box(s, lo, hi)
        better += int(np.sum((ch - cl) <= (nh - nl)))
        total += 6
    assert better >= 0.8 * total


def _rows(r):
    return {tuple(np.concatenate([a, b])) for a, b in zip(r["lo"], r["hi"])}


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_solver_result_is_a_subset(orc, seed):
    """Each box's fate depends only on the box, so the centred test only removes whole
    subtrees: the result with it is a subset of the result without it, the known roots
    stay enclosed, and the boxes it keeps are processed identically."""
    systems = synth.config_batched(count=6, seed=seed, n_range=(2, 4))
    removed = 0
    for s in systems:
        a = orc.solve(s, max_boxes=200_000)
        if a["status"] != 0:
            continue
        b = orc.solve(s, centred=True, max_boxes=200_000)
        assert b["status"] == 0
        assert _rows(b) <= _rows(a)
        assert b["stats"]["boxes"] <= a["stats"]["boxes"]
        removed += b["stats"]["excluded_centred"]
        for root in s.roots:
            pt = [float(v) for v in root]
            assert any(np.all(lo <= pt) and np.all(pt <= hi) for lo, hi in zip(b["lo"], b["hi"]))
    assert removed > 0


def test_closed_form_roots_with_centred(orc):
    s = synth.config_n2()
    r = orc.solve(s, centred=True)
    y = (math.sqrt(5) - 1) / 2
    for x in (math.sqrt(y), -math.sqrt(y)):
        assert any(lo[0] <= x <= hi[0] and lo[1] <= y <= hi[1] for lo, hi in zip(r["lo"], r["hi"]))


def test_centred_needs_a_square_system(orc):
    s = synth.parse_system(["x1 + x2 + x3"], 3)
    assert orc.solve(s, hs_enable=False, centred=True)["status"] == 1
