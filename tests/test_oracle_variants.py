"""Pins of the oracle's two split variants (Section 2.3 after eq 22; Algorithm 2).

Widest-coordinate bisection (split_mode = 1) in place of Algorithm 2's 2^n-way split:
* without contraction, on a box whose sides are equal, it accepts exactly the boxes the
  2^n split accepts, at n times the depth: interval evaluation is inclusion-monotone, so a
  cell of the 2^n grid survives its half-box ancestors exactly when it survives itself
  and its 2^n-split ancestors; a bisection of the narrowest side, a wrong half or a depth
  slip breaks the equality;
* at n = 1 the two splits are the same split, contraction included;
* known roots stay enclosed and the result does not depend on the processing order.

Two-box split on an extended-division gap (gap_split = 1):
* the textbook one-dimensional interval Newton step with extended division, in exact
  rationals: x^2 - 1 on [-2, 3] leaves [-2, 5/16] and [5/8, 3];
* on dyadic quadratic systems with boxes wide enough that M_ii contains 0, the sweep in
  exact rational interval arithmetic (same preconditioner) gives the rows' gaps; the
  oracle splits at the row with the widest one and its two boxes enclose the exact ones
  within a few hundred units in the last place; the other coordinates equal the hull
  sweep's;
* known roots stay enclosed and the result does not depend on the processing order.
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

import _dyadic as D
from paper_1802_00330_gb300 import synth


def _same(a, b, depth_scale=1):
    assert a["status"] == b["status"]
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
    assert np.array_equal(a["flags"], b["flags"])
    assert np.array_equal(a["depth"], depth_scale * b["depth"])


# ---- widest-coordinate bisection ---------------------------------------------------------

def test_bisection_equals_full_split_without_contraction(orc):
    systems = [synth.config_n2()] + synth.config_batched(count=8, seed=611, n_range=(2, 4))
    for s in systems:
        tol = float((s.box_hi[0] - s.box_lo[0]) / 2 ** 12)
        full = orc.solve(s, hs_enable=False, tol=tol)
        bis = orc.solve(s, hs_enable=False, tol=tol, split_mode=1)
        assert len(full["lo"]) > 0
        _same(bis, full, depth_scale=s.n_vars)
        assert bis["stats"]["boxes"] > full["stats"]["boxes"] / 2 ** s.n_vars


def test_bisection_is_the_full_split_in_one_dimension(orc):
    for eq, box in (("x1^2 - 2", (-3, 3)), ("x1^3 - 2*x1 + 0.5", (-2, 2.5)), ("x1^2 - 1", (-2, 3))):
        s = synth.parse_system([eq], 1, box=box, tol=1e-9)
        for kw in ({}, {"krawczyk": True}, {"hs_iters": 3}):
            _same(orc.solve(s, split_mode=1, **kw), orc.solve(s, **kw))


def test_bisection_keeps_known_roots(orc):
    s = synth.config_n2()
    r = orc.solve(s, split_mode=1)
    y = (math.sqrt(5) - 1) / 2
    for root in ((math.sqrt(y), y), (-math.sqrt(y), y)):
        inside = np.all((r["lo"] <= np.array(root) + 1e-15) & (np.array(root) - 1e-15 <= r["hi"]), axis=1)
        assert inside.any()
    assert orc.clusters(r["lo"], r["hi"])[0] == 2
    w = (r["hi"] - r["lo"]).max(axis=1)
    assert np.all(w[r["flags"] == 1] <= s.tol)
    for s in synth.config_batched(count=6, seed=612, n_range=(2, 4)):
        r = orc.solve(s, split_mode=1, tol=1e-5)
        z = np.array([float(v) for v in s.roots[0]])
        assert np.any(np.all((r["lo"] <= z) & (z <= r["hi"]), axis=1))


def test_bisection_is_order_independent(orc):
    for s in synth.config_batched(count=4, seed=613, n_range=(2, 4)):
        a = orc.solve(s, split_mode=1, tol=1e-5)
        for order, seed in ((1, 0), (2, 7)):
            _same(orc.solve(s, split_mode=1, tol=1e-5, order=order, order_seed=seed), a)


# ---- two-box split on a gap ----------------------------------------------------------------

def test_gap_step_textbook_newton_1d(orc):
    """x^2 - 1 on [-2, 3]: x = 1/2, f(x) = -3/4, F'(X) = [-4, 6] (mid 1, so B = 1);
    -3/4 / [-4, 6] = (-inf, -1/8] U [3/16, inf); x - that meets X in [-2, 5/16] and
    [5/8, 3] (all dyadic: exact)."""
    s = synth.parse_system(["x1^2 - 1"], 1)
    rc, boxes, row = orc.hs_gap_step(s, np.array([-2.0]), np.array([3.0]))
    assert rc == 3 and row == 0
    assert [(b[0][0], b[1][0]) for b in boxes] == [(-2.0, 0.3125), (0.625, 3.0)]
    # without the variant the same sweep returns the hull
    rc, lo, hi = orc.hs_step(s, np.array([-2.0]), np.array([3.0]))
    assert rc == 0 and (lo[0], hi[0]) == (-2.0, 3.0)


def _ext_pieces(S, Dd):
    """Exact extended division S / D for 0 in D (interior) and 0 not in S: two rays."""
    (s1, s2), (d1, d2) = S, Dd
    assert d1 < 0 < d2 and (s1 > 0 or s2 < 0)
    if s2 < 0:
        return [(None, s2 / d2), (s2 / d1, None)]
    return [(None, s1 / d1), (s1 / d2, None)]


def _exact_gap_sweep(a, bq, c, B, lo, hi):
    """Exact Gauss-Seidel sweep with extended division and the hull for later rows;
    returns (boxes, gaps) with gaps = {row: (gap, lower piece, upper piece)}, "empty"
    when a row leaves nothing, or None when a row's M_ii has an end exactly at 0 (a
    one-ray case outside this pin)."""
    n = len(a)
    X, x, J, M, r = D.exact_preconditioned(a, bq, c, B, lo, hi)
    Xp = list(X)
    gaps = {}
    for i in range(n):
        S = (r[i], r[i])
        for j in range(n):
            if j != i:
                S = D.iv_add(S, D.iv_mul(M[i][j], D.iv_sub(Xp[j], (x[j], x[j]))))
        Mi = M[i][i]
        if Mi[0] > 0 or Mi[1] < 0:
            Y = D.iv_sub((x[i], x[i]), D.iv_div(S, Mi))
            pieces = [(max(X[i][0], Y[0]), min(X[i][1], Y[1]))]
        elif S[0] <= 0 <= S[1]:
            pieces = [X[i]]            # 0 in S_i and in M_ii: the whole line (eq 10)
        else:
            if Mi[0] == 0 or Mi[1] == 0:
                return None
            pieces = []
            for p_lo, p_hi in _ext_pieces(S, Mi):
                y_lo = None if p_hi is None else x[i] - p_hi
                y_hi = None if p_lo is None else x[i] - p_lo
                pieces.append((X[i][0] if y_lo is None else max(X[i][0], y_lo),
                               X[i][1] if y_hi is None else min(X[i][1], y_hi)))
        pieces = sorted(p for p in pieces if p[0] <= p[1])
        if not pieces:
            return "empty"
        if len(pieces) == 2 and pieces[1][0] > pieces[0][1]:
            gaps[i] = (pieces[1][0] - pieces[0][1], pieces[0], pieces[1])
        Xp[i] = (pieces[0][0], pieces[-1][1])
    return Xp, gaps


def _near_empty(boxes):
    """An exactly empty row may survive outward rounding only as a sliver."""
    return all(np.min(b[1] - b[0]) <= 1e-9 * max(1.0, float(np.max(np.abs(b[0])))) for b in boxes)


def _encloses_close(lo, hi, exact, k=512):
    for j, (el, eh) in enumerate(exact):
        assert Q(float(lo[j])) <= el and eh <= Q(float(hi[j])), j
        for v, e in ((lo[j], el), (hi[j], eh)):
            assert abs(Q(float(v)) - e) <= Q(k) * Q(math.ulp(max(abs(float(e)), 1.0))), j


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gap_step_matches_exact_sweep(orc, n):
    rng = random.Random(9300 + n)
    split = 0
    for _ in range(80):
        s, a, bq, c, z = D.quadratic_system(rng, n)
        lo = np.array([float(zj) - rng.randint(64, 900) / 32 for zj in z])
        hi = np.array([float(zj) + rng.randint(64, 900) / 32 for zj in z])
        jl, jh = orc.jacobian(s, lo, hi)
        rc_b, B = orc.gj_inverse(0.5 * (jl + jh))
        if rc_b:
            continue
        ex = _exact_gap_sweep(a, bq, c, B, lo, hi)
        if ex is None:
            continue
        rc, boxes, row = orc.hs_gap_step(s, lo, hi)
        if ex == "empty":
            assert rc == 1 or (rc in (0, 3) and _near_empty(boxes))
            continue
        Xp, gaps = ex
        assert rc in (0, 3)
        if not gaps:
            continue
        ranked = sorted(gaps.items(), key=lambda kv: (-kv[1][0], kv[0]))
        best_row, (g, low, up) = ranked[0]
        if len(ranked) > 1 and ranked[0][1][0] - ranked[1][1][0] < Q(1, 1 << 30) * max(g, 1):
            continue   # two gaps too close to tell apart through rounding
        assert rc == 3 and row == best_row
        for box, piece in zip(boxes, (low, up)):
            exact = list(Xp)
            exact[best_row] = piece
            _encloses_close(box[0], box[1], exact)
        # every other coordinate is the hull sweep's
        rc_h, hlo, hhi = orc.hs_step(s, lo, hi)
        assert rc_h == 0
        for box in boxes:
            keep = [j for j in range(n) if j != row]
            assert np.array_equal(box[0][keep], hlo[keep]) and np.array_equal(box[1][keep], hhi[keep])
        split += 1
    assert split >= 3


def test_gap_split_solver_keeps_roots(orc):
    s = synth.parse_system(["x1^2 - 1"], 1, box=(-2, 3), tol=1e-10)
    r = orc.solve(s, gap_split=True)
    assert r["stats"]["gap_splits"] >= 1
    for root in (-1.0, 1.0):
        assert np.any((r["lo"][:, 0] <= root) & (root <= r["hi"][:, 0]))
    assert np.all(np.abs(np.abs(r["lo"][:, 0]) - 1) < 1e-9)
    s = synth.config_n2()
    g = orc.solve(s, gap_split=True)
    assert orc.clusters(g["lo"], g["hi"])[0] == 2
    splits = 0
    for s in synth.config_batched(count=8, seed=614, n_range=(2, 4)):
        r = orc.solve(s, gap_split=True, tol=1e-5)
        z = np.array([float(v) for v in s.roots[0]])
        assert np.any(np.all((r["lo"] <= z) & (z <= r["hi"]), axis=1))
        splits += r["stats"]["gap_splits"]
    assert splits > 0


def test_gap_split_is_order_independent(orc):
    for s in synth.config_batched(count=4, seed=615, n_range=(2, 4)):
        a = orc.solve(s, gap_split=True, tol=1e-5)
        for order, seed in ((1, 0), (2, 11)):
            _same(orc.solve(s, gap_split=True, tol=1e-5, order=order, order_seed=seed), a)
