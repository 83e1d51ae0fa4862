"""Pins of the oracle's interval primitives against exact rational arithmetic.

Each directed operation must equal the exact result rounded down (lower end) or up
(upper end), computed here with ``fractions.Fraction`` and ``math.nextafter`` --
a mechanism independent of fesetround.  Paper: Section 2.2 eq 5-10 and
Section 3.2 eq 25-27.
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

INF = math.inf


def rd(q: Q) -> float:
    d = float(q)
    return d if Q(d) <= q else math.nextafter(d, -INF)


def ru(q: Q) -> float:
    d = float(q)
    return d if Q(d) >= q else math.nextafter(d, INF)


def _vals(rng, count):
    out = [0.0, -0.0, 1.0, -1.0, 0.5, 3.0, -7.0, 1e-300, -2.5e-310, 1 + 2**-52, -(1 + 2**-52),
           0.1, -0.3, 1e16, 4.0]
    for _ in range(count):
        e = rng.randint(-40, 40)
        out.append(rng.uniform(-1, 1) * 2.0**e)
    return out


def _ivals(rng, count):
    vs = _vals(rng, 2 * count)
    out = []
    for a, b in zip(vs[0::2], vs[1::2]):
        out.append((min(a, b), max(a, b)))
    out += [(0.0, 0.0), (-1.0, 0.0), (0.0, 2.0), (-3.0, 5.0), (1.0, 1.0), (-2.0, -1e-3)]
    return out


def exact_mul(x, y):
    ps = [Q(a) * Q(b) for a in x for b in y]
    return min(ps), max(ps)


def test_add_sub_directed(orc):
    rng = random.Random(1)
    ivs = _ivals(rng, 120)
    for x in ivs:
        for y in rng.sample(ivs, 12):
            lo, hi = orc.iv_op(orc.OP_ADD, x, y)
            assert lo == rd(Q(x[0]) + Q(y[0])) and hi == ru(Q(x[1]) + Q(y[1]))
            lo, hi = orc.iv_op(orc.OP_SUB, x, y)
            assert lo == rd(Q(x[0]) - Q(y[1])) and hi == ru(Q(x[1]) - Q(y[0]))


def test_mul_directed(orc):
    rng = random.Random(2)
    ivs = _ivals(rng, 120)
    for x in ivs:
        for y in rng.sample(ivs, 12):
            lo, hi = orc.iv_op(orc.OP_MUL, x, y)
            elo, ehi = exact_mul(x, y)
            assert lo == rd(elo) and hi == ru(ehi), (x, y, lo, hi)


def test_div_directed(orc):
    rng = random.Random(3)
    ivs = _ivals(rng, 120)
    for x in ivs:
        for y in rng.sample(ivs, 12):
            if not (y[0] > 0 or y[1] < 0):
                with pytest.raises(ValueError):
                    orc.iv_op(orc.OP_DIV, x, y)
                continue
            lo, hi = orc.iv_op(orc.OP_DIV, x, y)
            qs = [Q(a) / Q(b) for a in x for b in y]
            assert lo == rd(min(qs)) and hi == ru(max(qs)), (x, y)


def _chain(x: float, k: int, r):
    p = x
    for _ in range(k - 1):
        p = r(Q(p) * Q(x))
    return p


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_pow_rule(orc, k):
    """Power rule: monotone chains per end; pinned to the chain computed with exact
    rationals, and to enclosure/tightness of the exact range of x^k."""
    rng = random.Random(10 + k)
    for x in _ivals(rng, 150):
        lo, hi = orc.iv_op(orc.OP_POW, x, k=k)
        a, b = Q(x[0]), Q(x[1])
        cands = [a**k, b**k] + ([Q(0)] if a <= 0 <= b else [])
        elo, ehi = min(cands), max(cands)
        assert lo <= elo and hi >= ehi                      # encloses the exact range
        if k % 2 == 0:
            if x[0] >= 0:
                want = (_chain(x[0], k, rd), _chain(x[1], k, ru))
            elif x[1] <= 0:
                want = (_chain(-x[1], k, rd), _chain(-x[0], k, ru))
            else:
                want = (0.0, _chain(max(-x[0], x[1]), k, ru))
        else:
            wl = _chain(x[0], k, rd) if x[0] >= 0 else -_chain(-x[0], k, ru)
            wh = _chain(x[1], k, ru) if x[1] >= 0 else -_chain(-x[1], k, rd)
            want = (wl, wh)
        assert (lo, hi) == want
        # each chain step loses at most one ulp: relative slack <= k * 2^-52
        mag = max(abs(elo), abs(ehi))
        if mag > 1e-280:
            assert elo - Q(lo) <= mag * Q(k, 2**52) and Q(hi) - ehi <= mag * Q(k, 2**52)


def test_pow_small_k(orc):
    assert orc.iv_op(orc.OP_POW, (-3.0, 2.0), k=0) == (1.0, 1.0)
    assert orc.iv_op(orc.OP_POW, (-3.0, 2.0), k=1) == (-3.0, 2.0)
    assert orc.iv_op(orc.OP_POW, (-3.0, 2.0), k=2) == (0.0, 9.0)
    assert orc.iv_op(orc.OP_POW, (-3.0, 2.0), k=3) == (-27.0, 8.0)


def _in_pieces(v: Q, pieces):
    for lo, hi in pieces:
        if (lo == -INF or Q(lo) <= v) and (hi == INF or v <= Q(hi)):
            return True
    return False


def test_extended_division_cases(orc):
    """eq 10: every quotient of points x in X, y in Y (y != 0) lies in the pieces; the
    finite ends are the outward-rounded exact quotients of the bounding endpoints."""
    cases = [
        ((-3.0, -1.0), (-2.0, 0.0), [(rd(Q(-1) / Q(-2)), INF)]),
        ((-3.0, -1.0), (-2.0, 5.0), [(-INF, ru(Q(-1) / Q(5))), (rd(Q(-1) / Q(-2)), INF)]),
        ((-3.0, -1.0), (0.0, 5.0), [(-INF, ru(Q(-1) / Q(5)))]),
        ((1.0, 3.0), (-2.0, 0.0), [(-INF, ru(Q(1) / Q(-2)))]),
        ((1.0, 3.0), (-2.0, 5.0), [(-INF, ru(Q(1) / Q(-2))), (rd(Q(1) / Q(5)), INF)]),
        ((1.0, 3.0), (0.0, 5.0), [(rd(Q(1) / Q(5)), INF)]),
        ((0.1, 0.3), (-0.7, 0.3), [(-INF, ru(Q(0.1) / Q(-0.7))), (rd(Q(0.1) / Q(0.3)), INF)]),
        ((-1.0, 2.0), (-1.0, 1.0), [(-INF, INF)]),
        ((0.0, 2.0), (0.0, 1.0), [(-INF, INF)]),
        ((1.0, 2.0), (0.0, 0.0), []),
        ((-2.0, -1.0), (-0.0, 0.0), []),
    ]
    for x, y, want in cases:
        got = orc.extdiv(x, y)
        assert got == want, (x, y, got)
    rng = random.Random(5)
    for x, y, _ in cases:
        pieces = orc.extdiv(x, y)
        for _ in range(200):
            xs = Q(rng.uniform(x[0], x[1]))
            ys = Q(rng.uniform(y[0], y[1]))
            if ys == 0:
                continue
            assert _in_pieces(xs / ys, pieces)


def test_extended_division_ordinary(orc):
    rng = random.Random(6)
    for x in _ivals(rng, 50):
        for y in _ivals(rng, 20):
            if not (y[0] > 0 or y[1] < 0):
                continue
            (lo, hi), = orc.extdiv(x, y)
            assert (lo, hi) == orc.iv_op(orc.OP_DIV, x, y)
