"""Exact-rational pin of the oracle's Gauss-Seidel sweep (Section 2.3 eq 21-22, Algorithm 4
for M and r, eq 10 for the division).

On the dyadic systems of `_dyadic`, J(X) is exact in doubles and f at the midpoint is exact,
so with the oracle's preconditioner B (any B is valid) the sweep can be carried out in exact
rational interval arithmetic: S_i = r_i + sum_{j != i} M_ij (X'_j - x_j) with X'_j the
updated coordinate for j < i, Y_i = x_i - S_i / M_ii, X'_i = X_i intersected with Y_i.  The
oracle's box must enclose the exact one (outward rounding is inclusion-monotone) and lie
within a few hundred units in the last place of it.  A transposed M, an index taken from the
wrong row, a fold that uses X_j instead of X'_j, or a sign slip in r each move an end by
about the box width times |M_ij| and fail.
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

import _dyadic as D


def _close(a, exact, k=256):
    scale = max(abs(float(exact)), 1.0)
    return abs(Q(float(a)) - exact) <= Q(k) * Q(math.ulp(scale))


def _exact_sweep(a, bq, c, B, lo, hi):
    """Exact Gauss-Seidel sweep; None when some M_ii contains 0 (not this pin's case),
    'empty' when an intersection is empty."""
    n = len(a)
    X, x, J, M, r = D.exact_preconditioned(a, bq, c, B, lo, hi)
    if any(M[i][i][0] <= 0 <= M[i][i][1] for i in range(n)):
        return None
    Xp = list(X)
    for i in range(n):
        S = (r[i], r[i])
        for j in range(n):
            if j != i:
                S = D.iv_add(S, D.iv_mul(M[i][j], D.iv_sub(Xp[j], (x[j], x[j]))))
        Y = D.iv_sub((x[i], x[i]), D.iv_div(S, M[i][i]))
        lo_i, hi_i = max(X[i][0], Y[0]), min(X[i][1], Y[1])
        if lo_i > hi_i:
            return "empty"
        Xp[i] = (lo_i, hi_i)
    return Xp


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_sweep_encloses_exact_sweep_around_root(orc, n):
    rng = random.Random(8100 + n)
    checked = 0
    for _ in range(10):
        s, a, bq, c, z = D.quadratic_system(rng, n)
        lo = np.array([float(zj) - rng.randint(1, 24) / 64 for zj in z])
        hi = np.array([float(zj) + rng.randint(1, 24) / 64 for zj in z])
        jl, jh = orc.jacobian(s, lo, hi)
        rc_b, B = orc.gj_inverse(0.5 * (jl + jh))
        assert rc_b == 0
        ex = _exact_sweep(a, bq, c, B, lo, hi)
        if ex is None:
            continue
        assert ex != "empty"           # the planted root is in X, hence in X'
        rc, ol, oh = orc.hs_step(s, lo, hi)
        assert rc == 0
        contracted = False
        for i in range(n):
            assert Q(float(ol[i])) <= ex[i][0] and ex[i][1] <= Q(float(oh[i])), i
            assert _close(ol[i], ex[i][0]) and _close(oh[i], ex[i][1]), (i, ol[i], float(ex[i][0]))
            assert Q(float(ol[i])) <= z[i] <= Q(float(oh[i]))
            contracted |= (ol[i], oh[i]) != (lo[i], hi[i])
        assert contracted
        checked += 1
    assert checked >= 6


@pytest.mark.parametrize("n", [2, 3, 4])
def test_sweep_off_root_boxes(orc, n):
    """Boxes shifted off the root (some still contain it): where the exact sweep empties
    the box the oracle may keep a sliver only within rounding; where it does not, the oracle
    keeps the box and encloses the exact one tightly (it never drops a box the exact sweep
    keeps)."""
    rng = random.Random(8200 + n)
    seen_empty = seen_kept = 0
    for _ in range(100):
        s, a, bq, c, z = D.quadratic_system(rng, n)
        off = [rng.choice([-1, 1]) * rng.randint(1, 16) / 64 for _ in range(n)]
        w = [rng.randint(1, 16) / 64 for _ in range(n)]
        lo = np.array([float(z[j]) + off[j] - w[j] for j in range(n)])
        hi = np.array([float(z[j]) + off[j] + w[j] for j in range(n)])
        jl, jh = orc.jacobian(s, lo, hi)
        rc_b, B = orc.gj_inverse(0.5 * (jl + jh))
        if rc_b != 0:
            continue
        ex = _exact_sweep(a, bq, c, B, lo, hi)
        if ex is None:
            continue
        rc, ol, oh = orc.hs_step(s, lo, hi)
        if ex == "empty":
            seen_empty += 1
            if rc == 0:   # kept only by rounding: some coordinate is a sliver at an end
                assert any(oh[i] - ol[i] <= 1e-12 * max(1.0, abs(ol[i])) for i in range(n))
            continue
        seen_kept += 1
        assert rc == 0
        for i in range(n):
            assert Q(float(ol[i])) <= ex[i][0] and ex[i][1] <= Q(float(oh[i])), i
            assert _close(ol[i], ex[i][0]) and _close(oh[i], ex[i][1])
    assert seen_empty >= 5 and seen_kept >= 3
