"""Pins of the oracle's Krawczyk step and of the solver with it as the contraction.

Paper: Section 2.3 eq 15-16.  With x the midpoint of X, B an approximate inverse of
mid J(X), K(X) = x - B f(x) + [I - B J(X)](X - x); every root of f in X lies in K(X),
and the iteration keeps X intersected with K(X).

Pins (none retypes the oracle's double-precision code):
  * a 1-D worked example, x^2 - 2 on [1, 2], against its exact rational value;
  * linear systems, where the step is one Newton step: K(X) is a tiny box around the
    solution (a dropped identity term keeps X's width, a wrong sign of B f(x) misses it);
  * systems with quadratic diagonal terms and dyadic data, where J(X) is exact in doubles
    and K(X) is computed in exact rational interval arithmetic from the same B: the
    oracle's K(X) encloses it within a few units in the last place (a transposed or
    mis-signed term moves an end by about the box width);
  * containment of the planted root, and solves that find every planted root.
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

import _dyadic as D
from paper_1802_00330_gb300 import synth


def _ulps_close(a, exact, k=64):
    """|a - exact| within k units in the last place of max(|exact|, 1)."""
    scale = max(abs(float(exact)), 1.0)
    return abs(Q(float(a)) - exact) <= Q(k) * Q(math.ulp(scale))


def test_square_minus_two_worked_example(orc):
    """f = x^2 - 2 on X = [1, 2]: x = 3/2, f(x) = 1/4, J(X) = [2, 4], mid J = 3,
    B = RN(1/3) = b.  Exactly, K(X) = 3/2 - b/4 + (1 - b [2, 4]) [-1/2, 1/2]
    = [3/2 - b/4 - m, 3/2 - b/4 + m] with m = max(|1 - 4b|, |1 - 2b|) / 2."""
    s = synth.parse_system(["x1^2 - 2"], 1)
    rc, ol, oh, kl, kh = orc.kr_step(s, [1.0], [2.0])
    assert rc == 0
    b = Q(1.0 / 3.0)
    m = max(abs(1 - 4 * b), abs(1 - 2 * b)) / 2
    lo_x, hi_x = Q(3, 2) - b / 4 - m, Q(3, 2) - b / 4 + m
    assert Q(float(kl[0])) <= lo_x and hi_x <= Q(float(kh[0]))
    assert _ulps_close(kl[0], lo_x, 4) and _ulps_close(kh[0], hi_x, 4)
    # K(X) lies inside X, so the intersection is K(X) itself and holds sqrt(2)
    assert (ol[0], oh[0]) == (kl[0], kh[0])
    assert ol[0] < math.sqrt(2.0) < oh[0]


@pytest.mark.parametrize("n", [2, 3, 5])
def test_linear_system_is_one_newton_step(orc, n):
    """f = A z - c: J(X) = A, B = A^-1 to rounding, so K(X) collapses onto the solution."""
    rng = random.Random(100 + n)
    for _ in range(6):
        s, z = D.linear_system(rng, n)
        lo = np.array([float(zj) - rng.choice([0.25, 0.5, 0.75]) for zj in z])
        hi = lo + 1.0
        rc, ol, oh, kl, kh = orc.kr_step(s, lo, hi)
        assert rc == 0
        for j in range(n):
            assert Q(float(kl[j])) <= z[j] <= Q(float(kh[j]))
            assert kh[j] - kl[j] <= 1e-12, (j, kl[j], kh[j])
            assert (ol[j], oh[j]) == (kl[j], kh[j])


def _exact_krawczyk(a, bq, c, B, lo, hi):
    """K(X) of eq 15 in exact rational interval arithmetic (x the exact midpoint)."""
    n = len(a)
    X, x, J, M, r = D.exact_preconditioned(a, bq, c, B, lo, hi)
    K = []
    for i in range(n):
        k = (x[i] - r[i], x[i] - r[i])
        for j in range(n):
            d = Q(1 if i == j else 0)
            k = D.iv_add(k, D.iv_mul(D.iv_sub((d, d), M[i][j]), D.iv_sub(X[j], (x[j], x[j]))))
        K.append(k)
    return K, J


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_quadratic_systems_exact_enclosure(orc, n):
    rng = random.Random(7000 + n)
    for _ in range(8):
        s, a, bq, c, z = D.quadratic_system(rng, n)
        lo = np.array([float(zj) - rng.randint(1, 24) / 64 for zj in z])
        hi = np.array([float(zj) + rng.randint(1, 24) / 64 for zj in z])
        jl, jh = orc.jacobian(s, lo, hi)
        rc_b, B = orc.gj_inverse(0.5 * (jl + jh))
        assert rc_b == 0
        K, J = _exact_krawczyk(a, bq, c, B, lo, hi)
        for i in range(n):   # J(X) of this family is exact in doubles
            for j in range(n):
                assert (Q(float(jl[i, j])), Q(float(jh[i, j]))) == J[i][j]
        rc, ol, oh, kl, kh = orc.kr_step(s, lo, hi)
        assert rc in (0, 1)
        for i in range(n):
            assert Q(float(kl[i])) <= K[i][0] and K[i][1] <= Q(float(kh[i])), i
            assert _ulps_close(kl[i], K[i][0]) and _ulps_close(kh[i], K[i][1]), (i, kl[i], float(K[i][0]))
            # the planted root is in X, so it is in K(X) and the step cannot drop the box
            assert Q(float(kl[i])) <= z[i] <= Q(float(kh[i]))
        assert rc == 0
        for i in range(n):
            assert ol[i] == max(lo[i], kl[i]) and oh[i] == min(hi[i], kh[i])


def test_box_without_root_can_be_dropped(orc):
    """x1^2 - 2 on [1.5, 2]: K(X) lies left of X (x = 1.75, f(x) = 1.0625 > 0), the
    intersection is empty and the step reports it."""
    s = synth.parse_system(["x1^2 - 2"], 1)
    rc, ol, oh, kl, kh = orc.kr_step(s, [1.5], [2.0])
    assert rc == 1
    assert kh[0] < 1.5


@pytest.mark.parametrize("n", [2, 3, 4])
def test_solve_finds_planted_roots(orc, n):
    """The solver with the Krawczyk step returns boxes of width <= tol, one of which
    encloses the planted root."""
    rng = random.Random(900 + n)
    for _ in range(3):
        s, a, bq, c, z = D.quadratic_system(rng, n)
        box_lo = np.full(n, -4.0)
        box_hi = np.full(n, 4.0)
        r = orc.solve(s, box_lo=box_lo, box_hi=box_hi, tol=1e-6, krawczyk=True, hs_iters=4)
        assert r["status"] == 0
        st = r["stats"]
        assert st["hs_applied"] > 0 and st["hs_contracted"] > 0
        found = any(all(Q(float(r["lo"][k, j])) <= z[j] <= Q(float(r["hi"][k, j])) for j in range(n))
                    for k in range(len(r["lo"])))
        assert found
        assert np.all(r["hi"] - r["lo"] <= 1e-6)


def test_solve_root_free_is_empty(orc):
    s = synth.parse_system(["x1^2 + x2^2 + 1", "x1 - x2"], 2, box=(-3, 3), tol=1e-6)
    r = orc.solve(s, krawczyk=True)
    assert r["status"] == 0 and len(r["lo"]) == 0


def test_krawczyk_off_is_the_gauss_seidel_solver(orc):
    """krawczyk = False leaves the solver as it was (same boxes as the default call)."""
    s = synth.config_n2()
    a = orc.solve(s)
    b = orc.solve(s, krawczyk=False)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
