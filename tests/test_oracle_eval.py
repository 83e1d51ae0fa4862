"""Pins of the oracle's evaluation, Jacobian, Gauss-Jordan inverse and Hansen-Sengupta
sweep against exact arithmetic, closed forms and textbook special cases.

Paper: Definition 1-2 (interval evaluation, exclusion), Section 2.3 eq 14, 17-22 and
Algorithm 3 (Hansen-Sengupta), Section 2.4 eq 23-24 (Gauss-Jordan), Algorithm 4.
"""

import math
import random
from fractions import Fraction as Q

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth


def _rand_box(rng, n, lo=-4.0, hi=4.0):
    blo, bhi = [], []
    for _ in range(n):
        w = math.exp(rng.uniform(math.log(1e-6), math.log(3.0)))
        c = rng.uniform(lo + w / 2, hi - w / 2)
        blo.append(c - w / 2)
        bhi.append(c + w / 2)
    return np.array(blo), np.array(bhi)


def _sample_points(rng, lo, hi, count):
    pts = [[Q(float(lo[j])) for j in range(len(lo))], [Q(float(hi[j])) for j in range(len(lo))]]
    for _ in range(count):
        pts.append([Q(rng.uniform(float(lo[j]), float(hi[j]))) for j in range(len(lo))])
    return pts


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


def _exact_df(s, pt, i, j):
    acc = Q(0)
    for t in s.terms_of(i):
        a = int(s.exps[t, j])
        if a == 0:
            continue
        m = Q(float(s.coef_lo[t])) * a
        for jj in range(s.n_vars):
            e = int(s.exps[t, jj]) - (1 if jj == j else 0)
            m *= pt[jj] ** e
        acc += m
    return acc


def test_eval_contains_point_values(orc):
    """Definition 1: F(X) contains f(x) for every x in X (exact rational f)."""
    s = synth.config_n6()
    rng = random.Random(7)
    for _ in range(60):
        lo, hi = _rand_box(rng, 6)
        flo, fhi = orc.eval_box(s, lo, hi)
        for pt in _sample_points(rng, lo, hi, 6):
            for i, v in enumerate(_exact_f(s, pt)):
                assert Q(flo[i]) <= v <= Q(fhi[i])


def test_eval_linear_is_tight(orc):
    """For f = 3x - 5y + 2z - 7 the natural extension is the exact range rounded outward
    (at most a few ulps wider)."""
    s = synth.parse_system(["3*x1 - 5*x2 + 2*x3 - 7"], 3)
    rng = random.Random(8)
    for _ in range(200):
        lo, hi = _rand_box(rng, 3)
        (flo,), (fhi,) = orc.eval_box(s, lo, hi)
        elo = 3 * Q(lo[0]) - 5 * Q(hi[1]) + 2 * Q(lo[2]) - 7
        ehi = 3 * Q(hi[0]) - 5 * Q(lo[1]) + 2 * Q(hi[2]) - 7
        assert Q(flo) <= elo and ehi <= Q(fhi)
        slack = Q(8 * 2**-52) * (abs(elo) + abs(ehi) + 30)
        assert elo - Q(flo) <= slack and Q(fhi) - ehi <= slack


def test_eval_power_not_repeated_product(orc):
    """x^2 on [-1, 1] is [0, 1] (power rule), not x*x = [-1, 1]."""
    s = synth.parse_system(["x1^2"], 1)
    assert orc.eval_box(s, [-1.0], [1.0]) == (np.array([0.0]), np.array([1.0]))


def test_f32_encloses_f64(orc):
    """The FP32 prefilter form encloses the FP64 evaluation, so any box it drops FP64
    drops too (the prefilter cannot change the result set)."""
    rng = random.Random(9)
    for s in (synth.config_n6(), synth.config_n10()):
        for _ in range(400):
            lo, hi = _rand_box(rng, s.n_vars, -2.0, 2.0)
            dlo, dhi = orc.eval_box(s, lo, hi)
            flo, fhi = orc.eval_box_f32(s, lo, hi)
            assert np.all(flo.astype(np.float64) <= dlo) and np.all(fhi.astype(np.float64) >= dhi)


def test_jacobian_contains_derivatives(orc):
    s = synth.config_n6()
    rng = random.Random(11)
    for _ in range(25):
        lo, hi = _rand_box(rng, 6)
        jl, jh = orc.jacobian(s, lo, hi)
        for pt in _sample_points(rng, lo, hi, 3):
            for i in range(6):
                for j in range(6):
                    v = _exact_df(s, pt, i, j)
                    assert Q(jl[i, j]) <= v <= Q(jh[i, j])


def test_jacobian_closed_form(orc):
    """d/dx (x^3 y - 2 x) = 3 x^2 y - 2 and d/dy = x^3 on a point box: exact values."""
    s = synth.parse_system(["x1^3*x2 - 2*x1", "x1 + x2"], 2)
    jl, jh = orc.jacobian(s, [2.0, 3.0], [2.0, 3.0])
    assert jl[0, 0] == jh[0, 0] == 34.0 and jl[0, 1] == jh[0, 1] == 8.0
    assert jl[1, 0] == jh[1, 0] == 1.0 and jl[1, 1] == jh[1, 1] == 1.0


def test_gj_inverse_matches_numpy(orc):
    rng = np.random.default_rng(12)
    for n in range(1, 13):
        for _ in range(5):
            a = rng.normal(size=(n, n)) + n * np.eye(n)
            rc, inv = orc.gj_inverse(a)
            assert rc == 0
            ref = np.linalg.inv(a)
            assert np.max(np.abs(inv - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_gj_inverse_pivoting_and_singular(orc):
    p = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 2.0], [4.0, 0.0, 0.0]])
    rc, inv = orc.gj_inverse(p)
    assert rc == 0 and np.array_equal(inv, np.array([[0, 0, 0.25], [1, 0, 0], [0, 0.5, 0]]))
    rc, _ = orc.gj_inverse(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert rc == 1
    rc, _ = orc.gj_inverse(np.zeros((3, 3)))
    assert rc == 1


def test_hs_one_dimension_is_interval_newton(orc):
    """n = 1: one sweep is X cap (x - f(x)/F'(X)).  f = x^2 - 2 on [1, 2]: x = 1.5,
    f(x) = 0.25, F'(X) = [2, 4], so the exact step is [1.375, 1.4375]."""
    s = synth.parse_system(["x1^2 - 2"], 1)
    rc, lo, hi = orc.hs_step(s, [1.0], [2.0])
    assert rc == 0
    assert lo[0] <= 1.375 and hi[0] >= 1.4375
    assert 1.375 - lo[0] < 1e-14 and hi[0] - 1.4375 < 1e-14


def _newton_1d_exact(coefs, a, b):
    """Exact interval Newton step for f = sum c_k x^k on [a, b] with the natural extension
    of f' (power rule, exact), returning the list of exact pieces of X cap N."""
    m = (a + b) / 2
    fm = sum(c * m**k for k, c in enumerate(coefs))
    dlo = dhi = Q(0)
    for k, c in enumerate(coefs):
        if k == 0:
            continue
        kk = k - 1
        if kk == 0:
            plo = phi = Q(1)
        elif kk % 2 == 0 and a < 0 < b:
            plo, phi = Q(0), max(a**kk, b**kk)
        else:
            plo, phi = min(a**kk, b**kk), max(a**kk, b**kk)
        t = [c * k * plo, c * k * phi]
        dlo += min(t)
        dhi += max(t)
    if dlo > 0 or dhi < 0:
        qs = [fm / dlo, fm / dhi]
        n_lo, n_hi = m - max(qs), m - min(qs)
        lo, hi = max(a, n_lo), min(b, n_hi)
        return [] if lo > hi else [(lo, hi)]
    return None  # extended-division case, not compared here


def test_hs_one_dimension_random(orc):
    rng = random.Random(13)
    done = 0
    while done < 60:
        coefs = [Q(rng.randint(-6, 6)) for _ in range(4)]
        if coefs[3] == 0:
            continue
        s = synth.parse_system([" + ".join(f"{int(c)}*x1^{k}" if k else f"{int(c)}"
                                           for k, c in enumerate(coefs))], 1)
        a = Q(rng.randint(-16, 15), 4)
        b = a + Q(rng.randint(1, 8), 8)
        exact = _newton_1d_exact(coefs, a, b)
        if exact is None:
            continue
        rc, lo, hi = orc.hs_step(s, [float(a)], [float(b)])
        if not exact:
            # exact step empty: outward rounding may keep a sliver but never more
            assert rc == 1 or (hi[0] - lo[0] < 1e-12)
        else:
            assert rc == 0
            (elo, ehi), = exact
            assert Q(lo[0]) <= elo and ehi <= Q(hi[0])
            assert elo - Q(lo[0]) < Q(1, 10**10) and Q(hi[0]) - ehi < Q(1, 10**10)
        done += 1


def test_hs_linear_system_converges(orc):
    """For a linear system A x = b one sweep from a box around the solution contains
    the exact solution and shrinks to a few ulps (J(X) = A is thin, B A ~ I)."""
    rng = np.random.default_rng(14)
    for n in (2, 3, 5, 8):
        a = rng.integers(-4, 5, size=(n, n)) + 9 * np.eye(n, dtype=int)
        xs = [Q(int(v), 8) for v in rng.integers(-8, 9, size=n)]
        lines = []
        for i in range(n):
            b = sum(int(a[i, j]) * xs[j] for j in range(n))
            terms = [f"{int(a[i, j])}*x{j + 1}" for j in range(n) if a[i, j] != 0]
            lines.append(" + ".join(terms) + f" + {-b}")
        s = synth.parse_system(lines, n)
        lo = np.array([float(v) - 0.25 for v in xs])
        hi = np.array([float(v) + 0.3 for v in xs])
        rc, ol, oh = orc.hs_step(s, lo, hi)
        assert rc == 0
        for j in range(n):
            assert Q(ol[j]) <= xs[j] <= Q(oh[j])
            assert oh[j] - ol[j] < 1e-12


def test_hs_preserves_planted_root(orc):
    """Algorithm 3 output property 1: a root in X stays in the contracted box."""
    s = synth.config_n6()
    r = s.roots[0]
    rng = random.Random(15)
    contracted = 0
    for _ in range(80):
        w = 10 ** rng.uniform(-5, 0)
        lo = np.array([float(v) - w * rng.uniform(0.05, 0.95) for v in r])
        hi = lo + w
        assert all(Q(lo[j]) <= r[j] <= Q(hi[j]) for j in range(6))
        rc, ol, oh = orc.hs_step(s, lo, hi)
        assert rc != 1
        if rc == 0:
            assert all(Q(ol[j]) <= r[j] <= Q(oh[j]) for j in range(6))
            contracted += int(np.any(ol != lo) or np.any(oh != hi))
    assert contracted > 0


def test_hs_drops_root_free_box(orc):
    """x^2 - 2 = 0 has no root in [2, 3]: exclusion by evaluation alone already, and the
    sweep also returns the empty set."""
    s = synth.parse_system(["x1^2 - 2"], 1)
    rc, _, _ = orc.hs_step(s, [2.0], [3.0])
    assert rc == 1


def test_hs_sweep_that_changes_nothing_changes_nothing_again(orc):
    """The premise of stopping a visit's sweeps at the first sweep that leaves the box
    unchanged: the sweep is a function of the box, so the next one is identical."""
    rng = random.Random(77)
    for s in (synth.config_n2(), synth.config_n6()):
        for _ in range(20):
            lo, hi = _rand_box(rng, s.n_vars, float(s.box_lo[0]), float(s.box_hi[0]))
            for _ in range(12):
                rc, nlo, nhi = orc.hs_step(s, lo, hi)
                if rc != 0:
                    break
                if np.array_equal(nlo, lo) and np.array_equal(nhi, hi):
                    rc2, nlo2, nhi2 = orc.hs_step(s, nlo, nhi)
                    assert rc2 == 0 and np.array_equal(nlo2, nlo) and np.array_equal(nhi2, nhi)
                    break
                lo, hi = nlo, nhi
