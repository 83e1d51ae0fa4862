"""Seeded systems with dyadic data whose interval Jacobian is exact in doubles, and exact
rational interval arithmetic, for pinning the oracle's contraction steps.

f_i(x) = sum_j a_ij x_j + b_i x_i^2 - c_i with integer a_ij (diagonally dominant), b_i in
{+-1/2, +-1}, a dyadic root z and c chosen so that f(z) = 0 exactly.  On a box with dyadic
ends J(X) = A + diag(2 b_i X_i) is exact in doubles, and f at the exact midpoint is exact.
"""

from fractions import Fraction as Q

from paper_1802_00330_gb300 import synth


def exact_residual(s, pt):
    """f(pt) of a parsed system in exact rational arithmetic."""
    out = []
    for i in range(s.n_eqs):
        acc = Q(0)
        for t in s.terms_of(i):
            assert s.coef_lo[t] == s.coef_hi[t]
            m = Q(float(s.coef_lo[t]))
            for j in range(s.n_vars):
                m *= pt[j] ** int(s.exps[t, j])
            acc += m
        out.append(acc)
    return out


def _const(v):
    v = float(v)
    return f" - {v!r}" if v >= 0 else f" + {-v!r}"


def quadratic_system(rng, n):
    """(system, a, b, c, z) of the family above."""
    a = [[rng.randint(-3, 3) for _ in range(n)] for _ in range(n)]
    for i in range(n):
        a[i][i] = rng.choice([-1, 1]) * rng.randint(n + 2, n + 5)
    bq = [Q(rng.choice([-2, -1, 1, 2]), 2) for _ in range(n)]
    z = [Q(rng.randint(-48, 48), 32) for _ in range(n)]
    c = [sum(a[i][j] * z[j] for j in range(n)) + bq[i] * z[i] ** 2 for i in range(n)]
    lines = []
    for i in range(n):
        terms = [f"{a[i][j]}*x{j + 1}" for j in range(n) if a[i][j]]
        terms.append(f"{float(bq[i])!r}*x{i + 1}^2")
        lines.append(" + ".join(terms).replace("+ -", "- ") + _const(c[i]))
    s = synth.parse_system(lines, n)
    assert all(v == 0 for v in exact_residual(s, z))
    return s, a, bq, c, z


def linear_system(rng, n, cond_max=50.0):
    """(system, z) for f = A x - c with integer A (diagonally dominant, not symmetric)."""
    import numpy as np
    while True:
        a = [[rng.randint(-4, 4) for _ in range(n)] for _ in range(n)]
        for i in range(n):
            a[i][i] = rng.choice([-1, 1]) * rng.randint(n + 3, n + 6)
        if np.linalg.cond(np.array(a, float)) < cond_max and not np.allclose(a, np.transpose(a)):
            break
    z = [Q(rng.randint(-64, 64), 32) for _ in range(n)]
    c = [sum(a[i][j] * z[j] for j in range(n)) for i in range(n)]
    lines = []
    for i in range(n):
        terms = [f"{a[i][j]}*x{j + 1}" for j in range(n) if a[i][j]]
        lines.append(" + ".join(terms).replace("+ -", "- ") + _const(c[i]))
    s = synth.parse_system(lines, n)
    assert all(v == 0 for v in exact_residual(s, z))
    return s, z


# ---- exact rational intervals (pairs (lo, hi) of Fractions) ------------------------------
def iv_add(x, y):
    return (x[0] + y[0], x[1] + y[1])


def iv_sub(x, y):
    return (x[0] - y[1], x[1] - y[0])


def iv_mul(x, y):
    p = [x[0] * y[0], x[0] * y[1], x[1] * y[0], x[1] * y[1]]
    return (min(p), max(p))


def iv_div(x, y):
    """x / y for 0 not in y."""
    assert y[0] > 0 or y[1] < 0
    p = [x[0] / y[0], x[0] / y[1], x[1] / y[0], x[1] / y[1]]
    return (min(p), max(p))


def exact_jacobian(a, bq, X):
    n = len(a)
    J = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i != j:
                J[i][j] = (Q(a[i][j]), Q(a[i][j]))
            else:
                e = sorted([a[i][i] + 2 * bq[i] * X[i][0], a[i][i] + 2 * bq[i] * X[i][1]])
                J[i][j] = (e[0], e[1])
    return J


def exact_preconditioned(a, bq, c, B, lo, hi):
    """(X, x, J, M, r) in exact arithmetic: x the exact midpoint, M = B J(X), r = B f(x),
    with B the given double matrix taken exactly."""
    n = len(a)
    X = [(Q(float(lo[j])), Q(float(hi[j]))) for j in range(n)]
    x = [(l + h) / 2 for l, h in X]
    J = exact_jacobian(a, bq, X)
    fx = [sum(a[i][j] * x[j] for j in range(n)) + bq[i] * x[i] ** 2 - c[i] for i in range(n)]
    Bq = [[Q(float(B[i, u])) for u in range(n)] for i in range(n)]
    M = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            acc = (Q(0), Q(0))
            for u in range(n):
                acc = iv_add(acc, iv_mul((Bq[i][u], Bq[i][u]), J[u][j]))
            M[i][j] = acc
    r = [sum(Bq[i][u] * fx[u] for u in range(n)) for i in range(n)]
    return X, x, J, M, r
