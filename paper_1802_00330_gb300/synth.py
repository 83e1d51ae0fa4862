"""Seeded synthetic polynomial systems shaped like the paper's workloads.

The paper (Section 4, Tables 9-10) solves bounded polynomial systems with n = 2..9
variables, sparse monomials of low degree and integer or floating coefficients on
boxes [-b, b]^n with b in {1, ..., 32}.  Its 55-system test set is not available, so
every workload here is synthetic: a random sparse system whose constant terms are set
so that a chosen point on a dyadic grid is an exact root ("planted root").

This module is shared by the CUDA path's tests and bench and by the oracle's tests.
It holds no interval arithmetic and nothing of the solver: it only draws exponent
vectors and coefficients and checks the planted root exactly with ``fractions``.

System layout (sparse monomial form, the solver's input format):
    n_vars, n_eqs         ints
    eq_offsets  int32[n_eqs + 1]   terms of equation i are [eq_offsets[i], eq_offsets[i+1])
    coef_lo     float64[n_terms]   coefficient interval lower end
    coef_hi     float64[n_terms]   coefficient interval upper end (== coef_lo when exact)
    exps        uint8[n_terms, n_vars]  exponent of each variable in each term
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

SEED_BASE = 1802_00330


@dataclass
class PolySystem:
    n_vars: int
    n_eqs: int
    eq_offsets: np.ndarray
    coef_lo: np.ndarray
    coef_hi: np.ndarray
    exps: np.ndarray
    box_lo: np.ndarray
    box_hi: np.ndarray
    tol: float
    roots: list = field(default_factory=list)  # known exact roots, each a tuple of Fractions
    name: str = ""

    @property
    def n_terms(self) -> int:
        return int(self.eq_offsets[-1])

    def terms_of(self, i: int):
        return range(int(self.eq_offsets[i]), int(self.eq_offsets[i + 1]))

    def eval_exact(self, point) -> list:
        """Exact value of every equation at a rational point (coefficients must be exact)."""
        pt = [Fraction(v) for v in point]
        out = []
        for i in range(self.n_eqs):
            s = Fraction(0)
            for t in self.terms_of(i):
                c = Fraction(float(self.coef_lo[t]))
                m = Fraction(1)
                for j in range(self.n_vars):
                    a = int(self.exps[t, j])
                    if a:
                        m *= pt[j] ** a
                s += c * m
            out.append(s)
        return out


def monomials(n: int, max_deg: int):
    """All non-constant exponent vectors of total degree <= max_deg, in a fixed order."""
    out = []
    for d in range(1, max_deg + 1):
        for combo in itertools.combinations_with_replacement(range(n), d):
            e = [0] * n
            for j in combo:
                e[j] += 1
            out.append(tuple(e))
    return out


def _make_system(n, eq_terms, max_deg, coef_draw, root, rng, box_b, tol, name,
                 max_tries=200):
    """Draw a sparse system with the given root.  eq_terms[i] = monomials in eq i
    including the constant term.  Redraws until every variable occurs and the
    Jacobian at the root has condition number < 1e8."""
    mons = monomials(n, max_deg)
    for _ in range(max_tries):
        rows_exps = []
        rows_coef = []
        for k in eq_terms:
            k_nc = min(k - 1, len(mons))
            idx = rng.choice(len(mons), size=k_nc, replace=False)
            idx.sort()
            exps = [mons[q] for q in idx]
            coefs = [coef_draw() for _ in exps]
            rows_exps.append(exps)
            rows_coef.append(coefs)
        used = np.zeros(n, bool)
        for exps in rows_exps:
            for e in exps:
                used |= np.array(e) > 0
        if not used.all():
            continue
        # Jacobian at the root (float64 is enough for a conditioning check).
        r = np.array([float(v) for v in root])
        J = np.zeros((len(eq_terms), n))
        for i, (exps, coefs) in enumerate(zip(rows_exps, rows_coef)):
            for e, c in zip(exps, coefs):
                for j in range(n):
                    if e[j]:
                        ee = list(e)
                        ee[j] -= 1
                        J[i, j] += float(c) * e[j] * np.prod(r ** np.array(ee))
        if len(eq_terms) == n:
            try:
                if not np.isfinite(np.linalg.cond(J)) or np.linalg.cond(J) >= 1e8:
                    continue
            except np.linalg.LinAlgError:
                continue
        # Constant term: minus the exact value of the drawn terms at the root.
        offs = [0]
        all_exps = []
        all_coef = []
        for exps, coefs in zip(rows_exps, rows_coef):
            s = Fraction(0)
            for e, c in zip(exps, coefs):
                m = Fraction(1)
                for j in range(n):
                    if e[j]:
                        m *= Fraction(root[j]) ** e[j]
                s += Fraction(c) * m
            const = -s
            if Fraction(float(const)) != const:
                break  # not exactly representable; redraw
            for e, c in zip(exps, coefs):
                all_exps.append(e)
                all_coef.append(float(c))
            all_exps.append(tuple([0] * n))
            all_coef.append(float(const))
            offs.append(len(all_exps))
        else:
            coef = np.array(all_coef, dtype=np.float64)
            sysm = PolySystem(
                n_vars=n, n_eqs=len(eq_terms),
                eq_offsets=np.array(offs, dtype=np.int32),
                coef_lo=coef.copy(), coef_hi=coef.copy(),
                exps=np.array(all_exps, dtype=np.uint8).reshape(len(all_exps), n),
                box_lo=np.full(n, -float(box_b)), box_hi=np.full(n, float(box_b)),
                tol=tol, roots=[tuple(Fraction(v) for v in root)], name=name)
            assert all(v == 0 for v in sysm.eval_exact(root))
            return sysm
    raise RuntimeError("could not draw a well-conditioned system")


def _grid_root(rng, n, half_range, step=Fraction(1, 8)):
    k = int(half_range / step)
    return [step * int(rng.integers(-k, k + 1)) for _ in range(n)]


def _int_coef(rng, lo=-5, hi=5):
    def draw():
        while True:
            c = int(rng.integers(lo, hi + 1))
            if c != 0:
                return c
    return draw


def config_n2() -> PolySystem:
    """x^2 + y^2 - 1 = 0, x^2 - y = 0 on [-2,2]^2, tol 1e-8 (two real roots,
    y = (sqrt5 - 1)/2, x = +-sqrt(y))."""
    exps = np.array([[2, 0], [0, 2], [0, 0], [2, 0], [0, 1]], dtype=np.uint8)
    coef = np.array([1.0, 1.0, -1.0, 1.0, -1.0])
    return PolySystem(n_vars=2, n_eqs=2, eq_offsets=np.array([0, 3, 5], dtype=np.int32),
                      coef_lo=coef.copy(), coef_hi=coef.copy(), exps=exps,
                      box_lo=np.array([-2.0, -2.0]), box_hi=np.array([2.0, 2.0]),
                      tol=1e-8, roots=[], name="n2_circle_parabola")


def config_n6(seed: int = SEED_BASE + 1) -> PolySystem:
    """6 equations x 8 monomials (7 drawn + constant), degree <= 3, integer coefficients
    in [-5,5]\\{0}, planted root on the 1/8 grid in [-3,3]^6, box [-4,4]^6, tol 1e-6."""
    rng = np.random.default_rng(seed)
    root = _grid_root(rng, 6, 3)
    return _make_system(6, [8] * 6, 3, _int_coef(rng), root, rng, 4, 1e-6, "n6_sparse_deg3")


def config_n10(seed: int = SEED_BASE + 2) -> PolySystem:
    """10 equations x 12 monomials, degree <= 4, coefficients k/2^20 uniform in [-1,1],
    planted root on the 1/8 grid in [-1.5,1.5]^10, box [-2,2]^10, tol 1e-6."""
    rng = np.random.default_rng(seed)
    root = _grid_root(rng, 10, Fraction(3, 2))

    def draw():
        while True:
            k = int(rng.integers(-(1 << 20), (1 << 20) + 1))
            if k != 0:
                return Fraction(k, 1 << 20)
    return _make_system(10, [12] * 10, 4, draw, root, rng, 2, 1e-6, "n10_sparse_deg4")


def config_batched(count: int = 4096, seed: int = SEED_BASE + 3, n_range=(2, 8)):
    """`count` systems: n ~ U{2..8}, m = n, 4-10 monomials per equation, degree <= 3,
    integer coefficients in [-5,5], planted root on the 1/8 grid in [-3,3]^n,
    box [-4,4]^n, tol 1e-6."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        nm = len(monomials(n, 3)) + 1
        eq_terms = [min(int(rng.integers(4, 11)), nm) for _ in range(n)]
        root = _grid_root(rng, n, 3)
        out.append(_make_system(n, eq_terms, 3, _int_coef(rng), root, rng, 4, 1e-6,
                                f"batched_{s}_n{n}"))
    return out


def config_served(duration_s: float = 60.0, rate: float = 2000.0,
                  seed: int = SEED_BASE + 4, n_range=(3, 12), max_requests=None):
    """Poisson arrivals (mean `rate` req/s over `duration_s`) of systems with
    n ~ U{3..12}, degree <= 4, 6-14 monomials per equation, integer coefficients in
    [-5,5], planted root on the 1/8 grid in [-1.5,1.5]^n, box [-2,2]^n, tol 1e-6.
    Returns (arrival_times_s, systems)."""
    rng = np.random.default_rng(seed)
    times = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        times.append(t)
        if max_requests is not None and len(times) >= max_requests:
            break
    systems = []
    for s in range(len(times)):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        nm = len(monomials(n, 4)) + 1
        eq_terms = [min(int(rng.integers(6, 15)), nm) for _ in range(n)]
        root = _grid_root(rng, n, Fraction(3, 2))
        systems.append(_make_system(n, eq_terms, 4, _int_coef(rng), root, rng, 2, 1e-6,
                                    f"served_{s}_n{n}"))
    return np.array(times), systems


def served_systems(count: int, seed: int = SEED_BASE + 5, n_range=(3, 12)):
    """The first `count` requests of the served recipe (n ~ U{3..12}, degree <= 4, 6-14
    monomials per equation, integer coefficients in [-5,5], planted root on the 1/8 grid
    in [-1.5,1.5]^n, box [-2,2]^n, tol 1e-6), drawn from a generator of their own so
    that request k is the same system whatever arrival process carries it."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        nm = len(monomials(n, 4)) + 1
        eq_terms = [min(int(rng.integers(6, 15)), nm) for _ in range(n)]
        root = _grid_root(rng, n, Fraction(3, 2))
        out.append(_make_system(n, eq_terms, 4, _int_coef(rng), root, rng, 2, 1e-6, f"request_{s}_n{n}"))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = SEED_BASE + 6):
    """Arrival times (seconds from 0) of `count` requests of a Poisson stream of mean
    `rate` requests per second: cumulative exponential gaps from a seeded generator."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def random_boxes(rng, n, count, lo=-4.0, hi=4.0, min_w=1e-6, max_w=2.0):
    """Random boxes inside [lo,hi]^n with widths log-uniform in [min_w, max_w]
    (dyadic-friendly values are not forced; endpoints are arbitrary doubles)."""
    w = np.exp(rng.uniform(np.log(min_w), np.log(max_w), size=(count, n)))
    c = rng.uniform(lo + w / 2, hi - w / 2)
    return c - w / 2, c + w / 2


def _dir_round(q: Fraction):
    """(largest double <= q, smallest double >= q) for an exact rational q."""
    import math
    d = float(q)
    lo = d if Fraction(d) <= q else math.nextafter(d, -math.inf)
    hi = d if Fraction(d) >= q else math.nextafter(d, math.inf)
    return lo, hi


def parse_system(lines, n_vars, box=None, tol=1e-6, name=""):
    """Build a system from plain-text equations such as ``2*x9^2 + x1*x2 - 1.1*x1 + 1``
    (variables x1..xn, terms in the written order, each equation = 0).  A decimal
    coefficient that is not a double becomes the tightest enclosing double interval."""
    import re
    offs = [0]
    exps, clo, chi = [], [], []
    for ln in lines:
        s = ln.replace(" ", "")
        if s[0] not in "+-":
            s = "+" + s
        for sign, body in re.findall(r"([+-])([^+-]+)", s):
            e = [0] * n_vars
            coef = Fraction(1)
            for f in body.split("*"):
                m = re.fullmatch(r"x(\d+)(?:\^(\d+))?", f)
                if m:
                    e[int(m.group(1)) - 1] += int(m.group(2) or 1)
                else:
                    coef *= Fraction(f)
            if sign == "-":
                coef = -coef
            lo, hi = _dir_round(coef)
            exps.append(e)
            clo.append(lo)
            chi.append(hi)
        offs.append(len(exps))
    if box is None:
        box = (-1.0, 1.0)
    return PolySystem(n_vars=n_vars, n_eqs=len(lines), eq_offsets=np.array(offs, np.int32),
                      coef_lo=np.array(clo), coef_hi=np.array(chi),
                      exps=np.array(exps, np.uint8).reshape(len(exps), n_vars),
                      box_lo=np.full(n_vars, float(box[0])), box_hi=np.full(n_vars, float(box[1])),
                      tol=tol, name=name)


def load_fixture(path):
    """Read a text fixture: 'vars n', 'box lo hi', optional 'round_boxes ...', 'eq ...'."""
    meta = {}
    eqs = []
    for raw in open(path):
        ln = raw.strip()
        if not ln or ln.startswith("#"):
            continue
        key, _, rest = ln.partition(" ")
        if key == "eq":
            eqs.append(rest)
        else:
            meta[key] = rest.split()
    n = int(meta["vars"][0])
    box = tuple(float(v) for v in meta["box"])
    s = parse_system(eqs, n, box=box, name=path)
    s.meta = meta
    return s
