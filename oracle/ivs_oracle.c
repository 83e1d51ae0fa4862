/*
 * ivs_oracle.c -- plain, slow, serial CPU oracle for the per-box sweep of the
 * interval branch-and-bound + Hansen-Sengupta solver (Lin & Chen, "An efficient
 * algorithm for global interval solution of nonlinear algebraic equations and its
 * GPGPU implementation").
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the package smoke check and the bench's
 * CPU-baseline leg.  The CUDA library neither includes nor links it, and it shares no
 * code with the CUDA library.
 *
 * Paper map:
 *   interval +, -, x, / ........ Section 2.2 eq 5-9, directed forms Section 3.2 eq 25-27
 *   extended division .......... Section 2.2 eq 10
 *   interval evaluation F(X) ... Section 2.2 Definition 1; exclusion test Definition 2
 *   Hansen-Sengupta sweep ...... Section 2.3 eq 14, 17-22; Algorithm 3
 *   interval matrix product .... Algorithm 4 (with outward rounding, eq 14's remark)
 *   Gauss-Jordan inverse ....... Section 2.4 eq 23-24
 *   split / driver ............. Algorithm 1, Algorithm 2
 * Readings where the paper is silent or garbled are stated at each function.
 *
 * Every directed operation is a single IEEE operation under fesetround(); point
 * operations use round-to-nearest.  Build: -O2 -frounding-math -ffp-contract=off.
 */
#include "ivs_oracle.h"

#include <fenv.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* FENV_ACCESS: gcc honours the dynamic rounding mode with -frounding-math; every
 * directed operation also goes through volatile operands and results. */

/* ------------------------------------------------------------------------------ */
/* Directed-rounding scalar operations (Section 3.2: "rd" and "ru").               */
/* ------------------------------------------------------------------------------ */

static double op_dir(int mode, int op, double a, double b) {
    volatile double x = a, y = b;
    volatile double r;
    fesetround(mode);
    switch (op) {
    case 0: r = x + y; break;
    case 1: r = x - y; break;
    case 2: r = x * y; break;
    default: r = x / y; break;
    }
    fesetround(FE_TONEAREST);
    return r;
}
static double add_rd(double a, double b) { return op_dir(FE_DOWNWARD, 0, a, b); }
static double add_ru(double a, double b) { return op_dir(FE_UPWARD, 0, a, b); }
static double sub_rd(double a, double b) { return op_dir(FE_DOWNWARD, 1, a, b); }
static double sub_ru(double a, double b) { return op_dir(FE_UPWARD, 1, a, b); }
static double mul_rd(double a, double b) { return op_dir(FE_DOWNWARD, 2, a, b); }
static double mul_ru(double a, double b) { return op_dir(FE_UPWARD, 2, a, b); }
static double div_rd(double a, double b) { return op_dir(FE_DOWNWARD, 3, a, b); }
static double div_ru(double a, double b) { return op_dir(FE_UPWARD, 3, a, b); }

static double dmin(double a, double b) { return b < a ? b : a; }
static double dmax(double a, double b) { return b > a ? b : a; }

typedef struct { double lo, hi; } ivl;

/* eq 25 */
static ivl iv_add(ivl x, ivl y) { ivl r = {add_rd(x.lo, y.lo), add_ru(x.hi, y.hi)}; return r; }
/* eq 26 */
static ivl iv_sub(ivl x, ivl y) { ivl r = {sub_rd(x.lo, y.hi), sub_ru(x.hi, y.lo)}; return r; }
/* eq 27: lower end = least of the four endpoint products rounded down, upper end =
 * greatest of them rounded up.  rd/ru are monotone, so rounding each product and then
 * taking min/max equals rounding the exact min/max. */
static ivl iv_mul(ivl x, ivl y) {
    double l1 = mul_rd(x.lo, y.lo), l2 = mul_rd(x.hi, y.lo), l3 = mul_rd(x.lo, y.hi), l4 = mul_rd(x.hi, y.hi);
    double u1 = mul_ru(x.lo, y.lo), u2 = mul_ru(x.hi, y.lo), u3 = mul_ru(x.lo, y.hi), u4 = mul_ru(x.hi, y.hi);
    ivl r = {dmin(dmin(l1, l2), dmin(l3, l4)), dmax(dmax(u1, u2), dmax(u3, u4))};
    return r;
}
/* eq 8-9 with 0 not in y.  Reading: the four endpoint quotients are rounded directly
 * (tighter than x * (1/y), and the same operation count on both sides). */
static ivl iv_div(ivl x, ivl y) {
    double l1 = div_rd(x.lo, y.lo), l2 = div_rd(x.hi, y.lo), l3 = div_rd(x.lo, y.hi), l4 = div_rd(x.hi, y.hi);
    double u1 = div_ru(x.lo, y.lo), u2 = div_ru(x.hi, y.lo), u3 = div_ru(x.lo, y.hi), u4 = div_ru(x.hi, y.hi);
    ivl r = {dmin(dmin(l1, l2), dmin(l3, l4)), dmax(dmax(u1, u2), dmax(u3, u4))};
    return r;
}

/* Powers.  The paper evaluates with +, -, x only (Section 3.2) and does not say how
 * x^k is formed.  Reading: the standard power rule, built from monotone chains
 * p <- x, then (k-1) times p <- r(p * x) with one rounding direction r, applied to
 * nonnegative arguments:
 *   k even: lo >= 0 -> [down(lo), up(hi)];  hi <= 0 -> [down(-hi), up(-lo)];
 *           otherwise [0, up(max(-lo, hi))]
 *   k odd : each end separately; a negative end v maps to -(opposite chain of -v). */
static double chain_rd(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = mul_rd(p, x); return p; }
static double chain_ru(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = mul_ru(p, x); return p; }

static ivl iv_pow(ivl x, int k) {
    ivl r;
    if (k == 0) { r.lo = 1.0; r.hi = 1.0; return r; }
    if (k == 1) return x;
    if ((k & 1) == 0) {
        if (x.lo >= 0) { r.lo = chain_rd(x.lo, k); r.hi = chain_ru(x.hi, k); }
        else if (x.hi <= 0) { r.lo = chain_rd(-x.hi, k); r.hi = chain_ru(-x.lo, k); }
        else { r.lo = 0.0; r.hi = chain_ru(dmax(-x.lo, x.hi), k); }
    } else {
        r.lo = x.lo >= 0 ? chain_rd(x.lo, k) : -chain_ru(-x.lo, k);
        r.hi = x.hi >= 0 ? chain_ru(x.hi, k) : -chain_rd(-x.hi, k);
    }
    return r;
}

/* Extended division x / y (eq 10, Hanson / Kahan), pieces with infinite ends.
 * Readings of the garbled table:
 *  - 0 not in y: ordinary division (iv_div).
 *  - 0 in x and 0 in y: the whole line.
 *  - y = [0,0] and 0 not in x: empty.
 *  - x entirely negative (hi < 0):  y = [c,0]: [hi/c, +inf);  c < 0 < d: (-inf, hi/d] u [hi/c, +inf);
 *                                   y = [0,d]: (-inf, hi/d].
 *  - x entirely positive (lo > 0):  y = [c,0]: (-inf, lo/c];  c < 0 < d: (-inf, lo/c] u [lo/d, +inf);
 *                                   y = [0,d]: [lo/d, +inf)   (eq 10's last case reads "lo <= 0",
 *                                   a typo for lo >= 0).
 *  Finite ends round outward: a lower end down, an upper end up.
 * Returns the number of pieces (0, 1 or 2). */
static int iv_extdiv(ivl x, ivl y, ivl *p) {
    const double inf = INFINITY;
    if (y.lo > 0 || y.hi < 0) { p[0] = iv_div(x, y); return 1; }
    if (x.lo <= 0 && x.hi >= 0) { p[0].lo = -inf; p[0].hi = inf; return 1; }
    if (y.lo == 0 && y.hi == 0) return 0;
    if (x.hi < 0) {
        if (y.hi == 0) { p[0].lo = div_rd(x.hi, y.lo); p[0].hi = inf; return 1; }
        if (y.lo == 0) { p[0].lo = -inf; p[0].hi = div_ru(x.hi, y.hi); return 1; }
        p[0].lo = -inf; p[0].hi = div_ru(x.hi, y.hi);
        p[1].lo = div_rd(x.hi, y.lo); p[1].hi = inf;
        return 2;
    }
    /* x.lo > 0 */
    if (y.hi == 0) { p[0].lo = -inf; p[0].hi = div_ru(x.lo, y.lo); return 1; }
    if (y.lo == 0) { p[0].lo = div_rd(x.lo, y.hi); p[0].hi = inf; return 1; }
    p[0].lo = -inf; p[0].hi = div_ru(x.lo, y.lo);
    p[1].lo = div_rd(x.lo, y.hi); p[1].hi = inf;
    return 2;
}

/* ------------------------------------------------------------------------------ */
/* Natural interval extension of the system (Definition 1)                         */
/* ------------------------------------------------------------------------------ */

/* One term c * prod_j X_j^{a_j}: the product folds left over j = 0..n-1 for the
 * variables with a_j > 0 (each factor by iv_pow), then the coefficient interval
 * multiplies the product.  A constant term is its coefficient interval. */
static ivl term_value(int n, const uint8_t *e, ivl c, const ivl *X) {
    int have = 0;
    ivl p = {0, 0};
    for (int j = 0; j < n; j++) {
        if (e[j] == 0) continue;
        ivl f = iv_pow(X[j], e[j]);
        p = have ? iv_mul(p, f) : f;
        have = 1;
    }
    if (!have) return c;
    return iv_mul(c, p);
}

/* F_i(X): left fold of interval additions over the terms of equation i in input order,
 * starting from the first term; an equation without terms is [0,0]. */
static void eval_system(const orc_system *s, const ivl *X, ivl *F) {
    for (int i = 0; i < s->n_eqs; i++) {
        ivl acc = {0, 0};
        int have = 0;
        for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
            ivl c = {s->coef_lo[t], s->coef_hi[t]};
            ivl v = term_value(s->n_vars, s->exps + (size_t)t * s->n_vars, c, X);
            acc = have ? iv_add(acc, v) : v;
            have = 1;
        }
        F[i] = acc;
    }
}

/* Definition 2: the box is a configuration of f_i iff 0 is in F_i(X).  A NaN end
 * proves nothing, so the box is dropped only when an end is a number on the wrong
 * side of 0. */
static int excluded(const ivl *F, int m) {
    for (int i = 0; i < m; i++)
        if (F[i].lo > 0 || F[i].hi < 0) return 1;
    return 0;
}

/* J_ij(X) = sum over terms t of equation i with a_tj > 0 of
 *           [down(c_lo a_tj), up(c_hi a_tj)] * X^(a_t - e_j),
 * folded left in term order (the same term rule as F); [0,0] when no term has x_j. */
static void jacobian(const orc_system *s, const ivl *X, ivl *J) {
    int n = s->n_vars;
    uint8_t e[256];
    for (int i = 0; i < s->n_eqs; i++) {
        for (int j = 0; j < n; j++) {
            ivl acc = {0, 0};
            int have = 0;
            for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
                const uint8_t *a = s->exps + (size_t)t * n;
                if (a[j] == 0) continue;
                ivl c = {mul_rd(s->coef_lo[t], (double)a[j]), mul_ru(s->coef_hi[t], (double)a[j])};
                memcpy(e, a, (size_t)n);
                e[j] -= 1;
                ivl v = term_value(n, e, c, X);
                acc = have ? iv_add(acc, v) : v;
                have = 1;
            }
            J[i * n + j] = acc;
        }
    }
}

/* ------------------------------------------------------------------------------ */
/* Gauss-Jordan inverse (Section 2.4), round to nearest                            */
/* ------------------------------------------------------------------------------ */

/* [C] = [A | I_n]; for k = 1..n: pick the pivot row as the first row i >= k holding
 * the largest |C_ik|, swap it into row k, divide row k by the pivot over columns
 * j = k..2n (eq 23), then for every other row i subtract C_ik * (row k) over columns
 * j = k+1..2n (eq 24) and set C_ik = 0.  The right half is then A^-1.
 * Readings: the printed loop bounds "k = 1..n-1" and "j = k+1" in eq 23 are taken as
 * k = 1..n and j = k..2n.  A zero or non-finite pivot means "singular". */
static int gj_inverse(int n, const double *A, double *B) {
    int w = 2 * n;
    double *C = (double *)malloc(sizeof(double) * (size_t)n * (size_t)w);
    if (!C) return 1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < w; j++)
            C[i * w + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int k = 0; k < n; k++) {
        int piv = k;
        double best = fabs(C[k * w + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(C[i * w + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > 0) || !isfinite(best)) { free(C); return 1; }
        if (piv != k)
            for (int j = 0; j < w; j++) { double t = C[k * w + j]; C[k * w + j] = C[piv * w + j]; C[piv * w + j] = t; }
        double p = C[k * w + k];
        for (int j = k; j < w; j++) C[k * w + j] = C[k * w + j] / p;
        for (int i = 0; i < n; i++) {
            if (i == k) continue;
            double f = C[i * w + k];
            for (int j = k + 1; j < w; j++) C[i * w + j] = C[i * w + j] - f * C[k * w + j];
            C[i * w + k] = 0.0;
        }
    }
    int bad = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            B[i * n + j] = C[i * w + n + j];
            if (!isfinite(B[i * n + j])) bad = 1;
        }
    free(C);
    return bad;
}

/* ------------------------------------------------------------------------------ */
/* Hansen-Sengupta sweep (Section 2.3, eq 14 and 17-22; Algorithm 3)               */
/* ------------------------------------------------------------------------------ */

static double midpoint(double lo, double hi) { return 0.5 * (lo + hi); }  /* eq 2.5, RN */

/* Centred (mean-value) form.  Section 2.3 eq 13 expands f about the point x:
 * f(y) = f(x) + J(xi)(y - x) with xi in X, so for every y in X and x = mid X,
 * f_i(y) lies in F_c,i(X) = f_i(x) + sum_j J_ij(X) (X_j - x_j).  Computed with the same
 * J(X), the same thin-box f(x) at the RN midpoint and the same outward operations as the
 * Hansen-Sengupta step; the sum is a left fold over j = 1..n starting from f_i(x). */
static void centred_form(const orc_system *s, const ivl *X, ivl *Fc) {
    int n = s->n_vars;
    size_t nn = (size_t)n * (size_t)n;
    ivl *J = (ivl *)malloc(sizeof(ivl) * nn);
    ivl *xc = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *fx = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    if (!J || !xc || !fx) {
        for (int i = 0; i < n; i++) { Fc[i].lo = -INFINITY; Fc[i].hi = INFINITY; }
    } else {
        jacobian(s, X, J);
        for (int j = 0; j < n; j++) { double m = midpoint(X[j].lo, X[j].hi); xc[j].lo = m; xc[j].hi = m; }
        eval_system(s, xc, fx);
        for (int i = 0; i < n; i++) {
            ivl acc = fx[i];
            for (int j = 0; j < n; j++) acc = iv_add(acc, iv_mul(J[i * n + j], iv_sub(X[j], xc[j])));
            Fc[i] = acc;
        }
    }
    free(J); free(xc); free(fx);
}

/* One Gauss-Seidel sweep on the preconditioned linearisation B f(x) + B J(X)(z - x) = 0:
 *   x   = mid(X) (round to nearest, the same midpoint used to split),
 *   B   = Gauss-Jordan inverse of mid(J(X)) (mid of each entry, round to nearest),
 *   M   = B J(X), r = B F(x) (Algorithm 4: products rounded outward, the lower sum
 *         accumulated downward and the upper sum upward, u = 1..n in order),
 *   for i = 1..n (eq 21, 22):
 *     S_i = r_i + sum_{j<i} M_ij (X'_j - x_j) + sum_{j>i} M_ij (X_j - x_j)   (left fold)
 *     Y_i = x_i - S_i / M_ii  (extended division, eq 10)
 *     X'_i = hull(X_i intersected with Y_i); empty -> the box holds no root.
 * Readings: Algorithm 3's "P_i = R(x) - sum", "N_i = x_i + P_i / M_ii" has the sign of
 * r wrong and drops its index; eq 21 is followed.  When Y_i has two pieces X'_i is the
 * hull of the two intersections.  A NaN in S_i or M_ii leaves X'_i = X_i.
 * Returns 0 (out written), 1 (empty), 2 (skipped: mid(J) singular or B non-finite).
 *
 * With kr = 1 the contraction is Krawczyk's instead (eq 15, 16), from the same x, B, M
 * and r: K_i = (x_i - r_i) + sum_j ((I - M)_ij (X_j - x_j)), a left fold over j = 1..n
 * with (I - M)_ij = [d_ij, d_ij] - M_ij (d the Kronecker delta), every row from the
 * incoming box X (no row uses another row's result), then X'_i = X_i intersected with
 * K_i; a NaN in K_i leaves X'_i = X_i, an empty intersection in any row drops the box.
 * K (if not NULL) receives K(X) before the intersection.
 *
 * With gap = 1 (the variant after eq 22: split the box where the extended division leaves
 * a gap, instead of taking the hull) a Gauss-Seidel row whose Y_i meets X_i in two
 * pieces records the gap between them, RN(lower end of the upper piece - upper end of
 * the lower piece); later rows still use the hull.  If some row left a gap wider than 0,
 * the row with the widest one (the first of equal ones) splits the swept box in two:
 * Xo takes the lower piece in that coordinate and Xo2 the upper one (*gap_row = the
 * row), and the return value is 3. */
static int hs_sweep(const orc_system *s, const ivl *X, ivl *Xo, int kr, ivl *K, int gap, ivl *Xo2,
                    int *gap_row) {
    int n = s->n_vars;
    size_t nn = (size_t)n * (size_t)n;
    ivl *J = (ivl *)malloc(sizeof(ivl) * nn);
    ivl *M = (ivl *)malloc(sizeof(ivl) * nn);
    double *A = (double *)malloc(sizeof(double) * nn);
    double *B = (double *)malloc(sizeof(double) * nn);
    ivl *xc = (ivl *)calloc((size_t)n, sizeof(ivl));
    ivl *fx = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *r = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    int status = 0;
    if (!J || !M || !A || !B || !xc || !fx || !r) { status = 2; goto done; }

    jacobian(s, X, J);
    for (size_t q = 0; q < nn; q++) {
        A[q] = midpoint(J[q].lo, J[q].hi);
        if (!isfinite(A[q])) { status = 2; goto done; }
    }
    if (gj_inverse(n, A, B)) { status = 2; goto done; }
    for (int j = 0; j < n; j++) { double m = midpoint(X[j].lo, X[j].hi); xc[j].lo = m; xc[j].hi = m; }
    eval_system(s, xc, fx);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            ivl acc = {0, 0};
            for (int u = 0; u < n; u++) {
                ivl b = {B[i * n + u], B[i * n + u]};
                acc = iv_add(acc, iv_mul(b, J[u * n + j]));
            }
            M[i * n + j] = acc;
        }
        ivl acc = {0, 0};
        for (int u = 0; u < n; u++) {
            ivl b = {B[i * n + u], B[i * n + u]};
            acc = iv_add(acc, iv_mul(b, fx[u]));
        }
        r[i] = acc;
    }
    for (int j = 0; j < n; j++) Xo[j] = X[j];
    if (kr) {
        int empty = 0;
        for (int i = 0; i < n; i++) {
            ivl Ki = iv_sub(xc[i], r[i]);
            for (int j = 0; j < n; j++) {
                ivl d = {i == j ? 1.0 : 0.0, i == j ? 1.0 : 0.0};
                Ki = iv_add(Ki, iv_mul(iv_sub(d, M[i * n + j]), iv_sub(X[j], xc[j])));
            }
            if (K) K[i] = Ki;
            if (isnan(Ki.lo) || isnan(Ki.hi)) continue;
            double a = dmax(X[i].lo, Ki.lo), b = dmin(X[i].hi, Ki.hi);
            if (a <= b) { Xo[i].lo = a; Xo[i].hi = b; }
            else empty = 1;
        }
        status = empty;
        goto done;
    }
    double best_gap = 0;
    int best_row = -1;
    ivl gap_lower = {0, 0}, gap_upper = {0, 0};
    for (int i = 0; i < n; i++) {
        ivl S = r[i];
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            S = iv_add(S, iv_mul(M[i * n + j], iv_sub(Xo[j], xc[j])));
        }
        ivl D = M[i * n + i];
        if (isnan(S.lo) || isnan(S.hi) || isnan(D.lo) || isnan(D.hi)) continue;
        ivl Np[2], piece[2];
        int np = iv_extdiv(S, D, Np);
        double lo = INFINITY, hi = -INFINITY;
        int any = 0;
        for (int q = 0; q < np; q++) {
            ivl Y = iv_sub(xc[i], Np[q]);
            double a = dmax(X[i].lo, Y.lo), b = dmin(X[i].hi, Y.hi);
            if (a <= b) { lo = dmin(lo, a); hi = dmax(hi, b); piece[any].lo = a; piece[any].hi = b; any++; }
        }
        if (!any) { status = 1; goto done; }
        if (gap && any == 2) {
            int u = piece[1].lo < piece[0].lo ? 0 : 1;   /* the upper piece */
            double g = piece[u].lo - piece[1 - u].hi;     /* round to nearest */
            if (g > best_gap) { best_gap = g; best_row = i; gap_lower = piece[1 - u]; gap_upper = piece[u]; }
        }
        Xo[i].lo = lo;
        Xo[i].hi = hi;
    }
    if (best_row >= 0) {
        for (int j = 0; j < n; j++) Xo2[j] = Xo[j];
        Xo[best_row] = gap_lower;
        Xo2[best_row] = gap_upper;
        *gap_row = best_row;
        status = 3;
    }
done:
    free(J); free(M); free(A); free(B); free(xc); free(fx); free(r);
    return status;
}

/* ------------------------------------------------------------------------------ */
/* Driver (Algorithm 1) with the split of Algorithm 2                              */
/* ------------------------------------------------------------------------------ */

struct orc_result {
    int status;
    int n;
    int64_t count, cap;
    double *lo, *hi;
    int32_t *flags, *depth;
    orc_stats st;
    int64_t depth_boxes[ORC_MAX_DEPTH_STATS], depth_kept[ORC_MAX_DEPTH_STATS];
};

typedef struct { double *lo, *hi; int32_t *depth; int64_t size, cap, head; } stack_t_;

static int stack_push(stack_t_ *q, int n, const double *lo, const double *hi, int32_t d) {
    if (q->size == q->cap) {
        int64_t nc = q->cap ? q->cap * 2 : 1024;
        double *nl = (double *)realloc(q->lo, sizeof(double) * (size_t)(nc * n));
        if (!nl) return 1;
        q->lo = nl;
        double *nh = (double *)realloc(q->hi, sizeof(double) * (size_t)(nc * n));
        if (!nh) return 1;
        q->hi = nh;
        int32_t *nd = (int32_t *)realloc(q->depth, sizeof(int32_t) * (size_t)nc);
        if (!nd) return 1;
        q->depth = nd;
        q->cap = nc;
    }
    memcpy(q->lo + q->size * n, lo, sizeof(double) * (size_t)n);
    memcpy(q->hi + q->size * n, hi, sizeof(double) * (size_t)n);
    q->depth[q->size] = d;
    q->size++;
    return 0;
}

static int result_push(orc_result *r, const ivl *X, int32_t flag, int32_t depth) {
    int n = r->n;
    if (r->count == r->cap) {
        int64_t nc = r->cap ? r->cap * 2 : 256;
        double *nl = (double *)realloc(r->lo, sizeof(double) * (size_t)(nc * n));
        if (!nl) return 1;
        r->lo = nl;
        double *nh = (double *)realloc(r->hi, sizeof(double) * (size_t)(nc * n));
        if (!nh) return 1;
        r->hi = nh;
        int32_t *nf = (int32_t *)realloc(r->flags, sizeof(int32_t) * (size_t)nc);
        if (!nf) return 1;
        r->flags = nf;
        int32_t *nd = (int32_t *)realloc(r->depth, sizeof(int32_t) * (size_t)nc);
        if (!nd) return 1;
        r->depth = nd;
        r->cap = nc;
    }
    for (int j = 0; j < n; j++) {
        /* canonical zero: -0 -> +0 */
        r->lo[r->count * n + j] = X[j].lo == 0 ? 0.0 : X[j].lo;
        r->hi[r->count * n + j] = X[j].hi == 0 ? 0.0 : X[j].hi;
    }
    r->flags[r->count] = flag;
    r->depth[r->count] = depth;
    r->count++;
    return 0;
}

static uint64_t splitmix(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int validate(const orc_system *s, const double *lo, const double *hi, const orc_options *o) {
    if (!s || !lo || !hi || !o) return 1;
    if (s->n_vars <= 0 || s->n_vars > 16 || s->n_eqs <= 0 || s->n_terms < 0) return 1;
    if (!s->eq_offsets || s->eq_offsets[0] != 0 || s->eq_offsets[s->n_eqs] != s->n_terms) return 1;
    for (int i = 0; i < s->n_eqs; i++) if (s->eq_offsets[i + 1] < s->eq_offsets[i]) return 1;
    for (int t = 0; t < s->n_terms; t++) {
        if (!isfinite(s->coef_lo[t]) || !isfinite(s->coef_hi[t]) || s->coef_lo[t] > s->coef_hi[t]) return 1;
        for (int j = 0; j < s->n_vars; j++) if (s->exps[(size_t)t * s->n_vars + j] > 15) return 1;
    }
    for (int j = 0; j < s->n_vars; j++) if (!isfinite(lo[j]) || !isfinite(hi[j]) || lo[j] > hi[j]) return 1;
    if ((o->hs_enable || o->centred) && s->n_eqs != s->n_vars) return 1;
    if (o->split_mode < 0 || o->split_mode > 1 || o->gap_split < 0 || o->gap_split > 1) return 1;
    if (!(o->tol >= 0) || !isfinite(o->tol) || o->hs_iters < 0 || o->max_depth < 0) return 1;
    return 0;
}

/* comparator context of the final sort: per thread, so solves may run concurrently */
static _Thread_local int cmp_box_n;
static _Thread_local const double *cmp_lo, *cmp_hi;
static int cmp_idx(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    for (int j = 0; j < cmp_box_n; j++) {
        double x = cmp_lo[a * cmp_box_n + j], y = cmp_lo[b * cmp_box_n + j];
        if (x < y) return -1;
        if (x > y) return 1;
        x = cmp_hi[a * cmp_box_n + j]; y = cmp_hi[b * cmp_box_n + j];
        if (x < y) return -1;
        if (x > y) return 1;
    }
    return 0;
}

/* Algorithm 1 termination (II) and the split for a box that survived evaluation and
 * contraction: accept it at the desired width, or when its widest coordinate cannot be
 * split in doubles, or return it flagged at the depth limit, or push its children --
 * Algorithm 2's 2^n children (child c takes the upper half of coordinate j when bit j
 * of c is set) or, with split_mode = 1, the two halves of its widest coordinate (the
 * first of equal widths).  Returns 0, or 1 when memory ran out. */
static int finish_box(orc_result *res, stack_t_ *q, const ivl *X, int n, int32_t depth, const orc_options *o,
                      double *mid, double *clo, double *chi, int *depth_cut) {
    double w = 0;
    int jw = 0;
    for (int j = 0; j < n; j++) {
        double wj = X[j].hi - X[j].lo;
        if (wj > w) { w = wj; jw = j; }
    }
    if (w <= o->tol) {
        if (result_push(res, X, ORC_ACCEPT_WIDTH, depth)) return 1;
        res->st.accepted++;
        return 0;
    }
    for (int j = 0; j < n; j++) mid[j] = midpoint(X[j].lo, X[j].hi);
    if (mid[jw] == X[jw].lo || mid[jw] == X[jw].hi) {
        if (result_push(res, X, ORC_ACCEPT_UNSPLITTABLE, depth)) return 1;
        res->st.accepted++;
        res->st.unsplittable++;
        return 0;
    }
    if (depth + 1 > o->max_depth) {
        /* depth cut: the box is returned unsplit, flagged, and the solve is incomplete */
        if (result_push(res, X, ORC_ACCEPT_DEPTH_LIMIT, depth)) return 1;
        *depth_cut = 1;
        return 0;
    }
    res->st.split++;
    if (o->split_mode == 1) {
        for (int c = 0; c < 2; c++) {
            for (int j = 0; j < n; j++) { clo[j] = X[j].lo; chi[j] = X[j].hi; }
            if (c) clo[jw] = mid[jw];
            else chi[jw] = mid[jw];
            if (stack_push(q, n, clo, chi, depth + 1)) return 1;
        }
        return 0;
    }
    for (int64_t c = 0; c < ((int64_t)1 << n); c++) {
        for (int j = 0; j < n; j++) {
            if ((c >> j) & 1) { clo[j] = mid[j]; chi[j] = X[j].hi; }
            else { clo[j] = X[j].lo; chi[j] = mid[j]; }
        }
        if (stack_push(q, n, clo, chi, depth + 1)) return 1;
    }
    return 0;
}

int orc_solve(const orc_system *s, const double *box_lo, const double *box_hi,
              const orc_options *o, orc_result **out) {
    *out = NULL;
    orc_result *res = (orc_result *)calloc(1, sizeof(orc_result));
    if (!res) return ORC_ERR_NOMEM;
    *out = res;
    if (validate(s, box_lo, box_hi, o)) { res->status = ORC_ERR_INVALID; return res->status; }
    int n = s->n_vars, m = s->n_eqs;
    res->n = n;
    stack_t_ q = {0};
    ivl *X = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *Xn = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *X2 = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *F = (ivl *)malloc(sizeof(ivl) * (size_t)m);
    double *clo = (double *)malloc(sizeof(double) * (size_t)n);
    double *chi = (double *)malloc(sizeof(double) * (size_t)n);
    double *mid = (double *)malloc(sizeof(double) * (size_t)n);
    uint64_t rng = o->order_seed;
    int status = ORC_OK, depth_cut = 0;
    if (!X || !Xn || !X2 || !F || !clo || !chi || !mid || stack_push(&q, n, box_lo, box_hi, o->root_depth)) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    while (q.size > q.head) {
        if (o->max_boxes > 0 && res->st.boxes >= o->max_boxes) { status = ORC_ERR_BUDGET; break; }
        int64_t k;
        if (o->order == 1) k = q.head;                     /* FIFO */
        else if (o->order == 2) k = q.head + (int64_t)(splitmix(&rng) % (uint64_t)(q.size - q.head));
        else k = q.size - 1;                               /* LIFO */
        int32_t depth = q.depth[k];
        for (int j = 0; j < n; j++) { X[j].lo = q.lo[k * n + j]; X[j].hi = q.hi[k * n + j]; }
        if (o->order == 1) {
            q.head++;
            if (q.head > 4096 && q.head * 2 > q.size) {     /* compact the consumed prefix */
                int64_t live = q.size - q.head;
                memmove(q.lo, q.lo + q.head * n, sizeof(double) * (size_t)(live * n));
                memmove(q.hi, q.hi + q.head * n, sizeof(double) * (size_t)(live * n));
                memmove(q.depth, q.depth + q.head, sizeof(int32_t) * (size_t)live);
                q.size = live;
                q.head = 0;
            }
        } else {
            int64_t last = q.size - 1;
            if (k != last) {
                memcpy(q.lo + k * n, q.lo + last * n, sizeof(double) * (size_t)n);
                memcpy(q.hi + k * n, q.hi + last * n, sizeof(double) * (size_t)n);
                q.depth[k] = q.depth[last];
            }
            q.size--;
        }
        res->st.boxes++;
        if (depth > res->st.max_depth_seen) res->st.max_depth_seen = depth;
        int dslot = depth < ORC_MAX_DEPTH_STATS ? depth : ORC_MAX_DEPTH_STATS - 1;
        res->depth_boxes[dslot]++;

        /* Algorithm 2, last step / Definition 2: drop boxes where some F_i excludes 0 */
        eval_system(s, X, F);
        if (excluded(F, m)) { res->st.excluded_eval++; continue; }

        /* optional second exclusion test: the centred form (eq 13) */
        if (o->centred) {
            centred_form(s, X, F);
            if (excluded(F, m)) { res->st.excluded_centred++; continue; }
        }

        /* Algorithm 1 step (III): Hansen-Sengupta contraction */
        int two = 0;   /* the sweep split the box at a gap: X and X2 go on */
        if (o->hs_enable && depth >= o->hs_min_depth) {
            int dropped = 0;
            for (int it = 0; it < (o->hs_iters > 0 ? o->hs_iters : 1); it++) {
                res->st.hs_applied++;
                int gap_row = -1;
                int rc = hs_sweep(s, X, Xn, o->krawczyk, NULL, o->gap_split && !o->krawczyk, X2, &gap_row);
                if (rc == 1) { dropped = 1; break; }
                if (rc == 2) { res->st.hs_singular++; break; }
                if (rc == 3) {
                    res->st.hs_contracted++;
                    res->st.gap_splits++;
                    memcpy(X, Xn, sizeof(ivl) * (size_t)n);
                    two = 1;
                    break;
                }
                int changed = 0;
                for (int j = 0; j < n; j++)
                    if (Xn[j].lo != X[j].lo || Xn[j].hi != X[j].hi) changed = 1;
                if (changed) res->st.hs_contracted++;
                memcpy(X, Xn, sizeof(ivl) * (size_t)n);
                /* iterated until the contraction stalls (Section 2.3): a sweep that leaves
                 * the box unchanged would leave it unchanged again */
                if (!changed) break;
            }
            if (dropped) { res->st.hs_empty++; continue; }
        }
        res->depth_kept[dslot]++;

        /* Algorithm 1 termination (II) and Algorithm 2's split, for X (and X2) */
        if (finish_box(res, &q, X, n, depth, o, mid, clo, chi, &depth_cut)) { status = ORC_ERR_NOMEM; goto done; }
        if (two && finish_box(res, &q, X2, n, depth, o, mid, clo, chi, &depth_cut)) {
            status = ORC_ERR_NOMEM;
            goto done;
        }
    }
done:
    if (status == ORC_OK && depth_cut) status = ORC_ERR_BUDGET;
    res->status = status;
    /* sort the accepted boxes lexicographically */
    if (res->count > 1) {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)res->count);
        double *nl = (double *)malloc(sizeof(double) * (size_t)(res->count * n));
        double *nh = (double *)malloc(sizeof(double) * (size_t)(res->count * n));
        int32_t *nf = (int32_t *)malloc(sizeof(int32_t) * (size_t)res->count);
        int32_t *nd = (int32_t *)malloc(sizeof(int32_t) * (size_t)res->count);
        if (idx && nl && nh && nf && nd) {
            for (int64_t i = 0; i < res->count; i++) idx[i] = i;
            cmp_box_n = n; cmp_lo = res->lo; cmp_hi = res->hi;
            qsort(idx, (size_t)res->count, sizeof(int64_t), cmp_idx);
            for (int64_t i = 0; i < res->count; i++) {
                memcpy(nl + i * n, res->lo + idx[i] * n, sizeof(double) * (size_t)n);
                memcpy(nh + i * n, res->hi + idx[i] * n, sizeof(double) * (size_t)n);
                nf[i] = res->flags[idx[i]];
                nd[i] = res->depth[idx[i]];
            }
            free(res->lo); free(res->hi); free(res->flags); free(res->depth);
            res->lo = nl; res->hi = nh; res->flags = nf; res->depth = nd;
            nl = nh = NULL; nf = nd = NULL;
        } else if (res->status == ORC_OK) {
            res->status = ORC_ERR_NOMEM;
        }
        free(idx); free(nl); free(nh); free(nf); free(nd);
    }
    free(q.lo); free(q.hi); free(q.depth);
    free(X); free(Xn); free(X2); free(F); free(clo); free(chi); free(mid);
    return res->status;
}

int64_t orc_result_count(const orc_result *r) { return r ? r->count : 0; }
int orc_result_status(const orc_result *r) { return r ? r->status : ORC_ERR_INVALID; }
void orc_result_boxes(const orc_result *r, double *lo, double *hi, int32_t *flags, int32_t *depth) {
    if (!r || r->count == 0) return;
    if (lo) memcpy(lo, r->lo, sizeof(double) * (size_t)(r->count * r->n));
    if (hi) memcpy(hi, r->hi, sizeof(double) * (size_t)(r->count * r->n));
    if (flags) memcpy(flags, r->flags, sizeof(int32_t) * (size_t)r->count);
    if (depth) memcpy(depth, r->depth, sizeof(int32_t) * (size_t)r->count);
}
void orc_result_stats(const orc_result *r, orc_stats *st) { if (r && st) *st = r->st; }
void orc_result_depth_stats(const orc_result *r, int64_t *boxes, int64_t *kept) {
    if (!r) return;
    memcpy(boxes, r->depth_boxes, sizeof(r->depth_boxes));
    memcpy(kept, r->depth_kept, sizeof(r->depth_kept));
}
void orc_result_free(orc_result *r) {
    if (!r) return;
    free(r->lo); free(r->hi); free(r->flags); free(r->depth); free(r);
}

/* ------------------------------------------------------------------------------ */
/* Exposed single operations for the tests                                         */
/* ------------------------------------------------------------------------------ */

int orc_iv_op(int op, double a_lo, double a_hi, double b_lo, double b_hi, int k, double *out) {
    ivl a = {a_lo, a_hi}, b = {b_lo, b_hi}, r;
    switch (op) {
    case 0: r = iv_add(a, b); break;
    case 1: r = iv_sub(a, b); break;
    case 2: r = iv_mul(a, b); break;
    case 3: if (!(b.lo > 0 || b.hi < 0)) return 1; r = iv_div(a, b); break;
    case 4: r = iv_pow(a, k); break;
    case 5: r.lo = -a.hi; r.hi = -a.lo; break;
    default: return 1;
    }
    out[0] = r.lo;
    out[1] = r.hi;
    return 0;
}

int orc_iv_extdiv(double x_lo, double x_hi, double y_lo, double y_hi, double *pieces) {
    ivl x = {x_lo, x_hi}, y = {y_lo, y_hi}, p[2];
    int np = iv_extdiv(x, y, p);
    for (int q = 0; q < np; q++) { pieces[2 * q] = p[q].lo; pieces[2 * q + 1] = p[q].hi; }
    return np;
}

void orc_eval(const orc_system *s, const double *lo, const double *hi, double *out_lo, double *out_hi) {
    ivl X[16];
    ivl *F = (ivl *)malloc(sizeof(ivl) * (size_t)s->n_eqs);
    if (!F) return;
    for (int j = 0; j < s->n_vars; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; }
    eval_system(s, X, F);
    for (int i = 0; i < s->n_eqs; i++) { out_lo[i] = F[i].lo; out_hi[i] = F[i].hi; }
    free(F);
}

void orc_jacobian(const orc_system *s, const double *lo, const double *hi, double *j_lo, double *j_hi) {
    ivl X[16];
    ivl *J = (ivl *)malloc(sizeof(ivl) * (size_t)s->n_eqs * (size_t)s->n_vars);
    if (!J) return;
    for (int j = 0; j < s->n_vars; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; }
    jacobian(s, X, J);
    for (int q = 0; q < s->n_eqs * s->n_vars; q++) { j_lo[q] = J[q].lo; j_hi[q] = J[q].hi; }
    free(J);
}

int orc_gj_inverse(int n, const double *a, double *inv) { return gj_inverse(n, a, inv); }

void orc_centred(const orc_system *s, const double *lo, const double *hi, double *out_lo, double *out_hi) {
    int n = s->n_vars;
    ivl *X = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    ivl *F = (ivl *)malloc(sizeof(ivl) * (size_t)n);
    if (X && F) {
        for (int j = 0; j < n; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; }
        centred_form(s, X, F);
        for (int i = 0; i < n; i++) { out_lo[i] = F[i].lo; out_hi[i] = F[i].hi; }
    }
    free(X); free(F);
}

int orc_hs_step(const orc_system *s, const double *lo, const double *hi, double *out_lo, double *out_hi) {
    ivl X[16], Xo[16];
    for (int j = 0; j < s->n_vars; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; }
    int rc = hs_sweep(s, X, Xo, 0, NULL, 0, NULL, NULL);
    if (rc == 0)
        for (int j = 0; j < s->n_vars; j++) { out_lo[j] = Xo[j].lo; out_hi[j] = Xo[j].hi; }
    return rc;
}

int orc_hs_gap_step(const orc_system *s, const double *lo, const double *hi, double *out_lo, double *out_hi,
                    double *out2_lo, double *out2_hi, int32_t *gap_row) {
    ivl X[16], Xo[16], X2[16];
    int g = -1;
    for (int j = 0; j < s->n_vars; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; }
    int rc = hs_sweep(s, X, Xo, 0, NULL, 1, X2, &g);
    if (rc == 0 || rc == 3)
        for (int j = 0; j < s->n_vars; j++) { out_lo[j] = Xo[j].lo; out_hi[j] = Xo[j].hi; }
    if (rc == 3)
        for (int j = 0; j < s->n_vars; j++) { out2_lo[j] = X2[j].lo; out2_hi[j] = X2[j].hi; }
    if (gap_row) *gap_row = g;
    return rc;
}

int orc_kr_step(const orc_system *s, const double *lo, const double *hi, double *out_lo, double *out_hi,
                double *k_lo, double *k_hi) {
    ivl X[16], Xo[16], K[16];
    int n = s->n_vars;
    for (int j = 0; j < n; j++) { X[j].lo = lo[j]; X[j].hi = hi[j]; K[j].lo = -INFINITY; K[j].hi = INFINITY; }
    int rc = hs_sweep(s, X, Xo, 1, K, 0, NULL, NULL);
    if (rc != 2)
        for (int j = 0; j < n; j++) { k_lo[j] = K[j].lo; k_hi[j] = K[j].hi; }
    if (rc == 0)
        for (int j = 0; j < n; j++) { out_lo[j] = Xo[j].lo; out_hi[j] = Xo[j].hi; }
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* FP32 outward evaluation (the prefilter form)                                    */
/* ------------------------------------------------------------------------------ */

typedef struct { float lo, hi; } fiv;

static float f_op(int mode, int op, float a, float b) {
    volatile float x = a, y = b;
    volatile float r;
    fesetround(mode);
    switch (op) {
    case 0: r = x + y; break;
    case 1: r = x - y; break;
    default: r = x * y; break;
    }
    fesetround(FE_TONEAREST);
    return r;
}
static float f_cvt(int mode, double v) {
    volatile double x = v;
    volatile float r;
    fesetround(mode);
    r = (float)x;
    fesetround(FE_TONEAREST);
    return r;
}
static float fmin_(float a, float b) { return b < a ? b : a; }
static float fmax_(float a, float b) { return b > a ? b : a; }
static fiv fiv_add(fiv x, fiv y) { fiv r = {f_op(FE_DOWNWARD, 0, x.lo, y.lo), f_op(FE_UPWARD, 0, x.hi, y.hi)}; return r; }
static fiv fiv_mul(fiv x, fiv y) {
    float l1 = f_op(FE_DOWNWARD, 2, x.lo, y.lo), l2 = f_op(FE_DOWNWARD, 2, x.hi, y.lo);
    float l3 = f_op(FE_DOWNWARD, 2, x.lo, y.hi), l4 = f_op(FE_DOWNWARD, 2, x.hi, y.hi);
    float u1 = f_op(FE_UPWARD, 2, x.lo, y.lo), u2 = f_op(FE_UPWARD, 2, x.hi, y.lo);
    float u3 = f_op(FE_UPWARD, 2, x.lo, y.hi), u4 = f_op(FE_UPWARD, 2, x.hi, y.hi);
    fiv r = {fmin_(fmin_(l1, l2), fmin_(l3, l4)), fmax_(fmax_(u1, u2), fmax_(u3, u4))};
    return r;
}
static float fchain(int mode, float x, int k) { float p = x; for (int i = 1; i < k; i++) p = f_op(mode, 2, p, x); return p; }
static fiv fiv_pow(fiv x, int k) {
    fiv r;
    if (k == 0) { r.lo = 1.0f; r.hi = 1.0f; return r; }
    if (k == 1) return x;
    if ((k & 1) == 0) {
        if (x.lo >= 0) { r.lo = fchain(FE_DOWNWARD, x.lo, k); r.hi = fchain(FE_UPWARD, x.hi, k); }
        else if (x.hi <= 0) { r.lo = fchain(FE_DOWNWARD, -x.hi, k); r.hi = fchain(FE_UPWARD, -x.lo, k); }
        else { r.lo = 0.0f; r.hi = fchain(FE_UPWARD, fmax_(-x.lo, x.hi), k); }
    } else {
        r.lo = x.lo >= 0 ? fchain(FE_DOWNWARD, x.lo, k) : -fchain(FE_UPWARD, -x.lo, k);
        r.hi = x.hi >= 0 ? fchain(FE_UPWARD, x.hi, k) : -fchain(FE_DOWNWARD, -x.hi, k);
    }
    return r;
}

/* The same operation sequence as eval_system, in float: the box and the coefficients
 * are first rounded outward to float.  Every float intermediate then contains the
 * matching double intermediate, so 0 outside the float F_i implies 0 outside the
 * double F_i. */
void orc_eval_f32(const orc_system *s, const double *lo, const double *hi, float *out_lo, float *out_hi) {
    fiv X[16];
    int n = s->n_vars;
    for (int j = 0; j < n; j++) { X[j].lo = f_cvt(FE_DOWNWARD, lo[j]); X[j].hi = f_cvt(FE_UPWARD, hi[j]); }
    for (int i = 0; i < s->n_eqs; i++) {
        fiv acc = {0, 0};
        int have = 0;
        for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
            fiv c = {f_cvt(FE_DOWNWARD, s->coef_lo[t]), f_cvt(FE_UPWARD, s->coef_hi[t])};
            const uint8_t *e = s->exps + (size_t)t * n;
            int hp = 0;
            fiv p = {0, 0};
            for (int j = 0; j < n; j++) {
                if (e[j] == 0) continue;
                fiv f = fiv_pow(X[j], e[j]);
                p = hp ? fiv_mul(p, f) : f;
                hp = 1;
            }
            fiv v = hp ? fiv_mul(c, p) : c;
            acc = have ? fiv_add(acc, v) : v;
            have = 1;
        }
        out_lo[i] = acc.lo;
        out_hi[i] = acc.hi;
    }
}


/* ---- root isolation and backtracking (post-processing of a result) ---------------- */

static int64_t uf_find(int64_t *par, int64_t a) {
    while (par[a] != a) a = par[a];
    return a;
}

static int boxes_touch(int n, const double *lo, const double *hi, int64_t a, int64_t b) {
    for (int j = 0; j < n; j++)
        if (!(lo[a * n + j] <= hi[b * n + j] && lo[b * n + j] <= hi[a * n + j])) return 0;
    return 1;
}

int64_t orc_clusters(int n, int64_t count, const double *lo, const double *hi, int64_t *label) {
    if (count <= 0) return 0;
    int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)count);
    if (!par) return -1;
    for (int64_t i = 0; i < count; i++) par[i] = i;
    for (int64_t i = 0; i < count; i++)
        for (int64_t k = i + 1; k < count; k++)
            if (boxes_touch(n, lo, hi, i, k)) {
                int64_t a = uf_find(par, i), b = uf_find(par, k);
                if (a != b) par[a < b ? b : a] = a < b ? a : b;   /* root = smallest index */
            }
    /* number the clusters in the order of their first (smallest) box */
    int64_t nc = 0;
    int64_t *num = (int64_t *)malloc(sizeof(int64_t) * (size_t)count);
    if (!num) { free(par); return -1; }
    for (int64_t i = 0; i < count; i++) num[i] = -1;
    for (int64_t i = 0; i < count; i++) {
        int64_t r = uf_find(par, i);
        if (num[r] < 0) num[r] = nc++;
        label[i] = num[r];
    }
    free(num);
    free(par);
    return nc;
}

static int cmp_cells_n;
static int cmp_cells(const void *pa, const void *pb) {
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    for (int j = 0; j < cmp_cells_n; j++) {
        if (a[j] < b[j]) return -1;
        if (a[j] > b[j]) return 1;
    }
    return 0;
}

int64_t orc_backtrack(int n, int64_t count, const double *lo, const double *hi, const double *d_lo,
                      const double *d_hi, int level, int64_t max_cells, int64_t *groups) {
    const int64_t side = (int64_t)1 << level;
    int64_t total = 0, cap = 0;
    int32_t *cells = NULL;
    int32_t a[16], b[16], cur[16];
    for (int64_t i = 0; i < count; i++) {
        int64_t m = 1;
        for (int j = 0; j < n; j++) {
            double w = ldexp(d_hi[j] - d_lo[j], -level);
            double tl = (lo[i * n + j] - d_lo[j]) / w, th = (hi[i * n + j] - d_lo[j]) / w;
            double fa = floor(tl), fb = ceil(th) - 1.0;
            double x = fa < fb ? fa : fb, y = fa < fb ? fb : fa;
            if (x < 0) x = 0;
            if (y > (double)(side - 1)) y = (double)(side - 1);
            if (y < x) y = x;   /* a box outside the grid: the nearest cell */
            if (x > (double)(side - 1)) x = y = (double)(side - 1);
            a[j] = (int32_t)x;
            b[j] = (int32_t)y;
            m *= (int64_t)(b[j] - a[j] + 1);
            if (m > max_cells) { free(cells); if (groups) *groups = -1; return -1; }
        }
        if (total + m > max_cells) { free(cells); if (groups) *groups = -1; return -1; }
        if (total + m > cap) {
            int64_t nc = (total + m) * 2;
            int32_t *nb = (int32_t *)realloc(cells, sizeof(int32_t) * (size_t)(nc * n));
            if (!nb) { free(cells); if (groups) *groups = -1; return -1; }
            cells = nb;
            cap = nc;
        }
        for (int j = 0; j < n; j++) cur[j] = a[j];
        for (int64_t q = 0; q < m; q++) {   /* odometer over the box's cell ranges */
            memcpy(cells + (size_t)(total * n), cur, sizeof(int32_t) * (size_t)n);
            total++;
            for (int j = 0; j < n; j++) {
                if (cur[j] < b[j]) { cur[j]++; break; }
                cur[j] = a[j];
            }
        }
    }
    cmp_cells_n = n;
    if (total > 1) qsort(cells, (size_t)total, sizeof(int32_t) * (size_t)n, cmp_cells);
    int64_t distinct = 0;
    for (int64_t i = 0; i < total; i++)
        if (i == 0 || cmp_cells(cells + (size_t)((i - 1) * n), cells + (size_t)(i * n)) != 0) {
            if (distinct != i) memcpy(cells + (size_t)(distinct * n), cells + (size_t)(i * n), sizeof(int32_t) * (size_t)n);
            distinct++;
        }
    if (groups) {
        /* cells touch when their indices differ by at most 1 in every coordinate: as the
         * closed unit boxes [i, i + 1] of index space */
        double *ul = (double *)malloc(sizeof(double) * (size_t)(distinct * n + 1));
        double *uh = (double *)malloc(sizeof(double) * (size_t)(distinct * n + 1));
        int64_t *lab = (int64_t *)malloc(sizeof(int64_t) * (size_t)(distinct + 1));
        if (!ul || !uh || !lab) {
            *groups = -1;
        } else {
            for (int64_t i = 0; i < distinct * n; i++) { ul[i] = (double)cells[i]; uh[i] = (double)cells[i] + 1.0; }
            *groups = orc_clusters(n, distinct, ul, uh, lab);
        }
        free(ul); free(uh); free(lab);
    }
    free(cells);
    return distinct;
}
