/*
 * ivs_oracle.h -- serial CPU oracle for the interval branch-and-bound +
 * Hansen-Sengupta solver of "An efficient algorithm for global interval solution
 * of nonlinear algebraic equations and its GPGPU implementation" (Lin, Chen).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this file: only the tests, the package's smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Every interval operation is one IEEE operation executed under fesetround(FE_DOWNWARD)
 * for a lower end and fesetround(FE_UPWARD) for an upper end (Section 3.2, eq 25-27).
 * Point operations (midpoints, widths, the Gauss-Jordan inverse) run in the default
 * round-to-nearest mode.  Build with -O2 -frounding-math -ffp-contract=off.
 */
#ifndef IVS_ORACLE_H
#define IVS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sparse monomial system: equation i owns terms [eq_offsets[i], eq_offsets[i+1]),
 * term t is [coef_lo[t], coef_hi[t]] * prod_j x_j^exps[t*n_vars + j]. */
typedef struct {
    int32_t n_vars, n_eqs, n_terms;
    const int32_t *eq_offsets;
    const double *coef_lo, *coef_hi;
    const uint8_t *exps;
} orc_system;

typedef struct {
    double tol;             /* accept when max_j RN(hi_j - lo_j) <= tol            */
    int32_t hs_enable;      /* 1: Hansen-Sengupta step on every kept box            */
    int32_t hs_min_depth;   /* HS only at depth >= hs_min_depth                     */
    int32_t hs_iters;       /* at most this many Gauss-Seidel sweeps per visit (>= 1);
                               they stop at the first sweep that changes nothing       */
    int32_t root_depth;     /* depth given to the initial box                       */
    int32_t max_depth;      /* a box that would split past it is returned flagged   */
    int32_t order;          /* 0 LIFO, 1 FIFO, 2 seeded random pop                  */
    uint64_t order_seed;
    int64_t max_boxes;      /* work budget: boxes processed (0 = unlimited)         */
    int32_t centred;        /* 1: after the natural form, drop boxes whose centred
                               (mean-value) form excludes 0 (needs n_eqs == n_vars)  */
    int32_t krawczyk;       /* 1: the contraction step is Krawczyk's operator
                               intersected with the box (eq 15, 16) instead of the
                               Gauss-Seidel sweep (eq 21, 22); same iteration rule     */
    int32_t split_mode;     /* 0: Algorithm 2's split of every coordinate (2^n children);
                               1: bisection of the widest coordinate only (2 children)  */
    int32_t gap_split;      /* 1: a Gauss-Seidel sweep whose extended division leaves a
                               gap inside X_i returns two boxes, one per piece (the
                               widest such gap over the rows), instead of the hull      */
} orc_options;

/* result flags per accepted box */
#define ORC_ACCEPT_WIDTH 1
#define ORC_ACCEPT_UNSPLITTABLE 2
#define ORC_ACCEPT_DEPTH_LIMIT 4   /* returned unsplit at max_depth; status ORC_ERR_BUDGET */

/* status */
#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOMEM 2
#define ORC_ERR_BUDGET 3

typedef struct {
    int64_t boxes;          /* boxes popped and processed                          */
    int64_t excluded_eval;  /* dropped because some F_i(X) does not contain 0      */
    int64_t hs_applied;     /* HS sweeps run                                       */
    int64_t hs_empty;       /* dropped because the HS sweep returned the empty set  */
    int64_t hs_contracted;  /* HS sweeps that changed the box                      */
    int64_t hs_singular;    /* HS skipped: mid(J) singular or B non-finite          */
    int64_t accepted;
    int64_t unsplittable;
    int64_t split;
    int32_t max_depth_seen;
    int64_t excluded_centred;  /* dropped because some centred form F_c,i(X) excludes 0 */
    int64_t gap_splits;     /* sweeps that returned two boxes (gap_split = 1)         */
} orc_stats;

typedef struct orc_result orc_result;

int orc_solve(const orc_system *sys, const double *box_lo, const double *box_hi,
              const orc_options *opt, orc_result **out);
int64_t orc_result_count(const orc_result *r);
int orc_result_status(const orc_result *r);
/* accepted boxes, sorted lexicographically by (lo_0, hi_0, lo_1, hi_1, ...), -0 -> +0 */
void orc_result_boxes(const orc_result *r, double *lo, double *hi, int32_t *flags, int32_t *depth);
void orc_result_stats(const orc_result *r, orc_stats *st);
/* per depth d (clamped to ORC_MAX_DEPTH_STATS-1): boxes processed at depth d and boxes
 * that survived evaluation (and HS, when applied) at depth d */
#define ORC_MAX_DEPTH_STATS 64
void orc_result_depth_stats(const orc_result *r, int64_t *boxes, int64_t *kept);
void orc_result_free(orc_result *r);

/* ---- single operations, exposed for the tests that pin them -------------------- */
/* op: 0 add, 1 sub, 2 mul, 3 div (0 not in y), 4 pow (k), 5 neg
 * out[0..1] = [lo, hi] */
int orc_iv_op(int op, double a_lo, double a_hi, double b_lo, double b_hi, int k, double *out);
/* extended division x / y (eq 10): returns number of pieces (0 = empty set,
 * 1 or 2); pieces[4] = {lo0, hi0, lo1, hi1}, infinite ends as +-INFINITY. */
int orc_iv_extdiv(double x_lo, double x_hi, double y_lo, double y_hi, double *pieces);
/* F(X): out_lo/out_hi[n_eqs] (natural interval extension, Definition 1) */
void orc_eval(const orc_system *sys, const double *lo, const double *hi, double *out_lo, double *out_hi);
/* F(X) in float with outward rounding of inputs and ops (the FP32 prefilter form) */
void orc_eval_f32(const orc_system *sys, const double *lo, const double *hi, float *out_lo, float *out_hi);
/* interval Jacobian J(X), row-major n_eqs x n_vars */
void orc_jacobian(const orc_system *sys, const double *lo, const double *hi, double *j_lo, double *j_hi);
/* Gauss-Jordan inverse with partial pivoting (Section 2.4); returns 0 ok, 1 singular */
int orc_gj_inverse(int n, const double *a, double *inv);
/* one Hansen-Sengupta sweep (Section 2.3, Algorithm 3):
 * returns 0 = box out (maybe unchanged), 1 = empty, 2 = skipped (singular) */
int orc_hs_step(const orc_system *sys, const double *lo, const double *hi, double *out_lo, double *out_hi);
/* Root isolation over a set of boxes (row-major lo/hi, count x n): clusters are the
 * connected components of "touch" (two boxes touch when lo_j <= hi'_j and lo'_j <= hi_j for
 * every j).  label[i] = cluster of box i, clusters numbered in the order of their first box.
 * Returns the number of clusters.  Plain O(count^2) union-find. */
int64_t orc_clusters(int n, int64_t count, const double *lo, const double *hi, int64_t *label);
/* Backtracking (Algorithm 5, read on the dyadic grid of the initial box): the number of
 * distinct cells of level `level` (cell width (d_hi - d_lo) / 2^level per coordinate) that
 * the boxes meet; per coordinate t = (x - d_lo) / w in round to nearest, cells from
 * floor(t_lo) to ceil(t_hi) - 1 (the two ends swapped when they cross), clamped to the grid.
 * *groups (if not NULL) = connected components of those cells, cells touching when their
 * indices differ by at most 1 in every coordinate (the roots isolated at that width).
 * Returns -1 when more than max_cells cells would be enumerated. */
int64_t orc_backtrack(int n, int64_t count, const double *lo, const double *hi, const double *d_lo,
                      const double *d_hi, int level, int64_t max_cells, int64_t *groups);
/* One Krawczyk step (eq 15, 16): K(X) into k_lo/k_hi (status 0 or 1), X intersected with
 * K(X) into out_lo/out_hi (status 0).  Status as orc_hs_step. */
int orc_kr_step(const orc_system *sys, const double *lo, const double *hi, double *out_lo, double *out_hi,
                double *k_lo, double *k_hi);
/* One Gauss-Seidel sweep with the two-box split of a gap (gap_split = 1): status as
 * orc_hs_step, or 3 when the sweep returns two boxes -- out (the lower piece of
 * coordinate *gap_row) and out2 (the upper piece); the other coordinates are equal. */
int orc_hs_gap_step(const orc_system *sys, const double *lo, const double *hi, double *out_lo, double *out_hi,
                    double *out2_lo, double *out2_hi, int32_t *gap_row);
/* centred form of every equation over the box (n_eqs == n_vars): out[i] = F_c,i(X) */
void orc_centred(const orc_system *sys, const double *lo, const double *hi, double *out_lo, double *out_hi);

#ifdef __cplusplus
}
#endif
#endif
