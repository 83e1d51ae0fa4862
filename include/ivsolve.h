/*
 * ivsolve.h -- C ABI of the GB300 (sm_103a) interval solver for bounded polynomial
 * systems: interval branch-and-bound with Hansen-Sengupta contraction, after
 * Lin & Chen, "An efficient algorithm for global interval solution of nonlinear
 * algebraic equations and its GPGPU implementation".
 *
 * Problem statement (Algorithm 1, In/Out): given polynomial equations f_1..f_m in
 * x_1..x_n, a box of variable regions [d_lo_j, d_hi_j] and a desired width, return
 * the boxes ("configurations") of that width that may contain a real solution.  Every
 * real solution in the initial box lies in some returned box; an empty result with
 * IVS_OK proves that the box holds no solution (Algorithm 1, termination (I)).
 *
 * Per box, in this order (each box's fate depends only on the box itself):
 *   1. natural interval extension F(X) with outward rounding (Definition 1, eq 25-27);
 *      drop the box if some F_i(X) does not contain 0 (Definition 2, Algorithm 2);
 *   2. optional Hansen-Sengupta sweep (Section 2.3 eq 14, 17-22; Algorithm 3, with the
 *      Gauss-Jordan preconditioner of Section 2.4 and the products of Algorithm 4);
 *      drop the box if the sweep returns the empty set;
 *   3. accept when max_j (hi_j - lo_j) <= tol (Algorithm 1 termination (II)), else split
 *      every coordinate at its midpoint into 2^n children (Algorithm 2).
 * Readings of garbled or silent passages are documented with the implementation.
 *
 * All pointers are HOST pointers unless stated.  Inputs are borrowed for the duration
 * of the call and copied.  Results are owned by the library until ivs_result_free /
 * ivs_plan_destroy.  Every function returns an int status (IVS_OK on success) unless
 * it returns a count; no function aborts the process.  A GPU is required: with no
 * device or no driver the calls return IVS_ERR_CUDA.
 */
#ifndef IVSOLVE_H
#define IVSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define IVS_OK 0
#define IVS_ERR_INVALID 1  /* n <= 0 or > 16; lo > hi; non-finite input; exponent > 15;
                              HS requested with m != n; bad option values          */
#define IVS_ERR_NOMEM 2    /* device or host allocation failed, or the work queue
                              cannot hold the boxes a step needs                    */
#define IVS_ERR_BUDGET 3   /* max_boxes, max_results or max_depth was hit: the result
                              is returned but flagged incomplete                    */
#define IVS_ERR_TIMEOUT 4  /* time_budget_s elapsed; result incomplete              */
#define IVS_ERR_CUDA 5     /* a CUDA call failed (message: ivs_last_error())        */

/* ---- per-box flags of accepted boxes ------------------------------------------ */
#define IVS_BOX_WIDTH 1          /* max width <= tol                                 */
#define IVS_BOX_UNSPLITTABLE 2   /* widest coordinate cannot be split in doubles     */
#define IVS_BOX_DEPTH_LIMIT 4    /* returned unsplit at max_depth (status BUDGET)    */

/* Sparse monomial system (the paper's equations with "integer or floating number
 * coefficients", Section 3.2).  Equation i owns terms [eq_offsets[i], eq_offsets[i+1]);
 * term t is [coef_lo[t], coef_hi[t]] * prod_j x_j^exps[t*n_vars + j].  A coefficient
 * that is not a double is given as the interval of the two doubles around it
 * (coef_hi may be NULL when every coefficient is exact: then coef_hi = coef_lo).
 * Limits: 1 <= n_vars <= 16, exponents <= 15, n_eqs >= 1. */
typedef struct ivs_system {
    int32_t n_vars, n_eqs, n_terms;
    const int32_t *eq_offsets;   /* n_eqs + 1 entries, eq_offsets[0] == 0             */
    const double *coef_lo;       /* n_terms                                           */
    const double *coef_hi;       /* n_terms or NULL                                   */
    const uint8_t *exps;         /* n_terms * n_vars, row-major                       */
} ivs_system;

typedef struct ivs_options {
    double tol;              /* accept width (>= 0)                                   */
    int32_t hs_enable;       /* 1: Hansen-Sengupta sweep on boxes that survive F(X)    */
    int32_t hs_min_depth;    /* sweep only at depth >= this (the paper starts late)    */
    int32_t hs_iters;        /* at most this many sweeps per visit (>= 1); they stop at
                                the first sweep that leaves the box unchanged (Section
                                2.3: iterated until the contraction stalls)             */
    int32_t prefilter_fp32;  /* 1: FP32 stage before FP64.  It carries float enclosures
                                of both ends of every FP64 intermediate, so it drops a
                                box only when FP64 would and keeps one only when FP64
                                would; undecided boxes run the FP64 evaluation.  Results
                                are identical with and without it.                     */
    int32_t root_depth;      /* depth of the initial box                               */
    int32_t max_depth;       /* a box that would split past it is returned with
                                IVS_BOX_DEPTH_LIMIT and status IVS_ERR_BUDGET          */
    int64_t max_boxes;       /* work budget in processed boxes, 0 = unlimited          */
    int64_t max_results;     /* accepted-box capacity, 0 = library default             */
    double time_budget_s;    /* wall-clock budget, 0 = unlimited                       */
    int32_t centred_form;    /* 1: after the natural form, a second exclusion test by
                                the centred (mean-value) form from the expansion of
                                Section 2.3 eq 13, F_c,i(X) = f_i(x) + sum_j J_ij(X)
                                (X_j - x_j) at x = mid X, folded over j = 1..n; a box
                                is dropped when some F_c,i(X) excludes 0.  Needs
                                n_eqs == n_vars.  0 (default): natural form only.       */
    int32_t krawczyk;        /* 1: the contraction of every sweep (hs_enable, hs_min_depth,
                                hs_iters as above) is Krawczyk's operator, Section 2.3
                                eq 15-16: K_i = (x_i - r_i) + sum_j ((I - M)_ij (X_j -
                                x_j)) with the sweep's x = mid X, M = B J(X), r = B f(x),
                                folded over j = 1..n, every row from the incoming box;
                                X_i becomes X_i intersected with K_i and the box is
                                dropped when one intersection is empty.  The counters
                                hs_* then count Krawczyk steps.  0 (default): the
                                Gauss-Seidel sweep of eq 21-22.                         */
    int32_t split_mode;      /* 0 (default): Algorithm 2's split of every coordinate at its
                                midpoint (2^n children).  1: bisection of the widest
                                coordinate only (the first of equal widths; 2 children,
                                depth + 1 per bisection)                                 */
    int32_t gap_split;       /* 1: a Gauss-Seidel sweep whose extended division (eq 10)
                                leaves a gap inside X_i returns two boxes, one per piece,
                                at the row with the widest gap RN(lower end of the upper
                                piece - upper end of the lower piece) (the first of equal
                                ones; later rows use the hull), instead of the hull
                                (Section 2.3, after eq 22).  Both boxes then take the
                                accept / split step; the visit's sweeps stop there.
                                Ignored with krawczyk = 1.                              */
} ivs_options;

typedef struct ivs_stats {
    int64_t boxes;              /* boxes processed (each of the 2^n children counts)   */
    int64_t excluded_prefilter; /* dropped by the FP32 stage                           */
    int64_t excluded_eval;      /* dropped by the FP64 evaluation                      */
    int64_t hs_applied;         /* HS sweeps run                                       */
    int64_t hs_empty;           /* dropped by an HS sweep                              */
    int64_t hs_contracted;      /* HS sweeps that changed the box                      */
    int64_t hs_singular;        /* HS skipped (mid J singular, or B non-finite)        */
    int64_t accepted;
    int64_t unsplittable;
    int64_t split;
    int32_t max_depth_seen;
    int32_t waves;              /* device sweeps over the queue                        */
    double device_ms;           /* device time of the solve                            */
    int64_t launches;           /* kernels the solve launched                          */
    int64_t eval64_boxes;       /* boxes that ran the FP64 evaluation                  */
    int64_t kept_shadow;        /* boxes the FP32 shadow proved FP64 would keep        */
    double queue_ms;            /* served requests: submit -> admission                */
    double solve_ms;            /* served requests: admission -> result ready          */
    int64_t excluded_centred;   /* dropped by the centred form (centred_form = 1)      */
    int64_t gap_splits;         /* sweeps that returned two boxes (gap_split = 1)      */
} ivs_stats;

typedef struct ivs_result ivs_result;
typedef struct ivs_plan ivs_plan;

/* Fills *o with defaults: tol 1e-6, HS on from depth 0, one sweep, FP32 prefilter on,
 * root_depth 0, max_depth 200, no box or time budget. */
void ivs_options_default(ivs_options *o);

/* Solve one system on the initial box [box_lo, box_hi] (n_vars doubles each).
 * On IVS_OK / IVS_ERR_BUDGET / IVS_ERR_TIMEOUT *out receives a result (free it with
 * ivs_result_free); on other errors *out is NULL.
 * ivs_solve and ivs_solve_batch keep the device memory, stream, pinned buffers and
 * instantiated CUDA graph of their last call (device 0) and build the next call from
 * them; calls from several threads are safe (each takes the kept set or makes its own).
 * ivs_release_cached frees what is kept. */
void ivs_release_cached(void);
int ivs_solve(const ivs_system *sys, const double *box_lo, const double *box_hi,
              const ivs_options *opt, ivs_result **out);

/* Solve n_sys independent systems in one device run (batching form: the queues of all
 * systems share every sweep).  box_lo[s] / box_hi[s] point to system s's box; opts is
 * one options struct per system (or a single struct when opts_stride == 0).
 * outs[s] receives system s's result.  Returns the first non-OK status among systems
 * (or an error of the run itself). */
int ivs_solve_batch(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                    const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                    ivs_result **outs);

int64_t ivs_result_count(const ivs_result *r);
int32_t ivs_result_n_vars(const ivs_result *r);
int ivs_result_status(const ivs_result *r);
/* Copies the accepted boxes, sorted lexicographically by (lo_0, hi_0, lo_1, ...),
 * -0 written as +0.  lo, hi: count * n_vars doubles (row-major); flags, depth: count
 * int32 each; any of them may be NULL. */
int ivs_result_boxes(const ivs_result *r, double *lo, double *hi, int32_t *flags, int32_t *depth);
int ivs_result_stats(const ivs_result *r, ivs_stats *st);
/* Per depth d = 0..63 (depths above 63 counted in slot 63): boxes processed at depth d;
 * boxes that survived the evaluation (and the contraction, when applied) there; boxes
 * that entered the contraction there.  With a split at every depth these are the
 * paper's boxes per round (round d + 1, Tables 1, 4, 7) and, with hs_min_depth, its
 * Hansen-Sengupta "origin" (entered) and "new" (survived) boxes (Tables 2, 5).  Each
 * array holds 64 int64; any may be NULL. */
int ivs_result_depth_stats(const ivs_result *r, int64_t *boxes, int64_t *kept, int64_t *entered_hs);
void ivs_result_free(ivs_result *r);

/* ---- device-resident plan: upload once, solve many times ---------------------- */
/* cfg fields left 0 take defaults.  workspace: optional caller-owned DEVICE buffer
 * (e.g. from a PyTorch allocation) of workspace_bytes; when NULL the plan allocates
 * its own with cudaMalloc.  stream: a cudaStream_t (NULL = the plan creates one). */
typedef struct ivs_plan_cfg {
    void *workspace;
    size_t workspace_bytes;
    void *stream;
    int64_t wave_children;   /* max children evaluated per sweep (0 = default)       */
    int32_t eval_blocks;     /* grid of the evaluation kernel (0 = auto)             */
    int32_t eval_threads;    /* block of the evaluation kernel (0 = auto)            */
    int32_t device;          /* CUDA device ordinal                                  */
    int32_t profile;         /* 1: time each kernel class with CUDA events           */
} ivs_plan_cfg;

/* Bytes of device workspace a plan with these systems needs for the given
 * wave_children and queue capacity (queue_parents boxes).  Lets a caller allocate. */
size_t ivs_workspace_bytes(int32_t n_sys, const ivs_system *systems, int64_t wave_children,
                           int64_t queue_parents, int64_t max_results);

int ivs_plan_create(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                    const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                    const ivs_plan_cfg *cfg, ivs_plan **out);
/* Runs a full solve of every system in the plan on the plan's stream and waits for it.
 * The plan's results are replaced on each run. */
int ivs_plan_run(ivs_plan *p);
/* Copies system s's result of the last run to the host. */
int ivs_plan_result(ivs_plan *p, int32_t s, ivs_result **out);
int ivs_plan_stats(ivs_plan *p, ivs_stats *st);   /* totals over all systems, last run */
/* System s's counters of the last run and its per-depth counts (as ivs_result_depth_stats)
 * without copying its boxes; any output may be NULL. */
int ivs_plan_depth_stats(ivs_plan *p, int32_t s, ivs_stats *st, int64_t *boxes, int64_t *kept, int64_t *entered_hs);
void ivs_plan_destroy(ivs_plan *p);

/* Autotuner of the batching form (no paper counterpart): for the given systems it runs
 * short trial solves (each system capped at trial_boxes processed boxes) with every
 * combination of wave_children in {2^20, 2^22, 2^24} and evaluation grids of {4, 8, 16}
 * blocks per SM (each timed as the faster of two runs after a warm-up), and writes to *best
 * (its other fields zero) the configuration with the largest wave_children among those
 * within 3% of the highest boxes/s (the capped trial runs fewer sweeps than a full solve,
 * so it undercounts the fixed cost per sweep), and its rate to *best_rate.  The choices
 * only schedule work: results do not depend on them. */
int ivs_autotune(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                 const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                 int64_t trial_boxes, ivs_plan_cfg *best, double *best_rate);

/* Per-kernel-class device time of the last run of a plan created with cfg.profile = 1
 * (CUDA events on the plan's stream around each launch).  Writes up to max entries and
 * returns how many classes exist.  Class names: "eval", "hs_n<k>", "control". */
typedef struct ivs_kernel_time {
    char name[24];
    int64_t launches;
    double ms;
} ivs_kernel_time;
int32_t ivs_plan_kernel_times(ivs_plan *p, ivs_kernel_time *out, int32_t max);

/* Microbenchmark of the directed-rounding arithmetic rate of the device (no paper
 * counterpart; it supplies the roofline denominator): kind 0 = FP64 (__dadd_rd /
 * __dmul_ru chains), kind 1 = FP32 (__fadd_rd / __fmul_ru), kind 2 / 3 = FP64 with only
 * 8 / 1 lanes of each warp active (counts only active-lane operations: shows whether
 * idle lanes cost FP64 issue time), kind 4 / 5 = FP64 division, directed (__ddiv_rd /
 * __ddiv_ru) / round to nearest.  Writes the rate in operations per second (one add,
 * multiply or division = one operation) and the kernel time. */
int ivs_probe_rate(int32_t kind, int32_t device, double *ops_per_s, double *ms);


/* ---- serving: continuous batching over one shared device queue ------------------- */
/* A server keeps one device-resident queue for every system in flight.  Requests that
 * arrive while others run are admitted between sweeps (one sweep = Algorithm 2's
 * evaluation of every child of the popped parents, then Algorithm 3 and the accept /
 * split step) as soon as a slot and queue memory are free: each request owns a region of
 * 64 * 2^n queue entries (reserve_factor scales it; at least min_region_entries), and
 * requests wait, in arrival order, until one is free.  Each sweep's children go to the
 * requests in flight in order of the boxes each has processed so far, fewest first (least
 * attained service: a request that needs little work finishes in few sweeps whatever
 * else is in flight; up to 4096 slots), or, with schedule = 1, in equal shares in an order
 * that rotates every sweep; a request whose region is more than half full takes one
 * parent per sweep.  Their sweeps share kernels; the schedule never changes a result.  A system is solved when none of its
 * boxes remain in the queue; its result (the same as ivs_solve's, bit for bit: each box's
 * fate depends only on the box) is then ready for ivs_server_poll / ivs_server_wait.
 * A request whose options set time_budget_s > 0 and that is still unsolved that long
 * after its admission is cancelled between two sweeps: its remaining boxes are removed
 * from its region at once, and it completes with IVS_ERR_TIMEOUT and the boxes it had
 * accepted so far.
 * Submissions and polls may come from any host thread; one worker thread drives the GPU. */
typedef struct ivs_server ivs_server;
typedef struct ivs_server_cfg {
    size_t workspace_bytes;   /* device memory for the shared queue (0 = 4 GiB); sweep
                                 staging and the result regions are allocated on top     */
    int64_t wave_children;    /* children per sweep (0 = 2^22)                            */
    int64_t results_per_slot; /* result capacity of one request (0 = 16384)               */
    int32_t max_slots;        /* systems in flight at once (0 = 1024)                     */
    int32_t max_vars;         /* largest n accepted (0 = 12, at most 16)                  */
    int32_t sweeps_per_step;  /* sweeps between admissions / completion checks (0 = 2)    */
    int32_t device;           /* CUDA device ordinal                                      */
    double reserve_factor;    /* scales the per-request queue reservation (0 = 1)         */
    int64_t min_region_entries; /* smallest queue region of a request, in entries (0 = no
                                 minimum beyond 64 * 2^n): a region that is more than half
                                 full gives its request one parent per sweep, so a larger
                                 region lets small requests finish in fewer sweeps        */
    int32_t schedule;         /* 0: least attained service first; 1: rotating equal shares */
} ivs_server_cfg;

typedef struct ivs_server_stats {
    int64_t submitted, admitted, completed, in_flight, waiting;
    int64_t steps, sweeps, boxes;
    double busy_s;            /* worker time with systems in flight                       */
    char last_error[160];     /* the worker's last error text ("" if none)                */
} ivs_server_stats;

void ivs_server_cfg_default(ivs_server_cfg *cfg);
int ivs_server_create(const ivs_server_cfg *cfg, ivs_server **out);
/* Copies the system, box and options (validated as for ivs_solve; n_vars <= max_vars)
 * and queues the request; *ticket identifies it. */
int ivs_server_submit(ivs_server *sv, const ivs_system *sys, const double *box_lo, const double *box_hi,
                      const ivs_options *opt, uint64_t *ticket);
/* IVS_OK with *out = NULL while pending; IVS_OK with *out = the result once done (the
 * caller then owns it: ivs_result_free); IVS_ERR_INVALID for an unknown ticket.  The
 * result's stats carry queue_ms (submit -> admission) and solve_ms (admission -> done). */
int ivs_server_poll(ivs_server *sv, uint64_t ticket, ivs_result **out);
/* Like poll but blocks up to timeout_s seconds (<= 0: no limit). */
int ivs_server_wait(ivs_server *sv, uint64_t ticket, double timeout_s, ivs_result **out);
int ivs_server_get_stats(ivs_server *sv, ivs_server_stats *st);
/* Stops the worker (requests not finished are dropped) and frees everything. */
void ivs_server_destroy(ivs_server *sv);

/* ---- root isolation and backtracking (after the solve; host only) ---------------- */
/* Section 3.4: the last round leaves many tiny configurations; merging them isolates the
 * real roots.  ivs_clusters groups boxes (row-major lo/hi, count x n_vars, any order, e.g.
 * the boxes of ivs_result_boxes) into the connected components of "touch" (boxes a and b
 * touch when lo_a,j <= hi_b,j and lo_b,j <= hi_a,j for every j); the boxes around one
 * isolated real root form one component, also when the root sits on split planes and its
 * boxes lie on several sides of them.  Writes the number of clusters; label[i] = cluster of
 * box i, clusters numbered in the order of their first box (NULL to skip); for the first
 * cl_cap clusters their hull in cl_lo / cl_hi (n_vars doubles each; NULL to skip).  A sweep
 * over the first coordinate: work grows with the pairs of boxes whose first coordinates
 * overlap; IVS_ERR_BUDGET beyond 4e9 such pairs.  No GPU needed. */
int ivs_clusters(int32_t n_vars, int64_t count, const double *lo, const double *hi, int64_t *n_clusters,
                 int64_t *label, double *cl_lo, double *cl_hi, int64_t cl_cap);
/* Algorithm 5 (backtracking a configuration to the round before), read on the dyadic grid
 * of the initial box [box_lo, box_hi] and applied `level` rounds up from the finest: the
 * number of distinct cells of that grid at level `level` (cell width (box_hi_j - box_lo_j) /
 * 2^level) that the boxes meet -- the "backtracking boxes" the paper tabulates per width.
 * Per coordinate t = (x - box_lo_j) / width in round to nearest (exact for dyadic data), a
 * box meets cells floor(t_lo) .. ceil(t_hi) - 1, the two ends swapped when they cross (a
 * box of width 0 on a cell boundary meets both cells), clamped to the grid.  A root on a
 * cell corner gives several cells.  *n_groups (NULL to skip) receives the connected
 * components of those cells, cells touching when their indices differ by at most 1 in
 * every coordinate: the roots isolated at that width (the paper's "N real interval roots,
 * width w").  IVS_ERR_BUDGET if more than max_cells cells would be enumerated.  No GPU
 * needed. */
int ivs_backtrack(int32_t n_vars, int64_t count, const double *lo, const double *hi, const double *box_lo,
                  const double *box_hi, int32_t level, int64_t max_cells, int64_t *n_cells, int64_t *n_groups);

/* The same two operations on the GPU (Section 3.4, Algorithm 5), with the same results:
 * ivs_clusters_gpu and ivs_backtrack_gpu take host rows like the functions above (copied
 * to device `device`, scratch allocated per call); ivs_plan_clusters and
 * ivs_plan_backtrack work on a plan's device-resident result of system s after
 * ivs_plan_run, with that system's initial box, on the plan's stream -- no host copy of
 * the boxes.  Cells are sorted on the device as 128-bit keys (coordinate 0 most
 * significant), so the GPU backtracking needs n_vars * level <= 127 (IVS_ERR_INVALID
 * beyond); groups and clusters come from a union-find over the candidate pairs that a
 * binary search over the sorted keys leaves (IVS_ERR_BUDGET above 4e9 pairs; as above,
 * above max_cells cells).  ivs_plan_clusters returns the count only. */
int ivs_clusters_gpu(int32_t n_vars, int64_t count, const double *lo, const double *hi, int64_t *n_clusters,
                     int64_t *label, double *cl_lo, double *cl_hi, int64_t cl_cap, int32_t device);
int ivs_backtrack_gpu(int32_t n_vars, int64_t count, const double *lo, const double *hi, const double *box_lo,
                      const double *box_hi, int32_t level, int64_t max_cells, int64_t *n_cells, int64_t *n_groups,
                      int32_t device);
int ivs_plan_backtrack(ivs_plan *p, int32_t s, int32_t level, int64_t max_cells, int64_t *n_cells,
                       int64_t *n_groups);
int ivs_plan_clusters(ivs_plan *p, int32_t s, int64_t *n_clusters);

/* ---- allocation-free solve ------------------------------------------------------ */
/* No counterpart in the paper: an entry point for callers that cannot allocate.
 * Processes whose device memory belongs to a pool they must not bypass (a framework's
 * caching allocator, a serving engine that reserved the GPU's memory up front), plug-ins
 * and callbacks running inside another runtime that forbids allocation, and real-time
 * loops that cannot afford cudaMalloc's implicit synchronisation cannot call cudaMalloc.
 * ivs_solve_noalloc solves one system like ivs_solve but allocates nothing: every byte
 * of device scratch comes from one fixed file-scope __device__ array of
 * IVS_NOALLOC_SCRATCH_BYTES inside the library (present on every GPU that loads the
 * library, until the process exits), host work uses static buffers and the stack, and it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Limits of the fixed buffers: n_vars <= 12, a compiled term table (equations plus
 * Jacobian) of at most 48 KiB / 2048 terms, and at most 16384 boxes held as results.
 * Larger systems are rejected with IVS_ERR_INVALID and a message in errbuf; a solve
 * whose queue outgrows the buffer returns IVS_ERR_NOMEM, and one with more accepted
 * boxes than out_cap or 16384 returns IVS_ERR_BUDGET with the first ones.
 *
 * Inputs (host pointers) as for ivs_solve.  stream: a cudaStream_t or NULL (the legacy
 * default stream); the call waits on it between sweeps and returns after the solve, so
 * a stream in capture mode is rejected with IVS_ERR_INVALID.  Outputs (host memory
 * owned by the caller): out_lo / out_hi receive up to out_cap boxes of n_vars doubles,
 * row-major and sorted as in ivs_result_boxes; out_flags (may be NULL) their IVS_BOX_*
 * flags; *out_count the number written; stats (may be NULL) the counters; errbuf (may be
 * NULL) a message of at most errbuf_len bytes, also kept as ivs_last_error().  Returns
 * an IVS_* status.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every
 * call shares the one array and it keeps the previous call's contents (the call clears
 * what must start at zero): calls that overlap on the GPU -- from several host threads
 * on different streams, or on one device from several processes' views of it -- race.
 * Host threads are serialised by a lock inside the library. */
#define IVS_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int ivs_solve_noalloc(const ivs_system *sys, const double *box_lo, const double *box_hi,
                      const ivs_options *opt, void *stream, double *out_lo, double *out_hi,
                      int32_t *out_flags, int64_t out_cap, int64_t *out_count, ivs_stats *stats,
                      char *errbuf, int32_t errbuf_len);

const char *ivs_status_str(int status);
const char *ivs_last_error(void);   /* thread-local text of the last error           */

#ifdef __cplusplus
}
#endif
#endif /* IVSOLVE_H */
