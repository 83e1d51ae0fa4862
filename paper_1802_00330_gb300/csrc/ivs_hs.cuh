// ivs_hs.cuh -- Hansen-Sengupta sweep and the accept / split step for the boxes that
// survived the evaluation (Section 2.3 eq 14, 17-22; Algorithm 3; Gauss-Jordan of
// Section 2.4; Algorithm 4 products; Algorithm 1 termination (II); Algorithm 2 split).
//
// Mapping: one block takes BB boxes at a time (32; 16 for n >= 15) from an atomic
// cursor, and its NW warps share the work of those boxes.  Lane b of every warp always
// works on box b, so each FP64 warp instruction carries BB different boxes; the warps
// split what is independent within a box: the n^2 + n polynomials of J(X) and f(x), the
// row updates of each Gauss-Jordan step, the columns of M = B J(X), and the
// Gauss-Seidel products.  What is serial within a box stays with its owner thread (warp 0,
// lane b): pivot choice, the intersections, accept / split; each Gauss-Seidel row's fold and
// extended division run on two threads, lower ends on warp 0 and upper ends on warp 1.
//
// Why: GB300's FP64 pipe charges a whole warp instruction whatever the number of active
// lanes, and a sweep has few boxes (often less than one warp per SM), so one thread per
// box leaves the kernel waiting on the dependent chain of a single box.  Sharing a box's
// independent work among warps shortens that chain without adding FP64 instructions.
// Every value is computed by the same operations in the same order as the serial
// definition, so the results are unchanged.  Matrices live in shared memory (structure
// of arrays over the chunk's boxes: element (k, b) at k * BB + b, conflict-free).
// Comparisons, sign tests, NaN and finiteness checks run on the integer pipes.
// Templated on n; the instantiations are spread over several translation units
// (ivs_hs_*.cu).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ivs_internal.h"
#include "ivs_interval.cuh"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

namespace ivs {

namespace cg = cooperative_groups;

namespace hsd {
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kCS = 4;          // CTAs per cluster in the cooperative form (8 measured no faster)
constexpr int kCoopMaxN = 12;   // the cooperative form exists for n <= 12
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }
__device__ __forceinline__ unsigned long long *stat_ptr(const SweepArgs &a, int sys, int slot) {
    return a.stats + (size_t)sys * ST_COUNT + slot;
}
__device__ __forceinline__ double midpoint_rn(double lo, double hi) { return __dmul_rn(0.5, __dadd_rn(lo, hi)); }
// integer-pipe predicates on doubles
__device__ __forceinline__ bool d_isnan(double x) {
    return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) > 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool d_finite(double x) {
    return (__double_as_longlong(x) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
}
// |x| as an ordered integer; NaN ranks below everything (never chosen as a pivot)
__device__ __forceinline__ long long d_abskey(double x) {
    const long long m = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
    return m > 0x7FF0000000000000LL ? -1 : m;
}
// numeric a <= b for non-NaN doubles (-0 == +0)
__device__ __forceinline__ bool d_le(double a, double b) {
    return d_key(a) <= d_key(b) || (d_iszero(a) && d_iszero(b));
}
// numerically equal (-0 == +0; NaN never equals)
__device__ __forceinline__ bool d_same(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b) || (d_iszero(a) && d_iszero(b));
}

// Shared-memory layout of a block: arrays of rows, each row BB values (one per box).
template <int N>
struct Cfg {
    static constexpr int BB = (N >= 15) ? 16 : 32;   // boxes per chunk
    static constexpr int NW = (N <= 3) ? 4 : 8;      // warps per block
    static constexpr int NT = NW * 32;
    // blocks per SM: three for n = 7, 8 (80 registers, a few bytes of spill; measured 3-4%
    // faster on the batch's wide sweeps than two at 128 registers; the narrow n = 6 sweeps
    // measured 2% slower with three), two up to n = 10, then one
    static constexpr int MIN_BLOCKS = (N == 7 || N == 8) ? 3 : (N <= 10) ? 2 : 1;
    // doubles
    static constexpr int XLO = 0;                    // N rows: box lo
    static constexpr int XHI = XLO + N * BB;         // N: box hi
    static constexpr int XC = XHI + N * BB;          // N: midpoint x = mid X
    static constexpr int YLO = XC + N * BB;          // N: Gauss-Seidel result lo
    static constexpr int YHI = YLO + N * BB;         // N: hi
    static constexpr int JM = YHI + N * BB;          // 2 N^2: J(X), then M = B J(X), then products
    static constexpr int FR = JM + 2 * N * N * BB;   // 2 N: f(x), then r = B f(x)
    static constexpr int GB = FR + 2 * N * BB;       // N^2: mid J(X), Gauss-Jordan, then B
    static constexpr int PIV = GB + N * N * BB;      // 1: pivot of the current step
    static constexpr int DOUBLES = PIV + BB;
    // ints
    static constexpr int I_ROWID = 0;                // N: original row of each storage column
    static constexpr int I_SLOT = N * BB;            // N: storage column of each original row
    static constexpr int I_SYS = 2 * N * BB;         // system of the box
    static constexpr int I_ITS = I_SYS + BB;         // HS sweeps the box gets
    static constexpr int I_JF = I_ITS + BB;          // J(X) and f(x) needed in this pass
    static constexpr int I_HS = I_JF + BB;           // HS sweep wanted in this pass
    static constexpr int I_CEN = I_HS + BB;          // centred-form test in this pass
    static constexpr int I_CEX = I_CEN + BB;         // the centred form excluded the box
    static constexpr int I_RUN = I_CEX + BB;         // box takes part in the current sweep:
                                                     // 1 Gauss-Seidel, 2 Krawczyk
    static constexpr int I_BAD = I_RUN + BB;         // singular preconditioner: sweep skipped
    static constexpr int I_EMPTY = I_BAD + BB;       // Gauss-Seidel left no point: box dropped
    static constexpr int INTS = I_EMPTY + BB;
    static constexpr size_t BYTES = ((size_t)DOUBLES * 8 + (size_t)INTS * 4 + 15) & ~(size_t)15;
};

// coordinate accessors over the chunk arrays (box b's column)
template <int BB>
struct BoxCol {
    const double *lo, *hi;
    __device__ __forceinline__ ivd operator()(unsigned j) const { return ivd{lo[j * BB], hi[j * BB]}; }
};
template <int BB>
struct ThinCol {
    const double *c;
    __device__ __forceinline__ ivd operator()(unsigned j) const {
        const double v = c[j * BB];
        return ivd{v, v};
    }
};

// J(X) from the derivative polynomials compiled on the host (units q < N^2), and f(x)
// at the midpoint x = mid X as a thin-box evaluation (units N^2 + i), for every box of
// the chunk with I_JF set, by all threads of the block.
// In the cooperative form (COOP) the cluster's CTAs share the units and every result is
// written into each CTA's copy of the chunk (distributed shared memory); the barrier in
// front keeps a fast CTA from overwriting J or f while a peer still reads the last pass's.
template <int N, bool COOP>
__device__ __forceinline__ void jf_block(const SweepArgs &a, const char *blob_smem, double *sd, const int *si,
                                         int t) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT;
    const int *jf = si + C::I_JF;
    int gt = t, GT = NT;
    if (COOP) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        gt = (int)cl.block_rank() * NT + t;
        GT = kCS * NT;
    }
    for (int e = gt; e < (N * N + N) * BB; e += GT) {
        const int q = e / BB, b = e % BB;
        if (!jf[b]) continue;
        const DevSys &S = a.tb.sys[si[C::I_SYS + b]];
        const SysTab Tb = make_tab(blob_smem ? blob_smem : a.tb.blobs + S.blob_off, S);
        ivd v;
        double *dst;
        if (q < N * N) {
            v = poly64(Tb, S.j_poly + q, BoxCol<BB>{sd + C::XLO + b, sd + C::XHI + b});
            dst = sd + C::JM + (2 * q) * BB + b;
        } else {
            const int i = q - N * N;
            v = poly64(Tb, S.f_poly + i, ThinCol<BB>{sd + C::XC + b});
            dst = sd + C::FR + (2 * i) * BB + b;
        }
        if (COOP) {
            cg::cluster_group cl = cg::this_cluster();
#pragma unroll
            for (int r = 0; r < kCS; r++) {
                double *d = cl.map_shared_rank(dst, r);
                d[0] = v.lo;
                d[BB] = v.hi;
            }
        } else {
            dst[0] = v.lo;
            dst[BB] = v.hi;
        }
    }
    if (COOP) cg::this_cluster().sync();
    else __syncthreads();
}

// rows per unit of the cooperative M = B J(X): the fewest that give every unit its own
// warp of the cluster
template <int N>
__host__ __device__ constexpr int coop_rows() {
    int r = 1;
    while ((N + 1) * ((N + r - 1) / r) > kCS * Cfg<N>::NW) r++;
    return r;
}

// Centred (mean-value) form from the expansion of Section 2.3 eq 13: for every y in X,
// f_i(y) lies in F_c,i(X) = f_i(x) + sum_j J_ij(X) (X_j - x_j), folded left over
// j = 1..n from f_i(x).  One equation per unit; sets I_CEX when some F_c,i excludes 0
// (a NaN end never excludes).  Uses the J(X) and f(x) of jf_block.
template <int N>
__device__ __forceinline__ void centred_block(double *sd, int *si, int t) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT;
    const double *J = sd + C::JM;
    const int *cen = si + C::I_CEN;
    for (int e = t; e < N * BB; e += NT) {
        const int i = e / BB, b = e % BB;
        if (!cen[b]) continue;
        ivd acc = {sd[C::FR + (2 * i) * BB + b], sd[C::FR + (2 * i + 1) * BB + b]};
#pragma unroll
        for (int j = 0; j < N; j++) {
            const double xc = sd[C::XC + j * BB + b];
            const ivd d = iv_sub(ivd{sd[C::XLO + j * BB + b], sd[C::XHI + j * BB + b]}, ivd{xc, xc});
            acc = iv_add(acc, iv_mul(ivd{J[(2 * (i * N + j)) * BB + b], J[(2 * (i * N + j) + 1) * BB + b]}, d));
        }
        if (d_pos(acc.lo) || d_neg(acc.hi)) atomicOr(&si[C::I_CEX + b], 1);
    }
    __syncthreads();
}

// One Gauss-Seidel sweep on B f(x) + B J(X)(z - x) = 0 (eq 14, 21, 22) for every box of
// the chunk with I_RUN set (J(X) and f(x) already computed), by all threads of the block.
// Leaves the result in Y and sets I_EMPTY (no root) or I_BAD (singular preconditioner:
// the sweep is skipped).
// Parts: gj_block (mid J(X), Gauss-Jordan, column order), m_block (M = B J(X), r = B f(x)),
// gs_block (Gauss-Seidel); each ends with a barrier.
template <int N>
__device__ __forceinline__ void gj_block(double *sd, int *si, int t) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT;
    double *J = sd + C::JM;   // interval (i, j): lo at (2 (i N + j)) BB, hi at (2 (i N + j) + 1) BB
    double *G = sd + C::GB;   // point (i, j) at (i N + j) BB
    const int *run = si + C::I_RUN;
    int *bad = si + C::I_BAD;

    // A = mid(J(X)), round to nearest
    for (int e = t; e < N * N * BB; e += NT) {
        const int q = e / BB, b = e % BB;
        if (!run[b]) continue;
        const double m = midpoint_rn(J[(2 * q) * BB + b], J[(2 * q + 1) * BB + b]);
        if (!d_finite(m)) atomicOr(&bad[b], 1);
        G[q * BB + b] = m;
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting (Section 2.4), in place: after step k storage
    // column k holds column rowid[k] of the right half [.|I]; entries of identity columns
    // not yet touched are 0 and their updates are exact no-ops, so they are skipped
    for (int k = 0; k < N; k++) {
        if (t < BB) {
            const int b = t;
            if (run[b] && !bad[b]) {
                int piv = k;
                long long best = d_abskey(G[(k * N + k) * BB + b]);
                bool sing = best < 0;          // NaN diagonal: the serial search keeps it
                if (!sing) {
                    for (int i = k + 1; i < N; i++) {
                        const long long v = d_abskey(G[(i * N + k) * BB + b]);
                        if (v > best) { best = v; piv = i; }
                    }
                    sing = best <= 0 || best >= 0x7FF0000000000000LL;   // zero, NaN or infinite
                }
                if (sing) {
                    bad[b] = 1;
                } else {
                    if (piv != k) {
#pragma unroll
                        for (int j = 0; j < N; j++) {
                            const double tmp = G[(k * N + j) * BB + b];
                            G[(k * N + j) * BB + b] = G[(piv * N + j) * BB + b];
                            G[(piv * N + j) * BB + b] = tmp;
                        }
                        const int r = si[C::I_ROWID + k * BB + b];
                        si[C::I_ROWID + k * BB + b] = si[C::I_ROWID + piv * BB + b];
                        si[C::I_ROWID + piv * BB + b] = r;
                    }
                    sd[C::PIV + b] = G[(k * N + k) * BB + b];
                }
            }
        }
        __syncthreads();
        // pivot row divided by the pivot (eq 23; its own column becomes 1 / pivot)
        for (int e = t; e < N * BB; e += NT) {
            const int j = e / BB, b = e % BB;
            if (!run[b] || bad[b]) continue;
            const double pv = sd[C::PIV + b];
            G[(k * N + j) * BB + b] = __ddiv_rn(j == k ? 1.0 : G[(k * N + j) * BB + b], pv);
        }
        __syncthreads();
        // elimination of column k from the other rows (eq 24), one row per unit
        for (int e = t; e < N * BB; e += NT) {
            const int i = e / BB, b = e % BB;
            if (i == k || !run[b] || bad[b]) continue;
            const double f = G[(i * N + k) * BB + b];
            const double rp = G[(k * N + k) * BB + b];
#pragma unroll
            for (int j = 0; j < N; j++)
                if (j != k)
                    G[(i * N + j) * BB + b] = __dsub_rn(G[(i * N + j) * BB + b], __dmul_rn(f, G[(k * N + j) * BB + b]));
            G[(i * N + k) * BB + b] = __dsub_rn(0.0, __dmul_rn(f, rp));
        }
        __syncthreads();
    }
    // storage column k is column rowid[k] of B: restore the column order
    if (t < BB) {
        const int b = t;
        if (run[b] && !bad[b]) {
#pragma unroll
            for (int k = 0; k < N; k++) si[C::I_SLOT + si[C::I_ROWID + k * BB + b] * BB + b] = k;
        }
    }
    __syncthreads();
    for (int e = t; e < N * BB; e += NT) {
        const int i = e / BB, b = e % BB;
        if (!run[b] || bad[b]) continue;
        double rowv[N];
#pragma unroll
        for (int u = 0; u < N; u++) rowv[u] = G[(i * N + si[C::I_SLOT + u * BB + b]) * BB + b];
        bool nf = false;
#pragma unroll
        for (int u = 0; u < N; u++) {
            nf |= !d_finite(rowv[u]);
            G[(i * N + u) * BB + b] = rowv[u];
        }
        if (nf) atomicOr(&bad[b], 1);
    }
    __syncthreads();
}

// M = B J(X) in place of J, one column per unit; r = B f(x) in place of f (unit N)
// (Algorithm 4, outward, u = 1..n in order; starting from the first product equals
// starting from [0,0]).  Cooperative form: units are (column, block of coop_rows rows)
// spread over the cluster, each holds its column in registers across a barrier before
// any entry is overwritten, and writes its entries into every CTA's copy.
template <int N, bool COOP>
__device__ __forceinline__ void m_block(double *sd, const int *si, int t) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT;
    double *J = sd + C::JM;
    const double *G = sd + C::GB;
    const int *run = si + C::I_RUN;
    const int *bad = si + C::I_BAD;
    if constexpr (COOP) {
        constexpr int RB = coop_rows<N>(), NH = (N + RB - 1) / RB, U = (N + 1) * NH;
        cg::cluster_group cl = cg::this_cluster();
        const int gt = (int)cl.block_rank() * NT + t;
        const int u = gt / BB, b = gt % BB;
        const bool on = u < U && run[b] && !bad[b];
        const int j = u / NH, h = u % NH;
        ivd col[N];
        if (on) {
#pragma unroll
            for (int v = 0; v < N; v++)
                col[v] = (j < N) ? ivd{J[(2 * (v * N + j)) * BB + b], J[(2 * (v * N + j) + 1) * BB + b]}
                                 : ivd{sd[C::FR + (2 * v) * BB + b], sd[C::FR + (2 * v + 1) * BB + b]};
        }
        cl.sync();   // every column is read before any entry is overwritten
        if (on) {
            const int i1 = min(N, (h + 1) * RB);
            for (int i = h * RB; i < i1; i++) {
                ivd acc = iv_smul(G[(i * N) * BB + b], col[0]);
#pragma unroll
                for (int v = 1; v < N; v++) acc = iv_add(acc, iv_smul(G[(i * N + v) * BB + b], col[v]));
                double *dst = (j < N) ? J + (2 * (i * N + j)) * BB + b : sd + C::FR + (2 * i) * BB + b;
#pragma unroll
                for (int r = 0; r < kCS; r++) {
                    double *d = cl.map_shared_rank(dst, r);
                    d[0] = acc.lo;
                    d[BB] = acc.hi;
                }
            }
        }
        cl.sync();
    } else {
    for (int e = t; e < (N + 1) * BB; e += NT) {
        const int j = e / BB, b = e % BB;
        if (!run[b] || bad[b]) continue;
        ivd col[N];
        if (j < N) {
#pragma unroll
            for (int u = 0; u < N; u++) col[u] = ivd{J[(2 * (u * N + j)) * BB + b], J[(2 * (u * N + j) + 1) * BB + b]};
        } else {
#pragma unroll
            for (int u = 0; u < N; u++) col[u] = ivd{sd[C::FR + (2 * u) * BB + b], sd[C::FR + (2 * u + 1) * BB + b]};
        }
        for (int i = 0; i < N; i++) {
            ivd acc = iv_smul(G[(i * N) * BB + b], col[0]);
#pragma unroll
            for (int u = 1; u < N; u++) acc = iv_add(acc, iv_smul(G[(i * N + u) * BB + b], col[u]));
            double *dst = (j < N) ? J + (2 * (i * N + j)) * BB + b : sd + C::FR + (2 * i) * BB + b;
            dst[0] = acc.lo;
            dst[BB] = acc.hi;
        }
    }
    __syncthreads();
    }
}

// The widest gap an owner thread's Gauss-Seidel rows left (gap_split): row, width and the
// two pieces of X_i; row -1 while there is none.  Lives in the owner's registers.
struct GapRec {
    bool on;
    int row;
    double w, llo, lhi, ulo, uhi;
};

// warps 0 and 1 alone (the two threads of a box in the Gauss-Seidel rows)
__device__ __forceinline__ void pair_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// Gauss-Seidel (eq 21-22).  Row i folds r_i and the products M_ij (Y_j - x_j), j != i,
// in order j = 1..n, into s_i; then Y_i = X_i meets x_i - s_i / M_ii (extended division).
// Work split:
// * the products with j > i use the box's own coordinates: formed up front, one (i, j)
//   pair per unit, and written over M_ij (nothing reads M_ij afterwards);
// * the terms with j < i join s_i as soon as Y_j is final: while row j's owners work on
//   row j + 1, the other warps add term j to the rows below j + 1 (s_i lives in place of
//   r_i, which Gauss-Seidel boxes do not read again);
// * row i itself belongs to two threads per box on two warps (two FP64 pipes): warp 0
//   takes the lower ends (rd), warp 1 the upper ends (ru) -- the last prefix term, the
//   j > i part of the fold, one quotient each, and their ends of the pieces x_i - q;
//   warp 0 then intersects with X_i (integer compares) and records the result.
// Every end is the same operation on the same operands as in the serial order, so the
// results are bit-identical to it.  With gr.on (the owner's box asks for the two-box
// split) a row whose Y_i meets X_i in two pieces records its gap RN(lower end of the
// upper piece - upper end of the lower piece) in gr when it is wider than the widest so
// far; the row itself still takes the hull.
template <int N>
__device__ __forceinline__ void gs_block(double *sd, int *si, int t, GapRec &gr) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT, NP = N * (N - 1) / 2;
    static_assert(NT >= 128, "the rows need warps 0 and 1 and at least one more");
    double *J = sd + C::JM;
    double *F = sd + C::FR;    // r_i, then the running fold s_i
    double *SX = sd + C::GB;   // lower ends of the row's pieces (B is not read any more)
    const int *run = si + C::I_RUN;
    const int *bad = si + C::I_BAD;
    int *empty = si + C::I_EMPTY;
    for (int e = t; e < N * BB; e += NT) {
        const int i = e / BB, b = e % BB;
        sd[C::YLO + i * BB + b] = sd[C::XLO + i * BB + b];
        sd[C::YHI + i * BB + b] = sd[C::XHI + i * BB + b];
    }
    for (int e = t; e < NP * BB; e += NT) {
        const int pr = e / BB, b = e % BB;
        if (run[b] != 1 || bad[b]) continue;
        int i = 0, r = pr;   // pair pr -> (i, j), j > i, row by row
        while (r >= N - 1 - i) {
            r -= N - 1 - i;
            i++;
        }
        const int j = i + 1 + r;
        const double xc = sd[C::XC + j * BB + b];
        const ivd d = iv_sub(ivd{sd[C::XLO + j * BB + b], sd[C::XHI + j * BB + b]}, ivd{xc, xc});
        const ivd p = iv_mul(ivd{J[(2 * (i * N + j)) * BB + b], J[(2 * (i * N + j) + 1) * BB + b]}, d);
        J[(2 * (i * N + j)) * BB + b] = p.lo;
        J[(2 * (i * N + j) + 1) * BB + b] = p.hi;
    }
    __syncthreads();
    for (int i = 0; i < N; i++) {
        if (t < 64) {
            const int b = t & 31, up = t >> 5;   // up = 0: lower ends, 1: upper ends
            const bool on = b < BB && run[b] == 1 && !bad[b] && !empty[b];
            if (on) {
                double v = F[(2 * i + up) * BB + b];
                if (i > 0) {   // term j = i - 1 with the final Y_{i-1}
                    const double xc = sd[C::XC + (i - 1) * BB + b];
                    const ivd d = iv_sub(ivd{sd[C::YLO + (i - 1) * BB + b], sd[C::YHI + (i - 1) * BB + b]},
                                         ivd{xc, xc});
                    const ivd m = {J[(2 * (i * N + i - 1)) * BB + b], J[(2 * (i * N + i - 1) + 1) * BB + b]};
                    v = up ? __dadd_ru(v, iv_mul_hi(m, d)) : __dadd_rd(v, iv_mul_lo(m, d));
                }
#pragma unroll
                for (int j = 0; j < N; j++) {
                    if (j <= i) continue;
                    v = up ? __dadd_ru(v, J[(2 * (i * N + j) + 1) * BB + b]) : __dadd_rd(v, J[(2 * (i * N + j)) * BB + b]);
                }
                F[(2 * i + up) * BB + b] = v;
            }
            pair_sync();
            ivd s = {0.0, 0.0}, D = {0.0, 0.0};
            bool ok = false;
            int kind = XD_NONE, np = 0;
            double xc = 0.0, yhi[2] = {0.0, 0.0};
            if (on) {
                s = ivd{F[(2 * i) * BB + b], F[(2 * i + 1) * BB + b]};
                D = ivd{J[(2 * (i * N + i)) * BB + b], J[(2 * (i * N + i) + 1) * BB + b]};
                ok = !(d_isnan(s.lo) || d_isnan(s.hi) || d_isnan(D.lo) || d_isnan(D.hi));
            }
            if (ok) {
                const ExtDiv xd = extdiv_setup(s, D);
                kind = xd.kind;
                xc = sd[C::XC + i * BB + b];
                ivd pc[2];
                if (up) {   // upper quotient; lower ends of the pieces x_i - pc
                    np = extdiv_pieces(kind, 0.0, __ddiv_ru(xd.un, xd.ud), pc);
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        if (q < np) SX[q * BB + b] = __dsub_rd(xc, pc[q].hi);
                } else {    // lower quotient; upper ends
                    np = extdiv_pieces(kind, __ddiv_rd(xd.ln, xd.ld), 0.0, pc);
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        if (q < np) yhi[q] = __dsub_ru(xc, pc[q].lo);
                }
            }
            pair_sync();
            if (ok && !up) {
                const double xlo = sd[C::XLO + i * BB + b], xhi = sd[C::XHI + i * BB + b];
                double lo = 0.0, hi = 0.0;
                bool any = false;
                double pa[2] = {0.0, 0.0}, pb[2] = {0.0, 0.0};   // the non-empty pieces
                int npc = 0;
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    if (q >= np) continue;
                    const double a0 = d_max(xlo, SX[q * BB + b]), b0 = d_min(xhi, yhi[q]);
                    if (d_le(a0, b0)) {
                        lo = any ? d_min(lo, a0) : a0;
                        hi = any ? d_max(hi, b0) : b0;
                        any = true;
                        if (npc == 0) { pa[0] = a0; pb[0] = b0; }
                        else { pa[1] = a0; pb[1] = b0; }
                        npc++;
                    }
                }
                if (!any) {
                    empty[b] = 1;
                } else {
                    if (gr.on && npc == 2) {
                        const bool zero_up = !d_le(pa[0], pa[1]);   // piece 1 starts below piece 0
                        const double llo = zero_up ? pa[1] : pa[0], lhi = zero_up ? pb[1] : pb[0];
                        const double ulo = zero_up ? pa[0] : pa[1], uhi = zero_up ? pb[0] : pb[1];
                        const double g = __dsub_rn(ulo, lhi);
                        if (g > gr.w) {
                            gr.w = g;
                            gr.row = i;
                            gr.llo = llo; gr.lhi = lhi; gr.ulo = ulo; gr.uhi = uhi;
                        }
                    }
                    sd[C::YLO + i * BB + b] = lo;
                    sd[C::YHI + i * BB + b] = hi;
                }
            }
        } else if (i > 0) {
            // term j = i - 1 of the rows below i (row i's own is with its owners), on
            // the warps of the other two sub-partitions first (warp w runs on
            // sub-partition w % 4; warps 0 and 1 hold the row)
            const int w = t >> 5, q = w & 3;
            const int rank = q >= 2 ? 2 * (w >> 2) + q - 2 : C::NW / 2 + 2 * ((w >> 2) - 1) + q;
            for (int e = rank * 32 + (t & 31); e < (N - 1 - i) * BB; e += NT - 64) {
                const int i2 = i + 1 + e / BB, b = e % BB;
                if (run[b] != 1 || bad[b] || empty[b]) continue;
                const double xc = sd[C::XC + (i - 1) * BB + b];
                const ivd d = iv_sub(ivd{sd[C::YLO + (i - 1) * BB + b], sd[C::YHI + (i - 1) * BB + b]}, ivd{xc, xc});
                const ivd p = iv_mul(ivd{J[(2 * (i2 * N + i - 1)) * BB + b], J[(2 * (i2 * N + i - 1) + 1) * BB + b]}, d);
                const ivd s = iv_add(ivd{F[(2 * i2) * BB + b], F[(2 * i2 + 1) * BB + b]}, p);
                F[(2 * i2) * BB + b] = s.lo;
                F[(2 * i2 + 1) * BB + b] = s.hi;
            }
        }
        __syncthreads();
    }
}

// Krawczyk step (eq 15-16) for the boxes with run == 2, after m_block: M = B J(X) sits in
// J's place and r = B f(x) in f's.  Row i: K_i = (x_i - r_i) + sum_j ([d_ij, d_ij] - M_ij)
// (X_j - x_j), folded over j = 1..n from the incoming box (rows are independent: one unit
// per row and box), then Y_i = X_i intersected with K_i; a NaN leaves Y_i = X_i, an empty
// intersection marks the box empty.  Runs after gs_block, which has set Y = X.
template <int N>
__device__ __forceinline__ void kr_block(double *sd, int *si, int t) {
    using C = Cfg<N>;
    constexpr int BB = C::BB, NT = C::NT;
    const double *J = sd + C::JM;
    const int *run = si + C::I_RUN;
    const int *bad = si + C::I_BAD;
    int *empty = si + C::I_EMPTY;
    for (int e = t; e < N * BB; e += NT) {
        const int i = e / BB, b = e % BB;
        if (run[b] != 2 || bad[b]) continue;
        const double xi = sd[C::XC + i * BB + b];
        ivd k = iv_sub(ivd{xi, xi}, ivd{sd[C::FR + (2 * i) * BB + b], sd[C::FR + (2 * i + 1) * BB + b]});
#pragma unroll
        for (int j = 0; j < N; j++) {
            const double dij = (i == j) ? 1.0 : 0.0;
            const ivd g = iv_sub(ivd{dij, dij}, ivd{J[(2 * (i * N + j)) * BB + b], J[(2 * (i * N + j) + 1) * BB + b]});
            const double xc = sd[C::XC + j * BB + b];
            const ivd d = iv_sub(ivd{sd[C::XLO + j * BB + b], sd[C::XHI + j * BB + b]}, ivd{xc, xc});
            k = iv_add(k, iv_mul(g, d));
        }
        if (d_isnan(k.lo) || d_isnan(k.hi)) continue;
        const double lo = d_max(sd[C::XLO + i * BB + b], k.lo), hi = d_min(sd[C::XHI + i * BB + b], k.hi);
        if (d_le(lo, hi)) {
            sd[C::YLO + i * BB + b] = lo;
            sd[C::YHI + i * BB + b] = hi;
        } else {
            atomicOr(&empty[b], 1);
        }
    }
    __syncthreads();
}
}  // namespace hsd

// The kernel body.  Independent form (COOP = false): every CTA takes its own chunks.
// Cooperative form (COOP = true, clusters of kCS CTAs, one CTA per SM): a cluster takes
// a chunk and its CTAs work on it together -- each keeps a full copy of the chunk's state
// and runs the serial parts itself (identical results on every copy), while J(X), f(x)
// and M = B J(X) are shared out over the cluster's warps.  A sweep with at most coop_max
// boxes runs in the cooperative form, larger ones in the independent form (the other
// kernel returns at once).
template <int N, bool COOP>
__device__ __forceinline__ void hs_body(const SweepArgs &a, int cache_blob, int64_t coop_max) {
    using namespace hsd;
    using C = Cfg<N>;
    constexpr int BB = C::BB;
    extern __shared__ __align__(16) char smem[];
    // chunk index, two slots used in turn: in the cooperative form the cluster's first CTA
    // writes the next chunk's slot while a peer may not yet have read the current one
    __shared__ long long s_base[2];
    const int t = threadIdx.x, lane = (int)lane_id();
    const size_t blob_bytes = cache_blob ? (size_t)a.blob_smem : 0;
    double *sd = reinterpret_cast<double *>(smem + blob_bytes);
    int *si = reinterpret_cast<int *>(sd + C::DOUBLES);

    WaveCtl *ctl = a.ctl;
    const int64_t count = ctl->surv_count[N];
    if (COOP ? count > coop_max : count <= coop_max) return;   // the other form's sweep
    int rank = 0, group = blockIdx.x;                         // group: this CTA or cluster
    if (COOP) {
        rank = (int)cg::this_cluster().block_rank();
        group = blockIdx.x / kCS;
    }
    if ((int64_t)group * BB >= count) return;   // not needed for this many boxes (whole clusters)
    if (cache_blob) {
        const DevSys &S0 = a.tb.sys[0];
        copy_blob(smem, a.tb.blobs + S0.blob_off, (uint32_t)S0.blob_bytes);   // visible after the next barrier
    }
    const char *blob_smem = cache_blob ? smem : nullptr;
    const Surv *list = a.surv + (size_t)N * a.surv_cap;
    const bool owner = t < BB;   // owner thread of box b = t
    for (int slot = 0;; slot ^= 1) {
        if (COOP) {
            cg::cluster_group cl = cg::this_cluster();
            if (rank == 0 && t == 0) {
                const long long v = (long long)atomicAdd((unsigned long long *)&ctl->hs_cursor[N], (unsigned long long)BB);
#pragma unroll
                for (int r = 0; r < kCS; r++) *cl.map_shared_rank(&s_base[slot], r) = v;
            }
            cl.sync();
        } else {
            if (t == 0) s_base[slot] = (long long)atomicAdd((unsigned long long *)&ctl->hs_cursor[N], (unsigned long long)BB);
            __syncthreads();
        }
        const long long base = s_base[slot];
        if (base >= count) break;
        // the owners fetch their boxes: child `child` of queue entry `parent`
        bool active = false, stopped = false, dropped = false, dropped_c = false;
        int sys = 0, depth = 0, its = 0, cen = 0;
        unsigned st_app = 0, st_con = 0, st_sing = 0, st_gap = 0;
        // a sweep that split the box at a gap: the upper piece of coordinate two_row
        bool two = false;
        int two_row = 0;
        double two_lo = 0.0, two_hi = 0.0;
        GapRec gr{false, -1, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (owner) {
            const int b = t;
            const long long idx = base + b;
            active = idx < count;
            if (active) {
                const Surv sv = list[idx];
                const int64_t pi = sv.parent;
                sys = a.q.sys[pi];
                const uint32_t meta = a.q.meta[pi];
                const bool root = (meta & kRootFlag) != 0;
                depth = (int)(meta & kDepthMask) + (root ? 0 : 1);
                const DevSys &S = a.tb.sys[sys];
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const bool up = (sv.child >> j) & 1u;
                    const double lo = up ? a.q.mid[j * a.q.cap + pi] : a.q.lo[j * a.q.cap + pi];
                    const double hi = up ? a.q.hi[j * a.q.cap + pi] : a.q.mid[j * a.q.cap + pi];
                    sd[C::XLO + j * BB + b] = lo;
                    sd[C::XHI + j * BB + b] = hi;
                    sd[C::XC + j * BB + b] = midpoint_rn(lo, hi);
                }
                if (S.hs_enable && depth >= S.hs_min_depth) its = S.hs_iters > 0 ? S.hs_iters : 1;
                cen = S.centred;
            }
            si[C::I_SYS + b] = sys;
            si[C::I_ITS + b] = its > cen ? its : cen;   // passes: the centred test needs J, f once
        }
        // passes while some box wants one (a block-wide vote; in the cooperative form every
        // CTA holds the same boxes, so all of them take the same number of passes)
        const int my_passes = owner ? (its > cen ? its : cen) : 0;
        int my_cen = 0, my_kr = 0;   // this owner's box takes the centred test / Krawczyk step
        for (int it = 0; __syncthreads_or(my_passes > it); it++) {
            // pass `it`: J(X), f(x); on the first pass the centred test (if asked), then
            // the Hansen-Sengupta sweep for the boxes that want one and were not excluded
            if (owner) {
                const int b = t;
                const bool jf = active && !stopped && it < si[C::I_ITS + b];
                si[C::I_JF + b] = jf ? 1 : 0;
                si[C::I_HS + b] = (jf && it < its) ? 1 : 0;
                my_cen = (jf && it == 0 && cen) ? 1 : 0;
                si[C::I_CEN + b] = my_cen;
                si[C::I_CEX + b] = 0;
                si[C::I_BAD + b] = 0;
                si[C::I_EMPTY + b] = 0;
#pragma unroll
                for (int k = 0; k < N; k++) si[C::I_ROWID + k * BB + b] = k;
            }
            __syncthreads();
            jf_block<N, COOP>(a, blob_smem, sd, si, t);
            if (__syncthreads_or(my_cen)) centred_block<N>(sd, si, t);
            if (owner) {
                const int b = t;
                const bool run = si[C::I_HS + b] && !si[C::I_CEX + b];
                si[C::I_RUN + b] = run ? (a.tb.sys[si[C::I_SYS + b]].krawczyk ? 2 : 1) : 0;
                my_kr = si[C::I_RUN + b] == 2 ? 1 : 0;
                st_app += run ? 1u : 0u;
                if (run && it == 0 && rank == 0)   // every CTA of a cluster runs this; one counts
                    atomicAdd(stat_ptr(a, sys, ST_DEPTH_HS + (depth < kDepthSlots ? depth : kDepthSlots - 1)), 1ull);
                if (si[C::I_CEX + b]) {
                    dropped_c = true;
                    stopped = true;
                }
            }
            if (owner) {
                gr.on = si[C::I_RUN + t] == 1 && a.tb.sys[si[C::I_SYS + t]].gap_split;
                gr.row = -1;
                gr.w = 0.0;
            }
            __syncthreads();
            gj_block<N>(sd, si, t);
            m_block<N, COOP>(sd, si, t);
            gs_block<N>(sd, si, t, gr);
            if (__syncthreads_or(my_kr)) kr_block<N>(sd, si, t);
            if (owner && si[C::I_RUN + t]) {
                const int b = t;
                if (si[C::I_EMPTY + b]) {
                    dropped = true;
                    stopped = true;
                } else if (si[C::I_BAD + b]) {
                    st_sing++;
                    stopped = true;
                } else {
                    bool changed = false;
#pragma unroll
                    for (int j = 0; j < N; j++) {
                        const double ylo = sd[C::YLO + j * BB + b], yhi = sd[C::YHI + j * BB + b];
                        changed |= !d_same(ylo, sd[C::XLO + j * BB + b]) || !d_same(yhi, sd[C::XHI + j * BB + b]);
                        sd[C::XLO + j * BB + b] = ylo;
                        sd[C::XHI + j * BB + b] = yhi;
                        sd[C::XC + j * BB + b] = midpoint_rn(ylo, yhi);
                    }
                    if (gr.row >= 0) {
                        // two boxes at the widest gap: this one keeps the lower piece, the
                        // upper one takes the accept / split step after it; no more sweeps
                        sd[C::XLO + gr.row * BB + b] = gr.llo;
                        sd[C::XHI + gr.row * BB + b] = gr.lhi;
                        sd[C::XC + gr.row * BB + b] = midpoint_rn(gr.llo, gr.lhi);
                        two = true;
                        two_row = gr.row;
                        two_lo = gr.ulo;
                        two_hi = gr.uhi;
                        changed = true;
                        st_gap = 1;
                        stopped = true;
                    }
                    st_con += changed ? 1u : 0u;
                    // iterated until the contraction stalls (Section 2.3): a sweep that
                    // leaves the box unchanged would leave it unchanged again
                    if (!changed) stopped = true;
                }
            }
            __syncthreads();
        }
        // Algorithm 1 termination (II) and the split, by warp 0 (lane b owns box b); in the
        // cooperative form only the cluster's first CTA writes.  A box split at a gap takes
        // a second pass with the upper piece in its gap coordinate.
        if (t < 32 && rank == 0) {
            const int b = t;
            const int passes = __any_sync(kFull, two) ? 2 : 1;
            for (int pass = 0; pass < passes; pass++) {
            const bool act = active && (pass == 0 || two);
            if (pass == 1 && two) {
                sd[C::XLO + two_row * BB + b] = two_lo;
                sd[C::XHI + two_row * BB + b] = two_hi;
            }
            int fate = 0;   // 0 none / dropped, 1 accepted, 2 new parent
            int flag = 0;
            int jw = 0;     // the widest coordinate (the first of equal widths)
            unsigned st_uns = 0, st_empty = 0, st_cex = 0;
            if (act) {
                const DevSys &S = a.tb.sys[sys];
                if (dropped_c) {
                    st_cex = 1;
                } else if (dropped) {
                    st_empty = 1;
                } else {
                    double w = 0.0;
#pragma unroll
                    for (int j = 0; j < N; j++) {
                        const double wj = __dsub_rn(sd[C::XHI + j * BB + b], sd[C::XLO + j * BB + b]);
                        if (d_key(wj) > d_key(w)) { w = wj; jw = j; }
                    }
                    if (d_key(w) <= d_key(S.tol)) {
                        fate = 1;
                        flag = 1;
                    } else {
                        const double lw = sd[C::XLO + jw * BB + b], hw = sd[C::XHI + jw * BB + b];
                        const double mw = midpoint_rn(lw, hw);
                        if (d_le(mw, lw) && d_le(lw, mw)) {
                            fate = 1;
                            flag = 2;
                            st_uns++;
                        } else if (d_le(mw, hw) && d_le(hw, mw)) {
                            fate = 1;
                            flag = 2;
                            st_uns++;
                        } else if (depth + 1 > S.max_depth) {
                            fate = 1;
                            flag = 4;
                        } else {
                            fate = 2;
                        }
                    }
                }
            }
            // accepted boxes, into the system's result region
            const int sys0 = __shfl_sync(kFull, sys, 0);
            const bool uniform = __all_sync(kFull, !act || sys == sys0);
            {
                const unsigned ma = __ballot_sync(kFull, fate == 1);
                long long k = -1;
                if (ma && uniform) {
                    unsigned long long pos = 0;
                    if (lane == 0) pos = atomicAdd(stat_ptr(a, sys0, ST_OUT), (unsigned long long)__popc(ma));
                    pos = __shfl_sync(kFull, pos, 0);
                    k = (long long)(pos + __popc(ma & lanemask_lt()));
                } else if (fate == 1) {
                    k = (long long)atomicAdd(stat_ptr(a, sys, ST_OUT), 1ull);
                }
                if (fate == 1) {
                    const DevSys &Ss = a.tb.sys[sys];
                    if (k < Ss.out_cap) {
                        const long long e = Ss.out_base + k;
#pragma unroll
                        for (int j = 0; j < N; j++) {
                            a.out.lo[j * a.out.cap + e] = sd[C::XLO + j * BB + b];
                            a.out.hi[j * a.out.cap + e] = sd[C::XHI + j * BB + b];
                        }
                        a.out.sys[e] = sys;
                        a.out.flags[e] = flag;
                        a.out.depth[e] = depth;
                    } else {
                        atomicOr(stat_ptr(a, sys, ST_FLAGS), (unsigned long long)kFlagResultOverflow);
                    }
                    if (flag == 4) atomicOr(stat_ptr(a, sys, ST_FLAGS), (unsigned long long)kFlagDepthCut);
                }
            }
            // new parents: the split midpoints are the box midpoints (Algorithm 2); with
            // bisection only the widest coordinate has one (mid = hi elsewhere) and the
            // meta word carries that coordinate
            const unsigned ms = __ballot_sync(kFull, fate == 2);
            if (ms) {
                unsigned long long pos = 0;
                if (lane == 0) pos = atomicAdd((unsigned long long *)&ctl->staged, (unsigned long long)__popc(ms));
                pos = __shfl_sync(kFull, pos, 0);
                if (fate == 2) {
                    const long long k = (long long)(pos + __popc(ms & lanemask_lt()));
                    if (k < a.stage.cap) {
                        const bool bis = a.tb.sys[sys].bisect != 0;
#pragma unroll
                        for (int j = 0; j < N; j++) {
                            const double lo = sd[C::XLO + j * BB + b], hi = sd[C::XHI + j * BB + b];
                            a.stage.lo[j * a.stage.cap + k] = lo;
                            a.stage.mid[j * a.stage.cap + k] = (bis && j != jw) ? hi : midpoint_rn(lo, hi);
                            a.stage.hi[j * a.stage.cap + k] = hi;
                        }
                        a.stage.sys[k] = sys;
                        a.stage.meta[k] = ((uint32_t)depth & kDepthMask) | (bis ? ((uint32_t)jw << kSplitShift) : 0u) |
                                          ((uint32_t)(bis ? 1 : N) << kFanShift);
                    } else {
                        ctl->error = 1;
                    }
                }
            }
            // statistics (new parents also enter the live count): one atomic per warp when
            // the warp holds a single system; the sweep's counters only in the first pass
            const bool p0 = pass == 0;
            if (p0 && fate != 0)   // survived evaluation and contraction at its depth
                atomicAdd(stat_ptr(a, sys, ST_DEPTH_KEPT + (depth < kDepthSlots ? depth : kDepthSlots - 1)), 1ull);
            unsigned v[10] = {p0 ? st_app : 0u, st_empty, p0 ? st_con : 0u, p0 ? st_sing : 0u,
                              (fate == 1 && flag != 4) ? 1u : 0u, st_uns, fate == 2 ? 1u : 0u, fate == 2 ? 1u : 0u,
                              st_cex, p0 ? st_gap : 0u};
            const int slot[10] = {ST_HS_APPLIED, ST_HS_EMPTY, ST_HS_CONTRACTED, ST_HS_SINGULAR, ST_ACCEPTED,
                                  ST_UNSPLITTABLE, ST_SPLIT, ST_LIVE, ST_EXCL_CENTRED, ST_GAP_SPLITS};
            if (uniform) {
#pragma unroll
                for (int q = 0; q < 10; q++) {
                    const unsigned tot = __reduce_add_sync(kFull, v[q]);
                    if (lane == 0 && tot) atomicAdd(stat_ptr(a, sys0, slot[q]), (unsigned long long)tot);
                }
            } else if (act) {
#pragma unroll
                for (int q = 0; q < 10; q++)
                    if (v[q]) atomicAdd(stat_ptr(a, sys, slot[q]), (unsigned long long)v[q]);
            }
            }
        }
        __syncthreads();   // the chunk's arrays and s_base are reused by the next chunk
    }
    if (COOP) cg::this_cluster().sync();   // no CTA leaves while a peer may still write to it
}

template <int N>
__global__ void __launch_bounds__(hsd::Cfg<N>::NT, hsd::Cfg<N>::MIN_BLOCKS)
    k_hs(SweepArgs a, int cache_blob, long long coop_max) {
    hs_body<N, false>(a, cache_blob, coop_max);
}

template <int N>
__global__ void __cluster_dims__(hsd::kCS, 1, 1) __launch_bounds__(hsd::Cfg<N>::NT, 1)
    k_hs_coop(SweepArgs a, int cache_blob, long long coop_max) {
    hs_body<N, true>(a, cache_blob, coop_max);
}

// ---- launcher -------------------------------------------------------------------

// largest dynamic shared memory a block may use (227 KB less the static s_base)
constexpr size_t kHsSmemLimit = 227 * 1024 - 64;
// a cooperative CTA asks for at least this much, so no two share an SM
constexpr size_t kOneCtaPerSm = 120 * 1024;

// resident clusters of the cooperative kernel for a shared memory size, queried once per
// size (the launchers may run on several host threads)
int coop_clusters_cached(const void *func, int num_sms, int threads, size_t smem, cudaError_t *err);

template <int N>
static cudaError_t launch_hs_n(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) {
    *kernels = 1;
    using C = hsd::Cfg<N>;
    // cache the term table in shared memory when the plan holds one system and it fits
    const bool cache = a.single && (size_t)a.blob_smem + C::BYTES <= kHsSmemLimit;
    const size_t smem = (cache ? (size_t)a.blob_smem : 0) + C::BYTES;
    long long coop_max = 0;
    if constexpr (N <= hsd::kCoopMaxN) {
      if (num_sms >= 2 * hsd::kCS) {
        // narrow sweeps: clusters of kCS CTAs, one per SM, one chunk per cluster that can
        // be resident at once (a wider sweep runs faster in the independent form)
        const size_t csmem = smem > kOneCtaPerSm ? smem : kOneCtaPerSm;
        cudaError_t e = allow_max_dynamic_smem((const void *)k_hs_coop<N>);
        if (e != cudaSuccess) return e;
        const int active_clusters = coop_clusters_cached((const void *)k_hs_coop<N>, num_sms, C::NT, csmem, &e);
        if (e != cudaSuccess) return e;
        if (active_clusters > 0) {
            coop_max = (long long)active_clusters * C::BB;
            k_hs_coop<N><<<active_clusters * hsd::kCS, C::NT, csmem, st>>>(a, cache ? 1 : 0, coop_max);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            *kernels = 2;
        }
      }
    }
    cudaError_t e = allow_max_dynamic_smem((const void *)k_hs<N>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;   // blocks per SM at this shared memory size
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hs<N>, C::NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_hs<N><<<num_sms * per_sm, C::NT, smem, st>>>(a, cache ? 1 : 0, coop_max);
    return cudaGetLastError();
}

}  // namespace ivs
