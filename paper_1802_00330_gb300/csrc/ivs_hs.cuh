// ivs_hs.cuh -- Hansen-Sengupta sweep and the accept / split step for the boxes that
// survived the evaluation (Section 2.3 eq 14, 17-22; Algorithm 3; Gauss-Jordan of
// Section 2.4; Algorithm 4 products; Algorithm 1 termination (II); Algorithm 2 split).
//
// Mapping: one thread per box, 32 boxes per warp taken from an atomic cursor so a
// sweep's boxes spread over every SM.  GB300's FP64 pipe retires 2 lane-operations per
// cycle per SM and charges a whole warp instruction whatever the number of active
// lanes, so every lane of every FP64 instruction carries a different box; two or three
// resident warps per SM already keep the pipe busy.  Matrices live in per-thread shared
// memory (structure of arrays, conflict-free); the system's term table is cached in
// shared memory when the plan holds one system.  Comparisons, sign tests, NaN and
// finiteness checks run on the integer pipes.  Templated on n; the instantiations are
// spread over several translation units (ivs_hs_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "ivs_internal.h"
#include "ivs_interval.cuh"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

namespace ivs {

namespace hsd {
constexpr unsigned kFull = 0xFFFFFFFFu;
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

// per-thread scratch (doubles, structure of arrays with the block's thread stride T)
template <int N>
struct Scratch {
    static constexpr int J = 0;              // 2 N N : J(X), then M = B J
    static constexpr int G = 2 * N * N;      // N N   : Gauss-Jordan matrix, then B
    static constexpr int X = 3 * N * N;      // 2 N   : box for the interpreter
    static constexpr int DOUBLES = X + 2 * N;
    static constexpr int INTS = 2 * N;       // row ids, then column slots
    static constexpr size_t BYTES = (size_t)DOUBLES * 8 + (size_t)INTS * 4;
};

struct BoxS {
    const double *X;
    int T;
    __device__ __forceinline__ ivd operator()(unsigned j) const { return ivd{X[(2 * j) * T], X[(2 * j + 1) * T]}; }
};
}  // namespace hsd

// One Gauss-Seidel sweep on B f(x) + B J(X)(z - x) = 0 (eq 14, 21, 22).
// Returns 0 (Xo written), 1 (empty), 2 (skipped: singular preconditioner).
template <int N>
__device__ int hs_sweep(const SysTab &Tb, const DevSys &S, const double *Xlo, const double *Xhi,
                        double *Xolo, double *Xohi, double *sm, int *smi, int T) {
    using namespace hsd;
    using L = Scratch<N>;
    double *J = sm + L::J * T;
    double *G = sm + L::G * T;
    double *X = sm + L::X * T;
    int *rowid = smi;
    int *slot_of = smi + N * T;
#pragma unroll
    for (int j = 0; j < N; j++) {
        X[(2 * j) * T] = Xlo[j];
        X[(2 * j + 1) * T] = Xhi[j];
    }
    // J(X) from the derivative polynomials compiled on the host
    for (int q = 0; q < N * N; q++) {
        const ivd v = poly64(Tb, S.j_poly + q, BoxS{X, T});
        J[(2 * q) * T] = v.lo;
        J[(2 * q + 1) * T] = v.hi;
    }
    // A = mid(J(X)), round to nearest
    bool bad = false;
    for (int q = 0; q < N * N; q++) {
        const double m = midpoint_rn(J[(2 * q) * T], J[(2 * q + 1) * T]);
        bad |= !d_finite(m);
        G[q * T] = m;
    }
    if (bad) return 2;
    // Gauss-Jordan with partial pivoting (Section 2.4), in place: after step k storage
    // column k holds column rowid[k] of the right half [.|I]; entries of identity columns
    // not yet touched are 0 and their updates are exact no-ops, so they are skipped
#pragma unroll
    for (int k = 0; k < N; k++) rowid[k * T] = k;
    for (int k = 0; k < N; k++) {
        int piv = k;
        long long best = d_abskey(G[(k * N + k) * T]);
        if (best < 0) return 2;            // NaN diagonal: the serial search keeps it, singular
        for (int i = k + 1; i < N; i++) {
            const long long v = d_abskey(G[(i * N + k) * T]);
            if (v > best) { best = v; piv = i; }
        }
        if (best <= 0 || best >= 0x7FF0000000000000LL) return 2;   // zero, NaN or infinite
        if (piv != k) {
#pragma unroll
            for (int j = 0; j < N; j++) {
                const double t = G[(k * N + j) * T];
                G[(k * N + j) * T] = G[(piv * N + j) * T];
                G[(piv * N + j) * T] = t;
            }
            const int t = rowid[k * T];
            rowid[k * T] = rowid[piv * T];
            rowid[piv * T] = t;
        }
        const double pv = G[(k * N + k) * T];
        const double rp = __ddiv_rn(1.0, pv);                           // eq 23 (identity column)
#pragma unroll
        for (int j = 0; j < N; j++)
            if (j != k) G[(k * N + j) * T] = __ddiv_rn(G[(k * N + j) * T], pv);   // eq 23
        G[(k * N + k) * T] = rp;
        for (int i = 0; i < N; i++) {                                  // eq 24
            if (i == k) continue;
            const double f = G[(i * N + k) * T];
#pragma unroll
            for (int j = 0; j < N; j++)
                if (j != k) G[(i * N + j) * T] = __dsub_rn(G[(i * N + j) * T], __dmul_rn(f, G[(k * N + j) * T]));
            G[(i * N + k) * T] = __dsub_rn(0.0, __dmul_rn(f, rp));
        }
    }
    // storage column k is column rowid[k] of B: restore the column order
#pragma unroll
    for (int k = 0; k < N; k++) slot_of[rowid[k * T] * T] = k;
    for (int i = 0; i < N; i++) {
        double rowv[N];
#pragma unroll
        for (int u = 0; u < N; u++) rowv[u] = G[(i * N + slot_of[u * T]) * T];
#pragma unroll
        for (int u = 0; u < N; u++) {
            bad |= !d_finite(rowv[u]);
            G[(i * N + u) * T] = rowv[u];
        }
    }
    if (bad) return 2;
    // x = mid(X); f(x) as a thin-box evaluation
    double xc[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        xc[j] = midpoint_rn(Xlo[j], Xhi[j]);
        X[(2 * j) * T] = xc[j];
        X[(2 * j + 1) * T] = xc[j];
    }
    ivd fx[N];
    for (int i = 0; i < N; i++) fx[i] = poly64(Tb, S.f_poly + i, BoxS{X, T});
    // M = B J(X) in place of J, column by column; r = B f(x) (Algorithm 4, outward,
    // u = 1..n in order; starting from the first product equals starting from [0,0])
    for (int j = 0; j < N; j++) {
        ivd col[N];
#pragma unroll
        for (int u = 0; u < N; u++) col[u] = ivd{J[(2 * (u * N + j)) * T], J[(2 * (u * N + j) + 1) * T]};
        for (int i = 0; i < N; i++) {
            ivd acc = iv_smul(G[(i * N) * T], col[0]);
#pragma unroll
            for (int u = 1; u < N; u++) acc = iv_add(acc, iv_smul(G[(i * N + u) * T], col[u]));
            J[(2 * (i * N + j)) * T] = acc.lo;
            J[(2 * (i * N + j) + 1) * T] = acc.hi;
        }
    }
    ivd r[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        ivd acc = iv_smul(G[(i * N) * T], fx[0]);
#pragma unroll
        for (int u = 1; u < N; u++) acc = iv_add(acc, iv_smul(G[(i * N + u) * T], fx[u]));
        r[i] = acc;
    }
    // Gauss-Seidel (eq 21-22)
#pragma unroll
    for (int j = 0; j < N; j++) { Xolo[j] = Xlo[j]; Xohi[j] = Xhi[j]; }
#pragma unroll
    for (int i = 0; i < N; i++) {
        ivd s = r[i];
#pragma unroll
        for (int j = 0; j < N; j++) {
            if (j == i) continue;
            const ivd mij = {J[(2 * (i * N + j)) * T], J[(2 * (i * N + j) + 1) * T]};
            const ivd d = iv_sub(ivd{Xolo[j], Xohi[j]}, ivd{xc[j], xc[j]});
            s = iv_add(s, iv_mul(mij, d));
        }
        const ivd D = {J[(2 * (i * N + i)) * T], J[(2 * (i * N + i) + 1) * T]};
        if (d_isnan(s.lo) || d_isnan(s.hi) || d_isnan(D.lo) || d_isnan(D.hi)) continue;
        ivd pc[2];
        const int np = iv_extdiv(s, D, pc);
        double lo = 0.0, hi = 0.0;
        bool any = false;
        for (int q = 0; q < np; q++) {
            const ivd Y = iv_sub(ivd{xc[i], xc[i]}, pc[q]);
            const double a0 = d_max(Xlo[i], Y.lo), b0 = d_min(Xhi[i], Y.hi);
            if (d_le(a0, b0)) {
                lo = any ? d_min(lo, a0) : a0;
                hi = any ? d_max(hi, b0) : b0;
                any = true;
            }
        }
        if (!any) return 1;
        Xolo[i] = lo;
        Xohi[i] = hi;
    }
    return 0;
}

template <int N>
__global__ void __launch_bounds__(128) k_hs(SweepArgs a) {
    using namespace hsd;
    using L = Scratch<N>;
    extern __shared__ __align__(16) char smem[];
    const int T = blockDim.x, tid = threadIdx.x;
    const size_t blob_bytes = a.single ? (size_t)a.blob_smem : 0;
    double *sm = reinterpret_cast<double *>(smem + blob_bytes) + tid;
    int *smi = reinterpret_cast<int *>(reinterpret_cast<double *>(smem + blob_bytes) + (size_t)L::DOUBLES * T) + tid;

    WaveCtl *ctl = a.ctl;
    const int64_t count = ctl->surv_count[N];
    if (count == 0) return;
    if (a.single) {
        const DevSys &S0 = a.tb.sys[0];
        copy_blob(smem, a.tb.blobs + S0.blob_off, (uint32_t)S0.blob_bytes);
        __syncthreads();
    }
    const Surv *list = a.surv + (size_t)N * a.surv_cap;
    const unsigned lane = lane_id();
    for (;;) {
        // each warp takes the next 32 boxes, so every SM gets a share of a small sweep
        unsigned long long ws = 0;
        if (lane == 0) ws = atomicAdd((unsigned long long *)&ctl->hs_cursor[N], 32ull);
        ws = __shfl_sync(kFull, ws, 0);
        if ((long long)ws >= count) break;
        const int64_t idx = (int64_t)ws + lane;
        const bool active = idx < count;
        int fate = 0;   // 0 none / dropped, 1 accepted, 2 new parent
        int flag = 0, sys = 0, depth = 0;
        double Xlo[N], Xhi[N], xm[N];
        unsigned st_app = 0, st_empty = 0, st_con = 0, st_sing = 0, st_uns = 0;
        if (active) {
            const Surv sv = list[idx];
            const int64_t pi = sv.parent;
            sys = a.q.sys[pi];
            const uint32_t meta = a.q.meta[pi];
            const bool root = (meta & kRootFlag) != 0;
            depth = (int)(meta & kDepthMask) + (root ? 0 : 1);
            const DevSys S = a.tb.sys[sys];
            const SysTab Tb = make_tab(a.single ? smem : a.tb.blobs + S.blob_off, S);
#pragma unroll
            for (int j = 0; j < N; j++) {
                const bool up = (sv.child >> j) & 1u;
                Xlo[j] = up ? a.q.mid[j * a.q.cap + pi] : a.q.lo[j * a.q.cap + pi];
                Xhi[j] = up ? a.q.hi[j * a.q.cap + pi] : a.q.mid[j * a.q.cap + pi];
            }
            bool dropped = false;
            if (S.hs_enable && depth >= S.hs_min_depth) {
                const int iters = S.hs_iters > 0 ? S.hs_iters : 1;
                for (int it = 0; it < iters; it++) {
                    st_app++;
                    double Ylo[N], Yhi[N];
                    const int rc = hs_sweep<N>(Tb, S, Xlo, Xhi, Ylo, Yhi, sm, smi, T);
                    if (rc == 1) { dropped = true; break; }
                    if (rc == 2) { st_sing++; break; }
                    bool changed = false;
#pragma unroll
                    for (int j = 0; j < N; j++) {
                        changed |= (__double_as_longlong(Ylo[j]) != __double_as_longlong(Xlo[j]) && !(d_iszero(Ylo[j]) && d_iszero(Xlo[j]))) ||
                                   (__double_as_longlong(Yhi[j]) != __double_as_longlong(Xhi[j]) && !(d_iszero(Yhi[j]) && d_iszero(Xhi[j])));
                        Xlo[j] = Ylo[j];
                        Xhi[j] = Yhi[j];
                    }
                    st_con += changed ? 1u : 0u;
                }
            }
            if (dropped) {
                st_empty++;
            } else {
                // Algorithm 1 termination (II): width test; otherwise split at midpoints
                double w = 0.0;
                int jw = 0;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double wj = __dsub_rn(Xhi[j], Xlo[j]);
                    if (d_key(wj) > d_key(w)) { w = wj; jw = j; }
                }
                if (d_key(w) <= d_key(S.tol)) {
                    fate = 1;
                    flag = 1;
                } else {
#pragma unroll
                    for (int j = 0; j < N; j++) xm[j] = midpoint_rn(Xlo[j], Xhi[j]);
                    double mw = xm[0], lw = Xlo[0], hw = Xhi[0];
#pragma unroll
                    for (int j = 1; j < N; j++)
                        if (j == jw) { mw = xm[j]; lw = Xlo[j]; hw = Xhi[j]; }
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
        const bool uniform = __all_sync(kFull, !active || sys == sys0);
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
                        a.out.lo[j * a.out.cap + e] = Xlo[j];
                        a.out.hi[j * a.out.cap + e] = Xhi[j];
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
        // new parents
        const unsigned ms = __ballot_sync(kFull, fate == 2);
        if (ms) {
            unsigned long long pos = 0;
            if (lane == 0) pos = atomicAdd((unsigned long long *)&ctl->staged, (unsigned long long)__popc(ms));
            pos = __shfl_sync(kFull, pos, 0);
            if (fate == 2) {
                const long long k = (long long)(pos + __popc(ms & lanemask_lt()));
                if (k < a.stage.cap) {
#pragma unroll
                    for (int j = 0; j < N; j++) {
                        a.stage.lo[j * a.stage.cap + k] = Xlo[j];
                        a.stage.mid[j * a.stage.cap + k] = xm[j];
                        a.stage.hi[j * a.stage.cap + k] = Xhi[j];
                    }
                    a.stage.sys[k] = sys;
                    a.stage.meta[k] = (uint32_t)depth & kDepthMask;
                } else {
                    ctl->error = 1;
                }
            }
        }
        // statistics (new parents also enter the live count): one atomic per warp when
        // the warp holds a single system
        unsigned v[8] = {st_app, st_empty, st_con, st_sing, (fate == 1 && flag != 4) ? 1u : 0u, st_uns,
                         fate == 2 ? 1u : 0u, fate == 2 ? 1u : 0u};
        const int slot[8] = {ST_HS_APPLIED, ST_HS_EMPTY, ST_HS_CONTRACTED, ST_HS_SINGULAR, ST_ACCEPTED,
                             ST_UNSPLITTABLE, ST_SPLIT, ST_LIVE};
        if (uniform) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const unsigned tot = __reduce_add_sync(kFull, v[q]);
                if (lane == 0 && tot) atomicAdd(stat_ptr(a, sys0, slot[q]), (unsigned long long)tot);
            }
        } else if (active) {
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (v[q]) atomicAdd(stat_ptr(a, sys, slot[q]), (unsigned long long)v[q]);
        }
    }
}

// ---- launcher -------------------------------------------------------------------

// threads per block: as many (up to 128) as keep the block within ~200 KB of shared memory
template <int N>
inline int hs_threads(size_t blob) {
    const size_t per = hsd::Scratch<N>::BYTES;
    int t = (int)(((200u * 1024u) - blob) / per);
    t = (t / 32) * 32;
    if (t > 128) t = 128;
    if (t < 32) t = 32;
    return t;
}

template <int N>
static cudaError_t launch_hs_n(const SweepArgs &a, int num_sms, cudaStream_t st) {
    static int per_sm = 0;             // blocks per SM, found once per configuration
    static size_t configured_smem = 0;
    const size_t blob = a.single ? (size_t)a.blob_smem : 0;
    const int T = hs_threads<N>(blob);
    const size_t smem = blob + (size_t)T * hsd::Scratch<N>::BYTES;
    if (per_sm == 0 || configured_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(k_hs<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int bl = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, k_hs<N>, T, smem);
        if (e != cudaSuccess) return e;
        per_sm = bl < 1 ? 1 : bl;
        configured_smem = smem;
    }
    k_hs<N><<<num_sms * per_sm, T, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ivs
