// ivs_kernels.cu -- the per-box sweep over the device queue (sm_103a): control,
// evaluation stages, and the sweep loop as one CUDA graph.
//
// Paper map: Definition 1-2 and Algorithm 2 (evaluation and exclusion of the 2^n children
// of each parent); Algorithm 1 (the loop M_k -> M_{k+1} until the queue is empty).  The
// Hansen-Sengupta stage and the accept / split step are in ivs_hs.cuh.  Every operation
// sequence matches the serial definition step for step (same fold orders, same
// roundings), so the sorted result set is identical to the serial solver's.
#include <cuda_runtime.h>

#include <mutex>

#include "ivs_internal.h"
#include "ivs_interval.cuh"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

namespace ivs {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kEvalThreads = 256;
constexpr int kEvalWarps = kEvalThreads / 32;
constexpr int kEval64Threads = 128;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ unsigned long long *stat_ptr(const SweepArgs &a, int sys, int slot) {
    return a.stats + (size_t)sys * ST_COUNT + slot;
}

// ------------------------------------------------------------------------------------
// sweep control
// ------------------------------------------------------------------------------------

// Pops K parents from the top of the queue, as many as fit: the K popped parents'
// children (2^n each, 1 for an initial box) must fit the sweep's budget W, and in the
// worst case (every child kept and split again) the queue must hold them:
// top - K + children <= cap.  One block scans the fan-outs of the top entries.
constexpr int kBeginThreads = 1024;
constexpr int kBeginPer = 64;       // entries per thread: a window of 65536 parents
constexpr size_t kBeginSmem = (size_t)kBeginThreads * kBeginPer;   // one byte per window entry
// Serving with per-system regions, one block.  Least attained service first (the
// default): the regions with entries are taken in order of the boxes their request has
// processed so far (fewest first; a bitonic sort of up to kLasMax slots in shared memory),
// and each pops as many parents as its region allows until the sweep's W children are
// used up -- requests that need little work finish in few sweeps, whatever else is in
// flight.  Fair share (rg.fair_share, or more than kLasMax slots): every region gets W
// divided by the regions with entries (at least one parent), in an order that rotates
// with the sweep count.  Either way a region pops breadth first while under half full
// and one parent at a time beyond; the schedule never changes a result.
constexpr int kLasMax = 4096;
__device__ void wave_begin_regions(const SweepArgs &a, unsigned long long *s_key) {
    __shared__ long long s_red[kBeginThreads];
    __shared__ long long s_active, s_total, s_run;
    const DevRegions &rg = a.rg;
    WaveCtl *c = a.ctl;
    const int t = threadIdx.x, S = rg.n;
    const int64_t waves = c->waves;
    if (t == 0) { s_active = 0; s_total = 0; s_run = 0; }
    __syncthreads();
    // entries each region holds after the last sweep
    long long act = 0, tot = 0;
    for (int sl = t; sl < S; sl += kBeginThreads) {
        const int64_t held = rg.rem[sl] + (int64_t)rg.cursor[sl];
        rg.rem[sl] = held;
        rg.cursor[sl] = 0;
        act += held > 0 ? 1 : 0;
        tot += held;
    }
    atomicAdd((unsigned long long *)&s_active, (unsigned long long)act);
    atomicAdd((unsigned long long *)&s_total, (unsigned long long)tot);
    __syncthreads();
    const bool las = !rg.fair_share && S <= kLasMax;
    const long long share = las ? a.wave_children : a.wave_children / (s_active > 0 ? s_active : 1);
    if (las) {
        // keys (boxes processed, slot), slots without entries last; sorted ascending
        int n2 = 1;
        while (n2 < S) n2 <<= 1;
        for (int q = t; q < n2; q += kBeginThreads) {
            unsigned long long key = ~0ull;
            if (q < S) {
                const unsigned long long done = a.stats[(size_t)q * ST_COUNT + ST_BOXES];
                const unsigned long long cap = 1ull << 40;
                key = ((rg.rem[q] > 0 ? (done < cap ? done : cap) : 2 * cap) << 13) | (unsigned long long)q;
            }
            s_key[q] = key;
        }
        __syncthreads();
        for (int kk = 2; kk <= n2; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int q = t; q < n2; q += kBeginThreads) {
                    const int l = q ^ j;
                    if (l > q) {
                        const unsigned long long x = s_key[q], y = s_key[l];
                        if (((q & kk) == 0) ? (y < x) : (x < y)) {
                            s_key[q] = y;
                            s_key[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
    }
    // position q serves slot order[q] (least served first) or (q + waves) % S (rotating);
    // chunks of kBeginThreads positions are scanned in order with a running total of children
    for (int q0 = 0; q0 < S; q0 += kBeginThreads) {
        const int q = q0 + t;
        long long want = 0, fan = 1, k = 0;
        int sl = -1;
        if (q < S) {
            sl = las ? (int)(s_key[q] & 8191ull) : (int)(((int64_t)q + waves) % S);
            const int64_t held = rg.rem[sl];
            if (held > 0) {
                const bool root = held == 1 && (a.q.meta[rg.base[sl]] & kRootFlag) != 0;
                fan = fan_out(a.tb.sys[sl], root ? kRootFlag : 0u);
                k = share / fan;
                if (k < 1) k = 1;
                if (k > held) k = held;
                if (fan > 1) {
                    // breadth while the region is less than half full, one parent at a time
                    // (depth first) beyond: a region of R entries then still holds about
                    // R / (2 fan) more levels of the depth-first walk
                    const long long breadth = (rg.cap[sl] / 2 - held) / (fan - 1);
                    if (k > breadth) k = breadth > 1 ? breadth : 1;
                    if (held + k * (fan - 1) > rg.cap[sl]) k = 0;   // even one parent may not fit
                }
                want = k * fan;
            }
        }
        // inclusive scan of the children wanted (Hillis-Steele over the block)
        s_red[t] = want;
        __syncthreads();
        for (int off = 1; off < kBeginThreads; off <<= 1) {
            const long long v = t >= off ? s_red[t - off] : 0;
            __syncthreads();
            s_red[t] += v;
            __syncthreads();
        }
        const long long before = s_run + s_red[t] - want;
        if (sl >= 0) {
            long long give = k;
            if (before + want > a.wave_children) {
                const long long left = a.wave_children - before;
                give = left > 0 ? left / fan : 0;
            }
            rg.prefix[sl] = give;   // parents popped; turned into a prefix below
            if (rg.rem[sl] > 0 && give == 0 && s_active == 1) c->error = 1;   // cannot progress
        }
        __syncthreads();
        if (t == kBeginThreads - 1) s_run += s_red[t];
        __syncthreads();
    }
    // prefix over slots in slot order; rem = entries left below the popped parents
    if (t == 0) {
        long long run = 0, kids = 0;
        for (int sl = 0; sl < S; sl++) {
            const long long k = rg.prefix[sl];
            rg.prefix[sl] = run;
            run += k;
            const bool root = rg.rem[sl] == 1 && (a.q.meta[rg.base[sl]] & kRootFlag) != 0;
            kids += k * fan_out(a.tb.sys[sl], root ? kRootFlag : 0u);
            rg.rem[sl] -= k;
        }
        rg.prefix[S] = run;
        if (run == 0 && s_total > 0) c->error = 1;
        c->top = s_total;
        c->base = s_total - run;
        c->k = run;
        c->children = kids;
        c->cursor = 0;
        c->staged = 0;
        for (int n = 0; n <= kMaxVars; n++) { c->surv_count[n] = 0; c->hs_cursor[n] = 0; }
        c->cand_count = 0;
        c->cand_cursor = 0;
        c->waves += 1;
    }
}

// queue index of the sweep's parent p
__device__ __forceinline__ int64_t parent_index(const SweepArgs &a, int64_t base, int64_t p) {
    if (a.rg.n == 0) return base + p;
    int lo = 0, hi = a.rg.n;   // the slot s with prefix[s] <= p < prefix[s + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.rg.prefix[mid] <= p) lo = mid;
        else hi = mid;
    }
    return a.rg.base[lo] + a.rg.rem[lo] + (p - a.rg.prefix[lo]);
}

__global__ void __launch_bounds__(kBeginThreads) k_wave_begin(SweepArgs a) {
    // log2 children of the window's entries; serving: the sort keys of the slots
    extern __shared__ __align__(8) unsigned char s_fan[];
    __shared__ long long s_sum[kBeginThreads];
    __shared__ long long s_first;
    if (a.rg.n > 0) {
        wave_begin_regions(a, reinterpret_cast<unsigned long long *>(s_fan));
        return;
    }
    WaveCtl *c = a.ctl;
    const int64_t top = c->top;
    const int t = threadIdx.x;
    if (a.single) {
        // one system: every entry has fan-out F = 2^n except the initial box (fan-out 1,
        // alone in the queue when popped), so the scan below reduces to a closed form
        if (t != 0) return;
        int64_t k = 0, children = 0;
        if (top > 0) {
            if (a.q.meta[top - 1] & kRootFlag) {
                k = 1;
                children = 1;
            } else {
                const int64_t F = fan_out(a.tb.sys[0], 0u);
                k = a.wave_children / F;
                const int64_t by_room = (a.q.cap - top) / (F - 1);
                k = k < by_room ? k : by_room;
                k = k < top ? k : top;
                children = k * F;
            }
        }
        if (k <= 0 && top > 0) c->error = 1;
        c->base = top - k;
        c->k = k;
        c->children = children;
        c->cursor = 0;
        c->staged = 0;
        for (int n = 0; n <= kMaxVars; n++) { c->surv_count[n] = 0; c->hs_cursor[n] = 0; }
        c->cand_count = 0;
        c->cand_cursor = 0;
        c->waves += 1;
        return;
    }
    const int64_t window = top < (int64_t)kBeginThreads * kBeginPer ? top : (int64_t)kBeginThreads * kBeginPer;
    // entry i (0-based from the top) is queue index top - 1 - i; its log2 children come
    // from its meta word (0 for an initial box), read once with coalesced loads
    for (int q = 0; q < kBeginPer; q++) {
        const int64_t i = (int64_t)q * kBeginThreads + t;
        if (i < window) {
            const uint32_t m = a.q.meta[top - 1 - i];
            s_fan[i] = (m & kRootFlag) ? 0 : (unsigned char)((m >> kFanShift) & kFanMask);
        }
    }
    __syncthreads();
    auto fan_of = [&](int64_t i) -> long long { return 1ll << s_fan[i]; };
    long long local = 0;
    for (int q = 0; q < kBeginPer; q++) {
        const int64_t i = (int64_t)t * kBeginPer + q;
        if (i < window) local += fan_of(i);
    }
    // inclusive scan of the per-thread sums (Hillis-Steele over the block)
    s_sum[t] = local;
    if (t == 0) s_first = window;
    __syncthreads();
    for (int off = 1; off < kBeginThreads; off <<= 1) {
        const long long v = t >= off ? s_sum[t - off] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    long long pre = s_sum[t] - local;   // children of the entries before this thread's
    const long long room = a.q.cap - top;
    for (int q = 0; q < kBeginPer; q++) {
        const int64_t i = (int64_t)t * kBeginPer + q;
        if (i >= window) break;
        pre += fan_of(i);
        if (pre > a.wave_children || pre - (i + 1) > room) {
            atomicMin(&s_first, (long long)i);
            break;
        }
    }
    __syncthreads();
    if (t != 0) return;
    const int64_t k = s_first;
    int64_t children = 0;
    if (k > 0) {
        // children of the first k entries: recompute from the scan
        const int tk = (int)((k - 1) / kBeginPer), qk = (int)((k - 1) % kBeginPer);
        long long pre2 = tk > 0 ? s_sum[tk - 1] : 0;
        for (int q = 0; q <= qk; q++) pre2 += fan_of((int64_t)tk * kBeginPer + q);
        children = pre2;
    }
    if (k <= 0 && top > 0) c->error = 1;
    c->base = top - k;
    c->k = k;
    c->children = children;
    c->cursor = 0;
    c->staged = 0;
    for (int n = 0; n <= kMaxVars; n++) { c->surv_count[n] = 0; c->hs_cursor[n] = 0; }
    c->cand_count = 0;
    c->cand_cursor = 0;
    c->waves += 1;
}

// Moves the sweep's new parents onto the queue.  In the sweep graph (use_cond) block 0
// also sets the WHILE condition: more sweeps while the queue is non-empty after this
// commit, no error occurred and the sweep limit is not reached (nothing after the commit
// changes any of them).
__global__ void k_commit(SweepArgs a, int n_max, cudaGraphConditionalHandle h, int use_cond) {
    const WaveCtl *c = a.ctl;
    const int64_t staged = c->staged, base = c->base;
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
        const bool more = base + staged > 0 && c->error == 0 && c->waves < c->wave_limit;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < staged; i += stride) {
        int64_t d = base + i;
        if (a.rg.n > 0) {   // into the parent's own region, above what stays there
            const int sl = a.stage.sys[i];
            d = a.rg.base[sl] + a.rg.rem[sl] + (int64_t)atomicAdd(&a.rg.cursor[sl], 1ull);
        }
        for (int j = 0; j < n_max; j++) {
            a.q.lo[j * a.q.cap + d] = a.stage.lo[j * a.stage.cap + i];
            a.q.mid[j * a.q.cap + d] = a.stage.mid[j * a.stage.cap + i];
            a.q.hi[j * a.q.cap + d] = a.stage.hi[j * a.stage.cap + i];
        }
        a.q.sys[d] = a.stage.sys[i];
        a.q.meta[d] = a.stage.meta[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->top = base + staged;
}

__global__ void k_seed_roots(SweepArgs a, const double *box_lo, const double *box_hi,
                             const int32_t *root_depth, int n_sys, int n_max) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
        for (int j = 0; j < n_max; j++) {
            a.q.lo[j * a.q.cap + s] = box_lo[(size_t)s * n_max + j];
            a.q.mid[j * a.q.cap + s] = box_hi[(size_t)s * n_max + j];   // a root's only
            a.q.hi[j * a.q.cap + s] = box_hi[(size_t)s * n_max + j];    // child is itself
        }
        a.q.sys[s] = s;
        a.q.meta[s] = kRootFlag | ((uint32_t)root_depth[s] & kDepthMask);
        a.stats[(size_t)s * ST_COUNT + ST_LIVE] = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        WaveCtl *c = a.ctl;
        c->top = n_sys;
        c->base = 0;
        c->k = 0;
        c->staged = 0;
        c->out_count = 0;
        c->cursor = 0;
        c->error = 0;
        c->waves = 0;
        c->cand_count = 0;
        c->cand_cursor = 0;
        c->wave_limit = 0x7FFFFFFFFFFFFFFFLL;
        for (int n = 0; n <= kMaxVars; n++) { c->surv_count[n] = 0; c->hs_cursor[n] = 0; }
    }
}

// Serving: appends `count` initial boxes (one per newly admitted system) on top of the
// queue between sweeps; one block.
__global__ void k_admit(SweepArgs a, const double *box_lo, const double *box_hi, const int32_t *slot,
                        const int32_t *root_depth, int count, int n_max) {
    const int64_t top = a.ctl->top;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        int64_t e = top + i;
        if (a.rg.n > 0) {   // the start of the system's own region
            const int sl = slot[i];
            e = a.rg.base[sl];
            a.rg.rem[sl] = 1;
            a.rg.cursor[sl] = 0;
        }
        for (int j = 0; j < n_max; j++) {
            a.q.lo[j * a.q.cap + e] = box_lo[(size_t)i * n_max + j];
            a.q.mid[j * a.q.cap + e] = box_hi[(size_t)i * n_max + j];
            a.q.hi[j * a.q.cap + e] = box_hi[(size_t)i * n_max + j];
        }
        a.q.sys[e] = slot[i];
        a.q.meta[e] = kRootFlag | ((uint32_t)root_depth[i] & kDepthMask);
        a.stats[(size_t)slot[i] * ST_COUNT + ST_LIVE] = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.ctl->top = top + count;
}

// Serving with regions: a cancelled slot's region is emptied (its entries leave the total).
__global__ void k_cancel_regions(SweepArgs a, const int32_t *cancel) {
    for (int sl = threadIdx.x; sl < a.rg.n; sl += blockDim.x) {
        if (!cancel[sl]) continue;
        const int64_t held = a.rg.rem[sl] + (int64_t)a.rg.cursor[sl];
        if (held) atomicAdd((unsigned long long *)&a.ctl->top, (unsigned long long)(-held));
        a.rg.rem[sl] = 0;
        a.rg.cursor[sl] = 0;
    }
}

// ------------------------------------------------------------------------------------
// evaluation of the children of each parent
// ------------------------------------------------------------------------------------

// Child c of the warp's parent: coordinate j is [lo_j, mid_j] when bit j of c is clear,
// [mid_j, hi_j] when set.  p[0|1|2][j] = lo / mid / hi in FP64; f[0..3][j] = rd32(lo),
// rd32(mid), ru32(mid), ru32(hi); e[0..5][j] = rd32 / ru32 of lo, mid, hi.
struct ChildCoord64 {
    const double (*p)[kMaxVars];
    unsigned c;
    __device__ __forceinline__ ivd operator()(unsigned j) const {
        const unsigned up = (c >> j) & 1u;
        return ivd{p[up][j], p[up + 1][j]};
    }
};
struct ChildCoord32 {
    const float (*f)[kMaxVars];
    unsigned c;
    __device__ __forceinline__ ivf operator()(unsigned j) const {
        const unsigned up = (c >> j) & 1u;
        return ivf{f[up][j], f[up + 2][j]};
    }
};
struct ChildCoordShadow {
    const float (*e)[kMaxVars];
    unsigned c;
    __device__ __forceinline__ shv operator()(unsigned j) const {
        const unsigned up = (c >> j) & 1u;
        return shv{e[2 * up][j], e[2 * up + 1][j], e[2 * up + 2][j], e[2 * up + 3][j]};
    }
};
// coordinate of factor f of a table entry: the half is bit f of the combination q
struct ComboCoordShadow {
    const float (*e)[kMaxVars];
    unsigned q;
    __device__ __forceinline__ shv operator()(unsigned j, int f) const {
        const unsigned up = (q >> f) & 1u;
        return shv{e[2 * up][j], e[2 * up + 1][j], e[2 * up + 2][j], e[2 * up + 3][j]};
    }
};
// box held in shared memory, structure of arrays with the given stride
struct BoxCoord {
    const double *X;
    int stride;
    __device__ __forceinline__ ivd operator()(unsigned j) const {
        return ivd{X[(2 * j) * stride], X[(2 * j + 1) * stride]};
    }
};

__device__ __forceinline__ void push_surv(const SweepArgs &a, WaveCtl *ctl, int n, bool keep, Surv sv) {
    const unsigned km = __ballot_sync(kFull, keep);
    if (!km) return;
    unsigned long long pos = 0;
    if (lane_id() == 0) pos = atomicAdd((unsigned long long *)&ctl->surv_count[n], (unsigned long long)__popc(km));
    pos = __shfl_sync(kFull, pos, 0);
    if (keep) {
        const unsigned long long k = pos + __popc(km & lanemask_lt());
        if ((long long)k < a.surv_cap) a.surv[(size_t)n * a.surv_cap + k] = sv;
        else ctl->error = 1;
    }
}

// undecided children for k_eval64 (warp-aggregated append)
__device__ __forceinline__ void push_cand(const SweepArgs &a, WaveCtl *ctl, bool cand, Surv sv) {
    const unsigned cm = __ballot_sync(kFull, cand);
    if (!cm) return;
    unsigned long long pos = 0;
    if (lane_id() == 0) pos = atomicAdd((unsigned long long *)&ctl->cand_count, (unsigned long long)__popc(cm));
    pos = __shfl_sync(kFull, pos, 0);
    if (cand) {
        const unsigned long long k = pos + __popc(cm & lanemask_lt());
        if ((long long)k < a.surv_cap) a.cand[k] = sv;
        else ctl->error = 1;
    }
}

// Children c0 + k G + r (k < K) of parent pi per thread, decided K at a time from the
// parent's table (decide_from_table_k), then appended to the survivor / candidate lists.
template <int K>
__device__ __forceinline__ void table_children(const SweepArgs &a, WaveCtl *ctl, const SysTab &T, const DevSys &S,
                                               const float4 *tv, uint32_t meta, int64_t pi, int n, unsigned fan,
                                               unsigned r, unsigned G, unsigned &cnt_pre, unsigned &cnt_sh) {
    for (unsigned c0 = 0; c0 < fan; c0 += K * G) {
        unsigned c[K];
        bool want[K];
        int d[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            c[k] = child_bits(S, meta, c0 + k * G + r);
            want[k] = c0 + k * G + r < fan;
        }
        decide_from_table_k<K>(T, S, tv, c, want, d);
#pragma unroll
        for (int k = 0; k < K; k++) {
            const bool keep = want[k] && d[k] == 1, cand = want[k] && d[k] == 2;
            cnt_pre += (want[k] && d[k] == 0) ? 1u : 0u;
            cnt_sh += keep ? 1u : 0u;
            push_surv(a, ctl, n, keep, Surv{(uint32_t)pi, c[k]});
            push_cand(a, ctl, cand, Surv{(uint32_t)pi, c[k]});
        }
    }
}

// The children of one parent, evaluated by a group of threads: one warp (GROUP = 32) or
// the whole block.  r = the thread's rank in the group, G = the group size; every
// thread of the group runs this with the same pi.  Three forms: the FP32 shadow (decides
// what FP64 would decide with certainty; the undecided rest go to k_eval64), the plain
// FP32 prefilter (its survivors go to k_eval64), or FP64 only.
template <bool BLOCK>
__device__ __forceinline__ void group_sync() {
    if (BLOCK) __syncthreads();
    else __syncwarp();
}

template <bool BLOCK>
__device__ __forceinline__ void eval_parent(const SweepArgs &a, WaveCtl *ctl, const char *s_blob, float4 *s_tv,
                                            double (*sp)[kMaxVars], float (*sf)[kMaxVars], float (*se)[kMaxVars],
                                            int *s_flag, int64_t pi, unsigned r, unsigned G) {
    const unsigned lane = lane_id();
    const int sys = a.q.sys[pi];
    const uint32_t meta = a.q.meta[pi];
    const DevSys S = a.tb.sys[sys];
    const SysTab T = make_tab(a.single ? s_blob : a.tb.blobs + S.blob_off, S);
    const bool root = (meta & kRootFlag) != 0;
    const int depth = (int)(meta & kDepthMask) + (root ? 0 : 1);
    // the parent leaves the queue; past the box budget its children are dropped (the
    // decision of rank 0, shared by the group)
    int over = 0;
    if (r == 0) {
        atomicAdd(stat_ptr(a, sys, ST_LIVE), ~0ull);
        if (S.max_boxes > 0) {
            const unsigned long long done = *(volatile unsigned long long *)stat_ptr(a, sys, ST_BOXES);
            if ((long long)done >= S.max_boxes) {
                atomicOr(stat_ptr(a, sys, ST_FLAGS), (unsigned long long)kFlagBudget);
                over = 1;
            }
        }
        if (BLOCK) *s_flag = over;
    }
    if (BLOCK) {
        __syncthreads();
        over = *s_flag;
    } else {
        over = __shfl_sync(kFull, over, 0);
    }
    if (over) {
        if (BLOCK) __syncthreads();   // s_flag is rewritten for the next parent
        return;
    }
    const int n = S.n;
    if ((int)r < n) {
        const double lo = a.q.lo[r * a.q.cap + pi];
        const double mid = a.q.mid[r * a.q.cap + pi];
        const double hi = a.q.hi[r * a.q.cap + pi];
        sp[0][r] = lo;
        sp[1][r] = mid;
        sp[2][r] = hi;
        const float lod = __double2float_rd(lo), lou = __double2float_ru(lo);
        const float mdd = __double2float_rd(mid), mdu = __double2float_ru(mid);
        const float hid = __double2float_rd(hi), hiu = __double2float_ru(hi);
        sf[0][r] = lod;
        sf[1][r] = mdd;
        sf[2][r] = mdu;
        sf[3][r] = hiu;
        se[0][r] = lod;
        se[1][r] = lou;
        se[2][r] = mdd;
        se[3][r] = mdu;
        se[4][r] = hid;
        se[5][r] = hiu;
    }
    group_sync<BLOCK>();
    const unsigned fan = (unsigned)fan_out(S, meta);
    unsigned cnt_pre = 0, cnt_ev = 0, cnt_64 = 0, cnt_sh = 0;
    // per-parent term-combination table: when the fan-out fills warps and it fits
    const bool use_tv = S.prefilter && S.shadow && S.n_tv > 0 && S.n_tv <= a.tv_stride && fan >= 32;
    if (use_tv) {
        for (int e = (int)r; e < S.n_tv; e += (int)G) {
            const uint32_t mp = T.tv_map[e];
            s_tv[e] = term_shadow(T, (int)(mp >> 8), ComboCoordShadow{se, mp & 255u});
        }
        group_sync<BLOCK>();
    }
    // K children per thread (c0 + k G + r, k < K) on the table path with a child-index
    // table when the fan-out fills K rounds of the group: K independent chains
    const bool cix_tab = use_tv && S.n_cix > 0;
    if (cix_tab && fan >= 4 * G) {
        table_children<4>(a, ctl, T, S, s_tv, meta, pi, n, fan, r, G, cnt_pre, cnt_sh);
    } else if (cix_tab && fan >= 2 * G) {
        table_children<2>(a, ctl, T, S, s_tv, meta, pi, n, fan, r, G, cnt_pre, cnt_sh);
    } else {
    for (unsigned c0 = 0; c0 < fan; c0 += G) {
        const bool active = c0 + r < fan;
        const unsigned c = child_bits(S, meta, c0 + r);
        bool keep = false, cand = false;
        if (active) {
            if (use_tv) {
                const int d = decide_from_table(T, S, s_tv, c);
                keep = d == 1;
                cand = d == 2;
                cnt_pre += d == 0 ? 1u : 0u;
                cnt_sh += keep ? 1u : 0u;
            } else if (S.prefilter && S.shadow) {
                const int d = decide_shadow(T, S, ChildCoordShadow{se, c});
                keep = d == 1;
                cand = d == 2;
                cnt_pre += d == 0 ? 1u : 0u;
                cnt_sh += keep ? 1u : 0u;
            } else if (S.prefilter) {
                cand = keep32(T, S, ChildCoord32{sf, c});
                cnt_pre += cand ? 0u : 1u;
            } else {
                cnt_64 += 1;
                keep = keep64(T, S, ChildCoord64{sp, c});
                cnt_ev += keep ? 0u : 1u;
            }
        }
        push_surv(a, ctl, n, keep, Surv{(uint32_t)pi, c});
        push_cand(a, ctl, cand, Surv{(uint32_t)pi, c});
    }
    }
    cnt_pre = __reduce_add_sync(kFull, cnt_pre);
    cnt_ev = __reduce_add_sync(kFull, cnt_ev);
    cnt_64 = __reduce_add_sync(kFull, cnt_64);
    cnt_sh = __reduce_add_sync(kFull, cnt_sh);
    if (lane == 0) {
        if (r == 0) {
            atomicAdd(stat_ptr(a, sys, ST_BOXES), (unsigned long long)fan);
            atomicMax(stat_ptr(a, sys, ST_MAX_DEPTH), (unsigned long long)depth);
            atomicAdd(stat_ptr(a, sys, ST_DEPTH_BOXES + (depth < kDepthSlots ? depth : kDepthSlots - 1)),
                      (unsigned long long)fan);
        }
        if (cnt_pre) atomicAdd(stat_ptr(a, sys, ST_EXCL_PREFILTER), (unsigned long long)cnt_pre);
        if (cnt_ev) atomicAdd(stat_ptr(a, sys, ST_EXCL_EVAL), (unsigned long long)cnt_ev);
        if (cnt_64) atomicAdd(stat_ptr(a, sys, ST_EVAL64), (unsigned long long)cnt_64);
        if (cnt_sh) atomicAdd(stat_ptr(a, sys, ST_KEEP_SHADOW), (unsigned long long)cnt_sh);
    }
    group_sync<BLOCK>();   // the parent's arrays are rewritten for the next parent
}

// Children of the popped parents.  A wide sweep gives each warp a parent at a time from
// a shared cursor (one lane per child, or two or four children per lane on the table
// path when the fan-out fills that many rounds); a narrow one (at most one parent per block)
// gives each block its parents and spreads a parent's table entries and children over
// all of the block's threads, so the few parents of the first and last sweeps finish
// sooner.  Both run the same per-child arithmetic.
__global__ void __launch_bounds__(kEvalThreads, 3) k_eval(SweepArgs a) {
    extern __shared__ __align__(16) char s_blob[];
    float4 *s_tv_base = reinterpret_cast<float4 *>(s_blob + (a.single ? a.blob_smem : 0));
    __shared__ double s_p[kEvalWarps][3][kMaxVars];
    __shared__ float s_f[kEvalWarps][4][kMaxVars];
    __shared__ float s_e[kEvalWarps][6][kMaxVars];
    __shared__ int s_flag;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    WaveCtl *ctl = a.ctl;
    const int64_t base = ctl->base, K = ctl->k;
    const bool block_mode = K <= (int64_t)gridDim.x;
    // blocks beyond what K parents need leave at once (the others take every parent), so
    // a small sweep does not pay for the whole grid
    if (block_mode ? (int64_t)blockIdx.x >= K : (int64_t)blockIdx.x * (blockDim.x >> 5) >= K) return;
    if (a.single) {
        const DevSys &S0 = a.tb.sys[0];
        copy_blob(s_blob, a.tb.blobs + S0.blob_off, (uint32_t)S0.blob_bytes);
        __syncthreads();
    }
    if (block_mode) {
        for (int64_t p = blockIdx.x; p < K; p += gridDim.x)
            eval_parent<true>(a, ctl, s_blob, s_tv_base, s_p[0], s_f[0], s_e[0], &s_flag, parent_index(a, base, p),
                              threadIdx.x, blockDim.x);
        return;
    }
    float4 *s_tv = s_tv_base + (size_t)w * a.tv_stride;
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&ctl->cursor, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= K) break;
        eval_parent<false>(a, ctl, s_blob, s_tv, s_p[w], s_f[w], s_e[w], &s_flag, parent_index(a, base, p), lane, 32u);
    }
}

// FP64 evaluation of the candidates (undecided by the FP32 stage), one thread each,
// 32 per warp from an atomic cursor so the work is dense and spread over all SMs.
__global__ void __launch_bounds__(kEval64Threads) k_eval64(SweepArgs a) {
    extern __shared__ __align__(16) char s_blob[];
    __shared__ double sX[2 * kMaxVars * kEval64Threads];
    const int T = blockDim.x, tid = threadIdx.x;
    double *X = sX + tid;
    WaveCtl *ctl = a.ctl;
    const int64_t count = ctl->cand_count;
    if ((int64_t)blockIdx.x * blockDim.x >= count) return;   // not needed for this many candidates
    if (a.single) {
        const DevSys &S0 = a.tb.sys[0];
        copy_blob(s_blob, a.tb.blobs + S0.blob_off, (uint32_t)S0.blob_bytes);
        __syncthreads();
    }
    const unsigned lane = lane_id();
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd((unsigned long long *)&ctl->cand_cursor, 32ull);
        base = __shfl_sync(kFull, base, 0);
        if ((long long)base >= count) break;
        const int64_t idx = (int64_t)base + lane;
        const bool active = idx < count;
        bool keep = false;
        int sys = 0, n = 0;
        Surv sv{0, 0};
        if (active) {
            sv = a.cand[idx];
            const int64_t pi = sv.parent;
            sys = a.q.sys[pi];
            const DevSys S = a.tb.sys[sys];
            const SysTab Tb = make_tab(a.single ? s_blob : a.tb.blobs + S.blob_off, S);
            n = S.n;
            for (int j = 0; j < n; j++) {
                const bool up = (sv.child >> j) & 1u;
                X[(2 * j) * T] = up ? a.q.mid[j * a.q.cap + pi] : a.q.lo[j * a.q.cap + pi];
                X[(2 * j + 1) * T] = up ? a.q.hi[j * a.q.cap + pi] : a.q.mid[j * a.q.cap + pi];
            }
            keep = keep64(Tb, S, BoxCoord{X, T});
        }
        const int sys0 = __shfl_sync(kFull, sys, 0);
        const int n0 = __shfl_sync(kFull, n, 0);
        const bool uniform = __all_sync(kFull, !active || (sys == sys0 && n == n0));
        if (uniform) {
            push_surv(a, ctl, n0, keep, sv);
            const unsigned na = __popc(__ballot_sync(kFull, active));
            const unsigned nk = __popc(__ballot_sync(kFull, keep));
            if (lane == 0) {
                atomicAdd(stat_ptr(a, sys0, ST_EVAL64), (unsigned long long)na);
                if (na - nk) atomicAdd(stat_ptr(a, sys0, ST_EXCL_EVAL), (unsigned long long)(na - nk));
            }
        } else if (active) {
            if (keep) {
                const unsigned long long k = atomicAdd((unsigned long long *)&ctl->surv_count[n], 1ull);
                if ((long long)k < a.surv_cap) a.surv[(size_t)n * a.surv_cap + k] = sv;
                else ctl->error = 1;
            }
            atomicAdd(stat_ptr(a, sys, ST_EVAL64), 1ull);
            if (!keep) atomicAdd(stat_ptr(a, sys, ST_EXCL_EVAL), 1ull);
        }
    }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------

static cudaError_t launch_hs(const SweepArgs &a, int n, int num_sms, cudaStream_t st, int *kernels) {
    switch (n) {
    case 1: return launch_hs_dim1(a, num_sms, st, kernels);
    case 2: return launch_hs_dim2(a, num_sms, st, kernels);
    case 3: return launch_hs_dim3(a, num_sms, st, kernels);
    case 4: return launch_hs_dim4(a, num_sms, st, kernels);
    case 5: return launch_hs_dim5(a, num_sms, st, kernels);
    case 6: return launch_hs_dim6(a, num_sms, st, kernels);
    case 7: return launch_hs_dim7(a, num_sms, st, kernels);
    case 8: return launch_hs_dim8(a, num_sms, st, kernels);
    case 9: return launch_hs_dim9(a, num_sms, st, kernels);
    case 10: return launch_hs_dim10(a, num_sms, st, kernels);
    case 11: return launch_hs_dim11(a, num_sms, st, kernels);
    case 12: return launch_hs_dim12(a, num_sms, st, kernels);
    case 13: return launch_hs_dim13(a, num_sms, st, kernels);
    case 14: return launch_hs_dim14(a, num_sms, st, kernels);
    case 15: return launch_hs_dim15(a, num_sms, st, kernels);
    case 16: return launch_hs_dim16(a, num_sms, st, kernels);
    default: return cudaErrorInvalidValue;
    }
}

// The answers live in a fixed table (no heap allocation, so the allocation-free entry
// point may launch through here too); when it is full, further shapes are queried each
// time instead of cached.
int coop_clusters_cached(const void *func, int num_sms, int threads, size_t smem, cudaError_t *err) {
    struct Known {
        const void *func;
        int num_sms, threads, dev, clusters;
        size_t smem;
    };
    constexpr int kSlots = 512;
    static std::mutex mu;
    static Known known[kSlots];
    static int used = 0;
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < used; i++) {
        const Known &k = known[i];
        if (k.func == func && k.num_sms == num_sms && k.threads == threads && k.smem == smem && k.dev == dev)
            return k.clusters;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)((num_sms / 4) * 4));
    lc.blockDim = dim3((unsigned)threads);
    lc.dynamicSmemBytes = smem;
    int nc = 0;
    *err = cudaOccupancyMaxActiveClusters(&nc, func, &lc);
    if (*err != cudaSuccess) return 0;
    if (used < kSlots) known[used++] = Known{func, num_sms, threads, dev, nc, smem};
    return nc;
}

size_t eval_smem_bytes(const SweepArgs &a) {
    return (size_t)(a.single ? a.blob_smem : 0) + (size_t)a.eval_warps * a.tv_stride * sizeof(float4);
}

cudaError_t allow_max_dynamic_smem(const void *func) {
    // The attribute is global to the kernel: every plan and server sets the same maximum,
    // so one whose launches need less never lowers it under another's captured graph.
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

cudaError_t configure_eval_kernels(const SweepArgs &a) {
    (void)a;
    cudaError_t e = allow_max_dynamic_smem((const void *)k_wave_begin);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem((const void *)k_eval);
    if (e != cudaSuccess) return e;
    return allow_max_dynamic_smem((const void *)k_eval64);
}

static cudaError_t launch_sweep_impl(const SweepArgs &a, const int *hs_dims, int n_hs_dims, int eval_blocks,
                                     int num_sms, cudaStream_t st, cudaEvent_t *ev, cudaGraphConditionalHandle h,
                                     int use_cond, int *kernels) {
    int count = 4;   // wave_begin, eval, eval64, commit
    // ev (optional): n_hs_dims + 5 events recorded between the stages
    const size_t blob = a.single ? (size_t)a.blob_smem : 0;
    if (ev) cudaEventRecord(ev[0], st);
    k_wave_begin<<<1, kBeginThreads, kBeginSmem, st>>>(a);
    if (ev) cudaEventRecord(ev[1], st);
    k_eval<<<eval_blocks, a.eval_warps * 32, eval_smem_bytes(a), st>>>(a);
    if (ev) cudaEventRecord(ev[2], st);
    k_eval64<<<num_sms * 4, kEval64Threads, blob, st>>>(a);
    if (ev) cudaEventRecord(ev[3], st);
    for (int q = 0; q < n_hs_dims; q++) {
        int kq = 0;
        cudaError_t e = launch_hs(a, hs_dims[q], num_sms, st, &kq);
        if (e != cudaSuccess) return e;
        count += kq;
        if (ev) cudaEventRecord(ev[4 + q], st);
    }
    k_commit<<<num_sms * 4, 256, 0, st>>>(a, a.max_fan_shift, h, use_cond);
    if (ev) cudaEventRecord(ev[4 + n_hs_dims], st);
    if (kernels) *kernels = count;
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs &a, const int *hs_dims, int n_hs_dims, int eval_blocks,
                         int eval_threads, int num_sms, cudaStream_t st, cudaEvent_t *ev, int *kernels) {
    (void)eval_threads;
    return launch_sweep_impl(a, hs_dims, n_hs_dims, eval_blocks, num_sms, st, ev, cudaGraphConditionalHandle{}, 0,
                             kernels);
}

cudaError_t build_sweep_graph(const SweepArgs &a, const int *hs_dims, int n_hs_dims, int eval_blocks,
                              int eval_threads, int num_sms, cudaGraph_t *out, int *kernels_per_sweep) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            (void)eval_threads;
            cudaError_t le = launch_sweep_impl(a, hs_dims, n_hs_dims, eval_blocks, num_sms, cs, nullptr, h, 1,
                                               kernels_per_sweep);
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(cs, &captured);
            if (e == cudaSuccess && le != cudaSuccess) e = le;
        }
    }
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    *out = g;
    return cudaSuccess;
}

cudaError_t launch_admit(const SweepArgs &a, const double *d_lo, const double *d_hi, const int32_t *d_slot,
                         const int32_t *d_depth, int count, int n_max, cudaStream_t st) {
    k_admit<<<1, 256, 0, st>>>(a, d_lo, d_hi, d_slot, d_depth, count, n_max);
    return cudaGetLastError();
}

cudaError_t launch_cancel_regions(const SweepArgs &a, const int32_t *d_cancel, cudaStream_t st) {
    k_cancel_regions<<<1, 1024, 0, st>>>(a, d_cancel);
    return cudaGetLastError();
}

cudaError_t launch_seed_roots(const SweepArgs &a, const double *d_box_lo, const double *d_box_hi,
                              const int32_t *d_root_depth, int n_sys, int n_max, cudaStream_t st) {
    int blocks = (n_sys + 255) / 256;
    if (blocks < 1) blocks = 1;
    k_seed_roots<<<blocks, 256, 0, st>>>(a, d_box_lo, d_box_hi, d_root_depth, n_sys, n_max);
    return cudaGetLastError();
}

}  // namespace ivs
