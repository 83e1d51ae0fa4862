// ivs_internal.h -- layouts shared by the host runtime and the kernels of the library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector_types.h>

namespace ivs {

constexpr int kMaxVars = 16;
constexpr int kMaxExp = 15;

// Parent-entry meta word: depth in the low 16 bits, ROOT flag (the entry is an initial
// box that is evaluated itself, fan-out 1, not split first).
constexpr uint32_t kRootFlag = 1u << 30;
constexpr uint32_t kDepthMask = 0xFFFFu;
// Bisection (split_mode 1): the coordinate a parent is split in, bits 16-19 of its meta
// word; its queue entry holds mid_j = hi_j in every other coordinate, so child c (bit
// `coordinate` of c) reads [lo_j, hi_j] there whatever the decoding.
constexpr int kSplitShift = 16;
constexpr uint32_t kSplitMask = 0xFu;
// log2 of a parent's number of children (n, or 1 when bisected), bits 20-24 of its meta
// word, so the sweep's pop can size parents from the meta word alone
constexpr int kFanShift = 20;
constexpr uint32_t kFanMask = 0x1Fu;

// per-system statistics slots (int64 counters on the device)
enum Stat : int {
    ST_BOXES = 0,
    ST_EXCL_PREFILTER,
    ST_EXCL_EVAL,
    ST_HS_APPLIED,
    ST_HS_EMPTY,
    ST_HS_CONTRACTED,
    ST_HS_SINGULAR,
    ST_ACCEPTED,
    ST_UNSPLITTABLE,
    ST_SPLIT,
    ST_MAX_DEPTH,
    ST_FLAGS,          // bit 0: results overflowed, bit 1: depth cut, bit 2: box budget hit
    ST_EVAL64,         // boxes that ran the FP64 evaluation
    ST_KEEP_SHADOW,    // boxes the FP32 shadow proved kept (no FP64 evaluation)
    ST_OUT,            // accepted boxes of the system (its result region holds min(this, out_cap))
    ST_LIVE,           // queue entries of the system (0 after a sweep: the system is solved)
    ST_EXCL_CENTRED,   // boxes the centred form dropped
    ST_GAP_SPLITS,     // sweeps that returned two boxes at an extended-division gap
    ST_DEPTH_BOXES,    // kDepthSlots slots: boxes processed at depth d (d >= 63 in the last)
    ST_DEPTH_KEPT = ST_DEPTH_BOXES + 64,   // 64 slots: boxes that survived evaluation and
                                           // contraction at depth d
    ST_DEPTH_HS = ST_DEPTH_KEPT + 64,      // 64 slots: boxes that entered the contraction
    ST_COUNT = ST_DEPTH_HS + 64
};
constexpr int kDepthSlots = 64;
constexpr int64_t kFlagResultOverflow = 1, kFlagDepthCut = 2, kFlagBudget = 4;

// Compiled system, resident on the device.  Its polynomials (the m equations F_i, then
// the m*n Jacobian entries J_ij row-major when m == n) live in one blob of the blob
// arena at blob_off (layout: ivs_tab.cuh).
struct DevSys {
    int32_t n, m;
    int32_t f_poly;        // first polynomial of F (local index, 0)
    int32_t j_poly;        // first polynomial of J (local index m), -1 if none
    double tol;
    int32_t hs_enable, hs_min_depth, hs_iters, max_depth;
    int32_t prefilter;
    int32_t shadow;        // FP32 shadow decisions allowed (no FP32 overflow possible)
    int64_t max_boxes;
    int64_t blob_off;      // byte offset of the system's blob
    int32_t n_terms, n_polys, n_facs, blob_bytes;
    int64_t out_base;      // the system's result region: entries [out_base, out_base + out_cap)
    int64_t out_cap;
    int32_t n_fterms;      // terms of the equations F_i
    int32_t n_tv;          // term-combination entries (0: no per-parent table)
    int32_t centred;       // 1: centred-form exclusion test before Hansen-Sengupta
    int32_t n_cix;         // child-index entries (n_fterms << n; 0: none)
    int32_t krawczyk;      // 1: Krawczyk contraction (eq 15-16) instead of Gauss-Seidel
    int32_t bisect;        // 1: widest-coordinate bisection (2 children) instead of 2^n
    int32_t gap_split;     // 1: two boxes at an extended-division gap (Gauss-Seidel only)
};

// children of a popped queue entry: 1 for an initial box, else 2 (bisection) or 2^n
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t fan_out(const DevSys &S, uint32_t meta) {
    return (meta & kRootFlag) ? 1 : (S.bisect ? 2 : ((int64_t)1 << S.n));
}
// child bits of the c-th child of an entry (bit j set: upper half of coordinate j)
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t child_bits(const DevSys &S, uint32_t meta, uint32_t c) {
    return (S.bisect && !(meta & kRootFlag)) ? (c << ((meta >> kSplitShift) & kSplitMask)) : c;
}

struct DevTables {
    const DevSys *sys;
    const char *blobs;     // blob arena (16-byte aligned blobs)
};

// Queue of parent boxes (boxes to split), structure of arrays with capacity `cap`:
// coordinate j of entry i at lo[j * cap + i] (likewise mid, hi).
struct DevQueue {
    double *lo, *mid, *hi;
    int32_t *sys;
    uint32_t *meta;
    int64_t cap;
};

// Accepted boxes (output list).
struct DevOut {
    double *lo, *hi;
    int32_t *sys;
    int32_t *flags;
    int32_t *depth;
    int64_t cap;
};

// Control block of the sweep loop (device memory).
struct WaveCtl {
    int64_t top;            // queue size
    int64_t base;           // first parent popped by this sweep
    int64_t k;              // parents popped by this sweep
    int64_t staged;         // new parents written to the staging queue
    int64_t out_count;      // accepted boxes written
    int32_t cursor;         // evaluation kernel's parent cursor
    int32_t error;          // sticky: 1 = queue full
    int64_t surv_count[kMaxVars + 1];   // survivors per n (index n)
    int64_t hs_cursor[kMaxVars + 1];    // Hansen-Sengupta kernels' work cursors
    int64_t cand_count;                 // FP32 survivors waiting for the FP64 evaluation
    int64_t cand_cursor;
    int64_t waves;
    int64_t wave_limit;     // the device loop stops when waves reaches it
    int64_t children;       // children the current sweep evaluates
};

// Serving: one queue region per system slot ("device-resident queues admitted by the
// memory they need").  Slot s owns entries [base[s], base[s] + cap[s]) of the queue.
// Between sweeps it holds rem[s] + cursor[s] entries; a sweep pops its top k[s] parents
// (prefix[s] = popped parents of the slots before s), leaving rem[s] below them, and its
// new parents go on top (cursor[s] counts them).  n == 0: one stack shared by all systems.
struct DevRegions {
    int64_t *base, *cap;
    int64_t *rem;
    int64_t *prefix;                 // [n + 1]
    unsigned long long *cursor;
    int32_t n;
    int32_t fair_share;              // 1: rotating fair share instead of least served first
};

// survivor of the evaluation: parent index in the queue, child index
struct Surv {
    uint32_t parent;
    uint32_t child;
};

}  // namespace ivs
