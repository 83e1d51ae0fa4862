// ivs_tab.cuh -- a compiled system's term table and the natural-form evaluators.
//
// Each system is compiled on the host into one contiguous blob (layout below) holding
// its polynomials: the m equations F_i, then (when m == n) the m*n Jacobian entries J_ij.
// A polynomial is a range of terms; a term is a coefficient interval and a list of
// factors (var << 4 | exponent, exponent >= 1) in increasing variable order.  Kernels
// read the blob from global memory or copy it once per block into shared memory.
//
// Evaluation follows Definition 1 with the operation order fixed once for every
// implementation: a term folds its factor powers left in variable order, then the
// coefficient interval multiplies the product; a polynomial folds its terms left in
// input order.
#pragma once
#include <cuda_runtime.h>

#include "ivs_internal.h"
#include "ivs_interval.cuh"

namespace ivs {

// byte layout of a system blob with T terms, P polynomials, F factors, TF terms in the
// equations F_i, E term-combination entries and CX child-index entries
struct BlobLayout {
    uint32_t cs, clo, chi, clo32, chi32, poly_off, tinfo, tv_off, tv_map, cix, fac, bytes;
};
__host__ __device__ inline BlobLayout blob_layout(int T, int P, int F, int TF = 0, int E = 0, int CX = 0) {
    BlobLayout L;
    uint32_t o = 0;
    L.cs = o;        o += 16u * T;
    L.clo = o;       o += 8u * T;
    L.chi = o;       o += 8u * T;
    L.clo32 = o;     o += 4u * T;
    L.chi32 = o;     o += 4u * T;
    L.poly_off = o;  o += 4u * (P + 1);
    L.tinfo = o;     o += 4u * T;
    L.tv_off = o;    o += 4u * (TF + 1);
    L.tv_map = o;    o += 4u * E;
    L.cix = o;       o += (2u * CX + 3u) & ~3u;
    L.fac = o;       o += (uint32_t)F;
    L.bytes = (o + 15u) & ~15u;
    return L;
}

// term info word: factor start << 5 | factor count, and bit 31 set when the coefficient
// interval is a point (c_lo == c_hi), which lets the FP64 product take two multiplies
// instead of a general interval product (the same numbers either way)
constexpr uint32_t kTermPoint = 1u << 31;
__host__ __device__ inline int term_nf(uint32_t info) { return (int)(info & 31u); }
__host__ __device__ inline int term_f0(uint32_t info) { return (int)((info & ~kTermPoint) >> 5); }
// the info word of a term whose factors start at `start` (count `cnt`) with coefficient
// interval [clo, chi]; every packer of term tables uses this one encoding
__host__ __device__ inline uint32_t term_info(uint32_t start, uint32_t cnt, double clo, double chi) {
    return (start << 5) | cnt | (clo == chi ? kTermPoint : 0u);
}

struct SysTab {
    const float4 *cs;        // {rd32(c_lo), ru32(c_lo), rd32(c_hi), ru32(c_hi)}
    const double *clo, *chi; // coefficient interval
    const float *clo32, *chi32;
    const int32_t *poly_off; // [P + 1] term ranges
    const uint32_t *tinfo;   // term info words (above)
    const int32_t *tv_off;   // [TF + 1]: first combination entry of each F term
    const uint32_t *tv_map;  // [E]: term << 8 | combination of its variables' halves
    const uint16_t *cix;     // [TF << n] (if present): entry of F term t for child c at (t << n) + c
    const uint8_t *fac;
};

__device__ __forceinline__ SysTab make_tab(const char *blob, const DevSys &S) {
    const BlobLayout L = blob_layout(S.n_terms, S.n_polys, S.n_facs, S.n_fterms, S.n_tv, S.n_cix);
    SysTab t;
    t.cs = reinterpret_cast<const float4 *>(blob + L.cs);
    t.clo = reinterpret_cast<const double *>(blob + L.clo);
    t.chi = reinterpret_cast<const double *>(blob + L.chi);
    t.clo32 = reinterpret_cast<const float *>(blob + L.clo32);
    t.chi32 = reinterpret_cast<const float *>(blob + L.chi32);
    t.poly_off = reinterpret_cast<const int32_t *>(blob + L.poly_off);
    t.tinfo = reinterpret_cast<const uint32_t *>(blob + L.tinfo);
    t.tv_off = reinterpret_cast<const int32_t *>(blob + L.tv_off);
    t.tv_map = reinterpret_cast<const uint32_t *>(blob + L.tv_map);
    t.cix = reinterpret_cast<const uint16_t *>(blob + L.cix);
    t.fac = reinterpret_cast<const uint8_t *>(blob + L.fac);
    return t;
}

// cooperative copy of a blob (bytes a multiple of 16) into shared memory
__device__ __forceinline__ void copy_blob(char *dst, const char *src, uint32_t bytes) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 16u; i += blockDim.x) d[i] = s[i];
}

// ---- evaluators over a coordinate accessor x(j) ----------------------------------------

template <class Coord>
__device__ __forceinline__ ivd term64(const SysTab &T, int t, const Coord &x) {
    const ivd cf = {T.clo[t], T.chi[t]};
    const uint32_t info = T.tinfo[t];
    const int nf = term_nf(info), f0 = term_f0(info);
    if (nf == 0) return cf;
    unsigned fc = T.fac[f0];
    ivd prod = iv_pow(x(fc >> 4), (int)(fc & 15u));
    for (int f = 1; f < nf; f++) {
        fc = T.fac[f0 + f];
        prod = iv_mul(prod, iv_pow(x(fc >> 4), (int)(fc & 15u)));
    }
    // a point coefficient c: [c,c] * prod equals c * prod (two products, not four);
    // the flag is the term's, so the lanes of a warp take the same branch
    return (info & kTermPoint) ? iv_smul(cf.lo, prod) : iv_mul(cf, prod);
}

template <class Coord>
__device__ __forceinline__ ivd poly64(const SysTab &T, int p, const Coord &x) {
    const int t0 = T.poly_off[p], t1 = T.poly_off[p + 1];
    if (t0 == t1) return ivd{0.0, 0.0};
    ivd acc = term64(T, t0, x);
    for (int t = t0 + 1; t < t1; t++) acc = iv_add(acc, term64(T, t, x));
    return acc;
}

template <class Coord>
__device__ __forceinline__ ivf poly32(const SysTab &T, int p, const Coord &x) {
    const int t0 = T.poly_off[p], t1 = T.poly_off[p + 1];
    ivf acc = {0.0f, 0.0f};
    for (int t = t0; t < t1; t++) {
        const ivf cf = {T.clo32[t], T.chi32[t]};
        const uint32_t info = T.tinfo[t];
        const int nf = term_nf(info), f0 = term_f0(info);
        ivf v;
        if (nf == 0) {
            v = cf;
        } else {
            unsigned fc = T.fac[f0];
            ivf prod = fv_pow(x(fc >> 4), (int)(fc & 15u));
            for (int f = 1; f < nf; f++) {
                fc = T.fac[f0 + f];
                prod = fv_mul(prod, fv_pow(x(fc >> 4), (int)(fc & 15u)));
            }
            v = fv_mul(cf, prod);
        }
        acc = (t == t0) ? v : fv_add(acc, v);
    }
    return acc;
}

template <class Coord>
__device__ __forceinline__ shv poly_shadow(const SysTab &T, int p, const Coord &x, bool &poison) {
    const int t0 = T.poly_off[p], t1 = T.poly_off[p + 1];
    shv acc = {0.f, 0.f, 0.f, 0.f};
    for (int t = t0; t < t1; t++) {
        const float4 ce = T.cs[t];
        const shv cf = {ce.x, ce.y, ce.z, ce.w};
        const uint32_t info = T.tinfo[t];
        const int nf = term_nf(info), f0 = term_f0(info);
        shv v;
        if (nf == 0) {
            v = cf;
        } else {
            unsigned fc = T.fac[f0];
            shv prod = sh_pow(x(fc >> 4), (int)(fc & 15u), poison);
            for (int f = 1; f < nf; f++) {
                fc = T.fac[f0 + f];
                prod = sh_mul(prod, sh_pow(x(fc >> 4), (int)(fc & 15u), poison), poison);
            }
            v = sh_mul(cf, prod, poison);
        }
        acc = (t == t0) ? v : sh_add(acc, v);
    }
    return acc;
}

// Definition 2 in FP64: false as soon as one F_i excludes 0 (NaN ends never exclude)
template <class Coord>
__device__ __forceinline__ bool keep64(const SysTab &T, const DevSys &S, const Coord &x) {
    for (int i = 0; i < S.m; i++) {
        const ivd F = poly64(T, S.f_poly + i, x);
        if (d_pos(F.lo) || d_neg(F.hi)) return false;
    }
    return true;
}

template <class Coord>
__device__ __forceinline__ bool keep32(const SysTab &T, const DevSys &S, const Coord &x) {
    for (int i = 0; i < S.m; i++) {
        const ivf F = poly32(T, S.f_poly + i, x);
        if (F.lo > 0.0f || F.hi < 0.0f) return false;
    }
    return true;
}

// FP32 shadow decision: 0 = FP64 would exclude, 1 = FP64 would keep, 2 = undecided
template <class Coord>
__device__ __forceinline__ int decide_shadow(const SysTab &T, const DevSys &S, const Coord &x) {
    bool undecided = false;
    for (int i = 0; i < S.m; i++) {
        bool poison = false;
        const shv F = poly_shadow(T, S.f_poly + i, x, poison);
        if (poison) { undecided = true; continue; }
        if (F.ld > 0.0f || F.hu < 0.0f) return 0;        // lo64 > 0 or hi64 < 0
        if (!(F.lu <= 0.0f && F.hd >= 0.0f)) undecided = true;
    }
    return undecided ? 2 : 1;
}

// ---- per-parent term-combination table (FP32 shadow) ------------------------------------
// Entry (t, q) is the shadow of term t over the child whose halves in the term's
// variables are the bits of q (bit f <-> the term's f-th factor): exactly what
// poly_shadow computes for term t of any such child.  A poisoned entry is stored as NaN,
// which then makes the equation's sum NaN: it neither excludes nor proves a keep.
template <class Coord>
__device__ __forceinline__ float4 term_shadow(const SysTab &T, int t, const Coord &x) {
    const float4 ce = T.cs[t];
    const uint32_t info = T.tinfo[t];
    const int nf = term_nf(info), f0 = term_f0(info);
    if (nf == 0) return ce;
    bool poison = false;
    unsigned fc = T.fac[f0];
    shv prod = sh_pow(x(fc >> 4, 0), (int)(fc & 15u), poison);
    for (int f = 1; f < nf; f++) {
        fc = T.fac[f0 + f];
        prod = sh_mul(prod, sh_pow(x(fc >> 4, f), (int)(fc & 15u), poison), poison);
    }
    const shv v = sh_mul(shv{ce.x, ce.y, ce.z, ce.w}, prod, poison);
    if (poison) {
        const float nan = __int_as_float(0x7FC00000);
        return make_float4(nan, nan, nan, nan);
    }
    return make_float4(v.ld, v.lu, v.hd, v.hu);
}

// FP32 shadow decision of child c from its parent's table tv (same result as
// decide_shadow on the child): 0 exclude, 1 keep, 2 undecided.  The entry of a term for
// the child is read from the child-index table when the blob has one (small n), else
// gathered from the child's bits in the term's variables.
__device__ __forceinline__ int decide_from_table(const SysTab &T, const DevSys &S, const float4 *tv, unsigned c) {
    bool undecided = false;
    for (int i = 0; i < S.m; i++) {
        const int t0 = T.poly_off[S.f_poly + i], t1 = T.poly_off[S.f_poly + i + 1];
        shv acc = {0.f, 0.f, 0.f, 0.f};
        for (int t = t0; t < t1; t++) {
            int e;
            if (S.n_cix > 0) {
                e = T.cix[((unsigned)t << S.n) + c];
            } else {
                const uint32_t info = T.tinfo[t];
                const int nf = term_nf(info), f0 = term_f0(info);
                unsigned q = 0;
                for (int f = 0; f < nf; f++) q |= ((c >> (T.fac[f0 + f] >> 4)) & 1u) << f;
                e = T.tv_off[t] + (int)q;
            }
            const float4 v = tv[e];
            const shv sv = {v.x, v.y, v.z, v.w};
            acc = (t == t0) ? sv : sh_add(acc, sv);
        }
        if (acc.ld > 0.0f || acc.hu < 0.0f) return 0;
        if (!(acc.lu <= 0.0f && acc.hd >= 0.0f)) undecided = true;   // also NaN (poison)
    }
    return undecided ? 2 : 1;
}

// The same decision for K children c[0..K) of one parent at once (child-index table
// present), each exactly as decide_from_table: the K sums of an equation are independent
// chains of loads and adds, so one thread overlaps their latencies.  An equation is
// evaluated while any wanted child is undecided; a decided child's sums are ignored.
// want[k] = false: c[k] is not a child (d[k] = 0).
template <int K>
__device__ __forceinline__ void decide_from_table_k(const SysTab &T, const DevSys &S, const float4 *tv,
                                                    const unsigned (&c)[K], const bool (&want)[K], int (&d)[K]) {
    int rs[K];      // -1: no equation excluded yet
    bool und[K];
    int open = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        rs[k] = want[k] ? -1 : 0;
        und[k] = false;
        open += want[k] ? 1 : 0;
    }
    for (int i = 0; i < S.m && open > 0; i++) {
        const int t0 = T.poly_off[S.f_poly + i], t1 = T.poly_off[S.f_poly + i + 1];
        shv acc[K];
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] = shv{0.f, 0.f, 0.f, 0.f};
        for (int t = t0; t < t1; t++) {
            const uint16_t *row = T.cix + ((unsigned)t << S.n);
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float4 v = tv[row[c[k]]];
                const shv s = {v.x, v.y, v.z, v.w};
                acc[k] = (t == t0) ? s : sh_add(acc[k], s);
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (rs[k] >= 0) continue;
            if (acc[k].ld > 0.0f || acc[k].hu < 0.0f) {
                rs[k] = 0;
                open--;
            } else if (!(acc[k].lu <= 0.0f && acc[k].hd >= 0.0f)) {
                und[k] = true;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) d[k] = rs[k] >= 0 ? rs[k] : (und[k] ? 2 : 1);
}

}  // namespace ivs
