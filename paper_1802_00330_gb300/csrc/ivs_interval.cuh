// ivs_interval.cuh -- device interval arithmetic with directed rounding (sm_103a).
//
// Section 3.2 (eq 25-27): every lower end is rounded down and every upper end up,
// using the hardware's directed-rounding instructions (__dadd_rd, __dmul_ru, ...).
// Products pick their two endpoint products from the operands' signs: rd and ru are
// monotone, so the lower end rd(min of the four products) equals rd of the product the
// sign case selects, and likewise for the upper end.  Only the case where both
// operands straddle 0 needs four products.  Sign tests and min/max of doubles run on
// the integer pipes (bit patterns), keeping the FP64 pipe for arithmetic.
#pragma once
#include <cstdint>

namespace ivs {

struct ivd { double lo, hi; };
struct ivf { float lo, hi; };

// ---- sign tests on bit patterns (no FP64 instruction) ----------------------------
// Numeric semantics: -0 counts as 0.  NaN is neither positive nor negative.
__device__ __forceinline__ bool d_pos(double x) {      // x > 0
    long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool d_neg(double x) {      // x < 0
    long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ULL &&
           (b & 0x7FFFFFFFFFFFFFFFLL) <= 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool d_nonneg(double x) { return !(d_neg(x)) && !isnan(x); }
__device__ __forceinline__ bool d_nonpos(double x) { return !(d_pos(x)) && !isnan(x); }
__device__ __forceinline__ bool d_iszero(double x) {
    return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) == 0;
}
// total order key for non-NaN doubles (-0 sorts below +0; numerically a tie)
__device__ __forceinline__ long long d_key(double x) {
    long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double d_min(double a, double b) { return d_key(b) < d_key(a) ? b : a; }
__device__ __forceinline__ double d_max(double a, double b) { return d_key(b) > d_key(a) ? b : a; }

__device__ __forceinline__ bool f_pos(float x) { return x > 0.0f; }
__device__ __forceinline__ bool f_neg(float x) { return x < 0.0f; }

// ---- FP64 interval operations ----------------------------------------------------
__device__ __forceinline__ ivd iv_add(ivd x, ivd y) { return {__dadd_rd(x.lo, y.lo), __dadd_ru(x.hi, y.hi)}; }
__device__ __forceinline__ ivd iv_sub(ivd x, ivd y) { return {__dsub_rd(x.lo, y.hi), __dsub_ru(x.hi, y.lo)}; }

__device__ __forceinline__ ivd iv_mul(ivd x, ivd y) {
    // classify by sign: x >= 0, x <= 0, or straddling (lo < 0 < hi)
    const bool xp = !d_neg(x.lo), xn = !d_pos(x.hi);
    const bool yp = !d_neg(y.lo), yn = !d_pos(y.hi);
    if (xp) {
        if (yp) return {__dmul_rd(x.lo, y.lo), __dmul_ru(x.hi, y.hi)};
        if (yn) return {__dmul_rd(x.hi, y.lo), __dmul_ru(x.lo, y.hi)};
        return {__dmul_rd(x.hi, y.lo), __dmul_ru(x.hi, y.hi)};
    }
    if (xn) {
        if (yp) return {__dmul_rd(x.lo, y.hi), __dmul_ru(x.hi, y.lo)};
        if (yn) return {__dmul_rd(x.hi, y.hi), __dmul_ru(x.lo, y.lo)};
        return {__dmul_rd(x.lo, y.hi), __dmul_ru(x.lo, y.lo)};
    }
    if (yp) return {__dmul_rd(x.lo, y.hi), __dmul_ru(x.hi, y.hi)};
    if (yn) return {__dmul_rd(x.hi, y.lo), __dmul_ru(x.lo, y.lo)};
    return {d_min(__dmul_rd(x.lo, y.hi), __dmul_rd(x.hi, y.lo)),
            d_max(__dmul_ru(x.lo, y.lo), __dmul_ru(x.hi, y.hi))};
}

// point b times interval y (b a double): two products
__device__ __forceinline__ ivd iv_smul(double b, ivd y) {
    if (!d_neg(b)) return {__dmul_rd(b, y.lo), __dmul_ru(b, y.hi)};
    return {__dmul_rd(b, y.hi), __dmul_ru(b, y.lo)};
}

// monotone chains for the power rule (argument >= 0)
__device__ __forceinline__ double chain_rd(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = __dmul_rd(p, x); return p; }
__device__ __forceinline__ double chain_ru(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = __dmul_ru(p, x); return p; }

// x^k, k >= 1 (power rule: even k folds the sign, odd k is monotone)
__device__ __forceinline__ ivd iv_pow(ivd x, int k) {
    if (k == 1) return x;
    if ((k & 1) == 0) {
        if (!d_neg(x.lo)) return {chain_rd(x.lo, k), chain_ru(x.hi, k)};
        if (!d_pos(x.hi)) return {chain_rd(-x.hi, k), chain_ru(-x.lo, k)};
        return {0.0, chain_ru(d_max(-x.lo, x.hi), k)};
    }
    double lo = !d_neg(x.lo) ? chain_rd(x.lo, k) : -chain_ru(-x.lo, k);
    double hi = !d_neg(x.hi) ? chain_ru(x.hi, k) : -chain_rd(-x.hi, k);
    return {lo, hi};
}

// ordinary division, 0 not in y: the two quotients the signs select
__device__ __forceinline__ ivd iv_div(ivd x, ivd y) {
    const bool xp = !d_neg(x.lo), xn = !d_pos(x.hi);
    if (d_pos(y.lo)) {           // y > 0
        if (xp) return {__ddiv_rd(x.lo, y.hi), __ddiv_ru(x.hi, y.lo)};
        if (xn) return {__ddiv_rd(x.lo, y.lo), __ddiv_ru(x.hi, y.hi)};
        return {__ddiv_rd(x.lo, y.lo), __ddiv_ru(x.hi, y.lo)};
    }
    // y < 0
    if (xp) return {__ddiv_rd(x.hi, y.hi), __ddiv_ru(x.lo, y.lo)};
    if (xn) return {__ddiv_rd(x.hi, y.lo), __ddiv_ru(x.lo, y.hi)};
    return {__ddiv_rd(x.hi, y.hi), __ddiv_ru(x.lo, y.hi)};
}

// Extended division (eq 10).  Writes up to two pieces (ends may be infinite) and
// returns their count: 0 = empty set.  Case table: 0 not in y -> ordinary division;
// 0 in x and 0 in y -> whole line; y = [0,0], 0 not in x -> empty; x < 0: y = [c,0] ->
// [hi/c, +inf), c < 0 < d -> (-inf, hi/d] u [hi/c, +inf), y = [0,d] -> (-inf, hi/d];
// x > 0: y = [c,0] -> (-inf, lo/c], c < 0 < d -> (-inf, lo/c] u [lo/d, +inf),
// y = [0,d] -> [lo/d, +inf).  Finite ends round outward.
__device__ __forceinline__ int iv_extdiv(ivd x, ivd y, ivd *p) {
    const double inf = __longlong_as_double(0x7FF0000000000000LL);
    if (d_pos(y.lo) || d_neg(y.hi)) { p[0] = iv_div(x, y); return 1; }
    if (!d_pos(x.lo) && !d_neg(x.hi)) { p[0] = {-inf, inf}; return 1; }
    const bool ylo0 = d_iszero(y.lo), yhi0 = d_iszero(y.hi);
    if (ylo0 && yhi0) return 0;
    if (d_neg(x.hi)) {
        if (yhi0) { p[0] = {__ddiv_rd(x.hi, y.lo), inf}; return 1; }
        if (ylo0) { p[0] = {-inf, __ddiv_ru(x.hi, y.hi)}; return 1; }
        p[0] = {-inf, __ddiv_ru(x.hi, y.hi)};
        p[1] = {__ddiv_rd(x.hi, y.lo), inf};
        return 2;
    }
    if (yhi0) { p[0] = {-inf, __ddiv_ru(x.lo, y.lo)}; return 1; }
    if (ylo0) { p[0] = {__ddiv_rd(x.lo, y.hi), inf}; return 1; }
    p[0] = {-inf, __ddiv_ru(x.lo, y.lo)};
    p[1] = {__ddiv_rd(x.lo, y.hi), inf};
    return 2;
}

// ---- FP32 interval operations (prefilter) -----------------------------------------
__device__ __forceinline__ ivf fv_add(ivf x, ivf y) { return {__fadd_rd(x.lo, y.lo), __fadd_ru(x.hi, y.hi)}; }
__device__ __forceinline__ ivf fv_mul(ivf x, ivf y) {
    const bool xp = !(x.lo < 0.0f), xn = !(x.hi > 0.0f);
    const bool yp = !(y.lo < 0.0f), yn = !(y.hi > 0.0f);
    if (xp) {
        if (yp) return {__fmul_rd(x.lo, y.lo), __fmul_ru(x.hi, y.hi)};
        if (yn) return {__fmul_rd(x.hi, y.lo), __fmul_ru(x.lo, y.hi)};
        return {__fmul_rd(x.hi, y.lo), __fmul_ru(x.hi, y.hi)};
    }
    if (xn) {
        if (yp) return {__fmul_rd(x.lo, y.hi), __fmul_ru(x.hi, y.lo)};
        if (yn) return {__fmul_rd(x.hi, y.hi), __fmul_ru(x.lo, y.lo)};
        return {__fmul_rd(x.lo, y.hi), __fmul_ru(x.lo, y.lo)};
    }
    if (yp) return {__fmul_rd(x.lo, y.hi), __fmul_ru(x.hi, y.hi)};
    if (yn) return {__fmul_rd(x.hi, y.lo), __fmul_ru(x.lo, y.lo)};
    return {fminf(__fmul_rd(x.lo, y.hi), __fmul_rd(x.hi, y.lo)),
            fmaxf(__fmul_ru(x.lo, y.lo), __fmul_ru(x.hi, y.hi))};
}
__device__ __forceinline__ float fchain_rd(float x, int k) { float p = x; for (int i = 1; i < k; i++) p = __fmul_rd(p, x); return p; }
__device__ __forceinline__ float fchain_ru(float x, int k) { float p = x; for (int i = 1; i < k; i++) p = __fmul_ru(p, x); return p; }
__device__ __forceinline__ ivf fv_pow(ivf x, int k) {
    if (k == 1) return x;
    if ((k & 1) == 0) {
        if (!(x.lo < 0.0f)) return {fchain_rd(x.lo, k), fchain_ru(x.hi, k)};
        if (!(x.hi > 0.0f)) return {fchain_rd(-x.hi, k), fchain_ru(-x.lo, k)};
        return {0.0f, fchain_ru(fmaxf(-x.lo, x.hi), k)};
    }
    float lo = !(x.lo < 0.0f) ? fchain_rd(x.lo, k) : -fchain_ru(-x.lo, k);
    float hi = !(x.hi < 0.0f) ? fchain_ru(x.hi, k) : -fchain_rd(-x.hi, k);
    return {lo, hi};
}

// ---- FP32 shadow of an FP64 interval computation -----------------------------------
// For an FP64 interval [L, H] the shadow holds float enclosures L in [ld, lu] and
// H in [hd, hu].  rd32 <= rd64 and ru64 <= ru32 pointwise, and all roundings are
// monotone, so each shadow operation below encloses the FP64 operation's result.  An
// operation whose FP64 sign case cannot be proven from the enclosures (an end within
// float rounding of 0 but not exactly 0) marks the shadow ambiguous ("poisoned").
struct shv { float ld, lu, hd, hu; };

__device__ __forceinline__ shv sh_add(shv a, shv b) {
    return {__fadd_rd(a.ld, b.ld), __fadd_ru(a.lu, b.lu), __fadd_rd(a.hd, b.hd), __fadd_ru(a.hu, b.hu)};
}

// enclosure [rd(min), ru(max)] of the exact product of two values with enclosures
// [ad, au] and [bd, bu]
__device__ __forceinline__ float2 enc_mul(float ad, float au, float bd, float bu) {
    const ivf r = fv_mul(ivf{ad, au}, ivf{bd, bu});
    return make_float2(r.lo, r.hi);
}

// sign class of an FP64 interval from its shadow: 1 = [L,H] >= 0 (L >= 0),
// 2 = [L,H] <= 0 (H <= 0), 3 = L < 0 < H, 0 = not provable
__device__ __forceinline__ int sh_class(const shv &x) {
    if (x.ld >= 0.0f) return 1;
    if (x.hu <= 0.0f) return 2;
    if (x.lu < 0.0f && x.hd > 0.0f) return 3;
    return 0;
}

// FP64 product: L = rd64(min of the 4 end products), H = ru64(max); the proven sign
// classes name the products that are the min and the max.
__device__ __forceinline__ shv sh_mul(shv x, shv y, bool &poison) {
    const int cx = sh_class(x), cy = sh_class(y);
    if (cx == 0 || cy == 0) { poison = true; return {0.f, 0.f, 0.f, 0.f}; }
    float2 l, h;
    if (cx == 1) {
        if (cy == 1) { l = enc_mul(x.ld, x.lu, y.ld, y.lu); h = enc_mul(x.hd, x.hu, y.hd, y.hu); }
        else if (cy == 2) { l = enc_mul(x.hd, x.hu, y.ld, y.lu); h = enc_mul(x.ld, x.lu, y.hd, y.hu); }
        else { l = enc_mul(x.hd, x.hu, y.ld, y.lu); h = enc_mul(x.hd, x.hu, y.hd, y.hu); }
    } else if (cx == 2) {
        if (cy == 1) { l = enc_mul(x.ld, x.lu, y.hd, y.hu); h = enc_mul(x.hd, x.hu, y.ld, y.lu); }
        else if (cy == 2) { l = enc_mul(x.hd, x.hu, y.hd, y.hu); h = enc_mul(x.ld, x.lu, y.ld, y.lu); }
        else { l = enc_mul(x.ld, x.lu, y.hd, y.hu); h = enc_mul(x.ld, x.lu, y.ld, y.lu); }
    } else {
        if (cy == 1) { l = enc_mul(x.ld, x.lu, y.hd, y.hu); h = enc_mul(x.hd, x.hu, y.hd, y.hu); }
        else if (cy == 2) { l = enc_mul(x.hd, x.hu, y.ld, y.lu); h = enc_mul(x.ld, x.lu, y.ld, y.lu); }
        else {
            const float2 l1 = enc_mul(x.ld, x.lu, y.hd, y.hu), l2 = enc_mul(x.hd, x.hu, y.ld, y.lu);
            const float2 h1 = enc_mul(x.ld, x.lu, y.ld, y.lu), h2 = enc_mul(x.hd, x.hu, y.hd, y.hu);
            l = make_float2(fminf(l1.x, l2.x), fminf(l1.y, l2.y));
            h = make_float2(fmaxf(h1.x, h2.x), fmaxf(h1.y, h2.y));
        }
    }
    return {l.x, l.y, h.x, h.y};
}

// x^k (k >= 1) by the power rule of iv_pow: each FP64 chain p <- r64(p * v) is enclosed
// by the down chain of the lower enclosure end and the up chain of the upper end.
__device__ __forceinline__ shv sh_pow(shv x, int k, bool &poison) {
    if (k == 1) return x;
    if ((k & 1) == 0) {
        if (x.ld >= 0.0f)
            return {fchain_rd(x.ld, k), fchain_ru(x.lu, k), fchain_rd(x.hd, k), fchain_ru(x.hu, k)};
        if (x.hu <= 0.0f)
            return {fchain_rd(-x.hu, k), fchain_ru(-x.hd, k), fchain_rd(-x.lu, k), fchain_ru(-x.ld, k)};
        if (x.lu < 0.0f && x.hd > 0.0f) {
            const float md = fmaxf(-x.lu, x.hd), mu = fmaxf(-x.ld, x.hu);
            return {0.0f, 0.0f, fchain_rd(md, k), fchain_ru(mu, k)};
        }
        poison = true;
        return {0.f, 0.f, 0.f, 0.f};
    }
    shv r;
    if (x.ld >= 0.0f) { r.ld = fchain_rd(x.ld, k); r.lu = fchain_ru(x.lu, k); }
    else if (x.lu < 0.0f) { r.ld = -fchain_ru(-x.ld, k); r.lu = -fchain_rd(-x.lu, k); }
    else { poison = true; return {0.f, 0.f, 0.f, 0.f}; }
    if (x.hd >= 0.0f) { r.hd = fchain_rd(x.hd, k); r.hu = fchain_ru(x.hu, k); }
    else if (x.hu < 0.0f) { r.hd = -fchain_ru(-x.hd, k); r.hu = -fchain_rd(-x.hu, k); }
    else { poison = true; return {0.f, 0.f, 0.f, 0.f}; }
    return r;
}

}  // namespace ivs
