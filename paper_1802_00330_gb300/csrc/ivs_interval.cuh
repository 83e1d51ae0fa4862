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

// Products select their endpoint operands from the operands' sign classes (integer
// selects) and always issue two round-down and two round-up multiplies: with one box
// per lane, branching on signs would diverge across the warp and every diverged path
// would re-issue its FP64 instructions at full warp cost.  The second pair only differs
// from the first when both operands straddle 0.  Classes: P = lo >= 0, else N = hi <= 0,
// else S (lo < 0 < hi); P is tested first, as in the serial definition.
// Endpoint operands of the product x y: the lower end is min(rd(la lb), rd(la2 lb2)),
// the upper end max(ru(ua ub), ru(ua2 ub2)); the second pair differs from the first only
// when both operands straddle 0 (`both`).
struct MulSel {
    double la, lb, la2, lb2, ua, ub, ua2, ub2;
    bool both;
};
__device__ __forceinline__ MulSel mul_sel(ivd x, ivd y) {
    const bool xp = !d_neg(x.lo), xn = !xp && !d_pos(x.hi), xs = !xp && !xn;
    const bool yp = !d_neg(y.lo), yn = !yp && !d_pos(y.hi), ys = !yp && !yn;
    MulSel m;
    m.both = xs && ys;
    // lower end: xP: (yP ? lo : hi) * y.lo;  xN: (yN ? hi : lo) * y.hi;
    //            xS: yN ? hi * lo : lo * hi (and hi * lo as well when y straddles)
    m.la = xp ? (yp ? x.lo : x.hi) : (yn ? x.hi : x.lo);
    m.lb = xp ? y.lo : (xn ? y.hi : (yn ? y.lo : y.hi));
    m.la2 = m.both ? x.hi : m.la;
    m.lb2 = m.both ? y.lo : m.lb;
    // upper end: xP: (yN ? lo : hi) * y.hi;  xN: (yP ? hi : lo) * y.lo;
    //            xS: yP ? hi * hi : lo * lo (and hi * hi as well when y straddles)
    m.ua = xp ? (yn ? x.lo : x.hi) : (xn ? (yp ? x.hi : x.lo) : (yp ? x.hi : x.lo));
    m.ub = xp ? y.hi : (xn ? y.lo : (yp ? y.hi : y.lo));
    m.ua2 = m.both ? x.hi : m.ua;
    m.ub2 = m.both ? y.hi : m.ub;
    return m;
}
__device__ __forceinline__ ivd iv_mul(ivd x, ivd y) {
    const MulSel m = mul_sel(x, y);
    const double l1 = __dmul_rd(m.la, m.lb), u1 = __dmul_ru(m.ua, m.ub);
    // the second pair only when some lane of the warp has both operands straddling 0
    // (for the other lanes it repeats the first pair, so their result is unchanged)
    if (__any_sync(__activemask(), m.both)) return {d_min(l1, __dmul_rd(m.la2, m.lb2)), d_max(u1, __dmul_ru(m.ua2, m.ub2))};
    return {l1, u1};
}
// the lower / upper end of iv_mul(x, y) alone (the same value, half the multiplies)
__device__ __forceinline__ double iv_mul_lo(ivd x, ivd y) {
    const MulSel m = mul_sel(x, y);
    const double l1 = __dmul_rd(m.la, m.lb);
    if (__any_sync(__activemask(), m.both)) return d_min(l1, __dmul_rd(m.la2, m.lb2));
    return l1;
}
__device__ __forceinline__ double iv_mul_hi(ivd x, ivd y) {
    const MulSel m = mul_sel(x, y);
    const double u1 = __dmul_ru(m.ua, m.ub);
    if (__any_sync(__activemask(), m.both)) return d_max(u1, __dmul_ru(m.ua2, m.ub2));
    return u1;
}

// point b times interval y (b a double): two products
__device__ __forceinline__ ivd iv_smul(double b, ivd y) {
    const bool neg = d_neg(b);
    return {__dmul_rd(b, neg ? y.hi : y.lo), __dmul_ru(b, neg ? y.lo : y.hi)};
}

__device__ __forceinline__ double d_abs(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL);
}
// -x by flipping the sign bit (exactly IEEE negation) on the integer pipe
__device__ __forceinline__ double d_negate(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// monotone chains for the power rule (argument >= 0)
__device__ __forceinline__ double chain_rd(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = __dmul_rd(p, x); return p; }
__device__ __forceinline__ double chain_ru(double x, int k) { double p = x; for (int i = 1; i < k; i++) p = __dmul_ru(p, x); return p; }

// x^k, k >= 1, by the power rule.  Even k: [down-chain(a), up-chain(b)] with
// (a, b) = (lo, hi) if lo >= 0, (-hi, -lo) if hi <= 0, (0, max(-lo, hi)) otherwise.
// Odd k, each end e: q <- e, then (k-1) times q <- r(q * |e|); since r(-z) = -r'(z)
// exactly, this equals chain(e) for e >= 0 and -chain'(-e) for e < 0 (chain' in the
// opposite direction), i.e. the serial rule, with no branch on the sign.
__device__ __forceinline__ ivd iv_pow(ivd x, int k) {
    if (k == 1) return x;
    if ((k & 1) == 0) {
        const bool p = !d_neg(x.lo), n = !p && !d_pos(x.hi);
        const double a = p ? x.lo : (n ? d_negate(x.hi) : 0.0);
        const double b = p ? x.hi : (n ? d_negate(x.lo) : d_max(d_negate(x.lo), x.hi));
        return {chain_rd(a, k), chain_ru(b, k)};
    }
    const double al = d_abs(x.lo), ah = d_abs(x.hi);
    double lo = x.lo, hi = x.hi;
    for (int i = 1; i < k; i++) {
        lo = __dmul_rd(lo, al);
        hi = __dmul_ru(hi, ah);
    }
    return {lo, hi};
}

// ordinary division, 0 not in y: one round-down and one round-up quotient, operands
// selected by the signs (y > 0: xP [lo/hi, hi/lo], xN [lo/lo, hi/hi], xS [lo/lo, hi/lo];
// y < 0: xP [hi/hi, lo/lo], xN [hi/lo, lo/hi], xS [hi/hi, lo/hi])
__device__ __forceinline__ void div_operands(ivd x, ivd y, double &ln, double &ld, double &un, double &ud) {
    const bool xp = !d_neg(x.lo), xn = !xp && !d_pos(x.hi);
    if (d_pos(y.lo)) {
        ln = x.lo;
        ld = xp ? y.hi : y.lo;
        un = x.hi;
        ud = xn ? y.hi : y.lo;
    } else {
        ln = x.hi;
        ld = xn ? y.lo : y.hi;
        un = x.lo;
        ud = xp ? y.lo : y.hi;
    }
}
__device__ __forceinline__ ivd iv_div(ivd x, ivd y) {
    double ln, ld, un, ud;
    div_operands(x, y, ln, ld, un, ud);
    return {__ddiv_rd(ln, ld), __ddiv_ru(un, ud)};
}

// Extended division (eq 10).  Writes up to two pieces (ends may be infinite) and
// returns their count: 0 = empty set.  Case table: 0 not in y -> ordinary division;
// 0 in x and 0 in y -> whole line; y = [0,0], 0 not in x -> empty; x < 0: y = [c,0] ->
// [hi/c, +inf), c < 0 < d -> (-inf, hi/d] u [hi/c, +inf), y = [0,d] -> (-inf, hi/d];
// x > 0: y = [c,0] -> (-inf, lo/c], c < 0 < d -> (-inf, lo/c] u [lo/d, +inf),
// y = [0,d] -> [lo/d, +inf).  Finite ends round outward.  Every case needs at most one
// round-down and one round-up quotient; both are issued once with selected operands.
// The case and the quotient operands: qd = rd(ln / ld), qu = ru(un / ud).
enum : int { XD_ORD, XD_WHOLE, XD_NONE, XD_UP, XD_DOWN, XD_TWO };   // [qd,qu] R {} [qd,inf) (-inf,qu] both
struct ExtDiv {
    double ln, ld, un, ud;
    int kind;
};
__device__ __forceinline__ ExtDiv extdiv_setup(ivd x, ivd y) {
    const bool ordinary = d_pos(y.lo) || d_neg(y.hi);
    const bool whole = !ordinary && !d_pos(x.lo) && !d_neg(x.hi);
    const bool ylo0 = d_iszero(y.lo), yhi0 = d_iszero(y.hi);
    const bool xneg = d_neg(x.hi);                    // else x > 0 in the extended cases
    ExtDiv e;
    div_operands(x, y, e.ln, e.ld, e.un, e.ud);
    if (!ordinary) {
        // rd quotient: x < 0: hi / c;  x > 0: lo / d.   ru quotient: x < 0: hi / d;  x > 0: lo / c
        e.ln = xneg ? x.hi : x.lo;
        e.ld = xneg ? y.lo : y.hi;
        e.un = xneg ? x.hi : x.lo;
        e.ud = xneg ? y.hi : y.lo;
    }
    e.kind = ordinary ? XD_ORD : whole ? XD_WHOLE : (ylo0 && yhi0) ? XD_NONE
           : yhi0 ? (xneg ? XD_UP : XD_DOWN) : ylo0 ? (xneg ? XD_DOWN : XD_UP) : XD_TWO;
    // a quotient the case does not use gets 1 / 1 (its operands may hold a zero divisor,
    // which would take the division's special-case path for nothing)
    if (e.kind == XD_WHOLE || e.kind == XD_NONE || e.kind == XD_DOWN) e.ln = e.ld = 1.0;
    if (e.kind == XD_WHOLE || e.kind == XD_NONE || e.kind == XD_UP) e.un = e.ud = 1.0;
    return e;
}
// the pieces from the two quotients; returns their count
__device__ __forceinline__ int extdiv_pieces(int kind, double qd, double qu, ivd *p) {
    const double inf = __longlong_as_double(0x7FF0000000000000LL);
    switch (kind) {
        case XD_ORD: p[0] = {qd, qu}; return 1;
        case XD_WHOLE: p[0] = {-inf, inf}; return 1;
        case XD_NONE: return 0;
        case XD_UP: p[0] = {qd, inf}; return 1;
        case XD_DOWN: p[0] = {-inf, qu}; return 1;
        default: p[0] = {-inf, qu}; p[1] = {qd, inf}; return 2;
    }
}
__device__ __forceinline__ int iv_extdiv(ivd x, ivd y, ivd *p) {
    const ExtDiv e = extdiv_setup(x, y);
    const double qd = __ddiv_rd(e.ln, e.ld), qu = __ddiv_ru(e.un, e.ud);
    return extdiv_pieces(e.kind, qd, qu, p);
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

// Enclosure [rd32(min), ru32(max)] of the exact product of two FP64 values whose signs
// are known (sa / sb: true for >= 0, false for <= 0) and whose enclosures are
// [ad, au], [bd, bu].  The enclosures are first clamped to the known sign; then the
// minimum is ad*bd (+,+), au*bd (+,-), ad*bu (-,+), au*bu (-,-) and the maximum the
// mirror choice: two multiplies, operands picked by selects (no divergence).
__device__ __forceinline__ float2 enc_mul_signed(float ad, float au, bool sa, float bd, float bu, bool sb) {
    ad = sa ? fmaxf(ad, 0.0f) : ad;
    au = sa ? au : fminf(au, 0.0f);
    bd = sb ? fmaxf(bd, 0.0f) : bd;
    bu = sb ? bu : fminf(bu, 0.0f);
    return make_float2(__fmul_rd(sb ? ad : au, sa ? bd : bu), __fmul_ru(sb ? au : ad, sa ? bu : bd));
}

// sign class of an FP64 interval from its shadow: 1 = P (L >= 0), 2 = N (H <= 0),
// 3 = S (L < 0 < H), 0 = not provable
__device__ __forceinline__ int sh_class(const shv &x) {
    if (x.ld >= 0.0f) return 1;
    if (x.hu <= 0.0f) return 2;
    if (x.lu < 0.0f && x.hd > 0.0f) return 3;
    return 0;
}

// FP64 product L = rd64(min of the four end products), H = ru64(max): the proven classes
// name the products (the same table as iv_mul); each is enclosed by enc_mul_signed.
// Ends' signs: lo is >= 0 in class P, <= 0 otherwise; hi is <= 0 in class N, >= 0 otherwise.
__device__ __forceinline__ shv sh_mul(shv x, shv y, bool &poison) {
    const int cx = sh_class(x), cy = sh_class(y);
    poison |= (cx == 0) | (cy == 0);
    const bool xp = cx == 1, xn = cx == 2, xs = cx == 3;
    const bool yp = cy == 1, yn = cy == 2, ys = cy == 3;
    const bool sxl = xp, sxh = !xn, syl = yp, syh = !yn;
    // lower: x end (yP ? lo : hi) when xP, (yN ? hi : lo) otherwise; y end lo when xP,
    // hi when xN, (yN ? lo : hi) when xS; second candidate (x.hi, y.lo) when both straddle
    const bool lxh = xp ? !yp : yn;
    const bool lyh = xp ? false : (xn ? true : !yn);
    const bool uxh = xp ? !yn : yp;
    const bool uyh = xp ? true : (xn ? false : yp);
    const bool ss = xs && ys;
    const float2 l1 = enc_mul_signed(lxh ? x.hd : x.ld, lxh ? x.hu : x.lu, lxh ? sxh : sxl,
                                     lyh ? y.hd : y.ld, lyh ? y.hu : y.lu, lyh ? syh : syl);
    const float2 l2 = enc_mul_signed(ss ? x.hd : (lxh ? x.hd : x.ld), ss ? x.hu : (lxh ? x.hu : x.lu),
                                     ss ? sxh : (lxh ? sxh : sxl), ss ? y.ld : (lyh ? y.hd : y.ld),
                                     ss ? y.lu : (lyh ? y.hu : y.lu), ss ? syl : (lyh ? syh : syl));
    const float2 h1 = enc_mul_signed(uxh ? x.hd : x.ld, uxh ? x.hu : x.lu, uxh ? sxh : sxl,
                                     uyh ? y.hd : y.ld, uyh ? y.hu : y.lu, uyh ? syh : syl);
    const float2 h2 = enc_mul_signed(ss ? x.hd : (uxh ? x.hd : x.ld), ss ? x.hu : (uxh ? x.hu : x.lu),
                                     ss ? sxh : (uxh ? sxh : sxl), ss ? y.hd : (uyh ? y.hd : y.ld),
                                     ss ? y.hu : (uyh ? y.hu : y.lu), ss ? syh : (uyh ? syh : syl));
    return {fminf(l1.x, l2.x), fminf(l1.y, l2.y), fmaxf(h1.x, h2.x), fmaxf(h1.y, h2.y)};
}

// x^k (k >= 1) by the power rule of iv_pow.  Even k: the class picks the chain operands
// (clamped to their known sign) and down / up chains enclose the FP64 chains.  Odd k:
// the FP64 end is the monotone q-chain of iv_pow, so the q-chain of the lower enclosure
// end rounded down and of the upper end rounded up enclose it, whatever the signs.
__device__ __forceinline__ shv sh_pow(shv x, int k, bool &poison) {
    if (k == 1) return x;
    if ((k & 1) == 0) {
        const int c = sh_class(x);
        poison |= c == 0;
        const bool p = c == 1, n = c == 2;
        const float ad = p ? x.ld : (n ? -x.hu : 0.0f);
        const float au = p ? x.lu : (n ? -x.hd : 0.0f);
        const float bd = p ? fmaxf(x.hd, 0.0f) : (n ? -fminf(x.lu, 0.0f) : fmaxf(-x.lu, x.hd));
        const float bu = p ? x.hu : (n ? -x.ld : fmaxf(-x.ld, x.hu));
        return {fchain_rd(ad, k), fchain_ru(au, k), fchain_rd(bd, k), fchain_ru(bu, k)};
    }
    float ld = x.ld, lu = x.lu, hd = x.hd, hu = x.hu;
    const float ald = fabsf(x.ld), alu = fabsf(x.lu), ahd = fabsf(x.hd), ahu = fabsf(x.hu);
    for (int i = 1; i < k; i++) {
        ld = __fmul_rd(ld, ald);
        lu = __fmul_ru(lu, alu);
        hd = __fmul_rd(hd, ahd);
        hu = __fmul_ru(hu, ahu);
    }
    return {ld, lu, hd, hu};
}

}  // namespace ivs
