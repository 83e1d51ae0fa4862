// ivs_hostcore.cu -- host-side pieces shared by the plan runtime (ivs_host.cu) and the
// serving runtime (ivs_server.cu): the thread-local error text, input validation, the
// compilation of a system into its term blob, and the workspace layout helpers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ivs_hostcore.h"
#include "ivs_tab.cuh"

namespace ivs {
namespace host {

// fixed per-thread buffer: recording an error allocates nothing
thread_local char g_last_error[512];

void set_error_text(const char *msg) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg ? msg : "");
}

int fail(int status, const std::string &msg) {
    set_error_text(msg.c_str());
    return status;
}



// ---- outward rounding on the host (exact, from an error-free product) --------------
// p = RN(c * a); e = fma(c, a, -p) is the exact error (Dekker/Ogita-Rump-Oishi
// TwoProduct), so the rounded-down product is p when e >= 0 and the next double below p
// otherwise; symmetric for rounding up.
double mul_down(double c, double a) {
    double p = c * a;
    double e = std::fma(c, a, -p);
    return e < 0 ? std::nextafter(p, -INFINITY) : p;
}
double mul_up(double c, double a) {
    double p = c * a;
    double e = std::fma(c, a, -p);
    return e > 0 ? std::nextafter(p, INFINITY) : p;
}
float to_float_down(double d) {
    float f = (float)d;
    if ((double)f > d) f = std::nextafter(f, -INFINITY);
    return f;
}
float to_float_up(double d) {
    float f = (float)d;
    if ((double)f < d) f = std::nextafter(f, INFINITY);
    return f;
}

// One system's polynomials before packing into a blob (local indices).
struct SysBuild {
    std::vector<int32_t> poly_off{0};
    std::vector<double> clo, chi;
    std::vector<uint32_t> tinfo;
    std::vector<uint8_t> fac;
};



void add_term(SysBuild &b, double clo, double chi, const uint8_t *e, int n) {
    b.clo.push_back(clo);
    b.chi.push_back(chi);
    const uint32_t start = (uint32_t)b.fac.size();
    uint32_t cnt = 0;
    for (int j = 0; j < n; j++)
        if (e[j]) {
            b.fac.push_back((uint8_t)((j << 4) | e[j]));
            cnt++;
        }
    b.tinfo.push_back(term_info(start, cnt, clo, chi));
}

// packs a built system into the blob arena and fills the blob fields of d
// Per-parent table of the FP32 stage: for each term of the equations, one entry per
// combination of its variables' halves (2^factors entries), when the total stays small.
constexpr int kMaxTermCombos = 2048;

void pack_blob(HostTables &h, const SysBuild &b, DevSys &d, int n_fterms) {
    const int T = (int)b.clo.size(), P = (int)b.poly_off.size() - 1, F = (int)b.fac.size();
    std::vector<int32_t> tv_off{0};
    std::vector<uint32_t> tv_map;
    bool tv_ok = true;
    for (int t = 0; t < n_fterms && tv_ok; t++) {
        const int nf = term_nf(b.tinfo[t]);
        if (nf > 8 || tv_off.back() + (1 << nf) > kMaxTermCombos) { tv_ok = false; break; }
        for (int q = 0; q < (1 << nf); q++) tv_map.push_back(((uint32_t)t << 8) | (uint32_t)q);
        tv_off.push_back(tv_off.back() + (1 << nf));
    }
    const int TF = tv_ok ? n_fterms : 0, E = tv_ok ? (int)tv_map.size() : 0;
    // child-index table: for each F term and each child c (n bits), its table entry
    // tv_off[t] + (c's bits in the term's variables); kept small (n <= 8, <= 16384 entries)
    std::vector<uint16_t> cix;
    if (TF > 0 && d.n <= 8 && (int64_t)TF << d.n <= 16384) {
        cix.resize((size_t)TF << d.n);
        for (int t = 0; t < TF; t++) {
            const int nf = term_nf(b.tinfo[t]), f0 = term_f0(b.tinfo[t]);
            for (int c = 0; c < (1 << d.n); c++) {
                unsigned q = 0;
                for (int f = 0; f < nf; f++) q |= ((unsigned)(c >> (b.fac[f0 + f] >> 4)) & 1u) << f;
                cix[((size_t)t << d.n) + c] = (uint16_t)(tv_off[t] + (int)q);
            }
        }
    }
    const int CX = (int)cix.size();
    const BlobLayout L = blob_layout(T, P, F, TF, E, CX);
    const size_t off = h.blobs.size();
    h.blobs.resize(off + L.bytes, 0);
    char *base = h.blobs.data() + off;
    for (int t = 0; t < T; t++) {
        const float4 cs = make_float4(to_float_down(b.clo[t]), to_float_up(b.clo[t]), to_float_down(b.chi[t]),
                                      to_float_up(b.chi[t]));
        std::memcpy(base + L.cs + 16u * t, &cs, 16);
        const float c32[2] = {to_float_down(b.clo[t]), to_float_up(b.chi[t])};
        std::memcpy(base + L.clo32 + 4u * t, &c32[0], 4);
        std::memcpy(base + L.chi32 + 4u * t, &c32[1], 4);
    }
    if (T) {
        std::memcpy(base + L.clo, b.clo.data(), 8u * T);
        std::memcpy(base + L.chi, b.chi.data(), 8u * T);
        std::memcpy(base + L.tinfo, b.tinfo.data(), 4u * T);
    }
    std::memcpy(base + L.poly_off, b.poly_off.data(), 4u * (P + 1));
    if (TF) {
        std::memcpy(base + L.tv_off, tv_off.data(), 4u * (TF + 1));
        std::memcpy(base + L.tv_map, tv_map.data(), 4u * E);
    }
    if (CX) std::memcpy(base + L.cix, cix.data(), 2u * CX);
    if (F) std::memcpy(base + L.fac, b.fac.data(), (size_t)F);
    d.blob_off = (int64_t)off;
    d.n_terms = T;
    d.n_polys = P;
    d.n_facs = F;
    d.n_fterms = TF;
    d.n_tv = E;
    d.n_cix = CX;
    d.blob_bytes = (int32_t)L.bytes;
}

int validate(const ivs_system *s, const double *lo, const double *hi, const ivs_options *o) {
    if (!s || !lo || !hi || !o) return fail(IVS_ERR_INVALID, "null argument");
    if (s->n_vars <= 0 || s->n_vars > kMaxVars) return fail(IVS_ERR_INVALID, "n_vars must be in 1..16");
    if (s->n_eqs <= 0 || s->n_terms < 0) return fail(IVS_ERR_INVALID, "n_eqs must be >= 1, n_terms >= 0");
    if (!s->eq_offsets || (s->n_terms > 0 && (!s->coef_lo || !s->exps)))
        return fail(IVS_ERR_INVALID, "null system array");
    if (s->eq_offsets[0] != 0 || s->eq_offsets[s->n_eqs] != s->n_terms)
        return fail(IVS_ERR_INVALID, "eq_offsets must run from 0 to n_terms");
    for (int i = 0; i < s->n_eqs; i++)
        if (s->eq_offsets[i + 1] < s->eq_offsets[i]) return fail(IVS_ERR_INVALID, "eq_offsets not monotone");
    for (int t = 0; t < s->n_terms; t++) {
        double a = s->coef_lo[t], b = s->coef_hi ? s->coef_hi[t] : a;
        if (!std::isfinite(a) || !std::isfinite(b) || a > b) return fail(IVS_ERR_INVALID, "bad coefficient");
        for (int j = 0; j < s->n_vars; j++)
            if (s->exps[(size_t)t * s->n_vars + j] > kMaxExp) return fail(IVS_ERR_INVALID, "exponent > 15");
    }
    for (int j = 0; j < s->n_vars; j++)
        if (!std::isfinite(lo[j]) || !std::isfinite(hi[j]) || lo[j] > hi[j])
            return fail(IVS_ERR_INVALID, "bad initial box");
    if (o->hs_enable && s->n_eqs != s->n_vars) return fail(IVS_ERR_INVALID, "HS needs n_eqs == n_vars");
    if (o->centred_form && s->n_eqs != s->n_vars)
        return fail(IVS_ERR_INVALID, "the centred form needs n_eqs == n_vars");
    if (!(o->tol >= 0) || !std::isfinite(o->tol)) return fail(IVS_ERR_INVALID, "tol must be finite and >= 0");
    if (o->hs_iters < 0 || o->max_depth < 0 || o->max_depth > 0xFFF0 || o->root_depth < 0 ||
        o->root_depth > o->max_depth)
        return fail(IVS_ERR_INVALID, "bad depth / iteration options");
    if (o->split_mode < 0 || o->split_mode > 1 || o->gap_split < 0 || o->gap_split > 1)
        return fail(IVS_ERR_INVALID, "split_mode must be 0 or 1, gap_split 0 or 1");
    return IVS_OK;
}

// F_i and J_ij polynomials of one system appended to the tables.  J_ij = sum over terms t
// of equation i with a_tj > 0 of [down(c_lo a_tj), up(c_hi a_tj)] x^(a_t - e_j), in term
// order; its factors keep the variable order of the term.
// The FP32 shadow may decide boxes only when no FP32 intermediate can overflow: every
// term's magnitude over the initial box, times the number of terms, stays below 1e30
// (float max ~3.4e38).  Otherwise the plain FP32 prefilter (sound under overflow) runs.
bool shadow_safe(const ivs_system *s, const double *lo, const double *hi) {
    const int n = s->n_vars;
    for (int i = 0; i < s->n_eqs; i++) {
        const int nt = s->eq_offsets[i + 1] - s->eq_offsets[i];
        for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
            double c = std::max(std::fabs(s->coef_lo[t]), std::fabs(s->coef_hi ? s->coef_hi[t] : s->coef_lo[t]));
            double b = c;
            for (int j = 0; j < n; j++) {
                const int a = s->exps[(size_t)t * n + j];
                const double m = std::max(std::fabs(lo[j]), std::fabs(hi[j]));
                for (int q = 0; q < a; q++) b *= std::max(m, 1.0);
            }
            if (!(b * (nt + 1) < 1e30)) return false;
        }
    }
    return true;
}

void compile_system(HostTables &h, const ivs_system *s, const ivs_options *o) {
    const int n = s->n_vars, m = s->n_eqs;
    SysBuild bld;
    DevSys d{};
    d.n = n;
    d.m = m;
    d.f_poly = 0;
    for (int i = 0; i < m; i++) {
        for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
            double clo = s->coef_lo[t], chi = s->coef_hi ? s->coef_hi[t] : clo;
            add_term(bld, clo, chi, s->exps + (size_t)t * n, n);
        }
        bld.poly_off.push_back((int32_t)bld.clo.size());
    }
    d.j_poly = -1;
    if (m == n) {
        d.j_poly = m;
        uint8_t e[kMaxVars];
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) {
                for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
                    const uint8_t *a = s->exps + (size_t)t * n;
                    if (a[j] == 0) continue;
                    double clo = s->coef_lo[t], chi = s->coef_hi ? s->coef_hi[t] : clo;
                    std::memcpy(e, a, (size_t)n);
                    e[j] -= 1;
                    add_term(bld, mul_down(clo, (double)a[j]), mul_up(chi, (double)a[j]), e, n);
                }
                bld.poly_off.push_back((int32_t)bld.clo.size());
            }
    }
    d.tol = o->tol + 0.0;   // -0 -> +0
    d.hs_enable = o->hs_enable ? 1 : 0;
    d.hs_min_depth = o->hs_min_depth;
    d.hs_iters = o->hs_iters > 0 ? o->hs_iters : 1;
    d.max_depth = o->max_depth;
    d.prefilter = o->prefilter_fp32 ? 1 : 0;
    d.shadow = 0;
    d.max_boxes = o->max_boxes;
    d.centred = o->centred_form ? 1 : 0;
    d.krawczyk = o->krawczyk ? 1 : 0;
    d.bisect = o->split_mode == 1 ? 1 : 0;
    d.gap_split = o->gap_split ? 1 : 0;
    pack_blob(h, bld, d, bld.poly_off[m]);
    h.sys.push_back(d);
}

const char *last_error() { return g_last_error; }


size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }



Layout layout_for(int n_sys, int n_max, int64_t W, int64_t Q, int64_t O) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.queue = take((size_t)Q * (3 * n_max * sizeof(double) + 2 * sizeof(int32_t)) + 4 * 256);
    L.stage = take((size_t)W * (3 * n_max * sizeof(double) + 2 * sizeof(int32_t)) + 4 * 256);
    L.surv = take((size_t)(n_max + 2) * W * sizeof(Surv));
    L.out = take((size_t)O * (2 * n_max * sizeof(double) + 3 * sizeof(int32_t)) + 4 * 256);
    L.ctl = take(sizeof(WaveCtl));
    L.stats = take((size_t)n_sys * ST_COUNT * sizeof(unsigned long long));
    L.roots = take((size_t)n_sys * (2 * n_max * sizeof(double) + sizeof(int32_t)) + 2 * 256);
    L.total = off;
    return L;
}

DevQueue carve_queue(char *base, int64_t cap, int n_max) {
    DevQueue q{};
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = base + off; off = align_up(off + bytes, 256); return p; };
    q.lo = (double *)take((size_t)cap * n_max * sizeof(double));
    q.mid = (double *)take((size_t)cap * n_max * sizeof(double));
    q.hi = (double *)take((size_t)cap * n_max * sizeof(double));
    q.sys = (int32_t *)take((size_t)cap * sizeof(int32_t));
    q.meta = (uint32_t *)take((size_t)cap * sizeof(uint32_t));
    q.cap = cap;
    return q;
}

DevOut carve_out(char *base, int64_t cap, int n_max) {
    DevOut o{};
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = base + off; off = align_up(off + bytes, 256); return p; };
    o.lo = (double *)take((size_t)cap * n_max * sizeof(double));
    o.hi = (double *)take((size_t)cap * n_max * sizeof(double));
    o.sys = (int32_t *)take((size_t)cap * sizeof(int32_t));
    o.flags = (int32_t *)take((size_t)cap * sizeof(int32_t));
    o.depth = (int32_t *)take((size_t)cap * sizeof(int32_t));
    o.cap = cap;
    return o;
}


void fill_sorted(ivs_result *r, int n, int64_t total, const std::vector<double> &lo, const std::vector<double> &hi,
                 const std::vector<int32_t> &flags, const std::vector<int32_t> &depth) {
    r->n = n;
    std::vector<int64_t> idx((size_t)total);
    for (int64_t k = 0; k < total; k++) idx[(size_t)k] = k;
    auto key = [&](int64_t k, int j, bool upper) {
        double v = (upper ? hi : lo)[(size_t)j * total + k];
        return v == 0 ? 0.0 : v;
    };
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
        for (int j = 0; j < n; j++) {
            double x = key(a, j, false), y = key(b, j, false);
            if (x != y) return x < y;
            x = key(a, j, true);
            y = key(b, j, true);
            if (x != y) return x < y;
        }
        return false;
    });
    r->lo.resize(idx.size() * n);
    r->hi.resize(idx.size() * n);
    r->flags.resize(idx.size());
    r->depth.resize(idx.size());
    for (size_t q = 0; q < idx.size(); q++) {
        for (int j = 0; j < n; j++) {
            r->lo[q * n + j] = key(idx[q], j, false);
            r->hi[q * n + j] = key(idx[q], j, true);
        }
        r->flags[q] = flags[idx[q]];
        r->depth[q] = depth[idx[q]];
    }
}

}  // namespace host
}  // namespace ivs
