// ivs_noalloc.cu -- a solve entry point that allocates nothing.
//
// Some callers cannot allocate device memory: processes whose device memory belongs to a
// pool they must not bypass (a framework's caching allocator, or a serving engine that
// reserved the GPU's memory up front), plug-ins and callbacks that run inside another
// runtime which forbids allocation, and real-time loops that cannot afford cudaMalloc's
// implicit synchronisation.  ivs_solve_noalloc serves them: it runs the same sweep
// kernels as ivs_solve, but every byte of device scratch (tables, queue, staging,
// survivor lists, result list, counters) comes from one file-scope __device__ array of
// IVS_NOALLOC_SCRATCH_BYTES, and the host side uses fixed static buffers and the stack.
// It calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.  The
// array exists on every GPU that loads the library, until the process exits.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ivsolve.h"
#include "ivs_hostcore.h"
#include "ivs_internal.h"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

namespace ivs {
namespace {

constexpr size_t kScratch = IVS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kNoallocMaxVars = 12;
constexpr uint32_t kMaxBlob = 48 * 1024;
constexpr int kMaxTerms = 2048;

// The scratch every call shares.  In host code `g_scratch` names a host-side stand-in,
// not a device address: kernels receive the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_scratch[kScratch];

std::mutex g_mu;                        // serialises host-side set-up and the static buffers
void *g_scratch_addr[kMaxDevices] = {};
alignas(16) char g_host_blob[kMaxBlob]; // compiled term table staged on the host
WaveCtl g_ctl;                          // host copy of the sweep control block
char *g_errbuf = nullptr;               // the current call's message buffer (caller's)
int32_t g_errlen = 0;

// the message goes to the caller's buffer and to the thread's ivs_last_error() text
int err(int status, const char *msg) {
    if (g_errbuf && g_errlen > 0) std::snprintf(g_errbuf, (size_t)g_errlen, "%s", msg);
    host::set_error_text(msg);
    return status;
}
int err_cuda(const char *what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return err(IVS_ERR_CUDA, msg);
}

// exact outward products and float conversions (error-free product: Dekker's TwoProduct)
double down_mul(double c, double a) { const double p = c * a, e = std::fma(c, a, -p); return e < 0 ? std::nextafter(p, -INFINITY) : p; }
double up_mul(double c, double a) { const double p = c * a, e = std::fma(c, a, -p); return e > 0 ? std::nextafter(p, INFINITY) : p; }
float f_down(double d) { float f = (float)d; if ((double)f > d) f = std::nextafter(f, -INFINITY); return f; }
float f_up(double d) { float f = (float)d; if ((double)f < d) f = std::nextafter(f, INFINITY); return f; }

// Terms of the system (F_i, then J_ij) in the order the blob stores them; `emit` receives
// (coef_lo, coef_hi, exponent vector) per term and `close` ends a polynomial.
template <class Emit, class Close>
void walk_terms(const ivs_system *s, Emit emit, Close close) {
    const int n = s->n_vars, m = s->n_eqs;
    uint8_t e[kMaxVars];
    for (int i = 0; i < m; i++) {
        for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
            const double clo = s->coef_lo[t], chi = s->coef_hi ? s->coef_hi[t] : clo;
            emit(clo, chi, s->exps + (size_t)t * n);
        }
        close();
    }
    if (m != n) return;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            for (int t = s->eq_offsets[i]; t < s->eq_offsets[i + 1]; t++) {
                const uint8_t *a = s->exps + (size_t)t * n;
                if (a[j] == 0) continue;
                const double clo = s->coef_lo[t], chi = s->coef_hi ? s->coef_hi[t] : clo;
                std::memcpy(e, a, (size_t)n);
                e[j] -= 1;
                emit(down_mul(clo, (double)a[j]), up_mul(chi, (double)a[j]), e);
            }
            close();
        }
}

// Packs the system into g_host_blob (layout of ivs_tab.cuh); false if it does not fit.
bool pack_static(const ivs_system *s, DevSys &d) {
    const int n = s->n_vars;
    int T = 0, P = 0, F = 0;
    walk_terms(s, [&](double, double, const uint8_t *e) {
        T++;
        for (int j = 0; j < n; j++) F += e[j] ? 1 : 0;
    }, [&]() { P++; });
    if (T > kMaxTerms) return false;
    const BlobLayout L = blob_layout(T, P, F);
    if (L.bytes > kMaxBlob) return false;
    std::memset(g_host_blob, 0, L.bytes);
    int t = 0, p = 0, f = 0;
    int32_t *poly_off = reinterpret_cast<int32_t *>(g_host_blob + L.poly_off);
    poly_off[0] = 0;
    walk_terms(s, [&](double clo, double chi, const uint8_t *e) {
        const float4 cs = make_float4(f_down(clo), f_up(clo), f_down(chi), f_up(chi));
        std::memcpy(g_host_blob + L.cs + 16u * t, &cs, 16);
        std::memcpy(g_host_blob + L.clo + 8u * t, &clo, 8);
        std::memcpy(g_host_blob + L.chi + 8u * t, &chi, 8);
        const float c32lo = f_down(clo), c32hi = f_up(chi);
        std::memcpy(g_host_blob + L.clo32 + 4u * t, &c32lo, 4);
        std::memcpy(g_host_blob + L.chi32 + 4u * t, &c32hi, 4);
        const uint32_t start = (uint32_t)f;
        uint32_t cnt = 0;
        for (int j = 0; j < n; j++)
            if (e[j]) {
                reinterpret_cast<uint8_t *>(g_host_blob)[L.fac + f] = (uint8_t)((j << 4) | e[j]);
                f++;
                cnt++;
            }
        const uint32_t info = term_info(start, cnt, clo, chi);
        std::memcpy(g_host_blob + L.tinfo + 4u * t, &info, 4);
        t++;
    }, [&]() { poly_off[++p] = t; });
    d.n_terms = T;
    d.n_polys = P;
    d.n_facs = F;
    d.n_fterms = 0;   // no per-parent combination table (the evaluation takes the direct path)
    d.n_tv = 0;
    d.blob_bytes = (int32_t)L.bytes;
    return true;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// lexicographic order of rows (lo_0, hi_0, lo_1, hi_1, ...)
bool row_less(const double *lo, const double *hi, int n, int64_t a, int64_t b) {
    for (int j = 0; j < n; j++) {
        if (lo[a * n + j] != lo[b * n + j]) return lo[a * n + j] < lo[b * n + j];
        if (hi[a * n + j] != hi[b * n + j]) return hi[a * n + j] < hi[b * n + j];
    }
    return false;
}
void row_swap(double *lo, double *hi, int32_t *fl, int n, int64_t a, int64_t b) {
    for (int j = 0; j < n; j++) {
        std::swap(lo[a * n + j], lo[b * n + j]);
        std::swap(hi[a * n + j], hi[b * n + j]);
    }
    if (fl) std::swap(fl[a], fl[b]);
}
// in-place heap sort of the caller's rows (no extra memory)
void sort_rows(double *lo, double *hi, int32_t *fl, int n, int64_t cnt) {
    auto sift = [&](int64_t root, int64_t end) {
        for (;;) {
            int64_t c = 2 * root + 1;
            if (c >= end) return;
            if (c + 1 < end && row_less(lo, hi, n, c, c + 1)) c++;
            if (!row_less(lo, hi, n, root, c)) return;
            row_swap(lo, hi, fl, n, root, c);
            root = c;
        }
    };
    for (int64_t i = cnt / 2 - 1; i >= 0; i--) sift(i, cnt);
    for (int64_t end = cnt - 1; end > 0; end--) {
        row_swap(lo, hi, fl, n, 0, end);
        sift(0, end);
    }
}

// the result list (structure of arrays in scratch) to row-major rows in scratch
__global__ void k_rows(DevOut o, int64_t count, int n, double *lo, double *hi, int32_t *flags) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < n; j++) {
            const double a = o.lo[j * o.cap + k], b = o.hi[j * o.cap + k];
            lo[k * n + j] = a == 0 ? 0.0 : a;   // -0 -> +0
            hi[k * n + j] = b == 0 ? 0.0 : b;
        }
        flags[k] = o.flags[k];
    }
}

}  // namespace
}  // namespace ivs

using namespace ivs;

extern "C" int ivs_solve_noalloc(const ivs_system *s, const double *box_lo, const double *box_hi,
                                 const ivs_options *o, void *stream_ptr, double *out_lo, double *out_hi,
                                 int32_t *out_flags, int64_t out_cap, int64_t *out_count, ivs_stats *stats,
                                 char *errbuf, int32_t errbuf_len) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_errbuf = errbuf;
    g_errlen = errbuf_len;
    if (errbuf && errbuf_len > 0) errbuf[0] = 0;
    if (out_count) *out_count = 0;
    if (!s || !box_lo || !box_hi || !o || !out_count || out_cap < 0 || (out_cap > 0 && (!out_lo || !out_hi)))
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: null or negative argument");
    const int n = s->n_vars, m = s->n_eqs;
    if (n <= 0 || n > kNoallocMaxVars)
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: n_vars must be in 1..12 (fixed scratch)");
    if (m <= 0 || s->n_terms < 0 || !s->eq_offsets || (s->n_terms > 0 && (!s->coef_lo || !s->exps)) ||
        s->eq_offsets[0] != 0 || s->eq_offsets[m] != s->n_terms)
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: malformed system");
    for (int i = 0; i < m; i++)
        if (s->eq_offsets[i + 1] < s->eq_offsets[i]) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: malformed system");
    for (int t = 0; t < s->n_terms; t++) {
        const double a = s->coef_lo[t], b = s->coef_hi ? s->coef_hi[t] : a;
        if (!std::isfinite(a) || !std::isfinite(b) || a > b) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: bad coefficient");
        for (int j = 0; j < n; j++)
            if (s->exps[(size_t)t * n + j] > kMaxExp) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: exponent > 15");
    }
    for (int j = 0; j < n; j++)
        if (!std::isfinite(box_lo[j]) || !std::isfinite(box_hi[j]) || box_lo[j] > box_hi[j])
            return err(IVS_ERR_INVALID, "ivs_solve_noalloc: bad initial box");
    if (o->hs_enable && m != n) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: HS needs n_eqs == n_vars");
    if (o->centred_form && m != n)
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: the centred form needs n_eqs == n_vars");
    if (!(o->tol >= 0) || !std::isfinite(o->tol) || o->hs_iters < 0 || o->max_depth < 0 || o->max_depth > 0xFFF0 ||
        o->root_depth < 0 || o->root_depth > o->max_depth || o->split_mode < 0 || o->split_mode > 1 ||
        o->gap_split < 0 || o->gap_split > 1)
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: bad options");

    DevSys d{};
    if (!pack_static(s, d))
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: term table exceeds the fixed 48 KiB table buffer");
    d.n = n;
    d.m = m;
    d.f_poly = 0;
    d.j_poly = m == n ? m : -1;
    d.tol = o->tol + 0.0;
    d.hs_enable = o->hs_enable ? 1 : 0;
    d.hs_min_depth = o->hs_min_depth;
    d.hs_iters = o->hs_iters > 0 ? o->hs_iters : 1;
    d.max_depth = o->max_depth;
    d.prefilter = o->prefilter_fp32 ? 1 : 0;
    d.shadow = 0;   // plain FP32 prefilter: sound whatever the magnitudes
    d.max_boxes = o->max_boxes;
    d.centred = o->centred_form ? 1 : 0;
    d.krawczyk = o->krawczyk ? 1 : 0;
    d.bisect = o->split_mode == 1 ? 1 : 0;
    d.gap_split = o->gap_split ? 1 : 0;

    // ---- set-up, once per device (with that device current) ----
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return err_cuda("cudaGetDevice", ce);
    if (dev < 0 || dev >= kMaxDevices) return err(IVS_ERR_CUDA, "ivs_solve_noalloc: device ordinal too large");
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        ce = cudaGetSymbolAddress(&ptr, g_scratch);
        if (ce != cudaSuccess || !ptr) return err_cuda("cudaGetSymbolAddress(scratch)", ce);
        g_scratch_addr[dev] = ptr;
    }
    char *base = (char *)g_scratch_addr[dev];
    cudaStream_t st = (cudaStream_t)stream_ptr;
    // the loop below waits on the stream between sweeps and copies into pageable host
    // memory, which a stream in capture mode does not allow
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ce = cudaStreamIsCapturing(st, &cap);
    if (ce != cudaSuccess) return err_cuda("cudaStreamIsCapturing", ce);
    if (cap != cudaStreamCaptureStatusNone)
        return err(IVS_ERR_INVALID, "ivs_solve_noalloc: the stream is in capture mode (the call synchronises it)");
    int sms = 0;
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return err_cuda("cudaDeviceGetAttribute", ce);

    // ---- carve the fixed scratch ----
    const int64_t W = std::max<int64_t>((int64_t)1 << 15, (int64_t)1 << n);      // children per sweep
    const int64_t O = std::min<int64_t>(std::max<int64_t>(out_cap, 1), (int64_t)1 << 14);   // results held
    const size_t per_parent = (size_t)3 * n * 8 + 8;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = up256(off + bytes); return base + at; };
    DevSys *d_sys = (DevSys *)take(sizeof(DevSys));
    char *d_blob = take((size_t)d.blob_bytes);
    double *d_lo = (double *)take((size_t)n * 8);
    double *d_hi = (double *)take((size_t)n * 8);
    int32_t *d_depth = (int32_t *)take(4);
    WaveCtl *d_ctl = (WaveCtl *)take(sizeof(WaveCtl));
    unsigned long long *d_stats = (unsigned long long *)take((size_t)ST_COUNT * 8);
    SweepArgs a{};
    auto carve_q = [&](int64_t cap) {
        DevQueue q{};
        q.lo = (double *)take((size_t)cap * n * 8);
        q.mid = (double *)take((size_t)cap * n * 8);
        q.hi = (double *)take((size_t)cap * n * 8);
        q.sys = (int32_t *)take((size_t)cap * 4);
        q.meta = (uint32_t *)take((size_t)cap * 4);
        q.cap = cap;
        return q;
    };
    a.stage = carve_q(W);
    a.surv = (Surv *)take((size_t)(n + 2) * W * sizeof(Surv));
    a.cand = a.surv + (size_t)(n + 1) * W;
    a.out.lo = (double *)take((size_t)O * n * 8);
    a.out.hi = (double *)take((size_t)O * n * 8);
    a.out.sys = (int32_t *)take((size_t)O * 4);
    a.out.flags = (int32_t *)take((size_t)O * 4);
    a.out.depth = (int32_t *)take((size_t)O * 4);
    a.out.cap = O;
    double *d_rows_lo = (double *)take((size_t)O * n * 8);
    double *d_rows_hi = (double *)take((size_t)O * n * 8);
    int32_t *d_rows_fl = (int32_t *)take((size_t)O * 4);
    const size_t q_overhead = 5 * 256;
    if (off + q_overhead >= kScratch) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: fixed scratch too small for this system");
    const int64_t Q = (int64_t)((kScratch - off - q_overhead) / per_parent);
    if (Q < 4 * W) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: fixed scratch too small for this system's queue");
    a.q = carve_q(Q);
    if (off > kScratch) return err(IVS_ERR_INVALID, "ivs_solve_noalloc: fixed scratch overflow");
    d.blob_off = 0;   // the blob arena starts at d_blob
    d.out_base = 0;
    d.out_cap = O;
    a.tb.sys = d_sys;
    a.tb.blobs = d_blob;
    a.ctl = d_ctl;
    a.stats = d_stats;
    a.surv_cap = W;
    a.wave_children = W;
    a.max_fan_shift = n;
    a.n_sys = 1;
    a.single = 1;
    a.blob_smem = d.blob_bytes;

    // ---- upload (pageable copies from static host buffers; no allocation) ----
    const int32_t rd = o->root_depth;
#define NA_TRY(x)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) return err_cuda(#x, e_);                                   \
    } while (0)
    NA_TRY(cudaMemcpyAsync(d_sys, &d, sizeof(DevSys), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_blob, g_host_blob, (size_t)d.blob_bytes, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_lo, box_lo, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_hi, box_hi, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_depth, &rd, 4, cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: clear what must start at zero
    NA_TRY(cudaMemsetAsync(d_stats, 0, (size_t)ST_COUNT * 8, st));
    choose_eval_layout(a, 0);
    NA_TRY(configure_eval_kernels(a));
    NA_TRY(launch_seed_roots(a, d_lo, d_hi, d_depth, 1, n, st));   // also resets the control block

    // ---- sweep loop (host-driven: a graph would have to be instantiated, which allocates) ----
    const int dims[1] = {n};
    int status = IVS_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        NA_TRY(launch_sweep(a, dims, 1, sms * 8, 256, sms, st, nullptr));
        NA_TRY(cudaMemcpyAsync(&g_ctl, d_ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaStreamSynchronize(st));
        if (g_ctl.error) { status = IVS_ERR_NOMEM; break; }
        if (g_ctl.top == 0) break;
        if (o->time_budget_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->time_budget_s) {
            status = IVS_ERR_TIMEOUT;
            break;
        }
    }
    unsigned long long hs[ST_COUNT];
    NA_TRY(cudaMemcpyAsync(hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    const int64_t produced = (int64_t)hs[ST_OUT];
    const int64_t held = std::min<int64_t>(produced, O);
    const int64_t give = std::min<int64_t>(held, out_cap);
    if (give > 0) {
        k_rows<<<(int)std::min<int64_t>((give + 255) / 256, 1024), 256, 0, st>>>(a.out, give, n, d_rows_lo, d_rows_hi, d_rows_fl);
        NA_TRY(cudaGetLastError());
        NA_TRY(cudaMemcpyAsync(out_lo, d_rows_lo, (size_t)give * n * 8, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaMemcpyAsync(out_hi, d_rows_hi, (size_t)give * n * 8, cudaMemcpyDeviceToHost, st));
        if (out_flags) NA_TRY(cudaMemcpyAsync(out_flags, d_rows_fl, (size_t)give * 4, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaStreamSynchronize(st));
        sort_rows(out_lo, out_hi, out_flags, n, give);
    }
#undef NA_TRY
    *out_count = give;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->boxes = (int64_t)hs[ST_BOXES];
        stats->excluded_prefilter = (int64_t)hs[ST_EXCL_PREFILTER];
        stats->excluded_eval = (int64_t)hs[ST_EXCL_EVAL];
        stats->excluded_centred = (int64_t)hs[ST_EXCL_CENTRED];
        stats->gap_splits = (int64_t)hs[ST_GAP_SPLITS];
        stats->hs_applied = (int64_t)hs[ST_HS_APPLIED];
        stats->hs_empty = (int64_t)hs[ST_HS_EMPTY];
        stats->hs_contracted = (int64_t)hs[ST_HS_CONTRACTED];
        stats->hs_singular = (int64_t)hs[ST_HS_SINGULAR];
        stats->accepted = (int64_t)hs[ST_ACCEPTED];
        stats->unsplittable = (int64_t)hs[ST_UNSPLITTABLE];
        stats->split = (int64_t)hs[ST_SPLIT];
        stats->max_depth_seen = (int32_t)hs[ST_MAX_DEPTH];
        stats->waves = (int32_t)g_ctl.waves;
        stats->eval64_boxes = (int64_t)hs[ST_EVAL64];
        stats->kept_shadow = (int64_t)hs[ST_KEEP_SHADOW];
    }
    if (status == IVS_OK && (hs[ST_FLAGS] != 0 || produced > give)) status = IVS_ERR_BUDGET;
    if (status == IVS_ERR_NOMEM) err(status, "ivs_solve_noalloc: the fixed queue filled up");
    if (status == IVS_ERR_TIMEOUT) err(status, "ivs_solve_noalloc: time budget exhausted");
    return status;
}
