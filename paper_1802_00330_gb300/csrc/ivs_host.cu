// ivs_host.cu -- host runtime behind include/ivsolve.h: input validation, compilation of
// each system into device tables (F and its Jacobian), the device workspace, the sweep
// loop over the device queue, and result collection.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ivsolve.h"
#include "ivs_internal.h"
#include "ivs_hostcore.h"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

using namespace ivs;
using namespace ivs::host;

namespace {
template <class T>
int upload(void *&cursor, const std::vector<T> &v, const T *&dst, cudaStream_t st) {
    dst = reinterpret_cast<const T *>(cursor);
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(cursor, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    cursor = (char *)cursor + align_up(std::max<size_t>(v.size() * sizeof(T), 1), 256);
    return IVS_OK;
}

const ivs_options *opt_at(const ivs_options *opts, int32_t stride, int s) {
    return stride == 0 ? opts : (const ivs_options *)((const char *)opts + (size_t)stride * s);
}
}  // namespace




struct ivs_plan {
    int n_sys = 0, n_max = 0, device = 0, num_sms = 0;
    int eval_blocks = 0, eval_threads = 256;
    std::vector<int> dims;                 // distinct n over systems (HS kernels to launch)
    std::vector<ivs_options> opts;
    std::vector<int> sys_n;
    std::vector<int64_t> sys_out_base, sys_out_cap;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *ws = nullptr;
    bool own_ws = false;
    size_t ws_bytes = 0;
    void *tables_mem = nullptr;
    size_t tables_bytes = 0;
    SweepArgs args{};
    int64_t wave_children = 0, queue_cap = 0, out_cap = 0;
    double *d_box_lo = nullptr, *d_box_hi = nullptr;
    int32_t *d_root_depth = nullptr;
    WaveCtl *h_ctl = nullptr;              // pinned
    std::vector<unsigned long long> h_stats;
    int run_status = IVS_OK;
    float last_ms = 0.f;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double time_budget_s = 0;
    int64_t launches = 0;
    // profiling: stage events of one sweep and accumulated times per kernel class
    bool profile = false;
    std::vector<cudaEvent_t> stage_ev;
    std::vector<double> class_ms;          // [0] eval, [1] control, [2] eval64, [3 + q] hs dim q
    std::vector<int64_t> class_launches;
    // graph path: the whole sweep loop as one conditional-WHILE graph
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_kernels = 0;                 // kernels per sweep of the graph body
    int64_t *h_wave_limit = nullptr;       // pinned
    std::vector<double> box_lo_h, box_hi_h;   // initial boxes, n_max per system
};


extern "C" {

void ivs_options_default(ivs_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->hs_enable = 1;
    o->hs_min_depth = 0;
    o->hs_iters = 1;
    o->prefilter_fp32 = 1;
    o->root_depth = 0;
    o->max_depth = 200;
    o->max_boxes = 0;
    o->max_results = 0;
    o->time_budget_s = 0;
}

const char *ivs_status_str(int s) {
    switch (s) {
    case IVS_OK: return "ok";
    case IVS_ERR_INVALID: return "invalid argument";
    case IVS_ERR_NOMEM: return "out of memory";
    case IVS_ERR_BUDGET: return "budget exhausted (result incomplete)";
    case IVS_ERR_TIMEOUT: return "time budget exhausted (result incomplete)";
    case IVS_ERR_CUDA: return "CUDA error";
    default: return "unknown status";
    }
}

const char *ivs_last_error(void) { return ivs::host::last_error(); }

size_t ivs_workspace_bytes(int32_t n_sys, const ivs_system *systems, int64_t W, int64_t Q, int64_t O) {
    int n_max = 1;
    for (int s = 0; s < n_sys; s++) n_max = std::max(n_max, (int)systems[s].n_vars);
    return layout_for(n_sys, n_max, W, Q, O).total;
}

void ivs_plan_destroy(ivs_plan *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->own_ws && p->ws) cudaFree(p->ws);
    if (p->tables_mem) cudaFree(p->tables_mem);
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (cudaEvent_t e : p->stage_ev) cudaEventDestroy(e);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->h_wave_limit) cudaFreeHost(p->h_wave_limit);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

}  // extern "C"

namespace {

bool same_args(const SweepArgs &x, const SweepArgs &y) {
    auto same_q = [](const DevQueue &a, const DevQueue &b) {
        return a.lo == b.lo && a.mid == b.mid && a.hi == b.hi && a.sys == b.sys && a.meta == b.meta && a.cap == b.cap;
    };
    return x.tb.sys == y.tb.sys && x.tb.blobs == y.tb.blobs && same_q(x.q, y.q) && same_q(x.stage, y.stage) &&
           x.out.lo == y.out.lo && x.out.hi == y.out.hi && x.out.sys == y.out.sys && x.out.flags == y.out.flags &&
           x.out.depth == y.out.depth && x.out.cap == y.out.cap && x.ctl == y.ctl && x.surv == y.surv &&
           x.surv_cap == y.surv_cap && x.cand == y.cand && x.stats == y.stats &&
           x.wave_children == y.wave_children && x.max_fan_shift == y.max_fan_shift && x.n_sys == y.n_sys &&
           x.single == y.single && x.blob_smem == y.blob_smem && x.tv_stride == y.tv_stride &&
           x.eval_warps == y.eval_warps && x.rg.n == y.rg.n;
}

// Builds a plan.  With `reuse` (a plan that is no longer needed) its stream, events,
// pinned buffers, device memory (when large enough) and instantiated graph (when the
// kernels' arguments come out the same) move into the new plan instead of being
// created again; the rest of `reuse` is freed.
int plan_create_impl(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                     const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                     const ivs_plan_cfg *cfg, ivs_plan *reuse, ivs_plan **out) {
    std::unique_ptr<ivs_plan, void (*)(ivs_plan *)> old(reuse, ivs_plan_destroy);
    if (!out) return fail(IVS_ERR_INVALID, "null out");
    *out = nullptr;
    if (n_sys <= 0 || !systems || !box_lo || !box_hi || !opts) return fail(IVS_ERR_INVALID, "bad arguments");
    ivs_plan_cfg c{};
    if (cfg) c = *cfg;
    std::unique_ptr<ivs_plan, void (*)(ivs_plan *)> p(new (std::nothrow) ivs_plan(), ivs_plan_destroy);
    if (!p) return fail(IVS_ERR_NOMEM, "host allocation");
    p->n_sys = n_sys;
    HostTables h;
    int64_t out_cap = 0;
    std::vector<double> roots_lo, roots_hi;
    std::vector<int32_t> root_depth;
    for (int s = 0; s < n_sys; s++) {
        const ivs_options *o = opt_at(opts, opts_stride, s);
        int rc = validate(&systems[s], box_lo[s], box_hi[s], o);
        if (rc) return fail(rc, "system " + std::to_string(s) + ": " + std::string(last_error()));
        p->n_max = std::max(p->n_max, (int)systems[s].n_vars);
        out_cap += o->max_results > 0 ? o->max_results : 0;
        p->opts.push_back(*o);
        p->sys_n.push_back(systems[s].n_vars);
        if (std::find(p->dims.begin(), p->dims.end(), systems[s].n_vars) == p->dims.end())
            p->dims.push_back(systems[s].n_vars);
        compile_system(h, &systems[s], o);
        (void)0;
        h.sys.back().shadow = (o->prefilter_fp32 && std::getenv("IVS_NO_SHADOW") == nullptr &&
                               shadow_safe(&systems[s], box_lo[s], box_hi[s])) ? 1 : 0;
        if (o->time_budget_s > 0)
            p->time_budget_s = p->time_budget_s > 0 ? std::min(p->time_budget_s, o->time_budget_s) : o->time_budget_s;
    }
    std::sort(p->dims.begin(), p->dims.end());
    for (int s = 0; s < n_sys; s++)
        for (int j = 0; j < p->n_max; j++) {
            p->box_lo_h.push_back(j < systems[s].n_vars ? box_lo[s][j] : 0.0);
            p->box_hi_h.push_back(j < systems[s].n_vars ? box_hi[s][j] : 0.0);
        }
    for (int s = 0; s < n_sys; s++) {
        for (int j = 0; j < p->n_max; j++) {
            bool in = j < systems[s].n_vars;
            roots_lo.push_back(in ? box_lo[s][j] : 0.0);
            roots_hi.push_back(in ? box_hi[s][j] : 0.0);
        }
        root_depth.push_back(opt_at(opts, opts_stride, s)->root_depth);
    }
    // each system owns a result region: max_results boxes, or a default
    out_cap = 0;
    for (int s = 0; s < n_sys; s++) {
        const ivs_options *o = opt_at(opts, opts_stride, s);
        const int64_t cap = o->max_results > 0 ? o->max_results : (n_sys == 1 ? ((int64_t)1 << 20) : ((int64_t)1 << 14));
        h.sys[s].out_base = out_cap;
        h.sys[s].out_cap = cap;
        out_cap += cap;
    }

    p->device = c.device;
    CUDA_TRY(cudaSetDevice(p->device));
    CUDA_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    ivs_plan *r = (old && old->device == p->device) ? old.get() : nullptr;
    if (r && r->stream) CUDA_TRY(cudaStreamSynchronize(r->stream));
    if (c.stream) {
        p->stream = (cudaStream_t)c.stream;
    } else if (r && r->own_stream) {
        std::swap(p->stream, r->stream);
        r->own_stream = false;
        p->own_stream = true;
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    if (r && r->ev0 && r->ev1) {
        std::swap(p->ev0, r->ev0);
        std::swap(p->ev1, r->ev1);
    } else {
        CUDA_TRY(cudaEventCreate(&p->ev0));
        CUDA_TRY(cudaEventCreate(&p->ev1));
    }
    if (r && r->h_ctl) std::swap(p->h_ctl, r->h_ctl);
    else CUDA_TRY(cudaMallocHost((void **)&p->h_ctl, sizeof(WaveCtl)));

    // workspace: wave size W, queue capacity Q, result capacity O
    const int64_t W = c.wave_children > 0 ? c.wave_children : (int64_t)1 << 22;
    int64_t Q;
    size_t fixed = layout_for(n_sys, p->n_max, W, 0, out_cap).total;
    const size_t per_parent = 3 * p->n_max * sizeof(double) + 2 * sizeof(int32_t);
    if (c.workspace) {
        if (c.workspace_bytes <= fixed + 64 * 1024) return fail(IVS_ERR_NOMEM, "workspace too small");
        Q = (int64_t)((c.workspace_bytes - fixed - 64 * 1024) / per_parent);
        p->ws = c.workspace;
    } else {
        size_t want = c.workspace_bytes > 0 ? c.workspace_bytes : fixed + per_parent * (size_t)(4 * W) + (1 << 20);
        Q = (int64_t)((want - fixed - 64 * 1024) / per_parent);
        if (Q < 16) return fail(IVS_ERR_NOMEM, "workspace too small");
        size_t total = layout_for(n_sys, p->n_max, W, Q, out_cap).total;
        if (r && r->own_ws && r->ws_bytes >= total) {
            std::swap(p->ws, r->ws);
            p->ws_bytes = r->ws_bytes;
            r->own_ws = false;
        } else {
            if (r && r->own_ws && r->ws) {   // too small: give it back before allocating
                cudaFree(r->ws);
                r->ws = nullptr;
                r->own_ws = false;
            }
            cudaError_t e = cudaMalloc(&p->ws, total);
            if (e != cudaSuccess) return fail(IVS_ERR_NOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
            p->ws_bytes = total;
        }
        p->own_ws = true;
    }
    if (Q < n_sys) return fail(IVS_ERR_NOMEM, "queue cannot hold the initial boxes");
    Layout L = layout_for(n_sys, p->n_max, W, Q, out_cap);
    char *ws = (char *)p->ws;
    SweepArgs &a = p->args;
    a.q = carve_queue(ws + L.queue, Q, p->n_max);
    a.stage = carve_queue(ws + L.stage, W, p->n_max);
    a.surv = (Surv *)(ws + L.surv);
    a.surv_cap = W;
    a.cand = a.surv + (size_t)(p->n_max + 1) * W;
    a.out = carve_out(ws + L.out, out_cap, p->n_max);
    a.ctl = (WaveCtl *)(ws + L.ctl);
    a.stats = (unsigned long long *)(ws + L.stats);
    a.wave_children = W;
    a.max_fan_shift = p->n_max;
    a.n_sys = n_sys;
    p->d_box_lo = (double *)(ws + L.roots);
    p->d_box_hi = p->d_box_lo + (size_t)n_sys * p->n_max;
    p->d_root_depth = (int32_t *)(p->d_box_hi + (size_t)n_sys * p->n_max);
    for (int s = 0; s < n_sys; s++) {
        p->sys_out_base.push_back(h.sys[s].out_base);
        p->sys_out_cap.push_back(h.sys[s].out_cap);
    }
    p->wave_children = W;
    p->queue_cap = Q;
    p->out_cap = out_cap;

    // tables: the DevSys array and the blob arena in one allocation
    const size_t sys_bytes = align_up(h.sys.size() * sizeof(DevSys), 256);
    const size_t tables_need = sys_bytes + std::max<size_t>(h.blobs.size(), 16);
    if (r && r->tables_mem && r->tables_bytes >= tables_need) {
        std::swap(p->tables_mem, r->tables_mem);
        p->tables_bytes = r->tables_bytes;
    } else {
        CUDA_TRY(cudaMalloc(&p->tables_mem, tables_need));
        p->tables_bytes = tables_need;
    }
    CUDA_TRY(cudaMemcpyAsync(p->tables_mem, h.sys.data(), h.sys.size() * sizeof(DevSys), cudaMemcpyHostToDevice,
                             p->stream));
    if (!h.blobs.empty())
        CUDA_TRY(cudaMemcpyAsync((char *)p->tables_mem + sys_bytes, h.blobs.data(), h.blobs.size(),
                                 cudaMemcpyHostToDevice, p->stream));
    a.tb.sys = (const DevSys *)p->tables_mem;
    a.tb.blobs = (const char *)p->tables_mem + sys_bytes;
    // one system: every kernel caches its blob in shared memory (if it fits)
    a.single = (n_sys == 1 && h.sys[0].blob_bytes <= 48 * 1024) ? 1 : 0;
    a.blob_smem = a.single ? h.sys[0].blob_bytes : 0;
    int max_tv = 0;
    for (const DevSys &d : h.sys)
        if (d.shadow) max_tv = std::max(max_tv, d.n_tv);
    if (std::getenv("IVS_NO_COMBO")) max_tv = 0;   // per-child shadow evaluation instead of tables
    choose_eval_layout(a, max_tv);
    CUDA_TRY(configure_eval_kernels(a));
    CUDA_TRY(cudaMemcpyAsync(p->d_box_lo, roots_lo.data(), roots_lo.size() * 8, cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaMemcpyAsync(p->d_box_hi, roots_hi.data(), roots_hi.size() * 8, cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaMemcpyAsync(p->d_root_depth, root_depth.data(), root_depth.size() * 4, cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));

    p->eval_threads = c.eval_threads > 0 ? c.eval_threads : 256;
    p->eval_blocks = c.eval_blocks > 0 ? c.eval_blocks : p->num_sms * 8;
    p->h_stats.assign((size_t)n_sys * ST_COUNT, 0);
    p->profile = c.profile != 0;
    if (p->profile) {
        p->stage_ev.resize(p->dims.size() + 5);
        for (auto &e : p->stage_ev) CUDA_TRY(cudaEventCreate(&e));
    }
    // profiling needs per-stage events, which a graph body cannot hold: host loop then
    p->use_graph = !p->profile && std::getenv("IVS_HOST_LOOP") == nullptr;
    if (p->use_graph) {
        if (r && r->h_wave_limit) std::swap(p->h_wave_limit, r->h_wave_limit);
        else CUDA_TRY(cudaMallocHost((void **)&p->h_wave_limit, sizeof(int64_t)));
        if (r && r->graph_exec && same_args(r->args, a) && r->dims == p->dims && r->eval_blocks == p->eval_blocks &&
            r->eval_threads == p->eval_threads && r->num_sms == p->num_sms) {
            std::swap(p->graph, r->graph);          // same kernels, same arguments: same graph
            std::swap(p->graph_exec, r->graph_exec);
            p->graph_kernels = r->graph_kernels;
        } else {
            CUDA_TRY(build_sweep_graph(a, p->dims.data(), (int)p->dims.size(), p->eval_blocks, p->eval_threads,
                                       p->num_sms, &p->graph, &p->graph_kernels));
            CUDA_TRY(cudaGraphInstantiate(&p->graph_exec, p->graph, 0));
        }
    }
    p->class_ms.assign(3 + p->dims.size(), 0.0);
    p->class_launches.assign(3 + p->dims.size(), 0);
    *out = p.release();
    return IVS_OK;
}

// ivs_solve / ivs_solve_batch keep the plan of their last call per device and build
// the next one from its resources
std::mutex g_cache_mu;
constexpr int kCacheDevices = 64;
ivs_plan *g_cache[kCacheDevices] = {};

ivs_plan *cache_take(int device) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (device < 0 || device >= kCacheDevices) return nullptr;
    ivs_plan *p = g_cache[device];
    g_cache[device] = nullptr;
    return p;
}

void cache_put(ivs_plan *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (p->device >= 0 && p->device < kCacheDevices && !g_cache[p->device]) {
            g_cache[p->device] = p;
            return;
        }
    }
    ivs_plan_destroy(p);
}

}  // namespace

extern "C" {

int ivs_plan_create(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                    const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                    const ivs_plan_cfg *cfg, ivs_plan **out) {
    return plan_create_impl(n_sys, systems, box_lo, box_hi, opts, opts_stride, cfg, nullptr, out);
}

void ivs_release_cached(void) {
    for (int d = 0; d < kCacheDevices; d++) ivs_plan_destroy(cache_take(d));
}

int ivs_plan_run(ivs_plan *p) {
    if (!p) return fail(IVS_ERR_INVALID, "null plan");
    CUDA_TRY(cudaSetDevice(p->device));
    SweepArgs &a = p->args;
    cudaStream_t st = p->stream;
    auto t0 = std::chrono::steady_clock::now();
    CUDA_TRY(cudaEventRecord(p->ev0, st));
    CUDA_TRY(cudaMemsetAsync(a.stats, 0, (size_t)p->n_sys * ST_COUNT * sizeof(unsigned long long), st));
    CUDA_TRY(launch_seed_roots(a, p->d_box_lo, p->d_box_hi, p->d_root_depth, p->n_sys, p->n_max, st));
    int status = IVS_OK;
    const int nd = (int)p->dims.size();
    std::fill(p->class_ms.begin(), p->class_ms.end(), 0.0);
    std::fill(p->class_launches.begin(), p->class_launches.end(), 0);
    p->launches = 1;
    if (p->use_graph) {
        // one graph launch runs sweeps until the queue is empty; with a time budget the
        // loop is cut into chunks of sweeps so the host can check the clock in between
        const int64_t chunk = p->time_budget_s > 0 ? 16 : ((int64_t)1 << 62);
        int64_t waves_done = 0;
        for (;;) {
            *p->h_wave_limit = waves_done + chunk;
            CUDA_TRY(cudaMemcpyAsync(&a.ctl->wave_limit, p->h_wave_limit, sizeof(int64_t), cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaGraphLaunch(p->graph_exec, st));
            CUDA_TRY(cudaEventRecord(p->ev1, st));
            // the control block and the counters in one round trip (the counters of the
            // last launch are the ones kept)
            CUDA_TRY(cudaMemcpyAsync(p->h_ctl, a.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaMemcpyAsync(p->h_stats.data(), a.stats, p->h_stats.size() * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            p->launches += (int64_t)p->graph_kernels * (p->h_ctl->waves - waves_done);
            waves_done = p->h_ctl->waves;
            if (p->h_ctl->error) { status = IVS_ERR_NOMEM; break; }
            if (p->h_ctl->top == 0) break;
            if (p->time_budget_s > 0) {
                double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > p->time_budget_s) { status = IVS_ERR_TIMEOUT; break; }
            }
        }
    } else {
        for (;;) {
            int kernels = 0;
            CUDA_TRY(launch_sweep(a, p->dims.data(), nd, p->eval_blocks, p->eval_threads, p->num_sms, st,
                                  p->profile ? p->stage_ev.data() : nullptr, &kernels));
            p->launches += kernels;
            CUDA_TRY(cudaMemcpyAsync(p->h_ctl, a.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (p->profile) {
                // classes: [0] eval (per child), [1] control, [2] eval64, [3 + q] hs dim q
                float t = 0;
                cudaEventElapsedTime(&t, p->stage_ev[1], p->stage_ev[2]);
                p->class_ms[0] += t;
                p->class_launches[0] += 1;
                cudaEventElapsedTime(&t, p->stage_ev[0], p->stage_ev[1]);
                p->class_ms[1] += t;
                cudaEventElapsedTime(&t, p->stage_ev[3 + nd], p->stage_ev[4 + nd]);
                p->class_ms[1] += t;
                p->class_launches[1] += 2;
                cudaEventElapsedTime(&t, p->stage_ev[2], p->stage_ev[3]);
                p->class_ms[2] += t;
                p->class_launches[2] += 1;
                for (int q = 0; q < nd; q++) {
                    cudaEventElapsedTime(&t, p->stage_ev[3 + q], p->stage_ev[4 + q]);
                    p->class_ms[3 + q] += t;
                    p->class_launches[3 + q] += 1;
                }
            }
            if (p->h_ctl->error) { status = IVS_ERR_NOMEM; break; }
            if (p->h_ctl->top == 0) break;
            if (p->time_budget_s > 0) {
                double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > p->time_budget_s) { status = IVS_ERR_TIMEOUT; break; }
            }
        }
    }
    if (!p->use_graph) {
        CUDA_TRY(cudaEventRecord(p->ev1, st));
        CUDA_TRY(cudaMemcpyAsync(p->h_stats.data(), a.stats, p->h_stats.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    CUDA_TRY(cudaEventElapsedTime(&p->last_ms, p->ev0, p->ev1));
    p->run_status = status;
    if (status == IVS_ERR_NOMEM) return fail(status, "work queue full: raise workspace or lower wave size");
    if (status == IVS_ERR_TIMEOUT) return fail(status, "time budget exhausted");
    return IVS_OK;
}

static void fill_stats(const ivs_plan *p, int s, ivs_stats *st) {
    const unsigned long long *v = p->h_stats.data() + (size_t)s * ST_COUNT;
    st->boxes += (int64_t)v[ST_BOXES];
    st->excluded_prefilter += (int64_t)v[ST_EXCL_PREFILTER];
    st->excluded_eval += (int64_t)v[ST_EXCL_EVAL];
    st->excluded_centred += (int64_t)v[ST_EXCL_CENTRED];
    st->gap_splits += (int64_t)v[ST_GAP_SPLITS];
    st->hs_applied += (int64_t)v[ST_HS_APPLIED];
    st->hs_empty += (int64_t)v[ST_HS_EMPTY];
    st->hs_contracted += (int64_t)v[ST_HS_CONTRACTED];
    st->hs_singular += (int64_t)v[ST_HS_SINGULAR];
    st->accepted += (int64_t)v[ST_ACCEPTED];
    st->unsplittable += (int64_t)v[ST_UNSPLITTABLE];
    st->split += (int64_t)v[ST_SPLIT];
    st->max_depth_seen = std::max(st->max_depth_seen, (int32_t)v[ST_MAX_DEPTH]);
    st->eval64_boxes += (int64_t)v[ST_EVAL64];
    st->kept_shadow += (int64_t)v[ST_KEEP_SHADOW];
    st->waves = (int32_t)p->h_ctl->waves;
    st->device_ms = p->last_ms;
    st->launches = p->launches;
}

}  // extern "C"

// The device-resident result region of system s after the last run (for the GPU root
// isolation in ivs_roots.cu): coordinate j of box i at lo[i + j * stride].
int plan_result_view(ivs_plan *p, int32_t s, const double **lo, const double **hi, int64_t *count, int64_t *stride,
                     int *n, const double **box_lo, const double **box_hi, cudaStream_t *st, int *device) {
    if (!p || s < 0 || s >= p->n_sys) return fail(IVS_ERR_INVALID, "bad plan or system index");
    const unsigned long long *sv = p->h_stats.data() + (size_t)s * ST_COUNT;
    *count = std::min<int64_t>((int64_t)sv[ST_OUT], p->sys_out_cap[s]);
    *lo = p->args.out.lo + p->sys_out_base[s];
    *hi = p->args.out.hi + p->sys_out_base[s];
    *stride = p->args.out.cap;
    *n = p->sys_n[s];
    *box_lo = p->box_lo_h.data() + (size_t)s * p->n_max;
    *box_hi = p->box_hi_h.data() + (size_t)s * p->n_max;
    *st = p->stream;
    *device = p->device;
    return IVS_OK;
}

extern "C" {

int ivs_plan_depth_stats(ivs_plan *p, int32_t s, ivs_stats *st, int64_t *boxes, int64_t *kept, int64_t *entered_hs) {
    if (!p || s < 0 || s >= p->n_sys) return fail(IVS_ERR_INVALID, "bad arguments");
    const unsigned long long *v = p->h_stats.data() + (size_t)s * ST_COUNT;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(p, s, st);
    }
    for (int q = 0; q < kDepthSlots; q++) {
        if (boxes) boxes[q] = (int64_t)v[ST_DEPTH_BOXES + q];
        if (kept) kept[q] = (int64_t)v[ST_DEPTH_KEPT + q];
        if (entered_hs) entered_hs[q] = (int64_t)v[ST_DEPTH_HS + q];
    }
    return IVS_OK;
}

int ivs_plan_stats(ivs_plan *p, ivs_stats *st) {
    if (!p || !st) return fail(IVS_ERR_INVALID, "null argument");
    std::memset(st, 0, sizeof(*st));
    for (int s = 0; s < p->n_sys; s++) fill_stats(p, s, st);
    return IVS_OK;
}

int ivs_plan_result(ivs_plan *p, int32_t s, ivs_result **out) {
    if (!p || !out || s < 0 || s >= p->n_sys) return fail(IVS_ERR_INVALID, "bad arguments");
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(p->device));
    const unsigned long long *sv = p->h_stats.data() + (size_t)s * ST_COUNT;
    const int64_t total = std::min<int64_t>((int64_t)sv[ST_OUT], p->sys_out_cap[s]);
    const int64_t base = p->sys_out_base[s];
    const int n = p->sys_n[s];
    std::vector<int32_t> flags(total), depth(total);
    std::vector<double> lo((size_t)total * n), hi((size_t)total * n);
    const DevOut &o = p->args.out;
    if (total > 0) {
        CUDA_TRY(cudaMemcpyAsync(flags.data(), o.flags + base, total * 4, cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(cudaMemcpyAsync(depth.data(), o.depth + base, total * 4, cudaMemcpyDeviceToHost, p->stream));
        // coordinate j of entry base + i at j * cap + base + i: one strided copy per array
        CUDA_TRY(cudaMemcpy2DAsync(lo.data(), (size_t)total * 8, o.lo + base, (size_t)o.cap * 8, (size_t)total * 8,
                                   (size_t)n, cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(cudaMemcpy2DAsync(hi.data(), (size_t)total * 8, o.hi + base, (size_t)o.cap * 8, (size_t)total * 8,
                                   (size_t)n, cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(cudaStreamSynchronize(p->stream));
    }
    std::unique_ptr<ivs_result> r(new (std::nothrow) ivs_result());
    if (!r) return fail(IVS_ERR_NOMEM, "host allocation");
    r->n = n;
    fill_sorted(r.get(), n, total, lo, hi, flags, depth);
    fill_stats(p, s, &r->st);
    for (int q = 0; q < kDepthSlots; q++) {
        r->depth_boxes[q] = (int64_t)sv[ST_DEPTH_BOXES + q];
        r->depth_kept[q] = (int64_t)sv[ST_DEPTH_KEPT + q];
        r->depth_hs[q] = (int64_t)sv[ST_DEPTH_HS + q];
    }
    const unsigned long long fl = p->h_stats[(size_t)s * ST_COUNT + ST_FLAGS];
    int status = p->run_status;
    if (status == IVS_OK && fl) status = IVS_ERR_BUDGET;
    r->status = status;
    *out = r.release();
    return IVS_OK;
}

int ivs_autotune(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                 const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                 int64_t trial_boxes, ivs_plan_cfg *best, double *best_rate) {
    if (n_sys <= 0 || !systems || !box_lo || !box_hi || !opts || !best || trial_boxes <= 0)
        return fail(IVS_ERR_INVALID, "bad arguments");
    std::vector<ivs_options> topt((size_t)n_sys);
    for (int s = 0; s < n_sys; s++) {
        topt[(size_t)s] = *opt_at(opts, opts_stride, s);
        topt[(size_t)s].max_boxes = trial_boxes;
        topt[(size_t)s].time_budget_s = 0;
    }
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const int64_t waves[3] = {(int64_t)1 << 20, (int64_t)1 << 22, (int64_t)1 << 24};
    const int per_sm[3] = {4, 8, 16};
    double rate[3][3];
    double top = -1.0;
    for (int wi = 0; wi < 3; wi++)
        for (int bi = 0; bi < 3; bi++) {
            rate[wi][bi] = -1.0;
            ivs_plan_cfg c{};
            c.wave_children = waves[wi];
            c.eval_blocks = sms * per_sm[bi];
            ivs_plan *p = nullptr;
            int rc = ivs_plan_create(n_sys, systems, box_lo, box_hi, topt.data(), (int32_t)sizeof(ivs_options), &c, &p);
            if (rc == IVS_ERR_NOMEM) continue;   // this size does not fit: try the others
            if (rc) return rc;
            rc = ivs_plan_run(p);                // warm-up (graph upload, caches)
            for (int rep = 0; rep < 2 && (rc == IVS_OK || rc == IVS_ERR_NOMEM); rep++) {   // the faster of two runs
                rc = ivs_plan_run(p);
                ivs_stats st{};
                ivs_plan_stats(p, &st);
                if (rc == IVS_OK && st.device_ms > 0)
                    rate[wi][bi] = std::max(rate[wi][bi], (double)st.boxes / (st.device_ms * 1e-3));
            }
            ivs_plan_destroy(p);
            if (rc != IVS_OK && rc != IVS_ERR_NOMEM) return rc;
            top = std::max(top, rate[wi][bi]);
        }
    if (top < 0) return fail(IVS_ERR_NOMEM, "no trial configuration fit");
    // within 3% of the fastest, the largest sweep: the trial caps every system's boxes, so
    // it runs fewer sweeps than the full solve and undercounts the fixed cost of each
    int bw = -1, bb = -1;
    for (int wi = 2; wi >= 0 && bw < 0; wi--)
        for (int bi = 0; bi < 3; bi++)
            if (rate[wi][bi] >= 0.97 * top && (bw < 0 || rate[wi][bi] > rate[bw][bb])) {
                bw = wi;
                bb = bi;
            }
    ivs_plan_cfg bc{};
    bc.wave_children = waves[bw];
    bc.eval_blocks = sms * per_sm[bb];
    *best = bc;
    if (best_rate) *best_rate = rate[bw][bb];
    return IVS_OK;
}

int32_t ivs_plan_kernel_times(ivs_plan *p, ivs_kernel_time *out, int32_t max) {
    if (!p) return 0;
    const int32_t total = (int32_t)p->class_ms.size();
    for (int32_t q = 0; q < total && q < max && out; q++) {
        std::string name = q == 0 ? "eval" : q == 1 ? "control" : q == 2 ? "eval64" : "hs_n" + std::to_string(p->dims[q - 3]);
        std::memset(out[q].name, 0, sizeof(out[q].name));
        std::strncpy(out[q].name, name.c_str(), sizeof(out[q].name) - 1);
        out[q].launches = p->class_launches[q];
        out[q].ms = p->class_ms[q];
    }
    return total;
}

int ivs_probe_rate(int32_t kind, int32_t device, double *ops_per_s, double *ms) {
    if (!ops_per_s || kind < 0 || kind > 5) return fail(IVS_ERR_INVALID, "bad arguments");
    CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    double ops = 0;
    float t = 0;
    CUDA_TRY(run_probe(kind, sms, &ops, &t));
    *ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
    return IVS_OK;
}

int64_t ivs_result_count(const ivs_result *r) { return r ? (int64_t)r->flags.size() : 0; }
int32_t ivs_result_n_vars(const ivs_result *r) { return r ? r->n : 0; }
int ivs_result_status(const ivs_result *r) { return r ? r->status : IVS_ERR_INVALID; }
int ivs_result_boxes(const ivs_result *r, double *lo, double *hi, int32_t *flags, int32_t *depth) {
    if (!r) return fail(IVS_ERR_INVALID, "null result");
    if (lo && !r->lo.empty()) std::memcpy(lo, r->lo.data(), r->lo.size() * 8);
    if (hi && !r->hi.empty()) std::memcpy(hi, r->hi.data(), r->hi.size() * 8);
    if (flags && !r->flags.empty()) std::memcpy(flags, r->flags.data(), r->flags.size() * 4);
    if (depth && !r->depth.empty()) std::memcpy(depth, r->depth.data(), r->depth.size() * 4);
    return IVS_OK;
}
int ivs_result_depth_stats(const ivs_result *r, int64_t *boxes, int64_t *kept, int64_t *entered_hs) {
    if (!r) return fail(IVS_ERR_INVALID, "null result");
    if (boxes) std::memcpy(boxes, r->depth_boxes, sizeof(r->depth_boxes));
    if (kept) std::memcpy(kept, r->depth_kept, sizeof(r->depth_kept));
    if (entered_hs) std::memcpy(entered_hs, r->depth_hs, sizeof(r->depth_hs));
    return IVS_OK;
}
int ivs_result_stats(const ivs_result *r, ivs_stats *st) {
    if (!r || !st) return fail(IVS_ERR_INVALID, "null argument");
    *st = r->st;
    return IVS_OK;
}
void ivs_result_free(ivs_result *r) { delete r; }

int ivs_solve_batch(int32_t n_sys, const ivs_system *systems, const double *const *box_lo,
                    const double *const *box_hi, const ivs_options *opts, int32_t opts_stride,
                    ivs_result **outs) {
    if (!outs) return fail(IVS_ERR_INVALID, "null outs");
    for (int s = 0; s < n_sys; s++) outs[s] = nullptr;
    ivs_plan *p = nullptr;
    int rc = plan_create_impl(n_sys, systems, box_lo, box_hi, opts, opts_stride, nullptr, cache_take(0), &p);
    if (rc) return rc;
    int run = ivs_plan_run(p);
    if (run != IVS_OK && run != IVS_ERR_TIMEOUT && run != IVS_ERR_NOMEM) {
        ivs_plan_destroy(p);
        return run;
    }
    int first = run;
    for (int s = 0; s < n_sys; s++) {
        rc = ivs_plan_result(p, s, &outs[s]);
        if (rc) {
            ivs_plan_destroy(p);
            return rc;
        }
        if (first == IVS_OK && outs[s]->status != IVS_OK) first = outs[s]->status;
    }
    cache_put(p);
    return first;
}

int ivs_solve(const ivs_system *sys, const double *box_lo, const double *box_hi, const ivs_options *opt,
              ivs_result **out) {
    if (!out) return fail(IVS_ERR_INVALID, "null out");
    const double *lo[1] = {box_lo};
    const double *hi[1] = {box_hi};
    return ivs_solve_batch(1, sys, lo, hi, opt, 0, out);
}

}  // extern "C"
