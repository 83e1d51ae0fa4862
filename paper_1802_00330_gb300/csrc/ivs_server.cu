// ivs_server.cu -- the serving form: continuous batching over one shared device queue.
//
// One worker thread drives the GPU.  Each step it (1) admits waiting requests into free
// slots while their queue reservations fit, appending their initial boxes to the shared
// queue, (2) runs a few sweeps through the same sweep graph as a plan (the queue mixes the
// boxes of every system in flight, so requests that arrive while others run share their
// kernels), and (3) hands back every system whose live-entry counter dropped to zero.
// Results equal ivs_solve's bit for bit: each box's fate depends only on the box.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ivsolve.h"
#include "ivs_hostcore.h"
#include "ivs_internal.h"
#include "ivs_kernels.cuh"
#include "ivs_tab.cuh"

using namespace ivs;
using namespace ivs::host;
using Clock = std::chrono::steady_clock;

namespace {

constexpr uint32_t kBlobSlot = 128 * 1024;   // term-table bytes per slot (n = 12, 14 terms of degree 4
                                             // per equation need about 50 KB)

struct Request {
    uint64_t ticket = 0;
    int n = 0, m = 0;
    std::vector<int32_t> off;
    std::vector<double> clo, chi;
    std::vector<uint8_t> exps;
    std::vector<double> lo, hi;
    ivs_options opt{};
    Clock::time_point t_submit, t_admit;
    int64_t reserve = 0;
    ivs_system view() const {
        ivs_system s{};
        s.n_vars = n;
        s.n_eqs = m;
        s.n_terms = off.empty() ? 0 : off.back();
        s.eq_offsets = off.data();
        s.coef_lo = clo.data();
        s.coef_hi = chi.data();
        s.exps = exps.data();
        return s;
    }
};

struct Slot {
    bool used = false;
    bool cancelled = false;   // time budget ran out: its boxes are being dropped
    DevSys dev{};
    Request req;
};

}  // namespace

struct ivs_server {
    ivs_server_cfg cfg{};
    int device = 0, num_sms = 0, n_max = 0;
    cudaStream_t stream = nullptr;
    void *ws = nullptr, *tables = nullptr;
    DevSys *d_sys = nullptr;
    char *d_blobs = nullptr;
    SweepArgs a{};
    std::vector<int> dims;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    WaveCtl *h_ctl = nullptr;
    unsigned long long *h_stats = nullptr;
    int64_t *h_limit = nullptr;
    double *h_rlo = nullptr, *h_rhi = nullptr;     // admission staging (pinned)
    int32_t *h_rslot = nullptr, *h_rdepth = nullptr;
    double *d_rlo = nullptr, *d_rhi = nullptr;
    int32_t *d_rslot = nullptr, *d_rdepth = nullptr;
    int32_t *d_cancel = nullptr;                   // per slot: 1 = its region is emptied
    int64_t *h_region = nullptr;                   // pinned: a slot's region base and size
    int64_t q_cap = 0, rps = 0;
    std::map<int64_t, int64_t> free_regions;       // queue entries not held by a slot: start -> size
    std::vector<std::pair<int64_t, int64_t>> region_of;   // per slot
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::atomic<int> active{0};

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> waiting;
    std::unordered_map<uint64_t, ivs_result *> done;
    std::unordered_map<uint64_t, int> state;       // 1 waiting/running, 2 done
    uint64_t next_ticket = 1;
    bool stop = false;
    ivs_server_stats stats{};
    std::thread worker;

    ~ivs_server();
    int init();
    void loop();
    int step(std::vector<std::pair<uint64_t, ivs_result *>> &finished);
    void fail_all_active(int status, std::vector<std::pair<uint64_t, ivs_result *>> &finished);
    bool region_alloc(int64_t size, int64_t *start);
    void region_free(int slot);
};

ivs_server::~ivs_server() {
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv_work.notify_all();
    if (worker.joinable()) worker.join();
    if (stream) cudaStreamSynchronize(stream);
    for (auto &kv : done) delete kv.second;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ws) cudaFree(ws);
    if (tables) cudaFree(tables);
    if (h_region) cudaFreeHost(h_region);
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_stats) cudaFreeHost(h_stats);
    if (h_limit) cudaFreeHost(h_limit);
    if (h_rlo) cudaFreeHost(h_rlo);
    if (h_rhi) cudaFreeHost(h_rhi);
    if (h_rslot) cudaFreeHost(h_rslot);
    if (h_rdepth) cudaFreeHost(h_rdepth);
    if (stream) cudaStreamDestroy(stream);
}

int ivs_server::init() {
    n_max = cfg.max_vars;
    const int S = cfg.max_slots;
    CUDA_TRY(cudaSetDevice(device));
    CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    const int64_t W = cfg.wave_children;
    rps = cfg.results_per_slot;
    const int64_t O = (int64_t)S * rps;
    const size_t per_parent = 3 * (size_t)n_max * sizeof(double) + 2 * sizeof(int32_t);
    // workspace_bytes buys the shared queue; staging, lists and result regions come on top
    q_cap = (int64_t)(cfg.workspace_bytes / per_parent);
    if (q_cap < W) return fail(IVS_ERR_NOMEM, "server workspace too small for one sweep of children");
    const Layout L = layout_for(S, n_max, W, q_cap, O);
    cudaError_t e = cudaMalloc(&ws, L.total);
    if (e != cudaSuccess) return fail(IVS_ERR_NOMEM, std::string("cudaMalloc server workspace: ") + cudaGetErrorString(e));
    char *base = (char *)ws;
    a.q = carve_queue(base + L.queue, q_cap, n_max);
    a.stage = carve_queue(base + L.stage, W, n_max);
    a.surv = (Surv *)(base + L.surv);
    a.surv_cap = W;
    a.cand = a.surv + (size_t)(n_max + 1) * W;
    a.out = carve_out(base + L.out, O, n_max);
    a.ctl = (WaveCtl *)(base + L.ctl);
    a.stats = (unsigned long long *)(base + L.stats);
    a.wave_children = W;
    a.max_fan_shift = n_max;
    a.n_sys = S;
    a.single = 0;
    a.blob_smem = 0;
    // system records, term tables and the admission staging (S initial boxes, slot ids
    // and depths) in a second allocation
    const size_t sys_bytes = align_up((size_t)S * sizeof(DevSys), 256);
    const size_t blob_bytes = (size_t)S * kBlobSlot;
    const size_t adm_bytes = align_up((size_t)S * (2 * (size_t)n_max * sizeof(double) + 2 * sizeof(int32_t)), 256);
    // per slot: cancel flag; the region arrays (base, cap, rem, prefix (S + 1), cursor)
    const size_t slot_bytes = align_up((size_t)S * sizeof(int32_t), 256) + (size_t)(5 * S + 1) * sizeof(int64_t);
    CUDA_TRY(cudaMalloc(&tables, sys_bytes + blob_bytes + adm_bytes + slot_bytes));
    CUDA_TRY(cudaMemsetAsync(tables, 0, sys_bytes + blob_bytes + adm_bytes + slot_bytes, stream));
    d_sys = (DevSys *)tables;
    d_blobs = (char *)tables + sys_bytes;
    d_rlo = (double *)(d_blobs + blob_bytes);
    d_rhi = d_rlo + (size_t)S * n_max;
    d_rslot = (int32_t *)(d_rhi + (size_t)S * n_max);
    d_rdepth = d_rslot + S;
    d_cancel = (int32_t *)(d_blobs + blob_bytes + adm_bytes);
    int64_t *rg_mem = (int64_t *)((char *)d_cancel + align_up((size_t)S * sizeof(int32_t), 256));
    if (q_cap > (int64_t)0xFFFFFFFFLL) return fail(IVS_ERR_INVALID, "server queue above 2^32 entries");
    // one queue region per slot, carved from the queue at admission
    a.rg.base = rg_mem;
    a.rg.cap = rg_mem + S;
    a.rg.rem = rg_mem + 2 * S;
    a.rg.cursor = (unsigned long long *)(rg_mem + 3 * S);
    a.rg.prefix = rg_mem + 4 * S;
    a.rg.n = S;
    a.rg.fair_share = cfg.schedule == 1 ? 1 : 0;
    free_regions[0] = q_cap;
    region_of.assign((size_t)S, {0, 0});
    CUDA_TRY(cudaMallocHost((void **)&h_region, 2 * (size_t)S * sizeof(int64_t)));
    a.tb.sys = d_sys;
    a.tb.blobs = d_blobs;
    CUDA_TRY(cudaMallocHost((void **)&h_ctl, sizeof(WaveCtl)));
    CUDA_TRY(cudaMallocHost((void **)&h_stats, (size_t)S * ST_COUNT * sizeof(unsigned long long)));
    CUDA_TRY(cudaMallocHost((void **)&h_limit, sizeof(int64_t)));
    CUDA_TRY(cudaMallocHost((void **)&h_rlo, (size_t)S * n_max * sizeof(double)));
    CUDA_TRY(cudaMallocHost((void **)&h_rhi, (size_t)S * n_max * sizeof(double)));
    CUDA_TRY(cudaMallocHost((void **)&h_rslot, (size_t)S * sizeof(int32_t)));
    CUDA_TRY(cudaMallocHost((void **)&h_rdepth, (size_t)S * sizeof(int32_t)));
    CUDA_TRY(cudaMemsetAsync(a.stats, 0, (size_t)S * ST_COUNT * sizeof(unsigned long long), stream));
    CUDA_TRY(launch_seed_roots(a, d_rlo, d_rhi, d_rdepth, 0, n_max, stream));   // empty queue, reset control
    choose_eval_layout(a, 2048);   // any admitted system's table fits (hostcore caps it at 2048)
    CUDA_TRY(configure_eval_kernels(a));
    for (int n = 1; n <= n_max; n++) dims.push_back(n);
    CUDA_TRY(build_sweep_graph(a, dims.data(), (int)dims.size(), num_sms * 8, 256, num_sms, &graph));
    CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    CUDA_TRY(cudaMemcpyAsync(h_ctl, a.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, stream));   // top = 0, waves = 0
    CUDA_TRY(cudaStreamSynchronize(stream));
    slots.resize(S);
    for (int s = S - 1; s >= 0; s--) free_slots.push_back(s);
    worker = std::thread([this] { loop(); });
    return IVS_OK;
}

void ivs_server::fail_all_active(int status, std::vector<std::pair<uint64_t, ivs_result *>> &finished) {
    for (int s = 0; s < (int)slots.size(); s++) {
        if (!slots[s].used) continue;
        ivs_result *r = new (std::nothrow) ivs_result();
        if (r) {
            r->status = status;
            r->n = slots[s].req.n;
        }
        finished.push_back({slots[s].req.ticket, r});
        slots[s].used = false;
        free_slots.push_back(s);
        region_free(s);
    }
    active = 0;
}

// first fit over the free queue segments
bool ivs_server::region_alloc(int64_t size, int64_t *start) {
    for (auto it = free_regions.begin(); it != free_regions.end(); ++it) {
        if (it->second < size) continue;
        *start = it->first;
        const int64_t rest = it->second - size;
        const int64_t at = it->first + size;
        free_regions.erase(it);
        if (rest > 0) free_regions[at] = rest;
        return true;
    }
    return false;
}

void ivs_server::region_free(int slot) {
    auto &rg = region_of[(size_t)slot];
    if (rg.second <= 0) return;
    int64_t st = rg.first, sz = rg.second;
    rg = {0, 0};
    auto nx = free_regions.lower_bound(st);
    if (nx != free_regions.end() && st + sz == nx->first) {   // merge with the next segment
        sz += nx->second;
        nx = free_regions.erase(nx);
    }
    if (nx != free_regions.begin()) {                        // and with the previous one
        auto pv = std::prev(nx);
        if (pv->first + pv->second == st) {
            pv->second += sz;
            return;
        }
    }
    free_regions[st] = sz;
}

// One step: admit, run sweeps, collect finished systems.  Returns a CUDA status.
int ivs_server::step(std::vector<std::pair<uint64_t, ivs_result *>> &finished) {
    // (1) requests past their time budget leave the queue at once: their entries are
    // dropped (their region is emptied), and they complete in this step (IVS_ERR_TIMEOUT)
    {
        const auto now0 = Clock::now();
        bool any = false;
        for (int s = 0; s < (int)slots.size(); s++) {
            Slot &sl = slots[s];
            if (!sl.used || sl.cancelled || !(sl.req.opt.time_budget_s > 0)) continue;
            if (std::chrono::duration<double>(now0 - sl.req.t_admit).count() <= sl.req.opt.time_budget_s) continue;
            sl.cancelled = true;
            any = true;
            CUDA_TRY(cudaMemsetAsync(d_cancel + s, 0x01, sizeof(int32_t), stream));
            CUDA_TRY(cudaMemsetAsync(a.stats + (size_t)s * ST_COUNT + ST_LIVE, 0, sizeof(unsigned long long), stream));
        }
        if (any) CUDA_TRY(launch_cancel_regions(a, d_cancel, stream));
    }
    // (2) admission
    std::vector<Request> admit;
    std::vector<int> admit_slot;
    {
        std::lock_guard<std::mutex> lk(mu);
        // admission by memory: a request waits until a slot and a queue region of its
        // reservation are free (in arrival order)
        int64_t start = 0;
        while (!waiting.empty() && !free_slots.empty() && region_alloc(waiting.front().reserve, &start)) {
            admit.push_back(std::move(waiting.front()));
            waiting.pop_front();
            admit_slot.push_back(free_slots.back());
            free_slots.pop_back();
            region_of[(size_t)admit_slot.back()] = {start, admit.back().reserve};
        }
    }
    int n_adm = 0;
    for (size_t q = 0; q < admit.size(); q++) {
        Request &rq = admit[q];
        const int s = admit_slot[q];
        HostTables h;
        const ivs_system sv = rq.view();
        compile_system(h, &sv, &rq.opt);
        DevSys d = h.sys[0];
        if ((uint32_t)d.blob_bytes > kBlobSlot) {
            ivs_result *r = new (std::nothrow) ivs_result();
            if (r) { r->status = IVS_ERR_INVALID; r->n = rq.n; }
            finished.push_back({rq.ticket, r});
            free_slots.push_back(s);
            region_free(s);
            continue;
        }
        d.shadow = (rq.opt.prefilter_fp32 && shadow_safe(&sv, rq.lo.data(), rq.hi.data())) ? 1 : 0;
        d.blob_off = (int64_t)s * kBlobSlot;
        d.out_base = (int64_t)s * rps;
        d.out_cap = rq.opt.max_results > 0 ? std::min<int64_t>(rq.opt.max_results, rps) : rps;
        CUDA_TRY(cudaMemcpyAsync(d_sys + s, &d, sizeof(DevSys), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d_blobs + d.blob_off, h.blobs.data(), h.blobs.size(), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemsetAsync(a.stats + (size_t)s * ST_COUNT, 0, ST_COUNT * sizeof(unsigned long long), stream));
        CUDA_TRY(cudaMemsetAsync(d_cancel + s, 0, sizeof(int32_t), stream));
        h_region[2 * s] = region_of[(size_t)s].first;
        h_region[2 * s + 1] = region_of[(size_t)s].second;
        CUDA_TRY(cudaMemcpyAsync(a.rg.base + s, &h_region[2 * s], sizeof(int64_t), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(a.rg.cap + s, &h_region[2 * s + 1], sizeof(int64_t), cudaMemcpyHostToDevice, stream));
        for (int j = 0; j < n_max; j++) {
            h_rlo[(size_t)n_adm * n_max + j] = j < rq.n ? rq.lo[j] : 0.0;
            h_rhi[(size_t)n_adm * n_max + j] = j < rq.n ? rq.hi[j] : 0.0;
        }
        h_rslot[n_adm] = s;
        h_rdepth[n_adm] = rq.opt.root_depth;
        n_adm++;
        rq.t_admit = Clock::now();
        slots[s].used = true;
        slots[s].cancelled = false;
        slots[s].dev = d;
        slots[s].req = std::move(rq);
        active++;
    }
    if (n_adm > 0) {
        CUDA_TRY(cudaMemcpyAsync(d_rlo, h_rlo, (size_t)n_adm * n_max * sizeof(double), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d_rhi, h_rhi, (size_t)n_adm * n_max * sizeof(double), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d_rslot, h_rslot, (size_t)n_adm * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d_rdepth, h_rdepth, (size_t)n_adm * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(launch_admit(a, d_rlo, d_rhi, d_rslot, d_rdepth, n_adm, n_max, stream));
        std::lock_guard<std::mutex> lk(mu);
        stats.admitted += n_adm;
    }
    if (active == 0) return IVS_OK;
    // (3) a few sweeps through the sweep graph
    const int64_t waves0 = h_ctl->waves;
    *h_limit = waves0 + cfg.sweeps_per_step;
    CUDA_TRY(cudaMemcpyAsync(&a.ctl->wave_limit, h_limit, sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaGraphLaunch(exec, stream));
    CUDA_TRY(cudaMemcpyAsync(h_ctl, a.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(h_stats, a.stats, slots.size() * ST_COUNT * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    {
        std::lock_guard<std::mutex> lk(mu);
        stats.steps++;
        stats.sweeps += h_ctl->waves - waves0;
    }
    if (h_ctl->error) {
        // the queue overflowed despite the reservations: fail the systems in flight, restart empty
        fail_all_active(IVS_ERR_NOMEM, finished);
        CUDA_TRY(launch_seed_roots(a, d_rlo, d_rhi, d_rdepth, 0, n_max, stream));
        CUDA_TRY(cudaMemsetAsync(a.rg.rem, 0, slots.size() * sizeof(int64_t), stream));
        CUDA_TRY(cudaMemsetAsync(a.rg.cursor, 0, slots.size() * sizeof(unsigned long long), stream));
        CUDA_TRY(cudaMemcpyAsync(h_ctl, a.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        return IVS_OK;
    }
    // finished systems: no box of theirs left in the queue
    for (int s = 0; s < (int)slots.size(); s++) {
        if (!slots[s].used) continue;
        const unsigned long long *v = h_stats + (size_t)s * ST_COUNT;
        if (v[ST_LIVE] != 0) continue;
        Request &rq = slots[s].req;
        const int n = rq.n;
        const int64_t cap = rq.opt.max_results > 0 ? std::min<int64_t>(rq.opt.max_results, rps) : rps;
        const int64_t total = std::min<int64_t>((int64_t)v[ST_OUT], cap);
        const int64_t base = (int64_t)s * rps;
        std::vector<int32_t> flags(total), depth(total);
        std::vector<double> lo((size_t)total * n), hi((size_t)total * n);
        if (total > 0) {
            CUDA_TRY(cudaMemcpyAsync(flags.data(), a.out.flags + base, total * 4, cudaMemcpyDeviceToHost, stream));
            CUDA_TRY(cudaMemcpyAsync(depth.data(), a.out.depth + base, total * 4, cudaMemcpyDeviceToHost, stream));
            for (int j = 0; j < n; j++) {
                CUDA_TRY(cudaMemcpyAsync(lo.data() + (size_t)j * total, a.out.lo + (size_t)j * a.out.cap + base, total * 8,
                                         cudaMemcpyDeviceToHost, stream));
                CUDA_TRY(cudaMemcpyAsync(hi.data() + (size_t)j * total, a.out.hi + (size_t)j * a.out.cap + base, total * 8,
                                         cudaMemcpyDeviceToHost, stream));
            }
            CUDA_TRY(cudaStreamSynchronize(stream));
        }
        ivs_result *r = new (std::nothrow) ivs_result();
        if (r) {
            fill_sorted(r, n, total, lo, hi, flags, depth);
            ivs_stats &st = r->st;
            st.boxes = (int64_t)v[ST_BOXES];
            st.excluded_prefilter = (int64_t)v[ST_EXCL_PREFILTER];
            st.excluded_eval = (int64_t)v[ST_EXCL_EVAL];
            st.excluded_centred = (int64_t)v[ST_EXCL_CENTRED];
            st.gap_splits = (int64_t)v[ST_GAP_SPLITS];
            for (int q = 0; q < kDepthSlots; q++) {
                r->depth_boxes[q] = (int64_t)v[ST_DEPTH_BOXES + q];
                r->depth_kept[q] = (int64_t)v[ST_DEPTH_KEPT + q];
                r->depth_hs[q] = (int64_t)v[ST_DEPTH_HS + q];
            }
            st.hs_applied = (int64_t)v[ST_HS_APPLIED];
            st.hs_empty = (int64_t)v[ST_HS_EMPTY];
            st.hs_contracted = (int64_t)v[ST_HS_CONTRACTED];
            st.hs_singular = (int64_t)v[ST_HS_SINGULAR];
            st.accepted = (int64_t)v[ST_ACCEPTED];
            st.unsplittable = (int64_t)v[ST_UNSPLITTABLE];
            st.split = (int64_t)v[ST_SPLIT];
            st.max_depth_seen = (int32_t)v[ST_MAX_DEPTH];
            st.eval64_boxes = (int64_t)v[ST_EVAL64];
            st.kept_shadow = (int64_t)v[ST_KEEP_SHADOW];
            const auto now = Clock::now();
            st.queue_ms = std::chrono::duration<double, std::milli>(rq.t_admit - rq.t_submit).count();
            st.solve_ms = std::chrono::duration<double, std::milli>(now - rq.t_admit).count();
            st.device_ms = st.solve_ms;
            r->status = slots[s].cancelled ? IVS_ERR_TIMEOUT
                        : ((v[ST_FLAGS] != 0 || (int64_t)v[ST_OUT] > cap) ? IVS_ERR_BUDGET : IVS_OK);
            std::lock_guard<std::mutex> lk(mu);
            stats.boxes += st.boxes;
        }
        finished.push_back({rq.ticket, r});
        slots[s].used = false;
        free_slots.push_back(s);
        region_free(s);
        active--;
    }
    return IVS_OK;
}

void ivs_server::loop() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !waiting.empty() || active > 0; });
            if (stop) return;
        }
        std::vector<std::pair<uint64_t, ivs_result *>> finished;
        const auto t0 = Clock::now();
        int rc = step(finished);
        if (rc != IVS_OK) fail_all_active(rc, finished);
        std::lock_guard<std::mutex> lk(mu);
        if (rc != IVS_OK) {
            std::strncpy(stats.last_error, last_error(), sizeof(stats.last_error) - 1);
            stats.last_error[sizeof(stats.last_error) - 1] = 0;
        }
        stats.busy_s += std::chrono::duration<double>(Clock::now() - t0).count();
        for (auto &f : finished) {
            done[f.first] = f.second;
            state[f.first] = 2;
            stats.completed++;
        }
        if (!finished.empty()) cv_done.notify_all();
        if (rc != IVS_OK) {
            // a CUDA failure: refuse what is still waiting
            for (auto &w : waiting) {
                ivs_result *r = new (std::nothrow) ivs_result();
                if (r) { r->status = IVS_ERR_CUDA; r->n = w.n; }
                done[w.ticket] = r;
                state[w.ticket] = 2;
                stats.completed++;
            }
            waiting.clear();
            cv_done.notify_all();
        }
    }
}

extern "C" {

void ivs_server_cfg_default(ivs_server_cfg *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->workspace_bytes = (size_t)4 << 30;
    c->wave_children = (int64_t)1 << 22;
    c->results_per_slot = 16384;
    c->max_slots = 1024;
    c->max_vars = 12;
    c->sweeps_per_step = 2;
    c->device = 0;
    c->reserve_factor = 1.0;
}

int ivs_server_create(const ivs_server_cfg *cfg, ivs_server **out) {
    if (!out) return fail(IVS_ERR_INVALID, "null out");
    *out = nullptr;
    ivs_server_cfg c;
    ivs_server_cfg_default(&c);
    if (cfg) {
        if (cfg->workspace_bytes) c.workspace_bytes = cfg->workspace_bytes;
        if (cfg->wave_children > 0) c.wave_children = cfg->wave_children;
        if (cfg->results_per_slot > 0) c.results_per_slot = cfg->results_per_slot;
        if (cfg->max_slots > 0) c.max_slots = cfg->max_slots;
        if (cfg->max_vars > 0) c.max_vars = cfg->max_vars;
        if (cfg->sweeps_per_step > 0) c.sweeps_per_step = cfg->sweeps_per_step;
        if (cfg->reserve_factor > 0) c.reserve_factor = cfg->reserve_factor;
        if (cfg->min_region_entries > 0) c.min_region_entries = cfg->min_region_entries;
        c.schedule = cfg->schedule;
        c.device = cfg->device;
    }
    if (c.max_vars > kMaxVars || c.max_slots > 65536 || c.schedule < 0 || c.schedule > 1 || c.wave_children < ((int64_t)1 << c.max_vars))
        return fail(IVS_ERR_INVALID, "bad server configuration");
    std::unique_ptr<ivs_server> sv(new (std::nothrow) ivs_server());
    if (!sv) return fail(IVS_ERR_NOMEM, "host allocation");
    sv->cfg = c;
    sv->device = c.device;
    const int rc = sv->init();
    if (rc != IVS_OK) return rc;
    *out = sv.release();
    return IVS_OK;
}

int ivs_server_submit(ivs_server *sv, const ivs_system *s, const double *box_lo, const double *box_hi,
                      const ivs_options *opt, uint64_t *ticket) {
    if (!sv || !ticket) return fail(IVS_ERR_INVALID, "null argument");
    const int rc = validate(s, box_lo, box_hi, opt);
    if (rc) return rc;
    if (s->n_vars > sv->cfg.max_vars) return fail(IVS_ERR_INVALID, "n_vars above the server's max_vars");
    Request rq;
    rq.n = s->n_vars;
    rq.m = s->n_eqs;
    rq.off.assign(s->eq_offsets, s->eq_offsets + s->n_eqs + 1);
    rq.clo.assign(s->coef_lo, s->coef_lo + s->n_terms);
    rq.chi.assign(s->coef_hi ? s->coef_hi : s->coef_lo, (s->coef_hi ? s->coef_hi : s->coef_lo) + s->n_terms);
    rq.exps.assign(s->exps, s->exps + (size_t)s->n_terms * s->n_vars);
    rq.lo.assign(box_lo, box_lo + s->n_vars);
    rq.hi.assign(box_hi, box_hi + s->n_vars);
    rq.opt = *opt;
    rq.reserve = std::max<int64_t>(std::max<int64_t>((int64_t)(64.0 * sv->cfg.reserve_factor *
                                                                 (double)((int64_t)1 << s->n_vars)),
                                                       sv->cfg.min_region_entries),
                                   ((int64_t)1 << s->n_vars) + 1);
    rq.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        rq.ticket = sv->next_ticket++;
        *ticket = rq.ticket;
        sv->state[rq.ticket] = 1;
        sv->waiting.push_back(std::move(rq));
        sv->stats.submitted++;
    }
    sv->cv_work.notify_one();
    return IVS_OK;
}

static int take_done(ivs_server *sv, uint64_t ticket, ivs_result **out) {
    auto it = sv->done.find(ticket);
    *out = it->second;
    sv->done.erase(it);
    sv->state.erase(ticket);
    if (!*out) return fail(IVS_ERR_NOMEM, "host allocation of a result");
    return IVS_OK;
}

int ivs_server_poll(ivs_server *sv, uint64_t ticket, ivs_result **out) {
    if (!sv || !out) return fail(IVS_ERR_INVALID, "null argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto st = sv->state.find(ticket);
    if (st == sv->state.end()) return fail(IVS_ERR_INVALID, "unknown ticket");
    if (st->second != 2) return IVS_OK;
    return take_done(sv, ticket, out);
}

int ivs_server_wait(ivs_server *sv, uint64_t ticket, double timeout_s, ivs_result **out) {
    if (!sv || !out) return fail(IVS_ERR_INVALID, "null argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] {
        auto st = sv->state.find(ticket);
        return st == sv->state.end() || st->second == 2;
    };
    if (sv->state.find(ticket) == sv->state.end()) return fail(IVS_ERR_INVALID, "unknown ticket");
    if (timeout_s > 0) {
        if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return IVS_OK;
    } else {
        sv->cv_done.wait(lk, ready);
    }
    if (sv->state.find(ticket) == sv->state.end()) return fail(IVS_ERR_INVALID, "unknown ticket");
    return take_done(sv, ticket, out);
}

int ivs_server_get_stats(ivs_server *sv, ivs_server_stats *st) {
    if (!sv || !st) return fail(IVS_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *st = sv->stats;
    st->waiting = (int64_t)sv->waiting.size();
    st->in_flight = sv->active.load();
    return IVS_OK;
}

void ivs_server_destroy(ivs_server *sv) { delete sv; }

}  // extern "C"
