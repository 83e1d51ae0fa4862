// ivs_hostcore.h -- host-side helpers shared by the plan and serving runtimes.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ivsolve.h"
#include "ivs_internal.h"
#include "ivs_kernels.cuh"

// a result handed to the caller (ivs_result_* accessors)
struct ivs_result {
    int status = IVS_OK;
    int n = 0;
    std::vector<double> lo, hi;          // row-major, sorted, -0 written as +0
    std::vector<int32_t> flags, depth;
    ivs_stats st{};
    int64_t depth_boxes[64] = {}, depth_kept[64] = {};   // per depth (the last slot: >= 63)
    int64_t depth_hs[64] = {};                             // boxes entering the contraction
};

namespace ivs {
namespace host {

// sorts rows given as column-major arrays (lo/hi: n columns of `total` entries) into
// r's row-major lexicographic order (lo_0, hi_0, lo_1, ...), -0 -> +0
void fill_sorted(ivs_result *r, int n, int64_t total, const std::vector<double> &lo, const std::vector<double> &hi,
                 const std::vector<int32_t> &flags, const std::vector<int32_t> &depth);

int fail(int status, const std::string &msg);   // records the thread's error text, returns status
void set_error_text(const char *msg);            // records the thread's error text (no allocation)
const char *last_error();

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ivs::host::fail(IVS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct HostTables {
    std::vector<DevSys> sys;
    std::vector<char> blobs;   // 16-byte aligned blobs (layout: ivs_tab.cuh)
};

// IVS_OK or IVS_ERR_INVALID (with the reason recorded)
int validate(const ivs_system *s, const double *lo, const double *hi, const ivs_options *o);
// appends the system's blob and DevSys (options folded in; shadow off)
void compile_system(HostTables &h, const ivs_system *s, const ivs_options *o);
// true when no FP32 shadow intermediate can overflow on this machine
bool shadow_safe(const ivs_system *s, const double *lo, const double *hi);

size_t align_up(size_t v, size_t a);
struct Layout {
    size_t queue, stage, surv, out, ctl, stats, roots, total;
};
Layout layout_for(int n_sys, int n_max, int64_t W, int64_t Q, int64_t O);
DevQueue carve_queue(char *base, int64_t cap, int n_max);
DevOut carve_out(char *base, int64_t cap, int n_max);

}  // namespace host
}  // namespace ivs
