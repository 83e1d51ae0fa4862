// ivs_kernels.cuh -- kernels of one sweep over the device queue, and their launchers.
//
// One sweep ("wave") pops up to K parent boxes from the top of the queue and runs:
//   k_wave_begin  : chooses K so that the worst case (every child kept) fits
//   k_eval        : one warp per parent, one lane per child box (Algorithm 2's split is
//                   implicit: child c takes the upper half of coordinate j when bit j of
//                   c is set); optional FP32 outward evaluation, then FP64 evaluation
//                   (Definition 1-2); survivors compacted with a warp ballot into a list
//                   per dimension n
//   k_hs<N>       : 32 survivors per block (narrow sweeps: per cluster of 4 blocks,
//   k_hs_coop<N>    k_hs_coop): Hansen-Sengupta sweeps (Algorithm 3) or Krawczyk steps
//                   (eq 15-16), then accept (Algorithm 1 (II)) or write the box as a
//                   new parent
//   k_commit      : moves the new parents onto the queue where the popped ones were
#pragma once
#include <cuda_runtime.h>

#include "ivs_internal.h"

namespace ivs {

struct SweepArgs {
    DevTables tb;
    DevQueue q;        // the queue
    DevQueue stage;    // new parents of this sweep
    DevOut out;
    WaveCtl *ctl;
    Surv *surv;        // survivor list of dimension n at surv + n * surv_cap
    int64_t surv_cap;
    Surv *cand;        // FP32 survivors (capacity surv_cap)
    unsigned long long *stats;   // [n_sys][ST_COUNT]
    int64_t wave_children;       // children a sweep may evaluate
    int32_t max_fan_shift;       // max n over the plan's systems
    int32_t n_sys;
    int32_t single;              // 1: one system; kernels cache its blob in shared memory
    int32_t blob_smem;           // bytes of that blob
    int32_t tv_stride;           // term-combination entries per warp region (0: no tables)
    int32_t eval_warps;          // warps per block of k_eval
    DevRegions rg;               // serving: per-system queue regions (rg.n == 0: shared stack)
};

// dynamic shared memory of k_eval (blob cache + the warps' combination tables) and the
// kernels' limits; tv_stride / eval_warps come from choose_eval_layout
size_t eval_smem_bytes(const SweepArgs &a);
cudaError_t configure_eval_kernels(const SweepArgs &a);
// raises a kernel's dynamic shared memory limit to the device maximum (idempotent)
cudaError_t allow_max_dynamic_smem(const void *func);
// picks eval_warps and tv_stride for the largest table `max_tv` of the plan's systems
inline void choose_eval_layout(SweepArgs &a, int max_tv) {
    const size_t budget = 200 * 1024 - (size_t)(a.single ? a.blob_smem : 0);
    int warps = 8;
    while (warps > 1 && (size_t)warps * (size_t)max_tv * 16 > budget) warps--;
    a.eval_warps = warps;
    a.tv_stride = ((size_t)max_tv * 16 <= budget) ? max_tv : 0;
}
// one sweep; ev (nullable) receives n_hs_dims + 5 stage events; *kernels (nullable) the
// number of kernels launched
cudaError_t launch_sweep(const SweepArgs &a, const int *hs_dims, int n_hs_dims, int eval_blocks,
                         int eval_threads, int num_sms, cudaStream_t st, cudaEvent_t *ev, int *kernels = nullptr);
// The sweep loop as one CUDA graph: a conditional WHILE node whose body is one sweep; its
// commit kernel keeps the condition set while the queue is non-empty, no error occurred
// and ctl->waves < ctl->wave_limit.  Kernels per iteration: 4 + n_hs_dims.
cudaError_t build_sweep_graph(const SweepArgs &a, const int *hs_dims, int n_hs_dims, int eval_blocks,
                              int eval_threads, int num_sms, cudaGraph_t *out, int *kernels_per_sweep = nullptr);
// directed-rounding rate microbenchmark (kind 0 FP64, 1 FP32); returns ops and fills ms
cudaError_t run_probe(int kind, int num_sms, double *ops, float *ms);
cudaError_t launch_seed_roots(const SweepArgs &a, const double *d_box_lo, const double *d_box_hi,
                              const int32_t *d_root_depth, int n_sys, int n_max, cudaStream_t st);
// serving with regions: empties the regions of the slots with d_cancel[s] != 0 (between
// sweeps) and lowers the queue total accordingly
cudaError_t launch_cancel_regions(const SweepArgs &a, const int32_t *d_cancel, cudaStream_t st);
// appends initial boxes of newly admitted systems (slot ids) on top of the queue, or at
// the start of each system's region
cudaError_t launch_admit(const SweepArgs &a, const double *d_lo, const double *d_hi, const int32_t *d_slot,
                         const int32_t *d_depth, int count, int n_max, cudaStream_t st);
// Hansen-Sengupta + accept/split kernels for dimension n (ivs_hs_*.cu); *kernels receives
// how many kernels the call launched (1, or 2 with the cooperative form)
cudaError_t launch_hs_dim1(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim2(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim3(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim4(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim5(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim6(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim7(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim8(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim9(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim10(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim11(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim12(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim13(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim14(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim15(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);
cudaError_t launch_hs_dim16(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels);

}  // namespace ivs
