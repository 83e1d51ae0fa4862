// ivs_probe.cu -- directed-rounding arithmetic rate of the device.  The roofline of the
// solver's kernels is the FP64 (or FP32) pipe, and its rate is measured here rather than
// taken from a datasheet: each thread runs 8 independent chains alternating a
// round-down add and a round-up multiply, so the pipe, not latency, bounds the loop.
#include <cuda_runtime.h>

#include "ivs_kernels.cuh"

namespace ivs {

constexpr int kProbeIters = 4096;
constexpr int kProbeChains = 8;

__global__ void k_probe_fp64(double seed, double *sink, int active_lanes) {
    if ((int)(threadIdx.x & 31u) >= active_lanes) return;
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = seed + c * 1e-3 + threadIdx.x * 1e-9;
    const double a = 1.0000000001, b = 1e-12;
    for (int i = 0; i < kProbeIters; i++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++) x[c] = __dmul_ru(__dadd_rd(x[c], b), a);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) s += x[c];
    if (s == 12345.678) sink[0] = s;   // never true; keeps the chains live
}

__global__ void k_probe_fp32(float seed, float *sink) {
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = seed + c * 1e-3f + threadIdx.x * 1e-7f;
    const float a = 1.0000001f, b = 1e-7f;
    for (int i = 0; i < kProbeIters; i++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++) x[c] = __fmul_ru(__fadd_rd(x[c], b), a);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) s += x[c];
    if (s == 12345.678f) sink[0] = s;
}

// directed (kind 4: alternating __ddiv_rd / __ddiv_ru) or round-to-nearest (kind 5)
// FP64 division, the same 8 independent chains per thread; values stay near 1
__global__ void k_probe_div(double seed, double *sink, int directed) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = seed + c * 1e-3 + threadIdx.x * 1e-9;
    const double a = 1.0000000001, b = 0.9999999999;
    for (int i = 0; i < kProbeIters / 8; i++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++)
            x[c] = directed ? __ddiv_ru(__ddiv_rd(x[c], a), b) : __ddiv_rn(__ddiv_rn(x[c], a), b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) s += x[c];
    if (s == 12345.678) sink[0] = s;
}

cudaError_t run_probe(int kind, int num_sms, double *ops, float *ms) {
    void *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int threads = 256, blocks = num_sms * 8;
    for (int rep = 0; rep < 3; rep++) {   // first launches warm up clocks and caches
        cudaEventRecord(a);
        if (kind == 0) k_probe_fp64<<<blocks, threads>>>(1.0, (double *)sink, 32);
        else if (kind == 4 || kind == 5) k_probe_div<<<blocks, threads>>>(1.0, (double *)sink, kind == 4);
        else if (kind >= 2) k_probe_fp64<<<blocks, threads>>>(1.0, (double *)sink, kind == 2 ? 8 : 1);
        else k_probe_fp32<<<blocks, threads>>>(1.0f, (float *)sink);
        cudaEventRecord(b);
    }
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    const int lanes = kind == 2 ? 8 : kind == 3 ? 1 : 32;
    *ops = (double)blocks * (threads / 32) * lanes * (kind >= 4 ? kProbeIters / 8 : kProbeIters) * kProbeChains * 2.0;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e;
}

}  // namespace ivs
