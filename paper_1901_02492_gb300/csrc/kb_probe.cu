// Roofline denominator of the search: the L2-to-SM bandwidth of the search's own
// access form, measured on the device it runs on.
//
// The search gathers 256-byte warp spans (32 lanes x 8 bytes) at scattered
// offsets; at full size most of them hit L2, few hit L1 and few go to HBM.  The
// probe streams exactly such spans over an L2-resident 64 MB buffer (smaller
// than the 129 MB L2, far larger than all L1s) from every SM, bypassing L1
// (ld.global.cg), and reports the bytes delivered per second.
#include <cuda_runtime.h>

#include "kb_internal.h"

namespace {

__global__ void gather_peak_kernel(const float2 *__restrict__ buf, unsigned mask, int iters, float *sink) {
    const int lane = threadIdx.x & 31;
    unsigned w = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 977u;
    float acc = 0.0f;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
        const unsigned off = ((w + (unsigned)it * 7919u) & mask) + lane;
        const float2 v = __ldcg(buf + off);
        acc += v.x + v.y;
    }
    if (acc == 1234.5f) sink[0] = acc;   // keeps the loads; never true for a zero buffer
}

}  // namespace

extern "C" int kb_measure_gather_peak(kb_ctx *ctx, double *gb_per_s) {
    if (!ctx || !gb_per_s) return KB_EINVAL;
    *gb_per_s = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const size_t elems = (size_t)64 << 20 >> 3;   // 64 MB of float2
    float2 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, elems * sizeof(float2) + 4096);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, elems * sizeof(float2) + 4096);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int blocks = ctx->sm_count * 8, threads = 256, iters = 4096;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first run warms L2
        cudaEventRecord(a);
        gather_peak_kernel<<<blocks, threads>>>(buf, (unsigned)(elems - 64) & ~31u, iters, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        const double bytes = (double)blocks * threads * iters * sizeof(float2);
        *gb_per_s = bytes / (best * 1e-3) / 1e9;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(sink);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        ctx->err = std::string("kb_measure_gather_peak: ") + cudaGetErrorString(e);
        return KB_ECUDA;
    }
    return KB_OK;
}
