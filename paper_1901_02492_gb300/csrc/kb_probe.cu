// Roofline denominator of the search: the L2-to-SM bandwidth of the search's own
// access form, measured on the device it runs on.
//
// For one (velocity, epoch) a warp of the search reads `warp_bytes` contiguous
// bytes (32 lanes x P loads of 8 bytes, lane-contiguous per load) starting at
// the shifted span's first pixel: an arbitrary multiple of 8 bytes, so a
// 256-byte load usually touches 9 sectors, not 8.  At full size most of these
// reads hit L2, few hit L1 and few go to HBM.  The probe issues exactly such
// reads over an L2-resident 64 MB buffer (smaller than the 129 MB L2, far larger
// than all L1s) from every SM, bypassing L1 (ld.global.cg), at offsets that are
// multiples of `align_bytes`, and reports the bytes delivered per second.
#include <cuda_runtime.h>

#include "kb_internal.h"

namespace {

template <int P>
__global__ void gather_peak_kernel(const float2 *__restrict__ buf, unsigned mask, unsigned align, int iters,
                                   float *sink) {
    const int lane = threadIdx.x & 31;
    unsigned w = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 977u;
    float acc = 0.0f;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
        // span start: a multiple of `align` elements (align a power of two)
        const unsigned off = ((w + (unsigned)it * 7919u) & mask & ~(align - 1u)) + lane;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float2 v = __ldcg(buf + off + 32 * p);
            acc += v.x + v.y;
        }
    }
    if (acc == 1234.5f) sink[0] = acc;   // keeps the loads; never true for a zero buffer
}

}  // namespace

extern "C" int kb_measure_gather_peak(kb_ctx *ctx, int warp_bytes, int align_bytes, double *gb_per_s) {
    if (!ctx || !gb_per_s) return KB_EINVAL;
    *gb_per_s = 0.0;
    if (warp_bytes != 256 && warp_bytes != 512 && warp_bytes != 1024) return KB_EINVAL;
    if (align_bytes < 8 || align_bytes > 4096 || (align_bytes & (align_bytes - 1))) return KB_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const size_t elems = (size_t)64 << 20 >> 3;   // 64 MB of float2
    const int P = warp_bytes / 256;
    // span starts in [0, elems / 2): every span of up to 128 float2 stays inside the buffer
    const unsigned mask = (unsigned)(elems / 2) - 1u;
    const unsigned align = (unsigned)(align_bytes / 8);
    float2 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, elems * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, elems * sizeof(float2));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int blocks = ctx->sm_count * 8, threads = 256, iters = 4096 / P;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first run warms L2
        cudaEventRecord(a);
        if (P == 1)
            gather_peak_kernel<1><<<blocks, threads>>>(buf, mask, align, iters, sink);
        else if (P == 2)
            gather_peak_kernel<2><<<blocks, threads>>>(buf, mask, align, iters, sink);
        else
            gather_peak_kernel<4><<<blocks, threads>>>(buf, mask, align, iters, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        const double bytes = (double)blocks * threads * iters * P * sizeof(float2);
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
