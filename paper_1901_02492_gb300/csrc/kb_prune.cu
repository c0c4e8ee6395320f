// Likelihood bound of a warp span for the thresholded search (Sec. 5.3, which
// plans to spend less time on low-likelihood trajectories).
//
// For one trajectory, over the epochs whose pixel is in the image, Cauchy-Schwarz
// gives Psi^2 = (sum_t psi_t)^2 <= (sum_t psi_t^2 / phi_t) (sum_t phi_t); an epoch
// with phi_t = 0 has psi_t = 0 (every weight of its PSF window is 0), and with
// Psi > 0 only the positive psi_t can raise it, so
//     nu^2 = Psi^2 / Phi <= sum_t max(psi_t, 0)^2 / phi_t,
// a sum of single-epoch SNRs squared.  This file builds, per epoch and row, the
// largest such term over every window of `span` columns (the pixels one warp of
// the search covers for one velocity and epoch):
//     R[e][y][x + span - 1] = max over x' in [x, x + span) of q_e(x', y),
//     q_e = max(psi, 0)^2 / phi  (0 where phi <= 0 or off the image),
// for x = -(span - 1) .. W - 1 (row pitch W + span - 1), from exactly the values
// the search sums (the FP32 planes, or the decoded 16-bit codes).  The search
// adds one R value per epoch at its shifted span; when the sum cannot reach
// nu_min^2, no pixel of the span can, and the span's gathers for that velocity
// are skipped.  q and the sums round upwards, so the bound stays a bound.
//
// Window maxima by the van Herk / Gil-Werman method: in blocks of `span` inputs
// a running maximum from each block's start (g) and from its end (h), and a
// window of `span` inputs [i, i + span) is max(h[i], g[i + span - 1]).
#include <cuda_runtime.h>
#include <math.h>

#include "kb_device.cuh"

namespace kb {

namespace {

using namespace dev;

constexpr int kTileOut = 2048;   // outputs (window positions) per CTA

template <int STORAGE>
__device__ __forceinline__ float snr2_of(const SnrArgs &a, int e, int y, int x) {
    if (x < 0 || x >= a.W) return 0.0f;
    const long long i = (long long)e * a.plane_elems + a.origin + (long long)y * a.pitch + x;
    float p, f;
    if constexpr (STORAGE == KB_F32) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(a.planes) + i);
        p = v.x;
        f = v.y;
    } else {
        // the decoded code, code * scale: exactly the value the search adds
        const float2 v = Store<STORAGE>::acc(make_float2(0.0f, 0.0f),
                                             __ldg(reinterpret_cast<const pair16 *>(a.planes) + i), a.scales[e]);
        p = v.x;
        f = v.y;
    }
    return (p > 0.0f && f > 0.0f) ? __fdiv_ru(__fmul_ru(p, p), f) : 0.0f;
}

template <int STORAGE>
__global__ void snr2_kernel(SnrArgs a) {
    extern __shared__ float sm[];
    const int span = a.span;
    const int e = blockIdx.z, y = blockIdx.y, X0 = blockIdx.x * kTileOut;
    const int RW = a.W + span - 1;
    // inputs of this tile: x = X0 - (span - 1) + li, li in [0, L), L a multiple of span
    const int L = (kTileOut + span - 1 + span - 1) / span * span;
    float *q = sm, *g = sm + L, *h = sm + 2 * L;
    const int xlo = X0 - (span - 1);
    for (int li = threadIdx.x; li < L; li += blockDim.x) q[li] = snr2_of<STORAGE>(a, e, y, xlo + li);
    __syncthreads();
    for (int b = threadIdx.x; b < L / span; b += blockDim.x) {
        const int s0 = b * span;
        float m = 0.0f;
        for (int i = 0; i < span; ++i) {
            m = fmaxf(m, q[s0 + i]);
            g[s0 + i] = m;
        }
        m = 0.0f;
        for (int i = span - 1; i >= 0; --i) {
            m = fmaxf(m, q[s0 + i]);
            h[s0 + i] = m;
        }
    }
    __syncthreads();
    float *out = a.out + ((long long)e * a.H + y) * RW;
    for (int lo = threadIdx.x; lo < kTileOut && X0 + lo < RW; lo += blockDim.x)
        out[X0 + lo] = fmaxf(h[lo], g[lo + span - 1]);
}

}  // namespace

cudaError_t launch_snr2(const SnrArgs &a, cudaStream_t st) {
    const int RW = a.W + a.span - 1;
    const dim3 grid((RW + kTileOut - 1) / kTileOut, a.H, a.N);
    const int L = (kTileOut + a.span - 1 + a.span - 1) / a.span * a.span;
    const size_t smem = (size_t)3 * L * sizeof(float);
    cudaError_t e;
    switch (a.storage) {
        case KB_F32:
            e = cudaFuncSetAttribute(snr2_kernel<KB_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_F32><<<grid, 256, smem, st>>>(a);
            break;
        case KB_BF16:
            e = cudaFuncSetAttribute(snr2_kernel<KB_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_BF16><<<grid, 256, smem, st>>>(a);
            break;
        case KB_F16:
            e = cudaFuncSetAttribute(snr2_kernel<KB_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_F16><<<grid, 256, smem, st>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace kb
