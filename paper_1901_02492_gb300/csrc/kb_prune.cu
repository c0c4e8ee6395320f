// Likelihood bound of a warp span for the thresholded search (Sec. 5.3, which
// plans to spend less time on low-likelihood trajectories).
//
// For one trajectory, over the epochs whose pixel is in the image, Cauchy-Schwarz
// gives Psi^2 = (sum_t psi_t)^2 <= (sum_t psi_t^2 / phi_t) (sum_t phi_t); an epoch
// with phi_t = 0 has psi_t = 0 (every weight of its PSF window is 0), and with
// Psi > 0 only the positive psi_t can raise it, so
//     nu^2 = Psi^2 / Phi <= sum_t max(psi_t, 0)^2 / phi_t,
// a sum of single-epoch SNRs squared.  A warp of the search covers `span`
// consecutive start pixels of one row for one velocity; shifted by an epoch's
// offset they read the columns [x, x + span).  Those columns lie inside the
// window [32 c, 32 c + span + 32) with c = floor(x / 32), so this file stores,
// per epoch and row, the largest such term over each of those windows:
//     R[e][y][c + span / 32] = max over x' in [32 c, 32 c + span + 32) of q_e(x', y),
//     q_e = max(psi, 0)^2 / phi  (0 where phi <= 0 or off the image),
// for c = -span / 32 .. floor((W - 1) / 32), from exactly the values the search
// sums (the FP32 planes, or the decoded 16-bit codes).  Aligned 32-column blocks
// make the planes 32 times smaller than one entry per column (26 MB for twelve
// 4096^2 epochs: they stay in L2), for a window 32 columns wider than the span.
// The search adds one R value per epoch at its shifted span; when the sum cannot
// reach nu_min^2, no pixel of the span can, and the span's gathers for that
// velocity are skipped.  q and the sums round upwards, so the bound stays a bound.
#include <cuda_runtime.h>
#include <math.h>

#include "kb_device.cuh"

namespace kb {

namespace {

using namespace dev;

constexpr int kThreads = 128;

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

// One CTA per (row, epoch): block maxima of q over 32 columns (one warp load per
// block, a warp max), then each output the maximum of span / 32 + 1 consecutive
// blocks.  q >= 0, so float bit patterns order like the floats.
template <int STORAGE>
__global__ void __launch_bounds__(kThreads) snr2_kernel(SnrArgs a) {
    extern __shared__ float blk[];
    const int e = blockIdx.y, y = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nblk = (a.W + 31) / 32, nb = a.span / 32;
    for (int c = warp; c < nblk; c += kThreads / 32) {
        const float q = snr2_of<STORAGE>(a, e, y, 32 * c + lane);
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(q));
        if (lane == 0) blk[c] = __uint_as_float(m);
    }
    __syncthreads();
    const int RWc = nblk + nb;
    float *out = a.out + ((long long)e * a.H + y) * RWc;
    for (int o = threadIdx.x; o < RWc; o += kThreads) {
        const int c = o - nb;   // the window's first block
        float m = 0.0f;
        for (int i = 0; i <= nb; ++i) {
            const int b = c + i;
            if (b >= 0 && b < nblk) m = fmaxf(m, blk[b]);
        }
        out[o] = m;
    }
}

}  // namespace

cudaError_t launch_snr2(const SnrArgs &a, cudaStream_t st) {
    if (a.span % 32 != 0) return cudaErrorInvalidValue;
    const dim3 grid(a.H, a.N);
    const size_t smem = (size_t)((a.W + 31) / 32) * sizeof(float);
    cudaError_t e;
    switch (a.storage) {
        case KB_F32:
            e = cudaFuncSetAttribute(snr2_kernel<KB_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_F32><<<grid, kThreads, smem, st>>>(a);
            break;
        case KB_BF16:
            e = cudaFuncSetAttribute(snr2_kernel<KB_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_BF16><<<grid, kThreads, smem, st>>>(a);
            break;
        case KB_F16:
            e = cudaFuncSetAttribute(snr2_kernel<KB_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) snr2_kernel<KB_F16><<<grid, kThreads, smem, st>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace kb
