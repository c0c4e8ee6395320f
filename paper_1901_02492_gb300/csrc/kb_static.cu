// kb_make_psi_phi_static: the likelihood images without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// psi/phi planes: code whose device memory is owned by another allocator (a
// framework's caching pool that must see every allocation), real-time loops in
// which cudaMalloc/cudaFree are not allowed because they can block or
// synchronise the device, or hosts with a fixed memory plan.  They bring their
// own input and output buffers; the only other memory the psi/phi kernel needs
// is a small table of per-epoch PSF taps, which here lives in a file-scope
// static device array instead of a buffer of a kb_stack.
//
// The array is part of the module image: every GPU that loads this library
// holds it (kStaticTapFloats floats = 256 KB) until the process exits, and all
// calls share it.  A call overwrites the part it uses before its kernel runs,
// so nothing in it has to start at zero; calls that overlap on the GPU (for
// example on two streams) race on it and must be ordered by the caller.
//
// The taps reach the array through a host staging buffer that every call
// rewrites, so a call on a stream that is being captured into a CUDA graph is
// refused (KB_EINVAL): a captured copy would read that buffer when the graph is
// replayed, by then holding another call's taps.  The array's device address is
// looked up on every call (cudaGetSymbolAddress allocates nothing and is cheap),
// so it stays right when the device's context is destroyed and created again
// and the module is loaded at another address.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "kb_internal.h"

namespace {

constexpr size_t kStaticTapFloats = 65536;   // 256 KB of PSF taps

// the scratch: per-epoch taps in the layout documented in kb_psiphi.cu
static __device__ __align__(256) float g_static_taps[kStaticTapFloats];

std::mutex g_mu;
float g_taps_host[kStaticTapFloats];     // host staging of one call's taps (guarded by g_mu)

bool is_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int kb_make_psi_phi_static(const float *sci, const float *var, const uint8_t *mask, const float *psf,
                                      int N, int H, int W, int K, float bright_max, float *out, void *stream) {
    kb::NvtxRange nvtx("kb_make_psi_phi_static");
    cudaStream_t st = (cudaStream_t)stream;
    // first, before any other CUDA call: a capturing stream is refused (see above)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return KB_EINVAL;
    }
    if (cap != cudaStreamCaptureStatusNone) return KB_EINVAL;
    if (!sci || !var || !psf || !out) return KB_EINVAL;
    if (N < 1 || N > KB_MAX_EPOCHS || H < 1 || W < 1 || H > KB_MAX_SIDE || W > KB_MAX_SIDE) return KB_EINVAL;
    if (K < 1 || K > KB_MAX_PSF || (K % 2) == 0) return KB_EINVAL;
    for (size_t i = 0; i < (size_t)N * K * K; ++i)
        if (!std::isfinite(psf[i])) return KB_EINVAL;
    if (!is_device(sci) || !is_device(var) || !is_device(out) || (mask && !is_device(mask))) return KB_EINVAL;

    // separable PSFs for every epoch take the two-pass kernel, as in kb_make_psi_phi
    bool sep = true;
    std::vector<std::vector<double>> fa(N), fb(N);
    for (int e = 0; e < N && sep; ++e) sep = kb::factor_psf(psf + (size_t)e * K * K, K, fa[e], fb[e]);
    const size_t nt = kb::taps_floats(N, K, sep);
    if (nt > kStaticTapFloats) return KB_EINVAL;   // more taps than the static scratch holds

    std::lock_guard<std::mutex> lock(g_mu);
    // the device address of the array on the current device (the host-side name
    // g_static_taps is only a stand-in, not an address a kernel may use)
    float *taps_dev = nullptr;
    if (cudaGetSymbolAddress((void **)&taps_dev, g_static_taps) != cudaSuccess || !taps_dev) {
        cudaGetLastError();
        return KB_ECUDA;
    }
    for (int e = 0; e < N; ++e) {
        const float *T = psf + (size_t)e * K * K;
        if (sep) {
            float *o = g_taps_host + (size_t)e * 4 * K;
            for (int i = 0; i < K; ++i) {
                o[2 * i] = (float)fa[e][i];
                o[2 * i + 1] = (float)(fa[e][i] * fa[e][i]);
                o[2 * K + 2 * i] = (float)fb[e][i];
                o[2 * K + 2 * i + 1] = (float)(fb[e][i] * fb[e][i]);
            }
        } else {
            float *o = g_taps_host + (size_t)e * 2 * K * K;
            for (int i = 0; i < K * K; ++i) {
                o[2 * i] = T[i];
                o[2 * i + 1] = (float)((double)T[i] * (double)T[i]);
            }
        }
    }
    // from pageable memory: the staging is consumed before this call returns
    if (cudaMemcpyAsync(taps_dev, g_taps_host, nt * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return KB_ECUDA;

    kb::PsiPhiArgs a;
    a.sci = sci;
    a.var = var;
    a.mask = mask;
    a.bright_max = std::isnan(bright_max) ? INFINITY : bright_max;
    a.N = N;
    a.H = H;
    a.W = W;
    a.pitch = W;                          // the caller's plain [N][H][W] layout
    a.plane_elems = (long long)H * W;
    a.origin = 0;
    a.K = K;
    a.separable = sep;
    a.taps = taps_dev;
    a.out = reinterpret_cast<float2 *>(out);
    a.maxbits = nullptr;
    return kb::launch_psi_phi(a, st) == cudaSuccess ? KB_OK : KB_ECUDA;
}
