// Host side of the C ABI declared in include/kb.h: argument checks, device
// memory and HBM-budget accounting, PSF analysis, the fixed-point trajectory
// offset table, and the launches of the stage (a) / stage (b) kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "kb_internal.h"

namespace {

// Sets the context's device for the duration of a call, restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(kb_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_fail(kb_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, KB_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// Device allocation under the context's HBM budget.
int dev_alloc(kb_ctx *ctx, size_t bytes, void **p, size_t *acct) {
    *p = nullptr;
    if (bytes == 0) return KB_OK;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->budget && ctx->in_use + bytes > ctx->budget)
            return fail(ctx, KB_ENOMEM, "HBM budget exceeded: %zu in use + %zu requested > %zu", ctx->in_use, bytes,
                        ctx->budget);
        ctx->in_use += bytes;
    }
    // from the context's pool, ordered on its internal stream; synchronising that
    // stream (not the device) makes the block usable from any stream
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->astream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->astream);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->in_use -= bytes;
        cudaGetLastError();
        if (*p) cudaFreeAsync(*p, ctx->astream);
        *p = nullptr;
        return fail(ctx, KB_ENOMEM, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    *acct += bytes;
    return KB_OK;
}

// Returns a block to the pool in the internal stream's order.  The caller has
// made that stream wait for the last work that used the block.
void dev_free(kb_ctx *ctx, void *p) {
    if (p) cudaFreeAsync(p, ctx->astream);
}

// Pinned host staging: reuse a cached block of at least `bytes`, else allocate.
cudaError_t host_alloc(kb_ctx *ctx, size_t bytes, void **p, size_t *cap) {
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        int best = -1;
        for (int i = 0; i < (int)ctx->host_cache.size(); ++i)
            if (ctx->host_cache[i].second >= bytes &&
                (best < 0 || ctx->host_cache[i].second < ctx->host_cache[best].second))
                best = i;
        if (best >= 0) {
            *p = ctx->host_cache[best].first;
            *cap = ctx->host_cache[best].second;
            ctx->host_cached -= *cap;
            ctx->host_cache.erase(ctx->host_cache.begin() + best);
            return cudaSuccess;
        }
    }
    *cap = bytes;
    return cudaMallocHost(p, bytes);
}

// Keeps up to 1 GiB of released staging for reuse (cudaFreeHost can stall the device).
void host_release(kb_ctx *ctx, void *p, size_t cap) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->host_cached + cap <= ((size_t)1 << 30)) {
            ctx->host_cache.emplace_back(p, cap);
            ctx->host_cached += cap;
            return;
        }
    }
    cudaFreeHost(p);
}

void dev_release(kb_ctx *ctx, size_t bytes) {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->in_use -= std::min(ctx->in_use, bytes);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}


// ---- fixed-point trajectory offsets (see include/kb.h) ----------------------
constexpr int64_t kVelOne = 1LL << 16;    // v_q units per px/day
constexpr int64_t kTimeOne = 1LL << 20;   // t_q units per day
constexpr int64_t kVelMax = 1LL << 28;    // |v| < 2^12 px/day
constexpr int64_t kTimeMax = 1LL << 26;   // t - t_min < 2^6 days

// floor((vq * tq + 2^35) / 2^36): round half up of v t, exact in 64-bit integers
inline int64_t offset_q(int64_t vq, int64_t tq) {
    int64_t num = vq * tq + (1LL << 35);
    int64_t q = num / (1LL << 36);           // truncates toward zero
    if ((num % (1LL << 36)) < 0) q -= 1;     // floor for negative remainders
    return q;
}

struct Plan {
    std::vector<int> epoch_of;   // time-order position -> epoch
    std::vector<int64_t> tq;     // per time-order position
    int n0 = 0;                  // leading positions with tq == 0
};

int plan_times(kb_ctx *ctx, const double *times, int N, Plan &pl) {
    for (int e = 0; e < N; ++e)
        if (!std::isfinite(times[e])) return fail(ctx, KB_EINVAL, "times[%d] is not finite", e);
    double tmin = *std::min_element(times, times + N);
    pl.epoch_of.resize(N);
    std::iota(pl.epoch_of.begin(), pl.epoch_of.end(), 0);
    std::stable_sort(pl.epoch_of.begin(), pl.epoch_of.end(), [&](int a, int b) { return times[a] < times[b]; });
    pl.tq.resize(N);
    pl.n0 = 0;
    for (int j = 0; j < N; ++j) {
        double dt = times[pl.epoch_of[j]] - tmin;
        if (!(dt * (double)kTimeOne < (double)kTimeMax))
            return fail(ctx, KB_EINVAL, "epoch span %.6g days exceeds the supported 64 days", dt);
        pl.tq[j] = llround(dt * (double)kTimeOne);
        if (pl.tq[j] == 0 && pl.n0 == j) pl.n0 = j + 1;
    }
    return KB_OK;
}

int quant_velocity(kb_ctx *ctx, double v, int64_t *q) {
    if (!std::isfinite(v) || !(fabs(v) * (double)kVelOne < (double)kVelMax))
        return fail(ctx, KB_EINVAL, "velocity %.6g px/day outside the supported |v| < 4096", v);
    *q = llround(v * (double)kVelOne);
    return KB_OK;
}

}  // namespace

namespace kb {
// ---- PSF analysis ------------------------------------------------------------
// A K x K kernel is separable when T(i, j) = a(i) b(j); the factors are read off
// the row and column through the largest tap and checked against every tap.
bool factor_psf(const float *T, int K, std::vector<double> &a, std::vector<double> &b) {
    int bi = 0, bj = 0;
    double best = 0.0;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j)
            if (fabs((double)T[i * K + j]) > best) {
                best = fabs((double)T[i * K + j]);
                bi = i;
                bj = j;
            }
    a.assign(K, 0.0);
    b.assign(K, 0.0);
    if (best == 0.0) return true;   // all-zero kernel: any factors of zero
    double piv = (double)T[bi * K + bj];
    for (int i = 0; i < K; ++i) a[i] = (double)T[i * K + bj];
    for (int j = 0; j < K; ++j) b[j] = (double)T[bi * K + j] / piv;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j)
            if (fabs(a[i] * b[j] - (double)T[i * K + j]) > 1e-6 * best) return false;
    return true;
}
}  // namespace kb

// =============================================================================
extern "C" {

int kb_init(kb_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return KB_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return KB_EINVAL;
    }
    kb_ctx *ctx = new kb_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete ctx;
        return KB_ECUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    e = cudaMemPoolCreate(&ctx->pool, &pp);
    if (e == cudaSuccess) {
        // freed blocks stay in the pool until the context is destroyed
        uint64_t keep = ~0ULL;
        e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->astream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        kb_destroy(ctx);
        return KB_ECUDA;
    }
    *out = ctx;
    return KB_OK;
}

void kb_destroy(kb_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->astream) {
        cudaStreamSynchronize(ctx->astream);
        cudaStreamDestroy(ctx->astream);
    }
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    for (auto &b : ctx->host_cache) cudaFreeHost(b.first);
    delete ctx;
}

const char *kb_last_error(const kb_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t kb_hbm_in_use(const kb_ctx *ctx) { return ctx ? ctx->in_use : 0; }

int kb_set_search_order(kb_ctx *ctx, int order) {
    if (!ctx) return KB_EINVAL;
    if (order < -1 || order > 2) return fail(ctx, KB_EINVAL, "order %d not in -1..2", order);
    ctx->search_order = order;
    return KB_OK;
}

int kb_set_search_swizzle(kb_ctx *ctx, int cols) {
    if (!ctx) return KB_EINVAL;
    if (cols < -1 || cols > 65535) return fail(ctx, KB_EINVAL, "swizzle %d not in -1..65535", cols);
    ctx->search_swizzle = cols;
    return KB_OK;
}

int kb_set_search_carveout(kb_ctx *ctx, int percent) {
    if (!ctx) return KB_EINVAL;
    if (percent < -1 || percent > 100) return fail(ctx, KB_EINVAL, "carveout %d not in -1..100", percent);
    ctx->search_carveout = percent;
    return KB_OK;
}

int kb_set_search_variant(kb_ctx *ctx, int variant) {
    if (!ctx) return KB_EINVAL;
    if (variant < 0 || variant > 8) return fail(ctx, KB_EINVAL, "search variant %d not in 0..8", variant);
    ctx->search_variant = variant;
    return KB_OK;
}

int kb_debug_build(void) {
#ifdef KB_DEBUG
    return 1;
#else
    return 0;
#endif
}

int kb_debug_word(kb_ctx *ctx, unsigned long long *word, int reset) {
    if (!ctx || !word) return fail(ctx, KB_EINVAL, "kb_debug_word: null argument");
    DeviceGuard g(ctx->device);
    cudaError_t e = kb::debug_word(word, reset != 0);
    if (e == cudaErrorNotSupported) return fail(ctx, KB_EINVAL, "kb_debug_word: not a KB_DEBUG build");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_debug_word");
    return KB_OK;
}

// ---- stacks ------------------------------------------------------------------

int kb_stack_create(kb_ctx *ctx, int N, int H, int W, int storage, kb_stack **out) {
    if (!ctx || !out) return KB_EINVAL;
    *out = nullptr;
    if (N < 1 || N > KB_MAX_EPOCHS || H < 1 || W < 1 || H > KB_MAX_SIDE || W > KB_MAX_SIDE)
        return fail(ctx, KB_EINVAL, "stack shape N=%d H=%d W=%d outside 1..%d x 1..%d x 1..%d", N, H, W,
                    KB_MAX_EPOCHS, KB_MAX_SIDE, KB_MAX_SIDE);
    if (storage != KB_F32 && storage != KB_BF16 && storage != KB_F16)
        return fail(ctx, KB_EINVAL, "unknown storage %d", storage);
    DeviceGuard g(ctx->device);
    kb_stack *s = new kb_stack();
    s->ctx = ctx;
    s->N = N;
    s->H = H;
    s->W = W;
    s->L = kb::make_layout(H, W);
    s->storage = storage;
    size_t plane = (size_t)s->L.plane_elems;
    int rc = dev_alloc(ctx, (size_t)N * plane * sizeof(float2), (void **)&s->f32, &s->bytes);
    if (rc == KB_OK && storage != KB_F32)
        rc = dev_alloc(ctx, (size_t)2 * N * plane * sizeof(kb::pair16), (void **)&s->q16, &s->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)N * sizeof(float2), (void **)&s->scales, &s->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)2 * N * sizeof(unsigned), (void **)&s->maxbits, &s->bytes);
    // The planes are cleared by the first kb_make_psi_phi, on its stream: a memset
    // here would run on the library's internal stream and queue behind whatever
    // kernels other streams have on the device.
    cudaError_t e = cudaSuccess;
    if (rc == KB_OK) e = cudaEventCreateWithFlags(&s->taps_done, cudaEventDisableTiming);
    if (rc == KB_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&s->used, cudaEventDisableTiming);
    if (rc == KB_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "kb_stack_create");
    if (rc != KB_OK) {
        kb_stack_free(s);
        return rc;
    }
    *out = s;
    return KB_OK;
}

void kb_stack_free(kb_stack *s) {
    if (!s) return;
    DeviceGuard g(s->ctx->device);
    kb_ctx *ctx = s->ctx;
    if (s->taps_done) {
        cudaEventSynchronize(s->taps_done);
        cudaStreamWaitEvent(ctx->astream, s->taps_done, 0);
        cudaEventDestroy(s->taps_done);
    }
    if (s->used) {
        cudaStreamWaitEvent(ctx->astream, s->used, 0);   // the last search that read the planes
        cudaEventDestroy(s->used);
    }
    dev_free(ctx, s->f32);
    dev_free(ctx, s->q16);
    dev_free(ctx, s->scales);
    dev_free(ctx, s->maxbits);
    dev_free(ctx, s->snr2);
    dev_free(ctx, s->taps);
    host_release(ctx, s->taps_host, s->taps_host_cap);
    dev_release(ctx, s->bytes);
    delete s;
}

int kb_make_psi_phi(kb_stack *s, const float *sci, const float *var, const uint8_t *mask, const float *psf, int K,
                    float bright_max, void *stream) {
    kb::NvtxRange nvtx("kb_make_psi_phi");
    if (!s) return KB_EINVAL;
    kb_ctx *ctx = s->ctx;
    if (!sci || !var || !psf) return fail(ctx, KB_EINVAL, "kb_make_psi_phi: sci, var and psf are required");
    if (K < 1 || K > KB_MAX_PSF || (K % 2) == 0)
        return fail(ctx, KB_EINVAL, "PSF size K=%d must be odd and in 1..%d", K, KB_MAX_PSF);
    DeviceGuard g(ctx->device);
    if (!is_device_ptr(sci) || !is_device_ptr(var) || (mask && !is_device_ptr(mask)))
        return fail(ctx, KB_EINVAL, "kb_make_psi_phi: sci, var and mask must be device pointers");
    const int N = s->N;
    for (size_t i = 0; i < (size_t)N * K * K; ++i)
        if (!std::isfinite(psf[i])) return fail(ctx, KB_EINVAL, "psf[%zu] is not finite", i);
    cudaStream_t st = (cudaStream_t)stream;

    // analyse the PSFs: separable for every epoch -> two-pass kernel
    bool sep = true;
    std::vector<std::vector<double>> fa(N), fb(N);
    for (int e = 0; e < N && sep; ++e) sep = kb::factor_psf(psf + (size_t)e * K * K, K, fa[e], fb[e]);
    size_t nt = kb::taps_floats(N, K, sep);
    if (nt > s->taps_floats) {
        if (s->taps_done) {
            cudaEventSynchronize(s->taps_done);
            cudaStreamWaitEvent(ctx->astream, s->taps_done, 0);
        }
        dev_free(ctx, s->taps);
        host_release(ctx, s->taps_host, s->taps_host_cap);
        dev_release(ctx, s->taps_floats * sizeof(float));
        s->bytes -= std::min(s->bytes, s->taps_floats * sizeof(float));
        s->taps = nullptr;
        s->taps_host = nullptr;
        s->taps_floats = 0;
        int rc = dev_alloc(ctx, nt * sizeof(float), (void **)&s->taps, &s->bytes);
        if (rc != KB_OK) return rc;
        cudaError_t e = host_alloc(ctx, nt * sizeof(float), (void **)&s->taps_host, &s->taps_host_cap);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocHost(taps)");
        s->taps_floats = nt;
    } else {
        cudaEventSynchronize(s->taps_done);   // previous upload finished reading the staging
    }
    float *th = s->taps_host;
    for (int e = 0; e < N; ++e) {
        const float *T = psf + (size_t)e * K * K;
        if (sep) {
            float *o = th + (size_t)e * 4 * K;
            for (int i = 0; i < K; ++i) {
                o[2 * i] = (float)fa[e][i];
                o[2 * i + 1] = (float)(fa[e][i] * fa[e][i]);
                o[2 * K + 2 * i] = (float)fb[e][i];
                o[2 * K + 2 * i + 1] = (float)(fb[e][i] * fb[e][i]);
            }
        } else {
            float *o = th + (size_t)e * 2 * K * K;
            for (int i = 0; i < K * K; ++i) {
                o[2 * i] = T[i];
                o[2 * i + 1] = (float)((double)T[i] * (double)T[i]);
            }
        }
    }
    cudaError_t e = cudaSuccess;
    if (!s->zeroed) {
        // once per stack: the zero borders (psi/phi only write the image's pixels); the
        // 16-bit copies are written whole by the quantize kernel
        e = cudaMemsetAsync(s->f32, 0, (size_t)N * s->L.plane_elems * sizeof(float2), st);
        if (e == cudaSuccess) s->zeroed = true;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->taps, th, nt * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->taps_done, st);
    bool q = s->q16 != nullptr;
    // per-epoch maxima: the 16-bit scales and the binary points of the exact rescoring sums
    if (e == cudaSuccess) e = cudaMemsetAsync(s->maxbits, 0, 2 * N * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_make_psi_phi upload");

    kb::PsiPhiArgs a;
    a.sci = sci;
    a.var = var;
    a.mask = mask;
    a.bright_max = std::isnan(bright_max) ? INFINITY : bright_max;
    a.N = N;
    a.H = s->H;
    a.W = s->W;
    a.pitch = s->L.pitch;
    a.plane_elems = s->L.plane_elems;
    a.origin = s->L.origin;
    a.K = K;
    a.separable = sep;
    a.taps = s->taps;
    a.out = s->f32;
    a.maxbits = s->maxbits;
    e = kb::launch_psi_phi(a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "psi/phi kernel");
    if (q) {
        e = kb::launch_quantize(s->f32, s->q16, s->scales, s->maxbits, N, s->L.plane_elems, s->storage, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "quantize kernel");
    }
    e = cudaEventRecord(s->used, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_make_psi_phi");
    s->filled = true;
    s->snr2_valid = false;   // the bound planes follow the psi/phi planes
    return KB_OK;
}

int kb_stack_copy_planes(const kb_stack *s, int which, void *dst, size_t dst_bytes, void *stream) {
    if (!s) return KB_EINVAL;
    kb_ctx *ctx = s->ctx;
    if (!dst) return fail(ctx, KB_EINVAL, "kb_stack_copy_planes: dst is NULL");
    if (!s->filled) return fail(ctx, KB_EINVAL, "kb_stack_copy_planes: the stack has no psi/phi yet");
    if (which == 2) {
        // the span bound planes of KB_PRUNE, as built (contiguous [N][H][(W + 31) / 32 + span / 32])
        if (!s->snr2 || !s->snr2_valid) return fail(ctx, KB_EINVAL, "the stack has no span bound planes");
        if (dst_bytes < s->snr2_bytes) return fail(ctx, KB_EINVAL, "dst_bytes %zu < %zu", dst_bytes, s->snr2_bytes);
        DeviceGuard g(ctx->device);
        cudaStream_t st = (cudaStream_t)stream;
        const bool dev = is_device_ptr(dst);
        cudaError_t e = cudaMemcpyAsync(dst, s->snr2, s->snr2_bytes, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaEventRecord(s->used, st);
        if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_stack_copy_planes");
        return KB_OK;
    }
    const void *src = which == 0 ? (const void *)s->f32 : (const void *)s->q16;
    size_t elem = which == 0 ? sizeof(float2) : sizeof(kb::pair16);
    if ((which != 0 && which != 1) || !src) return fail(ctx, KB_EINVAL, "stack has no planes of kind %d", which);
    size_t need = (size_t)s->N * s->H * s->W * elem;
    if (dst_bytes < need) return fail(ctx, KB_EINVAL, "dst_bytes %zu < %zu", dst_bytes, need);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    bool dev = is_device_ptr(dst);
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < s->N && e == cudaSuccess; ++ep) {
        const char *from = (const char *)src + (size_t)(ep * s->L.plane_elems + s->L.origin) * elem;
        char *to = (char *)dst + (size_t)ep * s->H * s->W * elem;
        e = cudaMemcpy2DAsync(to, (size_t)s->W * elem, from, (size_t)s->L.pitch * elem, (size_t)s->W * elem,
                              (size_t)s->H, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->used, st);
    if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_stack_copy_planes");
    return KB_OK;
}

int kb_stack_scales(const kb_stack *s, float *psi_scale, float *phi_scale) {
    if (!s || !psi_scale || !phi_scale) return KB_EINVAL;
    DeviceGuard g(s->ctx->device);
    if (!s->q16) {
        for (int e = 0; e < s->N; ++e) psi_scale[e] = phi_scale[e] = 1.0f;
        return KB_OK;
    }
    std::vector<float2> h(s->N);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), s->scales, s->N * sizeof(float2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s->ctx, e, "kb_stack_scales");
    for (int i = 0; i < s->N; ++i) {
        psi_scale[i] = h[i].x;
        phi_scale[i] = h[i].y;
    }
    return KB_OK;
}

// ---- offsets -----------------------------------------------------------------

int kb_offsets(const double *times, int N, const double *vx, const double *vy, int V, int32_t *dx, int32_t *dy) {
    if (!times || !vx || !vy || !dx || !dy || N < 1 || V < 1) return KB_EINVAL;
    Plan pl;
    int rc = plan_times(nullptr, times, N, pl);
    if (rc != KB_OK) return rc;
    std::vector<int64_t> tq(N);
    for (int j = 0; j < N; ++j) tq[pl.epoch_of[j]] = pl.tq[j];
    for (int v = 0; v < V; ++v) {
        int64_t qx, qy;
        if ((rc = quant_velocity(nullptr, vx[v], &qx)) != KB_OK) return rc;
        if ((rc = quant_velocity(nullptr, vy[v], &qy)) != KB_OK) return rc;
        for (int e = 0; e < N; ++e) {
            dx[(size_t)v * N + e] = (int32_t)offset_q(qx, tq[e]);
            dy[(size_t)v * N + e] = (int32_t)offset_q(qy, tq[e]);
        }
    }
    return KB_OK;
}

// ---- jobs --------------------------------------------------------------------

// candidates kept by a search for FP64 rescoring: k plus a margin that grows with
// the storage's rounding (bf16 2^-8, fp16 2^-11, fp32 2^-24); the certificate sends
// the pixels the margin does not cover to the exhaustive FP64 repair
static int job_kkeep(int topk, int flags, int storage) {
    if (!(flags & KB_RESCORE_FP64)) return topk;
    return topk + (storage == KB_BF16 ? std::max(2, topk / 2) : std::max(2, topk / 4));
}

// Device bytes of kb_stack_create + kb_make_psi_phi (an upper bound: the tap
// table is sized for the larger PSF form), and of kb_job_create: the same sums as
// those calls' allocations.
static size_t stack_bytes(int N, int H, int W, int storage, int K) {
    const size_t plane = (size_t)kb::make_layout(H, W).plane_elems;
    size_t b = (size_t)N * plane * sizeof(float2);
    if (storage != KB_F32) b += (size_t)2 * N * plane * sizeof(kb::pair16);
    b += (size_t)N * sizeof(float2) + (size_t)2 * N * sizeof(unsigned);
    // the tap table of whichever PSF form is larger (the form is known only from the PSF)
    b += std::max(kb::taps_floats(N, K, true), kb::taps_floats(N, K, false)) * sizeof(float);
    return b;
}

static size_t job_bytes(int H, int W, int N, int V, int topk, int flags) {
    const size_t npix = (size_t)H * W;
    size_t b = (size_t)V * N * sizeof(int2) + (size_t)V * sizeof(int) + (size_t)V * N * sizeof(uint32_t) +
               sizeof(int) + (size_t)N * sizeof(int) + (size_t)V * sizeof(float2) +
               npix * job_kkeep(topk, flags, KB_BF16) * sizeof(kb::Rec);
    if (flags & KB_RESCORE_FP64) b += npix * topk * sizeof(kb::Rec64) + npix * sizeof(int) + sizeof(int);
    return b;
}

int kb_estimate_bytes(int N, int H, int W, int storage, int K, int V, int topk, int flags, size_t *stack,
                      size_t *job) {
    if (N < 1 || N > KB_MAX_EPOCHS || H < 1 || W < 1 || H > KB_MAX_SIDE || W > KB_MAX_SIDE || K < 1 ||
        K > KB_MAX_PSF || (K % 2) == 0 || V < 1 || V > KB_MAX_VELOCITIES || topk < 1 || topk > KB_MAX_TOPK ||
        (storage != KB_F32 && storage != KB_BF16 && storage != KB_F16) || (flags & ~KB_RESCORE_FP64))
        return KB_EINVAL;
    if (stack) *stack = stack_bytes(N, H, W, storage, K);
    if (job) *job = job_bytes(H, W, N, V, topk, flags);
    return KB_OK;
}

int kb_job_create(kb_ctx *ctx, int H, int W, int N, int V, int topk, int flags, kb_job **out) {
    if (!ctx || !out) return KB_EINVAL;
    *out = nullptr;
    if (H < 1 || W < 1 || H > KB_MAX_SIDE || W > KB_MAX_SIDE || N < 1 || N > KB_MAX_EPOCHS || V < 1 ||
        V > KB_MAX_VELOCITIES || topk < 1 || topk > KB_MAX_TOPK)
        return fail(ctx, KB_EINVAL, "job shape H=%d W=%d N=%d V=%d topk=%d out of range", H, W, N, V, topk);
    if (flags & ~KB_RESCORE_FP64) return fail(ctx, KB_EINVAL, "unknown flags 0x%x", flags);
    DeviceGuard g(ctx->device);
    kb_job *j = new kb_job();
    j->ctx = ctx;
    j->H = H;
    j->W = W;
    j->Ncap = N;
    j->Vcap = V;
    j->kcap = topk;
    j->flags = flags;
    j->kkeep_cap = job_kkeep(topk, flags, KB_BF16);   // the largest margin
    size_t npix = (size_t)H * W;
    int rc = dev_alloc(ctx, (size_t)V * N * sizeof(int2), (void **)&j->offs, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)V * sizeof(int), (void **)&j->vorder, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)V * N * sizeof(uint32_t), (void **)&j->ptab, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, sizeof(int), (void **)&j->status, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)N * sizeof(int), (void **)&j->epoch_of, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)V * sizeof(float2), (void **)&j->vq, &j->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, npix * j->kkeep_cap * sizeof(kb::Rec), (void **)&j->recs, &j->bytes);
    if (rc == KB_OK && (flags & KB_RESCORE_FP64))
        rc = dev_alloc(ctx, npix * topk * sizeof(kb::Rec64), (void **)&j->recs64, &j->bytes);
    if (rc == KB_OK && (flags & KB_RESCORE_FP64)) rc = dev_alloc(ctx, npix * sizeof(int), (void **)&j->ulist, &j->bytes);
    if (rc == KB_OK && (flags & KB_RESCORE_FP64)) rc = dev_alloc(ctx, sizeof(int), (void **)&j->ucount, &j->bytes);
    if (rc == KB_OK) {
        // pinned staging: the tables of a search, then (16-byte aligned) the host copies of
        // the status word and the repaired-pixel count, written after each search
        const size_t tables = (size_t)V * N * sizeof(int2) + (size_t)V * sizeof(int) + (size_t)N * sizeof(int) +
                              (size_t)V * sizeof(float2) + (size_t)V * N * sizeof(uint32_t);
        const size_t hstat_off = (tables + 15) & ~(size_t)15;
        j->stage_bytes = hstat_off + 16;
        cudaError_t e = host_alloc(ctx, j->stage_bytes, &j->stage, &j->stage_cap);
        if (e == cudaSuccess) {
            j->hstat = reinterpret_cast<int *>(static_cast<char *>(j->stage) + hstat_off);
            j->hstat[0] = 0;
            j->hstat[1] = 0;
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->stage_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->rdone, cudaEventDisableTiming);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "kb_job_create");
    }
    if (rc != KB_OK) {
        kb_job_free(j);
        return rc;
    }
    *out = j;
    return KB_OK;
}

void kb_job_free(kb_job *j) {
    if (!j) return;
    DeviceGuard g(j->ctx->device);
    kb_ctx *ctx = j->ctx;
    if (j->stage_done) {
        cudaEventSynchronize(j->stage_done);
        cudaEventDestroy(j->stage_done);
    }
    if (j->done) {
        cudaStreamWaitEvent(ctx->astream, j->done, 0);   // the last search's kernels
        cudaEventDestroy(j->done);
    }
    if (j->rdone) {
        cudaStreamWaitEvent(ctx->astream, j->rdone, 0);  // the last results read
        cudaEventDestroy(j->rdone);
    }
    dev_free(ctx, j->offs);
    dev_free(ctx, j->vorder);
    dev_free(ctx, j->ptab);
    dev_free(ctx, j->status);
    dev_free(ctx, j->epoch_of);
    dev_free(ctx, j->vq);
    dev_free(ctx, j->recs);
    dev_free(ctx, j->recs64);
    dev_free(ctx, j->ulist);
    dev_free(ctx, j->ucount);
    dev_free(ctx, j->expand);
    host_release(ctx, j->stage, j->stage_cap);
    dev_release(ctx, j->bytes);
    delete j;
}

// Stream-ordered copies of the status word and the repaired-pixel count into the
// job's pinned host words, read by kb_job_wait / kb_job_repaired once job->done
// has completed (a synchronous read would wait behind other streams' work).
static cudaError_t readback_status(kb_job *job, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(job->hstat, job->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && job->rescored)
        e = cudaMemcpyAsync(job->hstat + 1, job->ucount, sizeof(int), cudaMemcpyDeviceToHost, st);
    return e;
}

// Distance along a Hilbert curve filling the 2^16 x 2^16 grid: at each level
// from the coarsest, the quadrant's index in the curve's visiting order, then the
// coordinates turned into the quadrant's own frame.
uint64_t hilbert_index(uint32_t x, uint32_t y) {
    const uint32_t n = 1u << 16;
    uint64_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {   // rotate the quadrant
            if (rx == 1) {
                x = s - 1 - (x & (s - 1));
                y = s - 1 - (y & (s - 1));
            }
            std::swap(x, y);
        }
        x &= s - 1;
        y &= s - 1;
    }
    return d;
}

// Validation, fixed-point offset table, processing order and upload of one
// search's tables (stream-ordered), and the kernels' argument blocks.  Shared by
// kb_search and kb_batch_create.
static int prepare_search(kb_job *job, const kb_stack *s, const double *times, const double *vx, const double *vy,
                          int V, int topk, float nu_min, int flags, cudaStream_t st, kb::SearchArgs &a,
                          kb::RescoreArgs &r, bool &rescore) {
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (!s || !times || !vx || !vy) return fail(ctx, KB_EINVAL, "kb_search: NULL argument");
    if (!s->filled) return fail(ctx, KB_EINVAL, "kb_search: the stack has no psi/phi yet (kb_make_psi_phi)");
    if (s->H != job->H || s->W != job->W || s->N > job->Ncap || V < 1 || V > job->Vcap || topk < 1 ||
        topk > job->kcap)
        return fail(ctx, KB_EINVAL, "kb_search: stack %dx%dx%d, V=%d, topk=%d do not fit the job (%dx%d, N<=%d, V<=%d, "
                    "topk<=%d)", s->N, s->H, s->W, V, topk, job->H, job->W, job->Ncap, job->Vcap, job->kcap);
    if ((flags & KB_RESCORE_FP64) && !(job->flags & KB_RESCORE_FP64))
        return fail(ctx, KB_EINVAL, "kb_search: rescoring requested but the job was created without it");
    if (flags & ~(KB_RESCORE_FP64 | KB_PRUNE)) return fail(ctx, KB_EINVAL, "unknown flags 0x%x", flags);
    if (std::isnan(nu_min)) return fail(ctx, KB_EINVAL, "nu_min is NaN");
    const int N = s->N;
    Plan pl;
    int rc = plan_times(ctx, times, N, pl);
    if (rc != KB_OK) return rc;
    std::vector<int64_t> qx(V), qy(V);
    for (int v = 0; v < V; ++v) {
        if ((rc = quant_velocity(ctx, vx[v], &qx[v])) != KB_OK) return rc;
        if ((rc = quant_velocity(ctx, vy[v], &qy[v])) != KB_OK) return rc;
    }

    // host tables in the pinned staging buffer (wait until its previous upload is done)
    cudaError_t e = cudaEventSynchronize(job->stage_done);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_search staging");
    // staging layout for this V, N: offs [V][N] | vq [V] | vorder [V] | epoch [N] (8-byte members first)
    int2 *h_offs = reinterpret_cast<int2 *>(job->stage);
    float2 *h_vq = reinterpret_cast<float2 *>(h_offs + (size_t)V * N);
    int *h_vorder = reinterpret_cast<int *>(h_vq + V);
    int *h_epoch = h_vorder + V;
    uint32_t *h_ptab = reinterpret_cast<uint32_t *>(h_epoch + N);
    for (int v = 0; v < V; ++v) {
        for (int j = 0; j < N; ++j)
            h_offs[(size_t)v * N + j] = make_int2((int)offset_q(qx[v], pl.tq[j]), (int)offset_q(qy[v], pl.tq[j]));
        h_vorder[v] = v;
        h_vq[v] = make_float2((float)((double)qx[v] / (double)kVelOne), (float)((double)qy[v] / (double)kVelOne));
    }
    // Processing order: by the offset at the latest epoch (dy, then dx).  The CTAs
    // resident at one time cover a band of start rows; in this order the rows of
    // every epoch's plane that a band reads are used by a contiguous run of
    // velocities, so the live set of all epochs stays in L2 instead of each
    // velocity re-fetching its rows from HBM.
    // Other orders (kb_set_search_order): along a Hilbert curve over the latest
    // offsets, so that velocities processed close together are close in both axes,
    // or the caller's order.
    {
        const int2 *last = h_offs + (N - 1);
        const int order = ctx->search_order < 0 ? 0 : ctx->search_order;
        if (order == 0) {
            std::stable_sort(h_vorder, h_vorder + V, [&](int a, int b) {
                int2 oa = last[(size_t)a * N], ob = last[(size_t)b * N];
                return oa.y < ob.y || (oa.y == ob.y && oa.x < ob.x);
            });
        } else if (order == 1) {
            int mnx = INT_MAX, mny = INT_MAX;
            for (int v = 0; v < V; ++v) {
                mnx = std::min(mnx, last[(size_t)v * N].x);
                mny = std::min(mny, last[(size_t)v * N].y);
            }
            std::vector<uint64_t> key(V);
            for (int v = 0; v < V; ++v) {
                const int2 o = last[(size_t)v * N];
                const uint32_t x = (uint32_t)std::min<int64_t>((int64_t)o.x - mnx, 65535);
                const uint32_t y = (uint32_t)std::min<int64_t>((int64_t)o.y - mny, 65535);
                key[v] = hilbert_index(x, y);
            }
            std::stable_sort(h_vorder, h_vorder + V, [&](int a, int b) { return key[a] < key[b]; });
        }
    }
    for (int j = 0; j < N; ++j) h_epoch[j] = pl.epoch_of[j];
    // producer table of the pipelined kernel: (dx, dy) as int16 pairs for the
    // non-reference epochs, in processing order (offsets beyond +-32767 are
    // outside any image the library accepts, so clamping keeps them outside)
    const int NJ = N - pl.n0;
    for (int i = 0; i < V; ++i)
        for (int jj = 0; jj < NJ; ++jj) {
            int2 o = h_offs[(size_t)h_vorder[i] * N + pl.n0 + jj];
            int ox = std::max(-32767, std::min(32767, o.x)), oy = std::max(-32767, std::min(32767, o.y));
            h_ptab[(size_t)i * NJ + jj] = ((uint32_t)oy << 16) | ((uint32_t)ox & 0xffffu);
        }
    e = cudaMemcpyAsync(job->offs, h_offs, (size_t)V * N * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(job->vorder, h_vorder, (size_t)V * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(job->epoch_of, h_epoch, (size_t)N * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(job->vq, h_vq, (size_t)V * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && NJ > 0)
        e = cudaMemcpyAsync(job->ptab, h_ptab, (size_t)V * NJ * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(job->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventRecord(job->stage_done, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_search upload");

    rescore = (flags & KB_RESCORE_FP64) != 0;
    const int kkeep = rescore ? job_kkeep(topk, flags, s->q16 ? s->storage : KB_F32) : topk;
    a.storage = s->q16 ? s->storage : KB_F32;
    a.planes = s->q16 ? (const void *)s->q16 : (const void *)s->f32;
    a.plane_elems = s->L.plane_elems;
    a.origin = s->L.origin;
    a.phase1 = (long long)N * s->L.plane_elems;
    a.planes_elems = (s->q16 ? 2LL : 1LL) * N * s->L.plane_elems;
    a.pad_x = s->L.pad_x;
    a.pad_y = s->L.pad_y;
    a.H = s->H;
    a.W = s->W;
    a.pitch = s->L.pitch;
    a.N = N;
    a.n0 = pl.n0;
    a.epoch_of = job->epoch_of;
    a.offs = job->offs;
    a.vorder = job->vorder;
    a.V = V;
    a.scales = s->scales;
    a.nu_min = nu_min;
    a.k = kkeep;
    a.out = job->recs;
    a.variant = ctx->search_variant;
    a.carveout = ctx->search_carveout;
    a.ptab = job->ptab;
    a.status = job->status;
    a.by0 = 0;
    a.nby = 0;
    // automatic tile order: super-columns of 8 tiles (12 x 4096^2, FP32, k = 8: 97.7 ms
    // against 117.4 ms row by row; 6 and 12 tiles within 1 %)
    a.swz = ctx->search_swizzle < 0 ? 8 : ctx->search_swizzle;
    a.cand_only = (flags & KB_RESCORE_FP64) ? 1 : 0;
    a.key_bits = 1;
    while ((1 << a.key_bits) < V) ++a.key_bits;
    a.snr2 = nullptr;           // set by kb_search for KB_PRUNE
    a.nu_min2_slack = 0.0f;
    if (rescore) {
        r.f32 = s->f32;
        r.plane_elems = a.plane_elems;
        r.origin = a.origin;
        r.H = s->H;
        r.W = s->W;
        r.pitch = s->L.pitch;
        r.N = N;
        r.epoch_of = job->epoch_of;
        r.offs = job->offs;
        r.maxbits = s->maxbits;
        r.cand = job->recs;
        r.kc = kkeep;
        r.k = topk;
        r.nu_min = (double)nu_min;
        r.out = job->recs64;
        r.V = V;
        r.unit = s->q16 ? (s->storage == KB_BF16 ? 0x1p-8 : 0x1p-11) : 0x1p-24;
        r.nu_key = 0;   // set once the search's list form is known
        r.ulist = job->ulist;
        r.ucount = job->ucount;
    }
    job->N = N;
    job->V = V;
    job->k = topk;
    job->kkeep = kkeep;
    job->storage = a.storage;
    job->rescored = rescore;
    return KB_OK;
}

int kb_search(kb_job *job, const kb_stack *s, const double *times, const double *vx, const double *vy, int V,
              int topk, float nu_min, int flags, void *stream) {
    kb::NvtxRange nvtx("kb_search");
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (job->owner) return fail(ctx, KB_EINVAL, "kb_search: the job belongs to a batch (kb_batch_free it first)");
    kb::SearchArgs a;
    kb::RescoreArgs r;
    bool rescore = false;
    // a results read still in flight (kb_results_async) must finish before the records change
    cudaStreamWaitEvent(st, job->rdone, 0);
    int rc = prepare_search(job, s, times, vx, vy, V, topk, nu_min, flags, st, a, r, rescore);
    if (rc != KB_OK) return rc;
    cudaError_t e;
    // KB_PRUNE: the span bound planes for the automatic shape's span, built on first use (and
    // after every kb_make_psi_phi) on this stream; only a positive nu_min can prune
    if ((flags & KB_PRUNE) && nu_min > 0.0f && a.variant == 0) {
        kb_stack *ms = const_cast<kb_stack *>(s);   // the bound planes are a cache of the stack
        const int span = kb::search_auto_span(a.storage, a.k);
        const size_t need = (size_t)ms->N * ms->H * ((ms->W + 31) / 32 + span / 32) * sizeof(float);
        if (ms->snr2 && ms->snr2_bytes != need) {
            cudaStreamWaitEvent(ctx->astream, ms->used, 0);
            dev_free(ctx, ms->snr2);
            dev_release(ctx, ms->snr2_bytes);
            ms->bytes -= std::min(ms->bytes, ms->snr2_bytes);
            ms->snr2 = nullptr;
            ms->snr2_bytes = 0;
            ms->snr2_valid = false;
        }
        if (!ms->snr2) {
            rc = dev_alloc(ctx, need, (void **)&ms->snr2, &ms->bytes);
            if (rc != KB_OK) return rc;
            ms->snr2_bytes = need;
            ms->snr2_valid = false;
        }
        if (!ms->snr2_valid || ms->snr2_span != span) {
            kb::SnrArgs b;
            b.planes = a.planes;
            b.storage = a.storage;
            b.scales = ms->scales;
            b.plane_elems = ms->L.plane_elems;
            b.origin = ms->L.origin;
            b.N = ms->N;
            b.H = ms->H;
            b.W = ms->W;
            b.pitch = ms->L.pitch;
            b.span = span;
            b.out = ms->snr2;
            e = kb::launch_snr2(b, st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "span bound kernel");
            ms->snr2_valid = true;
            ms->snr2_span = span;
        }
        a.snr2 = ms->snr2;
        a.nu_min2_slack = nu_min * nu_min;
    }
    if (a.variant >= 5)
        e = kb::launch_search_tma(a, st);
    else
        e = kb::launch_search(a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "search kernel");
    r.nu_key = kb::search_keys(a) ? a.key_bits : 0;
    if (rescore) {
        kb::NvtxRange nvtx_r("kb_rescore");
        e = cudaMemsetAsync(job->ucount, 0, sizeof(int), st);
        if (e == cudaSuccess) e = kb::launch_rescore(r, st);
        if (e == cudaSuccess) e = kb::launch_repair(r, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rescore kernels");
    }
    e = readback_status(job, st);
    if (e == cudaSuccess) e = cudaEventRecord(job->done, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->used, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_search");
    return KB_OK;
}

}  // extern "C"

// ---- batched searches --------------------------------------------------------
// Many searches (uneven stacks, epoch counts, grids, k) in one persistent launch
// per (storage, index width) group.  The work list holds one item per CTA tile
// of every search, {search, tile x, tile y, 0}; the persistent CTAs take items
// off it with an atomic counter.  Searches are ordered by per-tile cost
// (velocities x epochs), largest first, so the cheap tiles fill the tail; the
// tiles of one search stay in row-major order, so the CTAs resident at one time
// cover a band of rows of one stack, the L2 locality the one-search grid has.
// The launches (and the FP64 rescoring of the searches that ask for it) are
// captured once into a CUDA graph; kb_batch_run replays it.
struct kb_batch {
    kb_ctx *ctx = nullptr;
    std::vector<kb_job *> jobs;
    std::vector<const kb_stack *> stacks;
    std::vector<kb::SearchArgs> args;
    std::vector<kb::RescoreArgs> resc;       // searches with FP64 rescoring
    std::vector<int> resc_job;
    std::vector<kb_batch_group> groups;
    std::vector<std::vector<int>> group_jobs;
    std::vector<int4 *> group_items;          // device item list of each group
    kb::SearchArgs *d_args = nullptr;
    int *d_counters = nullptr;                // one per group
    int4 *d_items = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t cap2 = nullptr;              // second branch of the launch schedule
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t bytes = 0;
};

namespace {

int index_bits(const kb::SearchArgs &a) {
    const long long span = (a.storage == KB_F32 ? 1LL : 2LL) * a.N * a.plane_elems;
    return span < (1LL << 31) - 1 ? 32 : 64;
}

// Items of a group for one tile shape: whole searches, or (sample) a band of
// about `frac` of each search's rows from its middle.
void make_items(const kb_batch *b, int g, int variant, double frac, std::vector<int4> &out) {
    out.clear();
    const int span = kb::search_span(b->groups[g].storage, variant, b->groups[g].kmax), R = kb::kTileRows;
    for (int j : b->group_jobs[g]) {
        const kb::SearchArgs &a = b->args[j];
        const int tx = (a.W + span - 1) / span, ty = (a.H + R - 1) / R;
        int y0 = 0, y1 = ty;
        if (frac < 1.0) {
            const int n = std::max(1, std::min(ty, (int)std::ceil(ty * frac)));
            y0 = (ty - n) / 2;
            y1 = y0 + n;
        }
        // the one-search kernel's tile order: super-columns of a.swz tiles (0: rows), row by
        // row within each, so the CTAs working at one time cover a compact block
        const int sw = a.swz > 0 && a.swz < tx ? a.swz : tx;
        for (int s0 = 0; s0 < tx; s0 += sw)
            for (int by = y0; by < y1; ++by)
                for (int bx = s0; bx < std::min(tx, s0 + sw); ++bx) out.push_back(make_int4(j, bx, by, 0));
    }
}

// One group's searches with tile shape `variant`: schedule 0 runs the persistent
// kernel over the group's work list (n_items items) on `st`; schedule 1 launches
// the one-search kernel per search, over the middle `frac` of its row tiles (the
// rows make_items takes for the same frac), alternating between `st` and `st2`
// so that one search's CTAs start while the previous one drains.  The caller
// orders st2 after st before and joins it back after.
cudaError_t launch_group(const kb_batch *b, int g, int variant, int schedule, int n_items, double frac,
                         cudaStream_t st, cudaStream_t st2) {
    const kb_batch_group &G = b->groups[g];
    if (schedule == 0)
        return kb::launch_search_batch(b->d_args, b->group_items[g], n_items, b->d_counters + g, G.storage, variant,
                                       G.kmax, b->ctx->search_carveout, G.index_bits == 64, b->ctx->sm_count, st);
    cudaError_t e = cudaSuccess;
    int n = 0;
    for (int j : b->group_jobs[g]) {
        kb::SearchArgs a = b->args[j];
        a.variant = variant;
        if (frac < 1.0) {
            const int ty = (a.H + kb::kTileRows - 1) / kb::kTileRows;
            a.nby = std::max(1, std::min(ty, (int)std::ceil(ty * frac)));
            a.by0 = (ty - a.nby) / 2;
        }
        e = kb::launch_search(a, (n++ & 1) ? st2 : st);
        if (e != cudaSuccess) break;
    }
    return e;
}

// st2 waits for everything issued to st so far (fork), or st for st2 (join)
cudaError_t order_after(cudaStream_t waiter, cudaStream_t on, cudaEvent_t ev) {
    cudaError_t e = cudaEventRecord(ev, on);
    return e == cudaSuccess ? cudaStreamWaitEvent(waiter, ev, 0) : e;
}

}  // namespace

extern "C" {

int kb_batch_create(kb_ctx *ctx, int count, const kb_batch_item *items, int flags, kb_batch **out) {
    if (!ctx || !out) return KB_EINVAL;
    *out = nullptr;
    if (count < 1 || !items) return fail(ctx, KB_EINVAL, "kb_batch_create: empty batch");
    if (flags & ~KB_BATCH_AUTOTUNE) return fail(ctx, KB_EINVAL, "kb_batch_create: unknown flags 0x%x", flags);
    for (int i = 0; i < count; ++i) {
        kb_job *j = items[i].job;
        if (!j || j->ctx != ctx) return fail(ctx, KB_EINVAL, "kb_batch_create: item %d has no job of this context", i);
        if (j->owner) return fail(ctx, KB_EINVAL, "kb_batch_create: item %d's job belongs to another batch", i);
        for (int k = 0; k < i; ++k)
            if (items[k].job == j) return fail(ctx, KB_EINVAL, "kb_batch_create: items %d and %d share a job", k, i);
    }
    DeviceGuard dg(ctx->device);
    kb_batch *b = new kb_batch();
    b->ctx = ctx;
    auto bail = [&](int rc) {
        kb_batch_free(b);
        return rc;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create"));

    // tables of every search, uploaded on the batch's stream
    b->args.resize(count);
    for (int i = 0; i < count; ++i) {
        const kb_batch_item &it = items[i];
        kb::RescoreArgs r;
        bool rescore = false;
        int rc = prepare_search(it.job, it.stack, it.times, it.vx, it.vy, it.V, it.topk, it.nu_min, it.flags, b->cap,
                                b->args[i], r, rescore);
        if (rc != KB_OK) {
            std::string why = ctx->err;
            return bail(fail(ctx, rc, "kb_batch_create item %d: %s", i, why.c_str()));
        }
        b->jobs.push_back(it.job);
        b->stacks.push_back(it.stack);
        it.job->owner = b;
        if (rescore) {
            b->resc.push_back(r);
            b->resc_job.push_back(i);
        }
    }

    // Groups by (storage, index width, list length): the lists' shared memory
    // sets how many CTAs an SM holds, so each group's launch is sized for its
    // own k instead of the batch's largest.  Within a group, searches by
    // per-tile cost, largest first.
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)b->args[x].V * b->args[x].N > (long long)b->args[y].V * b->args[y].N;
    });
    for (int i : order) {
        const kb::SearchArgs &a = b->args[i];
        const int bits = index_bits(a);
        int g = 0;
        while (g < (int)b->groups.size() && !(b->groups[g].storage == a.storage && b->groups[g].index_bits == bits &&
                                              b->groups[g].kmax == a.k))
            ++g;
        if (g == (int)b->groups.size()) {
            kb_batch_group G;
            memset(&G, 0, sizeof G);
            G.storage = a.storage;
            G.index_bits = bits;
            G.variant = kb::default_variant(a.storage, a.k);
            G.kmax = a.k;
            b->groups.push_back(G);
            b->group_jobs.emplace_back();
        }
        b->group_jobs[g].push_back(i);
        b->groups[g].evals += (double)a.V * a.N * a.H * a.W;
    }
    const int G = (int)b->groups.size();

    // device arrays: search arguments, counters, and each group's item list at
    // its narrowest tile shape (64 pixels: the most items any shape needs)
    size_t n_items_max = 0;
    std::vector<size_t> cap_items(G);
    {
        std::vector<int4> tmp;
        for (int g = 0; g < G; ++g) {
            make_items(b, g, 2, 1.0, tmp);
            cap_items[g] = tmp.size();
            n_items_max += tmp.size();
        }
    }
    int rc = dev_alloc(ctx, (size_t)count * sizeof(kb::SearchArgs), (void **)&b->d_args, &b->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, (size_t)G * sizeof(int), (void **)&b->d_counters, &b->bytes);
    if (rc == KB_OK) rc = dev_alloc(ctx, n_items_max * sizeof(int4), (void **)&b->d_items, &b->bytes);
    if (rc != KB_OK) return bail(rc);
    for (int g = 0, off = 0; g < G; off += (int)cap_items[g], ++g) b->group_items.push_back(b->d_items + off);
    e = cudaMemcpyAsync(b->d_args, b->args.data(), (size_t)count * sizeof(kb::SearchArgs), cudaMemcpyHostToDevice,
                        b->cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create upload"));

    // Autotuner: time every tile shape, with both schedules (the persistent
    // work-list kernel and one launch per search), of each group on a band from
    // the middle of each search's rows (about 4e10 trajectory-epoch evaluations
    // per group, or everything when smaller) and keep the fastest.  Without it
    // the context's variant (1..4) or the default shape runs persistent.
    std::vector<int4> host;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (flags & KB_BATCH_AUTOTUNE) {
        e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        for (int g = 0; g < G && e == cudaSuccess; ++g) {
            const double frac = std::min(1.0, 4e10 / std::max(1.0, b->groups[g].evals));
            float best = INFINITY;
            for (int v = 1; v <= 4 && e == cudaSuccess; ++v) {
                make_items(b, g, v, frac, host);
                e = cudaMemcpyAsync(b->group_items[g], host.data(), host.size() * sizeof(int4),
                                    cudaMemcpyHostToDevice, b->cap);
                for (int sched = 0; sched < 2 && e == cudaSuccess; ++sched) {
                    float ms = 0.0f;
                    for (int rep = (v == 1 && sched == 0 ? 0 : 1); rep < 2 && e == cudaSuccess; ++rep) {
                        e = cudaMemsetAsync(b->d_counters + g, 0, sizeof(int), b->cap);   // rep 0: warm-up
                        if (e == cudaSuccess) e = cudaEventRecord(t0, b->cap);
                        if (e == cudaSuccess) e = order_after(b->cap2, b->cap, b->fork);
                        if (e == cudaSuccess)
                            e = launch_group(b, g, v, sched, (int)host.size(), frac, b->cap, b->cap2);
                        if (e == cudaSuccess) e = order_after(b->cap, b->cap2, b->join);
                        if (e == cudaSuccess) e = cudaEventRecord(t1, b->cap);
                        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                    }
                    (sched == 0 ? b->groups[g].tuned_ms : b->groups[g].tuned_ms_launch)[v] = ms;
                    if (e == cudaSuccess && ms < best) {
                        best = ms;
                        b->groups[g].variant = v;
                        b->groups[g].schedule = sched;
                    }
                }
            }
        }
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create autotune"));
    } else if (ctx->search_variant >= 1 && ctx->search_variant <= 4) {
        for (auto &Gr : b->groups) Gr.variant = ctx->search_variant;
    }

    // final item lists, then the captured graph
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        make_items(b, g, b->groups[g].variant, 1.0, host);
        b->groups[g].n_items = (long long)host.size();
        e = cudaMemcpyAsync(b->group_items[g], host.data(), host.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            b->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    }
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create items"));
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create capture"));
    cudaError_t ce = cudaMemsetAsync(b->d_counters, 0, (size_t)G * sizeof(int), b->cap);
    if (ce == cudaSuccess) ce = order_after(b->cap2, b->cap, b->fork);
    for (int g = 0; g < G && ce == cudaSuccess; ++g)
        ce = launch_group(b, g, b->groups[g].variant, b->groups[g].schedule, (int)b->groups[g].n_items, 1.0, b->cap,
                          b->cap2);
    if (ce == cudaSuccess) ce = order_after(b->cap, b->cap2, b->join);
    for (size_t i = 0; i < b->resc.size() && ce == cudaSuccess; ++i) {
        ce = cudaMemsetAsync(b->resc[i].ucount, 0, sizeof(int), b->cap);
        if (ce == cudaSuccess) ce = kb::launch_rescore(b->resc[i], b->cap);
        if (ce == cudaSuccess) ce = kb::launch_repair(b->resc[i], b->cap);
    }
    for (size_t i = 0; i < b->jobs.size() && ce == cudaSuccess; ++i) ce = readback_status(b->jobs[i], b->cap);
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (ce != cudaSuccess) e = ce;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "kb_batch_create graph"));
    *out = b;
    return KB_OK;
}

int kb_batch_run(kb_batch *b, void *stream) {
    kb::NvtxRange nvtx("kb_batch_run");
    if (!b) return KB_EINVAL;
    kb_ctx *ctx = b->ctx;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < b->jobs.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, b->jobs[i]->rdone, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
    for (size_t i = 0; i < b->jobs.size() && e == cudaSuccess; ++i) e = cudaEventRecord(b->jobs[i]->done, st);
    for (size_t i = 0; i < b->stacks.size() && e == cudaSuccess; ++i) e = cudaEventRecord(b->stacks[i]->used, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_batch_run");
    return KB_OK;
}

int kb_batch_groups(const kb_batch *b, kb_batch_group *out, int capacity, int *n_groups) {
    if (!b || !n_groups) return KB_EINVAL;
    *n_groups = (int)b->groups.size();
    if (out)
        for (int g = 0; g < std::min(capacity, *n_groups); ++g) out[g] = b->groups[g];
    return KB_OK;
}

void kb_batch_free(kb_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->ctx->device);
    if (b->cap) cudaStreamSynchronize(b->cap);
    for (kb_job *j : b->jobs) {
        if (j->done) cudaEventSynchronize(j->done);
        j->owner = nullptr;
    }
    if (b->cap2) cudaStreamSynchronize(b->cap2);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    dev_free(b->ctx, b->d_args);
    dev_free(b->ctx, b->d_counters);
    dev_free(b->ctx, b->d_items);
    dev_release(b->ctx, b->bytes);
    delete b;
}

// Enqueues the expansion of the job's records into `out` (device: directly;
// host: through the device staging buffer, each piece copied out in stream
// order) and records rdone.  Nothing waits on the host.  `whole` stages all
// records at once (one expansion, one copy: after the expansion only the copy
// engine is busy, so the copy overlaps whatever runs next); otherwise pieces of
// 2^22 records keep the staging small.
static int enqueue_results(kb_job *job, kb_result *out, size_t need, bool dev, bool whole, cudaStream_t st) {
    kb_ctx *ctx = job->ctx;
    // the job's last search must be complete before its records are read
    cudaStreamWaitEvent(st, job->done, 0);
    kb::ExpandArgs a;
    a.recs = job->rescored ? nullptr : job->recs;
    a.recs64 = job->rescored ? job->recs64 : nullptr;
    a.krec = job->kkeep;
    a.k = job->k;
    a.H = job->H;
    a.W = job->W;
    a.vq = job->vq;
    cudaError_t e;
    if (dev) {
        a.first = 0;
        a.count = (long long)need;
        a.out = out;
        e = kb::launch_expand(a, st);
        if (e == cudaSuccess) e = cudaEventRecord(job->rdone, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "expand kernel");
        return KB_OK;
    }
    const size_t chunk = whole ? need : std::min(need, (size_t)1 << 22);
    if (job->expand_cap < chunk) {
        cudaStreamWaitEvent(ctx->astream, job->done, 0);
        cudaStreamWaitEvent(ctx->astream, job->rdone, 0);   // a read still using the old staging
        dev_free(ctx, job->expand);
        dev_release(ctx, job->expand_cap * sizeof(kb_result));
        job->bytes -= std::min(job->bytes, job->expand_cap * sizeof(kb_result));
        job->expand = nullptr;
        job->expand_cap = 0;
        int rc = dev_alloc(ctx, chunk * sizeof(kb_result), (void **)&job->expand, &job->bytes);
        if (rc != KB_OK) return rc;
        job->expand_cap = chunk;
    }
    for (size_t first = 0; first < need; first += chunk) {
        size_t n = std::min(chunk, need - first);
        a.first = (long long)first;
        a.count = (long long)n;
        a.out = job->expand;
        e = kb::launch_expand(a, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + first, job->expand, n * sizeof(kb_result), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_results");
    }
    e = cudaEventRecord(job->rdone, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_results");
    return KB_OK;
}

int kb_results(kb_job *job, kb_result *out, size_t capacity, size_t *n_written, void *stream) {
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (job->k == 0) return fail(ctx, KB_EINVAL, "kb_results: no search has run on this job");
    size_t need = (size_t)job->H * job->W * job->k;
    if (n_written) *n_written = need;
    if (!out) return fail(ctx, KB_EINVAL, "kb_results: out is NULL");
    if (capacity < need) return fail(ctx, KB_ERANGE, "kb_results: capacity %zu < %zu records", capacity, need);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_ptr(out);
    int rc = enqueue_results(job, out, need, dev, false, st);
    if (rc != KB_OK || dev) return rc;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_results");
    return kb_job_wait(job);
}

int kb_results_async(kb_job *job, kb_result *out, size_t capacity, size_t *n_written, void *stream) {
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (job->k == 0) return fail(ctx, KB_EINVAL, "kb_results_async: no search has run on this job");
    size_t need = (size_t)job->H * job->W * job->k;
    if (n_written) *n_written = need;
    if (!out) return fail(ctx, KB_EINVAL, "kb_results_async: out is NULL");
    if (capacity < need)
        return fail(ctx, KB_ERANGE, "kb_results_async: capacity %zu < %zu records", capacity, need);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (!dev && at.type != cudaMemoryTypeHost)
        return fail(ctx, KB_EINVAL, "kb_results_async: out must be device or page-locked host memory");
    DeviceGuard g(ctx->device);
    return enqueue_results(job, out, need, dev, true, (cudaStream_t)stream);
}

int kb_results_compact_async(kb_job *job, kb_result_compact *out, size_t capacity, size_t *n_written,
                             void *stream) {
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (job->k == 0) return fail(ctx, KB_EINVAL, "kb_results_compact_async: no search has run on this job");
    const size_t need = (size_t)job->H * job->W * job->k;
    if (n_written) *n_written = need;
    if (!out) return fail(ctx, KB_EINVAL, "kb_results_compact_async: out is NULL");
    if (capacity < need)
        return fail(ctx, KB_ERANGE, "kb_results_compact_async: capacity %zu < %zu records", capacity, need);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (!dev && at.type != cudaMemoryTypeHost)
        return fail(ctx, KB_EINVAL, "kb_results_compact_async: out must be device or page-locked host memory");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamWaitEvent(st, job->done, 0);   // the job's last search
    const size_t bytes = need * sizeof(kb_result_compact);
    cudaError_t e = cudaSuccess;
    if (!job->rescored && job->kkeep == job->k) {
        // the search's own records: [H*W][k] of the same 16-byte layout
        e = cudaMemcpyAsync(out, job->recs, bytes, cudaMemcpyDefault, st);
    } else if (!job->rescored) {
        return fail(ctx, KB_EINVAL, "kb_results_compact_async: the job kept %d candidates for %d results",
                    job->kkeep, job->k);
    } else if (dev) {
        e = kb::launch_compact(job->recs64, (long long)need, out, st);
    } else {
        // through the job's staging buffer (counted in kb_result units)
        const size_t cap = (bytes + sizeof(kb_result) - 1) / sizeof(kb_result);
        if (job->expand_cap < cap) {
            cudaStreamWaitEvent(ctx->astream, job->done, 0);
            cudaStreamWaitEvent(ctx->astream, job->rdone, 0);
            dev_free(ctx, job->expand);
            dev_release(ctx, job->expand_cap * sizeof(kb_result));
            job->bytes -= std::min(job->bytes, job->expand_cap * sizeof(kb_result));
            job->expand = nullptr;
            job->expand_cap = 0;
            int rc = dev_alloc(ctx, cap * sizeof(kb_result), (void **)&job->expand, &job->bytes);
            if (rc != KB_OK) return rc;
            job->expand_cap = cap;
        }
        kb_result_compact *stage = reinterpret_cast<kb_result_compact *>(job->expand);
        e = kb::launch_compact(job->recs64, (long long)need, stage, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, stage, bytes, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(job->rdone, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_results_compact_async");
    return KB_OK;
}

int kb_filter_lightcurves(kb_job *job, const kb_stack *s, double nsigma, kb_filtered *out, size_t capacity,
                          size_t *n_written, void *stream) {
    kb::NvtxRange nvtx("kb_filter_lightcurves");
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (job->k == 0) return fail(ctx, KB_EINVAL, "kb_filter_lightcurves: no search has run on this job");
    if (!s || !s->filled || s->H != job->H || s->W != job->W || s->N != job->N)
        return fail(ctx, KB_EINVAL, "kb_filter_lightcurves: the stack is not the searched one (shape or psi/phi)");
    if (!(nsigma > 0.0) || !std::isfinite(nsigma))
        return fail(ctx, KB_EINVAL, "kb_filter_lightcurves: nsigma %g is not positive", nsigma);
    const size_t need = (size_t)job->H * job->W * job->k;
    if (n_written) *n_written = need;
    if (!out || !is_device_ptr(out)) return fail(ctx, KB_EINVAL, "kb_filter_lightcurves: out must be device memory");
    if (capacity < need) return fail(ctx, KB_ERANGE, "kb_filter_lightcurves: capacity %zu < %zu", capacity, need);
    DeviceGuard g(ctx->device);
    kb::FilterArgs a;
    a.f32 = s->f32;
    a.plane_elems = s->L.plane_elems;
    a.origin = s->L.origin;
    a.H = s->H;
    a.W = s->W;
    a.pitch = s->L.pitch;
    a.N = s->N;
    a.epoch_of = job->epoch_of;
    a.offs = job->offs;
    a.recs = job->rescored ? nullptr : job->recs;
    a.recs64 = job->rescored ? job->recs64 : nullptr;
    a.krec = job->kkeep;
    a.k = job->k;
    a.nsigma2 = nsigma * nsigma;
    a.out = out;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = kb::launch_filter(a, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->used, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_filter_lightcurves");
    return KB_OK;
}

int kb_stamps(kb_job *job, const float *sci, const uint8_t *mask, int N, int H, int W, const int32_t *x0,
              const int32_t *y0, const int32_t *vidx, int n, int radius, int mode, double aperture,
              const kb_moment_cuts *cuts, float *stamps, kb_moments *moments, void *stream) {
    kb::NvtxRange nvtx("kb_stamps");
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    if (job->k == 0) return fail(ctx, KB_EINVAL, "kb_stamps: no search has run on this job");
    if (N != job->N || H != job->H || W != job->W)
        return fail(ctx, KB_EINVAL, "kb_stamps: images %dx%dx%d are not the searched stack's %dx%dx%d", N, H, W,
                    job->N, job->H, job->W);
    if (radius < 0 || radius > KB_MAX_STAMP_RADIUS || (mode != KB_STAMP_MEAN && mode != KB_STAMP_MEDIAN) || n < 0 ||
        std::isnan(aperture))
        return fail(ctx, KB_EINVAL, "kb_stamps: radius %d, mode %d, aperture or count %d out of range", radius, mode, n);
    if (n == 0) return KB_OK;
    if (!sci || !stamps || !x0 || !y0 || !vidx || !is_device_ptr(sci) || !is_device_ptr(stamps) ||
        (mask && !is_device_ptr(mask)) || (moments && !is_device_ptr(moments)))
        return fail(ctx, KB_EINVAL, "kb_stamps: images, stamps and moments must be device memory, candidates host");
    std::vector<int4> cand(n);
    for (int i = 0; i < n; ++i) {
        if (x0[i] < 0 || x0[i] >= W || y0[i] < 0 || y0[i] >= H || vidx[i] < 0 || vidx[i] >= job->V)
            return fail(ctx, KB_EINVAL, "kb_stamps: candidate %d (%d, %d, v %d) outside the search", i, x0[i], y0[i],
                        vidx[i]);
        cand[i] = make_int4(x0[i], y0[i], vidx[i], 0);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int4 *dcand = nullptr;
    size_t acct = 0;
    int rc = dev_alloc(ctx, (size_t)n * sizeof(int4), (void **)&dcand, &acct);
    if (rc != KB_OK) return rc;
    kb::StampArgs a;
    a.sci = sci;
    a.mask = mask;
    a.N = N;
    a.H = H;
    a.W = W;
    a.epoch_of = job->epoch_of;
    a.offs = job->offs;
    a.cand = dcand;
    a.n = n;
    a.r = radius;
    a.mode = mode;
    a.aperture = aperture;
    a.cut = cuts != nullptr;
    if (cuts) a.cuts = *cuts;
    a.stamps = stamps;
    a.moments = moments;
    cudaError_t e = cudaMemcpyAsync(dcand, cand.data(), (size_t)n * sizeof(int4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = kb::launch_stamps(a, st);
    // the copy reads the host vector and the kernel the candidate list: both done before they go
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    dev_free(ctx, dcand);
    dev_release(ctx, acct);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_stamps");
    return KB_OK;
}

int kb_cluster(kb_ctx *ctx, const kb_result *cand, size_t n, const kb_cluster_params *p, int32_t *label,
               uint8_t *keep, uint8_t *core, size_t *n_groups, void *stream) {
    kb::NvtxRange nvtx("kb_cluster");
    if (!ctx || !p) return fail(ctx, KB_EINVAL, "kb_cluster: null context or parameters");
    if (n_groups) *n_groups = 0;
    if (n > ((size_t)1 << 29))
        return fail(ctx, KB_EINVAL, "kb_cluster: %zu candidates (at most 2^29)", n);
    auto pos_fin = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos_fin(p->w_pos) || !pos_fin(p->w_vel) || !pos_fin(p->eps) || p->min_samples < 1)
        return fail(ctx, KB_EINVAL, "kb_cluster: weights %g, %g, eps %g must be positive and finite, "
                    "min_samples %d >= 1", p->w_pos, p->w_vel, p->eps, p->min_samples);
    if (n == 0) return KB_OK;
    if (!cand || !label || !keep || !is_device_ptr(cand) || !is_device_ptr(label) || !is_device_ptr(keep) ||
        (core && !is_device_ptr(core)))
        return fail(ctx, KB_EINVAL, "kb_cluster: candidates and outputs must be device memory");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int T = 1;
    while (T < 2 * (int)n) T <<= 1;
    const size_t words = 2 * (size_t)T + 3 * n;   // owner, head | next, parent, bestidx
    const size_t bytes = 2 * n * sizeof(int4) + n * sizeof(unsigned long long) + words * sizeof(int) +
                         2 * sizeof(int) + 2 * n + 16;
    void *buf = nullptr;
    size_t acct = 0;
    int rc = dev_alloc(ctx, bytes, &buf, &acct);
    if (rc != KB_OK) return rc;
    kb::ClusterArgs a;
    a.cand = cand;
    a.n = (int)n;
    a.T = T;
    a.w_pos = p->w_pos;
    a.w_vel = p->w_vel;
    a.eps2 = p->eps * p->eps;
    // cells a little wider than eps: the rounding of the weighted coordinates
    // cannot put two neighbours more than one cell apart
    a.inv_side = 1.0 / (p->eps * (1.0 + 1.0 / 1048576.0));
    a.min_samples = p->min_samples;
    a.pts = reinterpret_cast<int4 *>(buf);
    a.cells = a.pts + n;
    unsigned long long *bestnu = reinterpret_cast<unsigned long long *>(a.cells + n);
    int *w = reinterpret_cast<int *>(bestnu + n);
    a.bestnu = bestnu;
    a.owner = w;
    a.head = w + T;
    a.next = w + 2 * (size_t)T;
    a.parent = a.next + n;
    a.bestidx = a.parent + n;
    a.count = reinterpret_cast<unsigned *>(a.bestidx + n);
    a.status = reinterpret_cast<int *>(a.count + 1);
    a.core = reinterpret_cast<uint8_t *>(a.status + 1);
    a.valid = a.core + n;
    a.label = label;
    a.keep = keep;
    a.core_out = core;
    unsigned hc[2] = {0u, 0u};
    cudaError_t e = kb::launch_cluster(a, ctx->sm_count, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, a.count, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    dev_free(ctx, buf);
    dev_release(ctx, acct);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_cluster");
    if (hc[1] == 1)
        return fail(ctx, KB_EINVAL, "kb_cluster: a weighted coordinate is beyond 2^30 eps (weights or eps unusable)");
    if (hc[1] != 0) return fail(ctx, KB_ECUDA, "kb_cluster: an internal loop bound was reached (status %u)", hc[1]);
    if (n_groups) *n_groups = hc[0];
    return KB_OK;
}

int kb_job_repaired(kb_job *job, size_t *n_pixels) {
    if (!job || !n_pixels) return KB_EINVAL;
    *n_pixels = 0;
    int rc = kb_job_wait(job);
    if (rc != KB_OK || !job->rescored) return rc;
    *n_pixels = (size_t)job->hstat[1];   // copied after the search's kernels (see readback_status)
    return KB_OK;
}

int kb_job_wait(kb_job *job) {
    if (!job) return KB_EINVAL;
    kb_ctx *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventSynchronize(job->done);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kb_job_wait");
    if (job->hstat[0] != 0)
        return fail(ctx, KB_ETIMEOUT, "a bounded device-side wait of the search gave up; results are invalid");
    return KB_OK;
}

}  // extern "C"
