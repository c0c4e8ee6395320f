// Stage (b): exhaustive trajectory search of Sec. 2.2 on sm_103a.
//
// For every start pixel (x0, y0) and every velocity v, the coadd of Sec. 2.1.5
//   Psi = sum_t psi_t(x0 + dx_vt, y0 + dy_vt),  Phi = sum_t phi_t(...)
// over the epochs whose pixel lies in the image, nu = Psi / sqrt(Phi), and the
// k best (nu desc, vidx asc) valid trajectories per start pixel.
//
// Work decomposition (GB300-first, not the paper's 32x16 thread blocks):
//   - a warp owns a row segment of 32*P start pixels (lane + 32 p) and runs the
//     whole velocity loop for them, so each pixel's top-k list stays in that
//     lane's registers and no cross-thread merge is needed;
//   - for one (velocity, epoch) the warp's P loads cover 32*P consecutive pixels
//     of one row of psi/phi: fully coalesced, no shared-memory staging needed
//     (there is no reuse across start pixels within one velocity);
//   - the velocity table (int16 dx, dy per epoch) is staged in shared memory in
//     chunks and read as warp-uniform broadcasts;
//   - epochs at t = t_min have offset 0 for every velocity: their contribution is
//     loaded once per pixel before the velocity loop;
//   - loads are issued four epochs at a time; when the whole 32*P span of every
//     epoch in the group lies inside the image (the common case) the group takes
//     an unpredicated path, otherwise per-lane predicates give exactly the
//     "outside contributes nothing" rule;
//   - (psi, phi) pairs are accumulated with packed add/fma.rn.f32x2; 16-bit
//     storage is unpacked and scaled by the epoch's power-of-two scales.
// The Psi/Phi of each kept trajectory are recomputed at the end by the same
// sequence of operations (bit-identical) together with nobs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "kb_internal.h"

namespace kb {

namespace {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int OFF_WORDS = 2048;   // packed offsets (8 KB) per velocity chunk

__device__ __forceinline__ unsigned long long as_u64(float2 v) {
    return *reinterpret_cast<unsigned long long *>(&v);
}
__device__ __forceinline__ float2 as_f2(unsigned long long u) { return *reinterpret_cast<float2 *>(&u); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
    return as_f2(d);
}

// storage traits: element type, load, accumulate
template <int STORAGE>
struct Store;

template <>
struct Store<KB_F32> {
    typedef float2 T;
    __device__ __forceinline__ static T load(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static T zero() { return make_float2(0.0f, 0.0f); }
    __device__ __forceinline__ static float2 acc(float2 a, T v, float2) { return add2(a, v); }
};

template <>
struct Store<KB_BF16> {
    typedef pair16 T;
    __device__ __forceinline__ static T load(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static T zero() { return 0u; }
    __device__ __forceinline__ static float2 acc(float2 a, T v, float2 s) {
        float2 f = make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
        return fma2(f, s, a);
    }
};

template <>
struct Store<KB_F16> {
    typedef pair16 T;
    __device__ __forceinline__ static T load(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static T zero() { return 0u; }
    __device__ __forceinline__ static float2 acc(float2 a, T v, float2 s) {
        __half2 h = *reinterpret_cast<__half2 *>(&v);
        return fma2(__half22float2(h), s, a);
    }
};

__device__ __forceinline__ int off_dx(uint32_t po) { return ((int)(po << 16)) >> 16; }
__device__ __forceinline__ int off_dy(uint32_t po) { return ((int)po) >> 16; }

// (nu desc, vidx asc)
__device__ __forceinline__ bool better(float an, int av, float bn, int bv) {
    return an > bn || (an == bn && av < bv);
}

template <int STORAGE, int P>
struct Ctx {
    typedef typename Store<STORAGE>::T T;
    const T *const *base;   // shared: plane base per time-ordered epoch
    const float2 *scale;    // shared: scale per time-ordered epoch
    int H, W, pitch, y, xw, lane;
};

// Loads of C consecutive time-ordered epochs (j0 .. j0+C-1) for one velocity.
template <int STORAGE, int P, int C>
__device__ __forceinline__ void gather_group(const Ctx<STORAGE, P> &c, const uint32_t *op, int j0, float2 (&acc)[P]) {
    typedef Store<STORAGE> S;
    typedef typename S::T T;
    int dx[C], dy[C];
    bool full = true;
#pragma unroll
    for (int q = 0; q < C; ++q) {
        uint32_t po = op[q];
        dx[q] = off_dx(po);
        dy[q] = off_dy(po);
        int ys = c.y + dy[q], xs = c.xw + dx[q];
        full &= ((unsigned)ys < (unsigned)c.H) && (xs >= 0) && (xs + 32 * P <= c.W);
    }
    T v[C][P];
    if (full) {   // warp-uniform
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const T *row = c.base[j0 + q] + (long long)(c.y + dy[q]) * c.pitch + (c.xw + dx[q] + c.lane);
#pragma unroll
            for (int p = 0; p < P; ++p) v[q][p] = S::load(row + 32 * p);
        }
    } else {
#pragma unroll
        for (int q = 0; q < C; ++q) {
            int ys = c.y + dy[q];
            bool rok = (unsigned)ys < (unsigned)c.H;
            const T *row = c.base[j0 + q] + (long long)(rok ? ys : 0) * c.pitch;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                int xx = c.xw + c.lane + 32 * p + dx[q];
                v[q][p] = S::zero();
                if (rok && (unsigned)xx < (unsigned)c.W) v[q][p] = S::load(row + xx);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
        float2 s = c.scale[j0 + q];
#pragma unroll
        for (int p = 0; p < P; ++p) acc[p] = S::acc(acc[p], v[q][p], s);
    }
}

template <int STORAGE, int P>
__global__ void __launch_bounds__(THREADS) search_kernel(SearchArgs a) {
    typedef Store<STORAGE> S;
    typedef typename S::T T;
    __shared__ const T *s_base[KB_MAX_EPOCHS];
    __shared__ float2 s_scale[KB_MAX_EPOCHS];
    // dynamic: packed offsets [OFF_WORDS] | velocity ids [OFF_WORDS] | lists nu [k][THREADS*P], vid [k][THREADS*P]
    extern __shared__ uint32_t s_dyn[];
    uint32_t *s_off = s_dyn;
    int *s_vid = reinterpret_cast<int *>(s_dyn + OFF_WORDS);
    float *s_ln = reinterpret_cast<float *>(s_dyn + 2 * OFF_WORDS);
    int *s_lv = reinterpret_cast<int *>(s_ln + a.k * THREADS * P);
    constexpr int LS = THREADS * P;   // list stride

    const int N = a.N, n0 = a.n0, NJ = N - n0, k = a.k;
    for (int j = threadIdx.x; j < N; j += THREADS) {
        int e = a.epoch_of[j];
        s_base[j] = reinterpret_cast<const T *>(a.planes) + (long long)e * a.plane_elems;
        s_scale[j] = (STORAGE == KB_F32) ? make_float2(1.0f, 1.0f) : a.scales[e];
    }
    for (int i = threadIdx.x; i < k * LS; i += THREADS) {
        s_ln[i] = -INFINITY;
        s_lv[i] = INT_MAX;
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y = blockIdx.y * WARPS + warp;
    const int xw = blockIdx.x * (32 * P);
    const bool active = y < a.H;

    Ctx<STORAGE, P> c;
    c.base = s_base;
    c.scale = s_scale;
    c.H = a.H;
    c.W = a.W;
    c.pitch = a.pitch;
    c.y = y;
    c.xw = xw;
    c.lane = lane;

    // the k-th entry of each list (admission threshold) lives in registers
    float thn[P];
    int thv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        thn[p] = -INFINITY;
        thv[p] = INT_MAX;
    }

    __syncthreads();
    // epochs at the reference time: offset 0 for every velocity
    float2 acc0[P];
#pragma unroll
    for (int p = 0; p < P; ++p) acc0[p] = make_float2(0.0f, 0.0f);
    if (active) {
        for (int j = 0; j < n0; ++j) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                int x = xw + lane + 32 * p;
                if (x < a.W) acc0[p] = S::acc(acc0[p], S::load(s_base[j] + (long long)y * a.pitch + x), s_scale[j]);
            }
        }
    }

    const int vchunk = min(a.V, OFF_WORDS / max(NJ, 1));
    for (int c0 = 0; c0 < a.V; c0 += vchunk) {
        const int nc = min(vchunk, a.V - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += THREADS) s_vid[i] = a.vorder[c0 + i];
        for (int i = threadIdx.x; i < nc * NJ; i += THREADS) {
            int vi = i / NJ, jj = i - vi * NJ;
            int2 o = a.offs[(long long)a.vorder[c0 + vi] * N + n0 + jj];
            int ox = max(-32767, min(32767, o.x)), oy = max(-32767, min(32767, o.y));
            s_off[i] = ((uint32_t)oy << 16) | ((uint32_t)ox & 0xffffu);
        }
        __syncthreads();
        if (!active) continue;
        for (int vi = 0; vi < nc; ++vi) {
            const int v = s_vid[vi];
            const uint32_t *op = s_off + vi * NJ;
            float2 acc[P];
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p] = acc0[p];
            int jj = 0;
            for (; jj + 4 <= NJ; jj += 4) gather_group<STORAGE, P, 4>(c, op + jj, n0 + jj, acc);
            for (; jj < NJ; ++jj) gather_group<STORAGE, P, 1>(c, op + jj, n0 + jj, acc);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float F = acc[p].y;
                if (!(F > 0.0f)) continue;
                float nu = acc[p].x * rsqrtf(F);
                if (!(nu >= a.nu_min)) continue;
                if (!better(nu, v, thn[p], thv[p])) continue;
                // insertion into this lane's sorted list (rare after the first velocities)
                float *ln = s_ln + p * THREADS + threadIdx.x;
                int *lv = s_lv + p * THREADS + threadIdx.x;
                int i = k - 1;
                while (i > 0) {
                    float pn = ln[(i - 1) * LS];
                    int pv = lv[(i - 1) * LS];
                    if (!better(nu, v, pn, pv)) break;
                    ln[i * LS] = pn;
                    lv[i * LS] = pv;
                    --i;
                }
                ln[i * LS] = nu;
                lv[i * LS] = v;
                thn[p] = ln[(k - 1) * LS];
                thv[p] = lv[(k - 1) * LS];
            }
        }
    }
    if (!active) return;

    // epilogue: recompute Psi, Phi (same operation sequence) and nobs of the kept entries
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int x = xw + lane + 32 * p;
        if (x >= a.W) continue;
        Rec *out = a.out + ((long long)y * a.W + x) * k;
        const float *ln = s_ln + p * THREADS + threadIdx.x;
        const int *lv = s_lv + p * THREADS + threadIdx.x;
        for (int i = 0; i < k; ++i) {
            Rec r;
            const int v = lv[i * LS];
            if (v == INT_MAX) {
                r.psi = 0.0f;
                r.phi = 0.0f;
                r.nu = -INFINITY;
                r.meta = kEmptyVidx;
            } else {
                const int2 *ov = a.offs + (long long)v * N;
                float2 acc = acc0[p];
                int nobs = n0;
                for (int j = n0; j < N; ++j) {
                    int2 o = __ldg(ov + j);
                    int xx = x + o.x, yy = y + o.y;
                    if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                        acc = S::acc(acc, S::load(s_base[j] + (long long)yy * a.pitch + xx), s_scale[j]);
                        ++nobs;
                    }
                }
                r.psi = acc.x;
                r.phi = acc.y;
                r.nu = ln[i * LS];
                r.meta = (uint32_t)v | ((uint32_t)nobs << 16);
            }
            reinterpret_cast<uint4 *>(out)[i] = *reinterpret_cast<uint4 *>(&r);
        }
    }
}

template <int STORAGE, int P>
cudaError_t launch_one(const SearchArgs &a, cudaStream_t st) {
    dim3 grid((a.W + 32 * P - 1) / (32 * P), (a.H + WARPS - 1) / WARPS);
    size_t smem = (size_t)2 * OFF_WORDS * 4 + (size_t)2 * a.k * THREADS * P * 4;
    cudaError_t err = cudaFuncSetAttribute(search_kernel<STORAGE, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    search_kernel<STORAGE, P><<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int STORAGE>
cudaError_t launch_storage(const SearchArgs &a, cudaStream_t st) {
    if (a.k <= 8) return launch_one<STORAGE, 4>(a, st);
    return launch_one<STORAGE, 2>(a, st);
}

}  // namespace

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, int /*sm_count*/) {
    switch (a.storage) {
        case KB_F32: return launch_storage<KB_F32>(a, st);
        case KB_BF16: return launch_storage<KB_BF16>(a, st);
        case KB_F16: return launch_storage<KB_F16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kb
