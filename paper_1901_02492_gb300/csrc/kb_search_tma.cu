// Stage (b), pipelined: exhaustive trajectory search of Sec. 2.2 with TMA.
//
// Same contract and results as search_kernel (kb_search.cu); this kernel moves
// the psi/phi gathers off the load/store units:
//   - a CTA owns CWARPS = 8 rows x 32*P columns of start pixels; one consumer
//     warp per row, lane + 32 p per pixel, and runs every velocity for them;
//   - for each (velocity, epoch) one producer warp issues a 3-D tiled TMA load
//     (cp.async.bulk.tensor) of the box of the plane that the whole tile reads
//     at that offset: 8 rows x (32 P + alignment) pixels, the tile shifted by
//     (dx, dy).  Rows or columns outside the planes are zero-filled by the TMA
//     unit; boxes that miss the image entirely are not fetched;
//   - the boxes go into an S-deep ring of shared-memory slots guarded by
//     mbarriers: "full" completes when the box has landed (transaction bytes),
//     "empty" when all consumer warps have read the slot;
//   - consumers read their row of the slot with conflict-free shared loads at
//     the box's alignment shift and accumulate (psi, phi) with packed f32x2 ops;
//   - every wait is bounded (clock64); a wait that gives up raises the job's
//     status word (KB_ETIMEOUT) and the kernel returns instead of spinning.
// The producer reads the per-(velocity, epoch) offsets from a table laid out in
// processing order, 32 entries per coalesced load, broadcast by shuffles.
#include <cuda.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "kb_device.cuh"

namespace kb {

namespace {

using namespace dev;

constexpr int CWARPS = 8;
constexpr int TTHREADS = (CWARPS + 1) * 32;
constexpr long long kWaitLimit = 4000000000LL;   // SM cycles (about 2 s) before a wait gives up

template <int STORAGE, int P>
struct Tile {
    typedef typename Store<STORAGE>::T T;
    static constexpr int AL = Store<STORAGE>::kAlign;
    static constexpr int BW = 32 * P + AL;                                        // box width (pixels)
    static constexpr uint32_t BOX_BYTES = (uint32_t)(CWARPS * BW * sizeof(T));
    static constexpr int SLOT = (int)((BOX_BYTES + 127u) & ~127u);                // 128-byte aligned slots
};

// shared-memory layout (bytes), host and device
struct TmaLayout {
    size_t slots, full, empty, flag, scale, epoch, ln, lv, total;
};
__host__ __device__ inline TmaLayout tma_layout(int S, int slot_bytes, int N, int k, int P) {
    TmaLayout L;
    L.slots = 0;
    L.full = (size_t)S * slot_bytes;
    L.empty = L.full + 8 * (size_t)S;
    L.flag = L.empty + 8 * (size_t)S;
    L.scale = (L.flag + 4 * (size_t)S + 7) & ~(size_t)7;
    L.epoch = L.scale + 8 * (size_t)N;
    L.ln = (L.epoch + 4 * (size_t)N + 15) & ~(size_t)15;
    L.lv = L.ln + 4 * (size_t)k * CWARPS * 32 * P;
    L.total = L.lv + 4 * (size_t)k * CWARPS * 32 * P;
    return L;
}

template <int STORAGE, int P, int S, int C>
__global__ void __launch_bounds__(TTHREADS) search_tma_kernel(const __grid_constant__ CUtensorMap tmap, SearchArgs a) {
    typedef Store<STORAGE> St;
    typedef typename St::T T;
    typedef Tile<STORAGE, P> Tl;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;

    const int N = a.N, n0 = a.n0, NJ = N - n0, k = a.k, V = a.V;
    const TmaLayout L = tma_layout(S, Tl::SLOT, N, k, P);
    unsigned char *slots = smem + L.slots;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.full);
    uint64_t *empty = reinterpret_cast<uint64_t *>(smem + L.empty);
    int *flag = reinterpret_cast<int *>(smem + L.flag);
    float2 *s_scale = reinterpret_cast<float2 *>(smem + L.scale);
    int *s_epoch = reinterpret_cast<int *>(smem + L.epoch);
    float *s_ln = reinterpret_cast<float *>(smem + L.ln);
    int *s_lv = reinterpret_cast<int *>(smem + L.lv);
    constexpr int LS = CWARPS * 32 * P;   // list stride

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0c = blockIdx.y * CWARPS;
    const int xw = blockIdx.x * (32 * P);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, CWARPS);
            flag[s] = -1;
        }
        s_abort = 0;
        fence_mbar_init();
    }
    for (int j = threadIdx.x; j < N; j += TTHREADS) {
        int e = a.epoch_of[j];
        s_epoch[j] = e;
        s_scale[j] = (STORAGE == KB_F32) ? make_float2(1.0f, 1.0f) : a.scales[e];
    }
    for (int i = threadIdx.x; i < k * LS; i += TTHREADS) {
        s_ln[i] = -INFINITY;
        s_lv[i] = INT_MAX;
    }
    __syncthreads();
    volatile int *abort_flag = &s_abort;
    const int items = V * NJ;

    if (warp == CWARPS) {
        // ---------------- producer warp: one TMA box per (velocity, epoch) ----------------
        int issued = 0;
        for (int b = 0; b < items && !*abort_flag; b += 32) {
            const uint32_t ent = (b + lane < items) ? __ldg(a.ptab + b + lane) : 0u;
            const int nb = min(32, items - b);
            for (int l = 0; l < nb; ++l) {
                const uint32_t po = __shfl_sync(0xffffffffu, ent, l);
                if (lane == 0) {
                    const int it = b + l, s = it % S;
                    bool go = true;
                    if (it >= S) go = mbar_wait(empty + s, (uint32_t)((it / S) - 1) & 1u, abort_flag, a.status, kWaitLimit);
                    if (go) {
                        const int dx = ((int)(po << 16)) >> 16, dy = ((int)po) >> 16;
                        const int jj = it % NJ;
                        const int ys = y0c + dy, xs = xw + dx;
                        const bool hit = (ys + CWARPS > 0) && (ys < a.H) && (xs + 32 * P > 0) && (xs < a.W);
                        if (hit) {
                            const int sh = xs & (Tl::AL - 1);
                            flag[s] = sh;
                            mbar_arrive_expect_tx(full + s, Tl::BOX_BYTES);
                            tma_load_3d(slots + (size_t)s * Tl::SLOT, &tmap, full + s, a.pad_x + xs - sh, a.pad_y + ys,
                                        s_epoch[n0 + jj]);
                        } else {
                            flag[s] = -1;
                            mbar_arrive(full + s);
                        }
                        issued = it + 1;
                    }
                }
                __syncwarp();
                if (*abort_flag) break;
            }
        }
        if (lane == 0 && *abort_flag) {
            // give the boxes still in flight a bounded time to land before the CTA can exit
            for (int it = max(0, issued - S); it < issued; ++it) {
                const long long t0 = clock64();
                while (!mbar_try_wait(full + it % S, (uint32_t)(it / S) & 1u) && clock64() - t0 < kWaitLimit) {
                }
            }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const int y = y0c + warp;
    const bool row_active = y < a.H;
    const T *rbase = reinterpret_cast<const T *>(slots) + warp * Tl::BW + lane;

    float2 acc0[P];
#pragma unroll
    for (int p = 0; p < P; ++p) acc0[p] = make_float2(0.0f, 0.0f);
    if (row_active) {
        const T *planes = reinterpret_cast<const T *>(a.planes);
        for (int j = 0; j < n0; ++j) {
            const T *src = planes + (long long)s_epoch[j] * a.plane_elems + a.origin + (long long)y * a.pitch + xw + lane;
#pragma unroll
            for (int p = 0; p < P; ++p) acc0[p] = St::acc(acc0[p], St::load(src + 32 * p), s_scale[j]);
        }
    }
    float thn[P];
    int thv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        thn[p] = -INFINITY;
        thv[p] = INT_MAX;
    }

    bool ok = true;
    for (int vi = 0; vi < V && ok; ++vi) {
        float2 acc[P];
#pragma unroll
        for (int p = 0; p < P; ++p) acc[p] = acc0[p];
        int jj = 0;
        for (; jj + C <= NJ && ok; jj += C) {
            const int it0 = vi * NJ + jj;
            T val[C][P];
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const int it = it0 + q, s = it % S;
                ok = ok && mbar_wait(full + s, (uint32_t)(it / S) & 1u, abort_flag, a.status, kWaitLimit);
                const int sh = ok ? flag[s] : -1;
                const T *src = rbase + (size_t)s * (Tl::SLOT / sizeof(T)) + sh;
#pragma unroll
                for (int p = 0; p < P; ++p) val[q][p] = (sh >= 0) ? src[32 * p] : St::zero();
            }
            __syncwarp();
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < C; ++q) mbar_arrive(empty + (it0 + q) % S);
            }
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const float2 sc = s_scale[n0 + jj + q];
#pragma unroll
                for (int p = 0; p < P; ++p) acc[p] = St::acc(acc[p], val[q][p], sc);
            }
        }
        for (; jj < NJ && ok; ++jj) {
            const int it = vi * NJ + jj, s = it % S;
            ok = mbar_wait(full + s, (uint32_t)(it / S) & 1u, abort_flag, a.status, kWaitLimit);
            const int sh = ok ? flag[s] : -1;
            const T *src = rbase + (size_t)s * (Tl::SLOT / sizeof(T)) + sh;
            T val[P];
#pragma unroll
            for (int p = 0; p < P; ++p) val[p] = (sh >= 0) ? src[32 * p] : St::zero();
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + s);
            const float2 sc = s_scale[n0 + jj];
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p] = St::acc(acc[p], val[p], sc);
        }
        if (!row_active) continue;
        const int v = __ldg(a.vorder + vi);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float F = acc[p].y;
            if (!(F > 0.0f)) continue;
            float nu = acc[p].x * rsqrtf(F);
            if (!(nu >= a.nu_min)) continue;
            if (!better(nu, v, thn[p], thv[p])) continue;
            float *ln = s_ln + p * (CWARPS * 32) + warp * 32 + lane;
            int *lv = s_lv + p * (CWARPS * 32) + warp * 32 + lane;
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
    if (!ok || !row_active) return;

    // epilogue: recompute Psi, Phi (same operation sequence) and nobs of the kept entries
    const T *planes = reinterpret_cast<const T *>(a.planes);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int x = xw + lane + 32 * p;
        if (x >= a.W) continue;
        Rec *out = a.out + ((long long)y * a.W + x) * k;
        const float *ln = s_ln + p * (CWARPS * 32) + warp * 32 + lane;
        const int *lv = s_lv + p * (CWARPS * 32) + warp * 32 + lane;
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
                    T val = St::zero();
                    if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                        val = St::load(planes + (long long)s_epoch[j] * a.plane_elems + a.origin + (long long)yy * a.pitch + xx);
                        ++nobs;
                    }
                    acc = St::acc(acc, val, s_scale[j]);
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <int STORAGE, int P, int S, int C>
cudaError_t launch_tma(const SearchArgs &a, cudaStream_t st) {
    typedef Tile<STORAGE, P> Tl;
    static_assert(32 * P <= kSpan, "tile span wider than the zero border");
    static_assert(Tl::BW <= 256, "TMA box dimension above 256");
    static_assert((Tl::BW * sizeof(typename Tl::T)) % 16 == 0, "box row not a multiple of 16 bytes");
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int es = (int)sizeof(typename Tl::T);
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)a.pitch, (cuuint64_t)(a.plane_elems / a.pitch), (cuuint64_t)a.N};
    cuuint64_t strides[2] = {(cuuint64_t)a.pitch * es, (cuuint64_t)a.plane_elems * es};
    cuuint32_t box[3] = {(cuuint32_t)Tl::BW, (cuuint32_t)CWARPS, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(&map, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                     const_cast<void *>(a.planes), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const TmaLayout L = tma_layout(S, Tl::SLOT, a.N, a.k, P);
    cudaError_t err = cudaFuncSetAttribute(search_tma_kernel<STORAGE, P, S, C>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (err != cudaSuccess) return err;
    dim3 grid((a.W + 32 * P - 1) / (32 * P), (a.H + CWARPS - 1) / CWARPS);
    search_tma_kernel<STORAGE, P, S, C><<<grid, TTHREADS, L.total, st>>>(map, a);
    return cudaGetLastError();
}

template <int STORAGE>
cudaError_t launch_tma_storage(const SearchArgs &a, cudaStream_t st) {
    switch (a.variant) {
        case 5: return launch_tma<STORAGE, 2, 8, 2>(a, st);
        case 6: return launch_tma<STORAGE, 2, 12, 4>(a, st);
        case 7: return launch_tma<STORAGE, 4, 8, 2>(a, st);
        case 8: return launch_tma<STORAGE, 4, 12, 4>(a, st);
        default: return launch_tma<STORAGE, 2, 12, 4>(a, st);
    }
}

}  // namespace

cudaError_t launch_search_tma(const SearchArgs &a, cudaStream_t st) {
    switch (a.storage) {
        case KB_F32: return launch_tma_storage<KB_F32>(a, st);
        case KB_BF16: return launch_tma_storage<KB_BF16>(a, st);
        case KB_F16: return launch_tma_storage<KB_F16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kb
