// Stage (b): exhaustive trajectory search of Sec. 2.2 on sm_103a.
//
// For every start pixel (x0, y0) and every velocity v, the coadd of Sec. 2.1.5
//   Psi = sum_t psi_t(x0 + dx_vt, y0 + dy_vt),  Phi = sum_t phi_t(...)
// over the epochs whose pixel lies in the image, nu = Psi / sqrt(Phi), and the
// k best (nu desc, vidx asc) valid trajectories per start pixel.
//
// Work decomposition (GB300-first, not the paper's 32x16 thread blocks):
//   - a CTA owns 8 rows x SPAN columns of start pixels, one warp per row; a lane
//     owns P loads' worth of pixels (FP32: pixel lane + 32 p; 16-bit: the pixel
//     pair 2 lane + 64 p, + 1) and runs the whole velocity loop for them.  The
//     admission threshold of each pixel's top-k (its k-th (nu, vidx)) is in
//     registers, the list of (nu, 16-bit velocity index) in shared memory.
//     Shared memory per CTA is kept small: the kernel is latency-bound (resident
//     warps set its throughput) and the SRAM left to L1 serves the early epochs'
//     gathers, which neighbouring velocities share;
//   - k <= 8: slot-major lists, each lane inserting into its own pixels' lists.
//     k > 8: pixel-major lists with an odd stride (k | 1), and when at most
//     kCoopMax lanes of a warp have a candidate for one pixel slot the warp
//     inserts each cooperatively (lane j holds slot j: one load, one ballot, one
//     shifted store) instead of one lane walking a long list while the others
//     wait; the epochs' last, partial load batch is predicated (one round trip);
//   - for one (velocity, epoch) a warp's loads cover SPAN consecutive pixels of
//     one plane row: fully coalesced 8-byte loads.  16-bit pairs are 8-byte
//     aligned because the planes also exist shifted by one pixel (the "phase 1"
//     copy) and odd shifts read that copy;
//   - the (velocity, epoch) table is staged per CTA in shared memory and checked
//     there once: each entry holds the element offset of the shifted row start
//     (epoch plane and phase included), a mask of the CTA's warps whose shifted
//     span overlaps the image, and the epoch's power-of-two scale exponents.
//     The inner loop is one broadcast load (a 16-byte pair of entries for FP32
//     and k > 8), one bit test, a select, the gathers and one packed f32x2
//     accumulate per pixel (16-bit: one mixed-precision FMA per value);
//   - spans that overlap the image only partly read the zero columns the planes
//     carry left and right of every row (kSpan wide); spans that miss it read a
//     small zero block that stays in L1, so off-image steps cost no memory
//     traffic and "outside contributes nothing" holds exactly;
//   - epochs at t = t_min have offset 0 for every velocity: their contribution is
//     loaded once per pixel before the velocity loop;
//   - velocities are processed in the order the host planner gives (sorted by
//     their latest-epoch offset, for L2 locality of the resident CTAs); ties in
//     nu are broken by the caller's velocity index, so the order changes no
//     result;
//   - CTAs take their tiles in super-columns a few tiles wide, row by row within
//     each, so the CTAs resident at one time cover a compact block of start
//     pixels and the late epochs' rows they read stay in L2 (row-by-row order
//     makes them span whole image rows, whose late-epoch windows fall out).
// The Psi/Phi of each kept trajectory are recomputed at the end by the same
// sequence of operations (bit-identical) together with nobs.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "kb_device.cuh"

namespace kb {

namespace {

using namespace dev;

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int TAB = 512;    // (velocity, epoch) entries staged per chunk (small: occupancy)
constexpr uint16_t kNoV = 0xFFFF;   // empty list slot (velocity indices are < 65535)

// zero block read by spans that miss the image (static device memory is zero-initialised)
__device__ __align__(16) float2 g_zero_block[4 * 32];

__device__ __forceinline__ float2 exp_scale(int e) {
    return make_float2(__int_as_float((e & 0xff) << 23), __int_as_float(((e >> 8) & 0xff) << 23));
}
__device__ __forceinline__ int scale_exp(float2 s) {
    return (int)((__float_as_uint(s.x) >> 23) & 0xff) | (int)(((__float_as_uint(s.y) >> 23) & 0xff) << 8);
}

// per-load traits: FP32 loads one pixel's (psi, phi), 16-bit loads two adjacent pixels' codes
template <int STORAGE>
struct Gather;
template <>
struct Gather<KB_F32> {
    typedef float2 LT;
    static constexpr int PIX = 1;
    __device__ __forceinline__ static void acc(float2 *a, LT v, float2) { a[0] = add2(a[0], v); }
};
template <int STORAGE>
struct Gather16 {
    typedef uint2 LT;
    static constexpr int PIX = 2;
    __device__ __forceinline__ static void acc(float2 *a, LT v, float2 s) {
        a[0] = Store<STORAGE>::acc(a[0], v.x, s);
        a[1] = Store<STORAGE>::acc(a[1], v.y, s);
    }
};
// BF16: mixed-precision fma.rn.f32.bf16 takes each code straight from its register
// half; the scale is a power of two (exactly a bf16), so code * scale is exact and
// the sum is rounded once -- the same FP32 result as unpacking and fma.rn.f32x2.
__device__ __forceinline__ void bf16_acc(float2 &a, uint32_t code, uint32_t sp16, uint32_t sf16) {
    asm("{\n\t.reg .b16 lo, hi, sp, sf;\n\t"
        "mov.b32 {lo, hi}, %2;\n\t"
        "cvt.u16.u32 sp, %3;\n\t"
        "cvt.u16.u32 sf, %4;\n\t"
        "fma.rn.f32.bf16 %0, lo, sp, %0;\n\t"
        "fma.rn.f32.bf16 %1, hi, sf, %1;\n\t}"
        : "+f"(a.x), "+f"(a.y)
        : "r"(code), "r"(sp16), "r"(sf16));
}
template <>
struct Gather<KB_BF16> {
    typedef uint2 LT;
    static constexpr int PIX = 2;
    __device__ __forceinline__ static void acc(float2 *a, LT v, float2 s) {
        // bf16 bit patterns of the two scales: the high halves of their float bits
        const uint32_t sp = __float_as_uint(s.x) >> 16, sf = __float_as_uint(s.y) >> 16;
        bf16_acc(a[0], v.x, sp, sf);
        bf16_acc(a[1], v.y, sp, sf);
    }
};
template <>
struct Gather<KB_F16> : Gather16<KB_F16> {};

// staged table entry: element offset (32 or 64 bit) and (warp mask | scale exponents << 16)
template <typename I>
struct Entry {
    I idx;
    int info;
};

// two consecutive table entries (the first at an even index) in one 16-byte load
template <typename E>
__device__ __forceinline__ void load_pair(const E *t, E &a, E &b) {
    if constexpr (sizeof(E) == 8) {
        const int4 w = *reinterpret_cast<const int4 *>(t);
        a.idx = w.x;
        a.info = w.y;
        b.idx = w.z;
        b.info = w.w;
    } else {
        a = t[0];
        b = t[1];
    }
}

// with k > 8, a warp's list insertions for one pixel slot are done cooperatively
// (the whole warp per candidate) when at most this many of its lanes insert, else
// by each lane alone
constexpr int kCoopMax = 3;

// One CTA tile (rows by * 8 .. +7, columns bx * SPAN .. +SPAN-1) of one search:
// the body of both the one-search kernel and the persistent batch kernel.
template <int STORAGE, int P, int C, bool PT, typename I>
__device__ __forceinline__ void search_tile(const SearchArgs &a, int bx, int by, float2 *s_scale, int4 *s_dyn4) {
    typedef Store<STORAGE> St;
    typedef typename St::T T;         // one pixel's (psi, phi)
    typedef Gather<STORAGE> G;
    typedef typename G::LT LT;        // one load
    typedef Entry<I> E;
    constexpr int PX = P * G::PIX;    // pixels per lane
    constexpr int SPAN = 32 * PX;     // pixels per warp row segment
    constexpr int LS = THREADS * PX;  // list columns (pixels) of the CTA

    // s_scale: per time-ordered epoch.  s_dyn4: table E [TAB] | velocity ids [TAB] |
    // list nu float [KP * LS] | list vidx u16 [KP * LS].  Column c = p * THREADS +
    // thread holds one pixel's list, best first; slot i of column c is at c * CS + i * IS.
    //   k <= 8 (PT false): slot-major, CS = 1, IS = LS, KP = k: each lane walks its
    //     own lists, consecutive lanes in consecutive banks.
    //   k > 8 (PT true): column-major with an odd stride, CS = KP = k | 1, IS = 1: a
    //     pixel's slots are contiguous for the warp-cooperative insertion, and lanes
    //     walking their own lists still hit distinct banks.
    E *s_tab = reinterpret_cast<E *>(s_dyn4);
    int *s_vid = reinterpret_cast<int *>(s_tab + TAB);
    const int N = a.N, n0 = a.n0, NJ = N - n0, k = a.k;
    const int KP = PT ? (a.k | 1) : a.k, CS = PT ? KP : 1, IS = PT ? 1 : LS;
    const int NJP = (NJ + 1) & ~1;   // table row stride: even, so entries pair into 16-byte loads
    float *s_ln = reinterpret_cast<float *>(s_vid + TAB);
    uint16_t *s_lv = reinterpret_cast<uint16_t *>(s_ln + KP * LS);

    for (int j = threadIdx.x; j < N; j += THREADS)
        s_scale[j] = (STORAGE == KB_F32) ? make_float2(1.0f, 1.0f) : exp_scale(scale_exp(a.scales[a.epoch_of[j]]));
    for (int i = threadIdx.x; i < KP * LS; i += THREADS) {
        s_ln[i] = -INFINITY;
        s_lv[i] = kNoV;
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y0 = by * WARPS;
    const int y = y0 + warp;
    const int xw = bx * SPAN;
    const bool active = y < a.H;
    const T *planes = reinterpret_cast<const T *>(a.planes);
    // element index of this lane's first pixel within a plane (even for 16-bit storage)
    const I tb = (I)(a.origin + (long long)y * a.pitch + xw + lane * G::PIX);
    const LT *zero = reinterpret_cast<const LT *>(g_zero_block) + lane;

    float thn[PX];
    int thv[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        thn[p] = -INFINITY;
        thv[p] = kNoV;
    }
    __syncthreads();

    // epochs at the reference time: offset 0 for every velocity (pixels past W read the zero columns)
    float2 acc0[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) acc0[p] = make_float2(0.0f, 0.0f);
    if (active) {
        for (int j = 0; j < n0; ++j) {
            const LT *src = reinterpret_cast<const LT *>(planes + (long long)a.epoch_of[j] * a.plane_elems + tb);
#pragma unroll
            for (int p = 0; p < P; ++p) G::acc(acc0 + p * G::PIX, __ldg(src + 32 * p), s_scale[j]);
        }
    }

    const int vchunk = min(a.V, TAB / max(NJP, 1));
    for (int c0 = 0; c0 < a.V; c0 += vchunk) {
        const int nc = min(vchunk, a.V - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += THREADS) s_vid[i] = a.vorder[c0 + i];
        for (int i = threadIdx.x; i < nc * NJ; i += THREADS) {
            const int vi = i / NJ, jj = i - vi * NJ;   // entry (vi, jj) at vi * NJP + jj
            const int j = n0 + jj;
            const int ep = a.epoch_of[j];
            const int2 o = a.offs[(long long)a.vorder[c0 + vi] * N + j];
            const int ox = max(-32767, min(32767, o.x)), oy = max(-32767, min(32767, o.y));
            int mask = 0;
            if (xw + ox + SPAN > 0 && xw + ox < a.W) {   // the span overlaps the image's columns
#pragma unroll
                for (int w = 0; w < WARPS; ++w)
                    if ((unsigned)(y0 + w + oy) < (unsigned)a.H) mask |= 1 << w;
            }
            long long g = (long long)ep * a.plane_elems + (long long)oy * a.pitch + ox;
            if (STORAGE != KB_F32 && (ox & 1)) g += a.phase1 - 1;   // odd shift: the phase-1 copy
            E e;
            e.idx = (I)g;
            e.info = mask | ((STORAGE == KB_F32 ? 0 : scale_exp(a.scales[ep])) << 16);
            s_tab[vi * NJP + jj] = e;
        }
        __syncthreads();
        if (!active) continue;
        for (int vi = 0; vi < nc; ++vi) {
            const int v = s_vid[vi];
            const E *tab = s_tab + vi * NJP;
            float2 acc[PX];
#pragma unroll
            for (int p = 0; p < PX; ++p) acc[p] = acc0[p];
            if constexpr (!PT) {
                // epochs in batches of C loads in flight, then one at a time
                int jj = 0;
                for (; jj + C <= NJ; jj += C) {
                    LT val[C][P];
                    int sx[C];
#pragma unroll
                    for (int q = 0; q < C; q += 2) {
                        // entries in pairs (one 16-byte shared load) for FP32; the 16-bit
                        // kernels, held to 48 registers, spill with the pair live and load singly
                        E t[2];
                        if constexpr (STORAGE == KB_F32) {
                            load_pair(tab + jj + q, t[0], t[1]);
                        } else {
                            t[0] = tab[jj + q];
                            t[1] = tab[jj + q + 1];
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            sx[q + h] = t[h].info >> 16;
                            const LT *src = ((t[h].info >> warp) & 1)
                                                ? reinterpret_cast<const LT *>(planes + (t[h].idx + tb)) : zero;
#pragma unroll
                            for (int p = 0; p < P; ++p) val[q + h][p] = __ldg(src + 32 * p);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        const float2 sc = exp_scale(sx[q]);
#pragma unroll
                        for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q][p], sc);
                    }
                }
                for (; jj < NJ; ++jj) {
                    const E t = tab[jj];
                    const LT *src =
                        ((t.info >> warp) & 1) ? reinterpret_cast<const LT *>(planes + (t.idx + tb)) : zero;
                    LT val[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) val[p] = __ldg(src + 32 * p);
                    const float2 sc = exp_scale(t.info >> 16);
#pragma unroll
                    for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[p], sc);
                }
            } else {
                // every batch of C predicated (warp-uniform): the remainder costs one
                // round trip instead of one per epoch, for more registers
                for (int jj = 0; jj < NJ; jj += C) {
                    LT val[C][P];
                    int sx[C];
#pragma unroll
                    for (int q = 0; q < C; q += 2) {
                        if (jj + q < NJ) {
                            E t[2];
                            load_pair(tab + jj + q, t[0], t[1]);   // the second may be row padding
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                if (jj + q + h < NJ) {
                                    sx[q + h] = t[h].info >> 16;
                                    const LT *src = ((t[h].info >> warp) & 1)
                                                        ? reinterpret_cast<const LT *>(planes + (t[h].idx + tb))
                                                        : zero;
#pragma unroll
                                    for (int p = 0; p < P; ++p) val[q + h][p] = __ldg(src + 32 * p);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        if (jj + q < NJ) {
                            const float2 sc = exp_scale(sx[q]);
#pragma unroll
                            for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q][p], sc);
                        }
                    }
                }
            }
            // scoring: one warp-uniform test gates the (divergent, rarer) list insertions
            float nu[PX];
            bool cand[PX];
            bool any = false;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const float F = acc[p].y;
                nu[p] = acc[p].x * rsqrtf(F);
                cand[p] = (F > 0.0f) && (nu[p] >= a.nu_min) && better(nu[p], v, thn[p], thv[p]);
                any |= cand[p];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                unsigned m = 0;
                if constexpr (PT) {
                    m = __ballot_sync(0xffffffffu, cand[p]);
                    if (m == 0) continue;
                }
                if (!PT || __popc(m) > kCoopMax) {
                    // each lane inserts into its own list, walking up from the last slot
                    if (cand[p]) {
                        float *ln = s_ln + (p * THREADS + threadIdx.x) * CS;
                        uint16_t *lv = s_lv + (p * THREADS + threadIdx.x) * CS;
                        int i = k - 1;
                        while (i > 0) {
                            const float pn = ln[(i - 1) * IS];
                            const int pv = lv[(i - 1) * IS];
                            if (!better(nu[p], v, pn, pv)) break;
                            ln[i * IS] = pn;
                            lv[i * IS] = (uint16_t)pv;
                            --i;
                        }
                        ln[i * IS] = nu[p];
                        lv[i * IS] = (uint16_t)v;
                        thn[p] = ln[(k - 1) * IS];
                        thv[p] = lv[(k - 1) * IS];
                    }
                } else {
                    // few lanes: the warp inserts their candidates one at a time, lane j
                    // holding slot j of the list (one load, one ballot, one store)
                    do {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const float nn = __shfl_sync(0xffffffffu, nu[p], src);
                        const int col = p * THREADS + warp * 32 + src;
                        float *ln = s_ln + col * KP;
                        uint16_t *lv = s_lv + col * KP;
                        float en = -INFINITY;
                        int ev = kNoV;
                        if (lane < k) {
                            en = ln[lane];
                            ev = lv[lane];
                        }
                        // first slot the candidate beats (exists: it beats the last slot)
                        const unsigned bm = __ballot_sync(0xffffffffu, lane < k && better(nn, v, en, ev));
                        const int pos = __ffs(bm) - 1;
                        const float upn = __shfl_up_sync(0xffffffffu, en, 1);
                        const int upv = __shfl_up_sync(0xffffffffu, ev, 1);
                        const float wn = lane == pos ? nn : (lane > pos ? upn : en);
                        const int wv = lane == pos ? v : (lane > pos ? upv : ev);
                        if (lane >= pos && lane < k) {
                            ln[lane] = wn;
                            lv[lane] = (uint16_t)wv;
                        }
                        const float tn = __shfl_sync(0xffffffffu, wn, k - 1);
                        const int tv = __shfl_sync(0xffffffffu, wv, k - 1);
                        if (lane == src) {
                            thn[p] = tn;
                            thv[p] = tv;
                        }
                    } while (m);
                }
                if constexpr (PT) __syncwarp();   // lists written above are read by other lanes later
            }
        }
    }
    if (!active) return;

    // epilogue: recompute Psi, Phi (same operation sequence) and nobs of the kept entries;
    // every off-image epoch added a zero in the main loop, so it adds a zero here too
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        const int x = xw + (G::PIX == 1 ? lane + 32 * p : 2 * lane + 64 * (p / 2) + (p & 1));
        if (x >= a.W) continue;
        Rec *out = a.out + ((long long)y * a.W + x) * k;
        const float *ln = s_ln + (p * THREADS + threadIdx.x) * CS;
        const uint16_t *lv = s_lv + (p * THREADS + threadIdx.x) * CS;
        for (int i = 0; i < k; ++i) {
            Rec r;
            const int v = lv[i * IS];
            if (v == kNoV) {
                r.psi = 0.0f;
                r.phi = 0.0f;
                r.nu = -INFINITY;
                r.meta = kEmptyVidx;
            } else {
                const int2 *ov = a.offs + (long long)v * N;
                float2 acc = acc0[p];
                int nobs = n0;
                for (int j = n0; j < N; ++j) {
                    const int2 o = __ldg(ov + j);
                    const int xx = x + o.x, yy = y + o.y;
                    T val = St::zero();
                    if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                        val = St::load(planes + (long long)a.epoch_of[j] * a.plane_elems + a.origin +
                                       (long long)yy * a.pitch + xx);
                        ++nobs;
                    }
                    acc = St::acc(acc, val, s_scale[j]);
                }
                r.psi = acc.x;
                r.phi = acc.y;
                r.nu = ln[i * IS];
                r.meta = (uint32_t)v | ((uint32_t)nobs << 16);
            }
            reinterpret_cast<uint4 *>(out)[i] = *reinterpret_cast<uint4 *>(&r);
        }
    }
}

// Resident CTAs per SM the register allocation is held to (0: no hold).  The
// shapes with one 8-byte load per lane and epoch, with the plain remainder loop
// (used for k <= 8, where registers decide how many CTAs an SM holds): the
// 16-bit one is held to 5 (48 registers), which measured faster than 4 despite
// the L1 the fifth CTA displaces; the FP32 one reaches 48 registers by itself
// and spills when held to it.  With the predicated remainder (k > 8, where the
// lists' shared memory limits the SM to 2-3 CTAs): 3 (85 registers).  The wider
// shapes: 2.  The batch kernel, which keeps its search's arguments in shared
// memory rather than the parameter bank and so needs more registers, is held to
// 3 for the narrow shapes and 2 for the wide ones.
template <int STORAGE, int P, bool PT>
constexpr int min_ctas() {
    constexpr bool narrow = STORAGE == KB_F32 ? P <= 2 : P <= 1;
    if (!narrow) return 2;
    if (PT) return 3;
    return STORAGE == KB_F32 ? 0 : 5;
}

template <int STORAGE, int P>
constexpr int min_ctas_batch() {
    return (STORAGE == KB_F32 ? P <= 2 : P <= 1) ? 3 : 2;
}

template <int STORAGE, int P, int C, bool PT, typename I>
__global__ void __launch_bounds__(THREADS, min_ctas<STORAGE, P, PT>()) search_kernel(SearchArgs a) {
    __shared__ float2 s_scale[KB_MAX_EPOCHS];
    extern __shared__ int4 s_dyn4[];
    int bx = blockIdx.x, by = blockIdx.y;
    if (a.swz > 0 && a.swz < (int)gridDim.x) {
        // CTAs start roughly in linear order: deal the tiles out in super-columns of
        // swz tiles, row by row within each (the last super-column may be narrower)
        const int gx = gridDim.x, lin = blockIdx.y * gx + blockIdx.x;
        const int per = a.swz * gridDim.y, s = lin / per, r = lin - s * per;
        const int w = min(a.swz, gx - s * a.swz);
        by = r / w;
        bx = s * a.swz + (r - by * w);
    }
    search_tile<STORAGE, P, C, PT, I>(a, bx, a.by0 + by, s_scale, s_dyn4);
}

// Persistent batch search: CTAs take (job, tile) work items from an atomic
// counter until the list is exhausted, copying the item's job descriptor into
// shared memory first.  The item list is ordered by cost (largest first), so
// uneven stacks, grids and epoch counts balance across the SMs.
template <int STORAGE, int P, int C, bool PT, typename I>
__global__ void __launch_bounds__(THREADS, min_ctas_batch<STORAGE, P>()) search_batch_kernel(const SearchArgs *jobs, const int4 *items, int n_items,
                                                             int *counter) {
    __shared__ float2 s_scale[KB_MAX_EPOCHS];
    __shared__ SearchArgs s_job;
    __shared__ int s_it;
    extern __shared__ int4 s_dyn4[];
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= n_items) break;
        const int4 w = items[it];
        for (int i = threadIdx.x; i < (int)(sizeof(SearchArgs) / sizeof(int)); i += THREADS)
            reinterpret_cast<int *>(&s_job)[i] = reinterpret_cast<const int *>(jobs + w.x)[i];
        __syncthreads();
        search_tile<STORAGE, P, C, PT, I>(s_job, w.y, w.z, s_scale, s_dyn4);
        __syncthreads();
    }
}

template <int STORAGE, int P, int C, bool PT, typename I>
cudaError_t launch_pt(const SearchArgs &a, cudaStream_t st, int sm_count) {
    constexpr int SPAN = 32 * P * Gather<STORAGE>::PIX;
    static_assert(SPAN <= kSpan, "warp span wider than the zero columns");
    auto kern = search_kernel<STORAGE, P, C, PT, I>;
    dim3 grid((a.W + SPAN - 1) / SPAN, a.nby > 0 ? a.nby : (a.H + WARPS - 1) / WARPS);
    size_t smem = (size_t)TAB * (sizeof(Entry<I>) + sizeof(int)) +
                  (size_t)(PT ? (a.k | 1) : a.k) * THREADS * P * Gather<STORAGE>::PIX * (sizeof(float) + sizeof(uint16_t));
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // Shared-memory carveout: it trades resident CTAs against the L1 that the early
    // epochs' gathers reuse across velocities.  Automatic: the driver's choice up to
    // k = 8; longer lists take 58 % (measured on the 12 x 4096^2 workload: k = 12
    // runs 1.25x faster than with the driver's choice).
    int carve = a.carveout;
    if (carve < 0 && a.k > 8) carve = 58;
    if (err == cudaSuccess && carve >= 0)
        err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    if (a.waves > 0) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (err != cudaSuccess) return err;
    // bands of `waves` resident waves of CTAs, one launch each (see kb_set_search_waves)
    const int band = per_sm > 0 ? max(1, (int)((long long)a.waves * per_sm * sm_count / grid.x)) : (int)grid.y;
    const int by_end = a.by0 + (int)grid.y;
    for (int b0 = a.by0; b0 < by_end; b0 += band) {
        SearchArgs ab = a;
        ab.by0 = b0;
        ab.nby = min(band, by_end - b0);
        kern<<<dim3(grid.x, ab.nby), THREADS, smem, st>>>(ab);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// lists longer than 8 take the predicated-remainder form (see min_ctas)
template <int STORAGE, int P, int C, typename I>
cudaError_t launch_one(const SearchArgs &a, cudaStream_t st, int sm_count) {
    if (a.k > 8) return launch_pt<STORAGE, P, C, true, I>(a, st, sm_count);
    return launch_pt<STORAGE, P, C, false, I>(a, st, sm_count);
}

template <int STORAGE, int P, int C>
cudaError_t launch_idx(const SearchArgs &a, cudaStream_t st, int sm_count) {
    // 32-bit element offsets when every plane of both phases fits
    const long long span = (STORAGE == KB_F32 ? 1LL : 2LL) * a.N * a.plane_elems;
    if (span < (1LL << 31) - 1) return launch_one<STORAGE, P, C, int>(a, st, sm_count);
    return launch_one<STORAGE, P, C, long long>(a, st, sm_count);
}

// Shapes: (loads per lane P, epochs per load batch C); a 16-bit load is two pixels.
template <int STORAGE>
cudaError_t launch_storage(const SearchArgs &a, cudaStream_t st, int sm_count) {
    if constexpr (STORAGE == KB_F32) {
        switch (a.variant) {
            case 1: return launch_idx<STORAGE, 4, 4>(a, st, sm_count);
            case 2: return launch_idx<STORAGE, 2, 4>(a, st, sm_count);
            case 3: return launch_idx<STORAGE, 4, 8>(a, st, sm_count);
            default: return launch_idx<STORAGE, 2, 8>(a, st, sm_count);
        }
    } else {
        switch (a.variant) {
            case 1: return launch_idx<STORAGE, 2, 4>(a, st, sm_count);
            case 2: return launch_idx<STORAGE, 1, 4>(a, st, sm_count);
            case 3: return launch_idx<STORAGE, 2, 8>(a, st, sm_count);
            default: return launch_idx<STORAGE, 1, 8>(a, st, sm_count);
        }
    }
}

template <int STORAGE, int P, int C, bool PT, typename I>
cudaError_t launch_batch_pt(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int kmax,
                            int carve, int sm_count, cudaStream_t st) {
    size_t smem = (size_t)TAB * (sizeof(Entry<I>) + sizeof(int)) +
                  (size_t)(PT ? (kmax | 1) : kmax) * THREADS * P * Gather<STORAGE>::PIX * (sizeof(float) + sizeof(uint16_t));
    auto kern = search_batch_kernel<STORAGE, P, C, PT, I>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (carve < 0 && kmax > 8) carve = 58;   // the rule of the one-search launch
    if (err == cudaSuccess && carve >= 0)
        err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    int per_sm = 0;
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (err != cudaSuccess) return err;
    // persistent grid: every SM filled with as many CTAs as it can hold
    const int grid = sm_count * (per_sm > 0 ? per_sm : 1);
    kern<<<grid, THREADS, smem, st>>>(jobs, items, n_items, counter);
    return cudaGetLastError();
}

template <int STORAGE, int P, int C, typename I>
cudaError_t launch_batch_one(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int kmax,
                             int carve, int sm_count, cudaStream_t st) {
    if (kmax > 8) return launch_batch_pt<STORAGE, P, C, true, I>(jobs, items, n_items, counter, kmax, carve, sm_count, st);
    return launch_batch_pt<STORAGE, P, C, false, I>(jobs, items, n_items, counter, kmax, carve, sm_count, st);
}

template <int STORAGE, int P, int C>
cudaError_t launch_batch_idx(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int kmax,
                             int carve, bool idx64, int sm_count, cudaStream_t st) {
    if (idx64)
        return launch_batch_one<STORAGE, P, C, long long>(jobs, items, n_items, counter, kmax, carve, sm_count, st);
    return launch_batch_one<STORAGE, P, C, int>(jobs, items, n_items, counter, kmax, carve, sm_count, st);
}

template <int STORAGE>
cudaError_t launch_batch_storage(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int variant,
                                 int kmax, int carve, bool idx64, int sm_count, cudaStream_t st) {
    if constexpr (STORAGE == KB_F32) {
        switch (variant) {
            case 1: return launch_batch_idx<STORAGE, 4, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 2: return launch_batch_idx<STORAGE, 2, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 3: return launch_batch_idx<STORAGE, 4, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            default: return launch_batch_idx<STORAGE, 2, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
        }
    } else {
        switch (variant) {
            case 1: return launch_batch_idx<STORAGE, 2, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 2: return launch_batch_idx<STORAGE, 1, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 3: return launch_batch_idx<STORAGE, 2, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            default: return launch_batch_idx<STORAGE, 1, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
        }
    }
}

}  // namespace

int search_span(int storage, int variant) {
    // loads per lane P of the shape, times 32 lanes, times pixels per load
    static const int p32[5] = {2, 4, 2, 4, 2}, p16[5] = {1, 2, 1, 2, 1};
    const int v = (variant >= 1 && variant <= 4) ? variant : 0;
    return storage == KB_F32 ? 32 * p32[v] : 64 * p16[v];
}

cudaError_t launch_search_batch(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int storage,
                                int variant, int kmax, int carve, bool idx64, int sm_count, cudaStream_t st) {
    switch (storage) {
        case KB_F32: return launch_batch_storage<KB_F32>(jobs, items, n_items, counter, variant, kmax, carve, idx64, sm_count, st);
        case KB_BF16: return launch_batch_storage<KB_BF16>(jobs, items, n_items, counter, variant, kmax, carve, idx64, sm_count, st);
        case KB_F16: return launch_batch_storage<KB_F16>(jobs, items, n_items, counter, variant, kmax, carve, idx64, sm_count, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, int sm_count) {
    switch (a.storage) {
        case KB_F32: return launch_storage<KB_F32>(a, st, sm_count);
        case KB_BF16: return launch_storage<KB_BF16>(a, st, sm_count);
        case KB_F16: return launch_storage<KB_F16>(a, st, sm_count);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kb
