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
//     pair 2 lane + 64 p, + 1) and runs the whole velocity loop for them;
//   - for one (velocity, epoch) a warp's loads cover SPAN consecutive pixels of
//     one plane row: fully coalesced 8-byte loads.  16-bit pairs are 8-byte
//     aligned because the planes also exist shifted by one pixel (the "phase 1"
//     copy) and odd shifts read that copy;
//   - the (velocity, epoch) table is staged per CTA in shared memory and checked
//     there once: each entry holds the element offset of the shifted row start
//     (epoch plane and phase included), a mask of the CTA's warps whose shifted
//     span overlaps the image, and for 16-bit storage the epoch's two
//     power-of-two scales as bf16 bit patterns (the FMA's scale operand).  The
//     inner loop per entry is one broadcast load, one mask test selecting the
//     entry's offset or the offset of a zero block, one wide multiply-add for
//     the address, the gathers and one packed f32x2 add per pixel (16-bit: one
//     mixed-precision FMA per value);
//   - spans that overlap the image only partly read the zero columns the planes
//     carry left and right of every row (kSpan wide); spans that miss it read the
//     zero columns left of row 0 of plane 0, which stay in L1, so off-image steps
//     cost no memory traffic and "outside contributes nothing" holds exactly;
//   - epochs at t = t_min have offset 0 for every velocity: their contribution is
//     loaded once per pixel before the velocity loop;
//   - velocities are processed in the order the host planner gives (sorted by
//     their latest-epoch offset, for L2 locality of the resident CTAs); ties in
//     nu are broken by the caller's velocity index, so the order changes no
//     result;
//   - CTAs take their tiles in super-columns a few tiles wide, row by row within
//     each, so the CTAs resident at one time cover a compact block of start
//     pixels and the late epochs' rows they read stay in L2;
//   - top-k: each pixel's list of (nu, 16-bit velocity index), best first, is in
//     shared memory (slot-major: slot i of list column c at c + i * LS, so the
//     lanes of a warp touch distinct banks); the k-th entry is mirrored in
//     registers as the admission threshold.  A trajectory that beats its pixel's
//     threshold is not inserted at once: the warp appends it to a queue in
//     shared memory (ballot + popc), and when 32 or more are pending every lane
//     inserts one.  Candidates arrive at scattered velocities for the 64-128
//     pixels of a warp, so inserting on arrival keeps the warp busy for one
//     lane's insertion at almost every velocity; batched, the lanes insert
//     together.  Lists up to 8 long insert by rank (all slots loaded at once,
//     then the tail shifted); longer ones walk up from the last slot.
// The Psi/Phi of each kept trajectory are recomputed at the end by the same
// sequence of operations (bit-identical) together with nobs.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "kb_device.cuh"

namespace kb {

#ifdef KB_DEBUG
// KB_DEBUG: the first out-of-bounds access of the search kernels, (site << 56) | offset
__device__ unsigned long long g_debug_word;
#endif

cudaError_t debug_word(unsigned long long *word, bool reset) {
#ifdef KB_DEBUG
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(word, g_debug_word, sizeof(*word));
    if (e == cudaSuccess && reset) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_debug_word, &zero, sizeof(zero));
    }
    return e;
#else
    (void)word;
    (void)reset;
    return cudaErrorNotSupported;
#endif
}

namespace {

#ifdef KB_DEBUG
__device__ __noinline__ void debug_record(int site, long long at) {
    atomicCAS(&g_debug_word, 0ull, ((unsigned long long)site << 56) | ((unsigned long long)at & 0x00ffffffffffffffull));
}
#endif

// One load of a gather from the planes.  KB_DEBUG builds check that it lies inside
// the planes' allocation (elems pixels of type T from `planes`); one outside is
// recorded with its site and read as zero.
template <typename LT, typename T>
__device__ __forceinline__ LT gather(const LT *src, const T *planes, long long elems, int site) {
#ifdef KB_DEBUG
    const long long at = (long long)((const char *)src - (const char *)planes);
    if (at < 0 || at + (long long)sizeof(LT) > elems * (long long)sizeof(T)) {
        debug_record(site, at);
        return LT{};
    }
#else
    (void)planes;
    (void)elems;
    (void)site;
#endif
    return __ldg(src);
}

// KB_DEBUG builds: index i must lie in [0, n) (site 5: offset-table entry, 6: list column)
__device__ __forceinline__ bool debug_in(long long i, long long n, int site) {
#ifdef KB_DEBUG
    if (i < 0 || i >= n) {
        debug_record(site, i);
        return false;
    }
#else
    (void)i;
    (void)n;
    (void)site;
#endif
    return true;
}

using namespace dev;

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr uint16_t kNoV = 0xFFFF;   // empty list slot (velocity indices are < 65535)
constexpr int kRankMax = 8;         // lists up to this long insert by rank, longer ones by walking

// (velocity, epoch) entries staged per chunk (small: occupancy); the 16-bit
// entries are twice as large and their CTAs hold twice the pixels
template <int STORAGE>
__host__ __device__ constexpr int tab_entries() { return STORAGE == KB_F32 ? 512 : 256; }

__device__ __forceinline__ float2 exp_scale(int e) {
    return make_float2(__int_as_float((e & 0xff) << 23), __int_as_float(((e >> 8) & 0xff) << 23));
}
__device__ __forceinline__ int scale_exp(float2 s) {
    return (int)((__float_as_uint(s.x) >> 23) & 0xff) | (int)(((__float_as_uint(s.y) >> 23) & 0xff) << 8);
}
// Scale operand of a 16-bit load: the bf16 bit patterns of the epoch's two
// power-of-two scales, psi in the low half and phi in the high half (a power of
// two is exactly a bf16).  Unused for FP32.
__device__ __forceinline__ uint32_t sc_of(float2 s) {
    return (__float_as_uint(s.x) >> 16) | (__float_as_uint(s.y) & 0xffff0000u);
}

// per-load traits: FP32 loads one pixel's (psi, phi), 16-bit loads two adjacent pixels' codes
template <int STORAGE>
struct Gather;
template <>
struct Gather<KB_F32> {
    typedef float2 LT;
    static constexpr int PIX = 1;
    __device__ __forceinline__ static void acc(float2 *a, LT v, uint32_t) { a[0] = add2(a[0], v); }
};
// BF16: mixed-precision fma.rn.f32.bf16 takes each code and each scale straight from
// its register half; the scale is a power of two, so code * scale is exact and the
// sum is rounded once -- the same FP32 result as unpacking and fma.rn.f32x2.
__device__ __forceinline__ void bf16_acc(float2 &a, uint32_t code, uint32_t sc) {
    asm("{\n\t.reg .b16 lo, hi, sp, sf;\n\t"
        "mov.b32 {lo, hi}, %2;\n\t"
        "mov.b32 {sp, sf}, %3;\n\t"
        "fma.rn.f32.bf16 %0, lo, sp, %0;\n\t"
        "fma.rn.f32.bf16 %1, hi, sf, %1;\n\t}"
        : "+f"(a.x), "+f"(a.y)
        : "r"(code), "r"(sc));
}
template <>
struct Gather<KB_BF16> {
    typedef uint2 LT;
    static constexpr int PIX = 2;
    __device__ __forceinline__ static void acc(float2 *a, LT v, uint32_t sc) {
        bf16_acc(a[0], v.x, sc);
        bf16_acc(a[1], v.y, sc);
    }
};
// FP16: the codes converted to FP32 and fused with the scales (fma.rn.f32x2)
template <>
struct Gather<KB_F16> {
    typedef uint2 LT;
    static constexpr int PIX = 2;
    __device__ __forceinline__ static void acc(float2 *a, LT v, uint32_t sc) {
        const float2 s = make_float2(__uint_as_float(sc << 16), __uint_as_float(sc & 0xffff0000u));
        a[0] = Store<KB_F16>::acc(a[0], v.x, s);
        a[1] = Store<KB_F16>::acc(a[1], v.y, s);
    }
};

// staged table entry: element offset (32 or 64 bit), the mask of the CTA's warps
// whose shifted span overlaps the image, and for 16-bit storage the epoch's scale
// operand (16 bytes: one shared load)
template <typename I, bool SC>
struct Entry;
template <typename I>
struct Entry<I, false> {
    I idx;
    int info;
};
template <>
struct Entry<int, true> {
    int idx;
    int info;
    uint32_t sc, pad;
};
template <>
struct Entry<long long, true> {
    long long idx;
    int info;
    uint32_t sc;
};
// FP32 planes, 32-bit offsets, no pruning: compact 4-byte entries (search_tile), twice as
// many per chunk of the table in the same shared bytes
template <int STORAGE, typename I, bool PRUNE>
__host__ __device__ constexpr bool compact_entries() { return STORAGE == KB_F32 && sizeof(I) == 4 && !PRUNE; }
template <int STORAGE, typename I, bool PRUNE>
__host__ __device__ constexpr int table_entries() {
    return compact_entries<STORAGE, I, PRUNE>() ? 2 * tab_entries<STORAGE>() : tab_entries<STORAGE>();
}
template <int STORAGE, typename I, bool PRUNE>
__host__ __device__ constexpr size_t table_entry_bytes() {
    return compact_entries<STORAGE, I, PRUNE>() ? sizeof(int) : sizeof(Entry<I, STORAGE != KB_F32>);
}
template <typename I>
__device__ __forceinline__ uint32_t entry_sc(const Entry<I, false> &) { return 0u; }
template <typename I>
__device__ __forceinline__ uint32_t entry_sc(const Entry<I, true> &e) { return e.sc; }

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

// Insert (cn, cv) into the list of column `col` (slot i at col + i * LS), if it
// beats the list's last entry.  Lists up to kRankMax long: every slot is loaded
// at once, the candidate's rank is the number of entries better than it, and the
// entries below it move down one slot.  Longer lists: a walk up from the last slot.
template <bool LONG>
__device__ __forceinline__ void list_insert(float *s_ln, uint16_t *s_lv, int col, int k, int LS, float cn, int cv) {
    float *ln = s_ln + col;
    uint16_t *lv = s_lv + col;
    if constexpr (!LONG) {
        float en[kRankMax];
        int ev[kRankMax];
        int pos = 0;
#pragma unroll
        for (int i = 0; i < kRankMax; ++i) {
            en[i] = -INFINITY;
            ev[i] = kNoV;
            if (i < k) {
                en[i] = ln[i * LS];
                ev[i] = lv[i * LS];
            }
            pos += (i < k && better(en[i], ev[i], cn, cv)) ? 1 : 0;
        }
        if (pos < k) {
#pragma unroll
            for (int i = kRankMax - 1; i > 0; --i)
                if (i < k && i > pos) {
                    ln[i * LS] = en[i - 1];
                    lv[i * LS] = (uint16_t)ev[i - 1];
                }
            ln[pos * LS] = cn;
            lv[pos * LS] = (uint16_t)cv;
        }
    } else {
        int i = k - 1;
        if (!better(cn, cv, ln[i * LS], lv[i * LS])) return;
        while (i > 0) {
            const float pn = ln[(i - 1) * LS];
            const int pv = lv[(i - 1) * LS];
            if (!better(cn, cv, pn, pv)) break;
            ln[i * LS] = pn;
            lv[i * LS] = (uint16_t)pv;
            --i;
        }
        ln[i * LS] = cn;
        lv[i * LS] = (uint16_t)cv;
    }
}

// Insert the warp's n pending candidates {nu bits, vidx | (p * 32 + lane) << 16}
// into their pixels' lists, then reload every lane's register thresholds.  Each
// round takes 32 entries, one per lane; entries of one pixel are inserted one
// after the other (match_any groups them), so a list is written by one lane at a
// time.  A candidate that no longer beats its list's last entry is dropped.  The
// result does not depend on the order of insertion: a list ends as the k best of
// everything offered to it under (nu desc, vidx asc).
template <int PX, bool LONG>
__device__ __forceinline__ void flush_queue(const uint2 *q, int n, float *s_ln, uint16_t *s_lv, int k, int LS,
                                            int warp, int lane, float *thn, int *thv) {
    for (int b = 0; b < n; b += 32) {
        bool pend = b + lane < n;
        uint2 e = make_uint2(0u, 0u);
        if (pend) e = q[b + lane];
        const float cn = __uint_as_float(e.x);
        const int cv = (int)(e.y & 0xffffu);
        const int pc = (int)(e.y >> 16);
        const int col = (pc >> 5) * THREADS + warp * 32 + (pc & 31);
        // at most 32 sub-rounds: each inserts at least the lowest pending lane of every group
        for (;;) {
            if (!__any_sync(0xffffffffu, pend)) break;
            const unsigned grp = __match_any_sync(0xffffffffu, pend ? pc : 256 + lane);
            if (pend && lane == __ffs(grp) - 1) {
                pend = false;
                if (debug_in(col, LS, 6)) list_insert<LONG>(s_ln, s_lv, col, k, LS, cn, cv);
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        const int c = p * THREADS + warp * 32 + lane;
        thn[p] = s_ln[c + (k - 1) * LS];
        thv[p] = s_lv[c + (k - 1) * LS];
    }
}

// Candidate lists of a search that only feeds the FP64 rescoring (KEYS): one
// 32-bit key per slot.  With b = a.key_bits bits for a velocity index, the high
// 32 - b bits hold nu's order-preserving FP32 encoding (sign bit flipped for
// nu >= 0, every bit flipped below) rounded upwards to a multiple of 2^b, and the
// low b bits hold 2^b - 1 - vidx, so that a larger key is a better (nu desc,
// vidx asc) candidate and one unsigned compare orders two of them.  The lists
// take 4 bytes a slot instead of 6, and the rescoring gets an upper bound on the
// reduced-precision nu of every trajectory left out: the last kept key's value (a
// trajectory outside has a smaller key, so its rounded-up nu is at most that
// value).  A key's value hi and the value lo one step of 2^b below it in the
// encoding bracket the unrounded nu: lo < nu <= hi.  Empty slots are key 0, below
// the key of every finite nu (whose encoding is at least 2^23).
constexpr int kKeyMax = 16;   // longest candidate list in key form

__device__ __forceinline__ uint32_t nu_key(float nu, int v, int b) {
    const uint32_t u = __float_as_uint(nu), m = (1u << b) - 1u;
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    const uint32_t q = (ord >> b) + ((ord & m) ? 1u : 0u);   // finite nu: q << b <= encoding of +inf
    return (q << b) | (m - (uint32_t)v);
}

// Rank insertion of key ck into the key list of column `col` (k <= kKeyMax slots,
// best first), if it beats the list's last entry.
__device__ __forceinline__ void key_insert(uint32_t *s_lk, int col, int k, int LS, uint32_t ck) {
    uint32_t *lk = s_lk + col;
    if (!(ck > lk[(k - 1) * LS])) return;
    uint32_t e[kKeyMax];
    int pos = 0;
#pragma unroll
    for (int i = 0; i < kKeyMax; ++i) {
        e[i] = i < k ? lk[i * LS] : 0u;
        pos += (i < k && e[i] > ck) ? 1 : 0;
    }
#pragma unroll
    for (int i = kKeyMax - 1; i > 0; --i)
        if (i < k && i > pos) lk[i * LS] = e[i - 1];
    lk[pos * LS] = ck;
}

// flush_queue for key lists: entries {key, (p * 32 + lane) << 16}
template <int PX>
__device__ __forceinline__ void flush_keys(const uint2 *q, int n, uint32_t *s_lk, int k, int LS, int warp, int lane,
                                           uint32_t *thk) {
    for (int b = 0; b < n; b += 32) {
        bool pend = b + lane < n;
        uint2 e = make_uint2(0u, 0u);
        if (pend) e = q[b + lane];
        const int pc = (int)(e.y >> 16);
        const int col = (pc >> 5) * THREADS + warp * 32 + (pc & 31);
        for (;;) {   // at most 32 sub-rounds, as in flush_queue
            if (!__any_sync(0xffffffffu, pend)) break;
            const unsigned grp = __match_any_sync(0xffffffffu, pend ? pc : 256 + lane);
            if (pend && lane == __ffs(grp) - 1) {
                pend = false;
                if (debug_in(col, LS, 6)) key_insert(s_lk, col, k, LS, e.x);
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int p = 0; p < PX; ++p) thk[p] = s_lk[p * THREADS + warp * 32 + lane + (k - 1) * LS];
}

// One CTA tile (rows by * 8 .. +7, columns bx * SPAN .. +SPAN-1) of one search:
// the body of both the one-search kernel and the persistent batch kernel.
// LONG: lists longer than kRankMax (walk insertion, predicated last load batch).
// PRUNE: before a velocity's gathers, each warp adds its shifted span's bound
// (one value per epoch from the span bound planes, kb_prune.cu: L2-resident, one
// per 32 columns) and skips the velocity when the bound cannot reach nu_min^2
// (the results do not change).
// KEYS: candidate lists in key form for the FP64 rescoring (a.cand_only, k <= kKeyMax).
template <int STORAGE, int P, int C, bool LONG, typename I, bool PRUNE, bool KEYS = false>
__device__ __forceinline__ void search_tile(const SearchArgs &a, int bx, int by, float2 *s_scale, int4 *s_dyn4) {
    typedef Store<STORAGE> St;
    typedef typename St::T T;         // one pixel's (psi, phi)
    typedef Gather<STORAGE> G;
    typedef typename G::LT LT;        // one load
    typedef Entry<I, STORAGE != KB_F32> E;
    // Compact entries (FP32 planes, 32-bit offsets, no pruning): one 4-byte offset per
    // (velocity, epoch), four to a 16-byte shared load.  The planes' zero rows above and
    // below make every warp's row of a band that overlaps the image's rows valid, so no
    // per-warp mask is needed; a band that misses the image gets the offset of the CTA's
    // rows of zeros above row 0 of plane 0 (any warp lands in them).
    constexpr bool CE = compact_entries<STORAGE, I, PRUNE>();
    static_assert(!CE || C % 4 == 0, "compact entries are read four at a time");
    static_assert(WARPS <= kPadRows, "a band of warps' rows must fit the planes' zero rows");
    constexpr int TAB = table_entries<STORAGE, I, PRUNE>();
    constexpr size_t EB = table_entry_bytes<STORAGE, I, PRUNE>();
    constexpr int PX = P * G::PIX;    // pixels per lane
    constexpr int SPAN = 32 * PX;     // pixels per warp row segment
    constexpr int LS = THREADS * PX;  // list columns (pixels) of the CTA
    constexpr int QCAP = 32 * (PX + 1);   // < 32 pending after a flush, + one velocity's candidates

    // s_scale: per time-ordered epoch.  s_dyn4: table E [TAB] | (PRUNE) bound offsets I [TAB] |
    // velocity ids [TAB] | list nu float [k * LS] | list vidx u16 [k * LS] | (8-byte aligned)
    // per-warp queues uint2 [WARPS][QCAP].
    E *s_tab = reinterpret_cast<E *>(s_dyn4);
    I *s_rid = reinterpret_cast<I *>(reinterpret_cast<char *>(s_dyn4) + TAB * EB);
    int *s_vid = reinterpret_cast<int *>(s_rid + (PRUNE ? TAB : 0));
    const int N = a.N, n0 = a.n0, NJ = N - n0, k = a.k;
    // table row stride: even, so that entries pair into 16-byte loads; compact entries: a
    // multiple of 4, four to a 16-byte load
    const int NJP = CE ? (NJ + 3) & ~3 : (NJ + 1) & ~1;
    int *s_tab4 = reinterpret_cast<int *>(s_dyn4);
    float *s_ln = reinterpret_cast<float *>(s_vid + TAB);
    uint16_t *s_lv = reinterpret_cast<uint16_t *>(s_ln + k * LS);
    uint32_t *s_lk = reinterpret_cast<uint32_t *>(s_vid + TAB);   // KEYS: the lists instead
    constexpr size_t kSlotBytes = KEYS ? sizeof(uint32_t) : sizeof(float) + sizeof(uint16_t);
    uint2 *s_q = reinterpret_cast<uint2 *>(s_dyn4) +
                 ((TAB * (EB + sizeof(int) + (PRUNE ? sizeof(I) : 0)) + (size_t)k * LS * kSlotBytes + 7) / 8);

    for (int j = threadIdx.x; j < N; j += THREADS)
        s_scale[j] = (STORAGE == KB_F32) ? make_float2(1.0f, 1.0f) : exp_scale(scale_exp(a.scales[a.epoch_of[j]]));
    for (int i = threadIdx.x; i < k * LS; i += THREADS) {
        if constexpr (KEYS) {
            s_lk[i] = 0u;
        } else {
            s_ln[i] = -INFINITY;
            s_lv[i] = kNoV;
        }
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y0 = by * WARPS;
    const int y = y0 + warp;
    const int xw = bx * SPAN;
    const bool active = y < a.H;
    const T *planes = reinterpret_cast<const T *>(a.planes);
    // element index of this lane's first pixel within a plane (even for 16-bit storage)
    const I tb = (I)(a.origin + (long long)y * a.pitch + xw + lane * G::PIX);
    // per-thread base: an entry's loads start at planes_t + idx; zidx instead lands on
    // this lane's pixels among the zero columns left of row 0 of plane 0 (kSpan >= the
    // 128 elements a lane reads there)
    const T *planes_t = planes + tb;
    const I zidx = (I)(lane * G::PIX) - tb;
    const unsigned wbit = 1u << warp;
    uint2 *q = s_q + warp * QCAP;
    int qn = 0;                       // pending candidates of this warp (warp-uniform)
    const unsigned lt_mask = (1u << lane) - 1u;

    float thn[PX];
    int thv[PX];
    uint32_t thk[PX];   // KEYS: the thresholds as keys
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        thn[p] = -INFINITY;
        thv[p] = kNoV;
        thk[p] = 0u;
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
            for (int p = 0; p < P; ++p)
                G::acc(acc0 + p * G::PIX, gather(src + 32 * p, planes, a.planes_elems, 1), sc_of(s_scale[j]));
        }
    }

    // PRUNE: a bound row holds one value per 32 columns, (W + 31) / 32 + SPAN / 32 of them,
    // the value for a span starting at column x at (x >> 5) + SPAN / 32; the reference
    // epochs' share is fixed
    const long long RW = (long long)(a.W + 31) / 32 + SPAN / 32;
    float b0 = 0.0f;
    if constexpr (PRUNE) {
        if (active)
            for (int j = 0; j < n0; ++j)
                b0 = __fadd_ru(b0, __ldg(a.snr2 + ((long long)a.epoch_of[j] * a.H + y) * RW + (xw >> 5) + SPAN / 32));
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
            if constexpr (CE) {
                // a warp's loads start at its lane base plus the offset; rows 0..WARPS-1 of the
                // allocation are zero (the pad rows above plane 0), one per warp
                const long long zero_rows = -(a.origin + (long long)y0 * a.pitch + xw);
                if (debug_in(vi * NJP + jj, TAB, 5)) s_tab4[vi * NJP + jj] = (int)(mask ? g : zero_rows);
            } else {
                E e;
                e.idx = (I)g;
                e.info = mask;
                if constexpr (STORAGE != KB_F32) e.sc = sc_of(exp_scale(scale_exp(a.scales[ep])));
                if (debug_in(vi * NJP + jj, TAB, 5)) s_tab[vi * NJP + jj] = e;
            }
            if constexpr (PRUNE)   // the CTA's first row; a warp adds warp * RW
                s_rid[vi * NJP + jj] = mask ? (I)(((long long)ep * a.H + y0 + oy) * RW + ((xw + ox) >> 5) + SPAN / 32)
                                            : (I)0;
        }
        __syncthreads();
        if (!active) continue;
        for (int vi = 0; vi < nc; ++vi) {
            const int v = s_vid[vi];
            const E *tab = s_tab + vi * NJP;
            if constexpr (PRUNE) {
                // the span's bound on nu^2, rounded upwards, lane 0's sum for the whole warp
                float b = 0.0f;
                const I *rid = s_rid + vi * NJP;
                for (int jj = lane; jj < NJ; jj += 32)
                    if (tab[jj].info & wbit) b = __fadd_ru(b, __ldg(a.snr2 + rid[jj] + (long long)warp * RW));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) b = __fadd_ru(b, __shfl_xor_sync(0xffffffffu, b, o));
                b = __shfl_sync(0xffffffffu, b, 0);
                if (__fmul_ru(__fadd_ru(b, b0), 1.0f + 0x1p-14f) < a.nu_min2_slack) continue;
            }
            float2 acc[PX];
#pragma unroll
            for (int p = 0; p < PX; ++p) acc[p] = acc0[p];
            if constexpr (CE && !LONG) {
                // epochs in batches of C loads in flight (offsets four to a shared load), then
                // one at a time
                const int *tab4 = s_tab4 + vi * NJP;
                int jj = 0;
                for (; jj + C <= NJ; jj += C) {
                    LT val[C][P];
#pragma unroll
                    for (int q4 = 0; q4 < C; q4 += 4) {
                        const int4 o = *reinterpret_cast<const int4 *>(tab4 + jj + q4);
                        const int oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const LT *src = reinterpret_cast<const LT *>(planes_t + oo[h]);
#pragma unroll
                            for (int p = 0; p < P; ++p) val[q4 + h][p] = gather(src + 32 * p, planes, a.planes_elems, 2);
                        }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < C; ++q2) {
#pragma unroll
                        for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q2][p], 0u);
                    }
                }
                for (; jj < NJ; ++jj) {
                    const LT *src = reinterpret_cast<const LT *>(planes_t + tab4[jj]);
                    LT val[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) val[p] = gather(src + 32 * p, planes, a.planes_elems, 3);
#pragma unroll
                    for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[p], 0u);
                }
            } else if constexpr (CE) {
                // LONG: every batch of C predicated (warp-uniform), the row padding read but unused
                const int *tab4 = s_tab4 + vi * NJP;
                for (int jj = 0; jj < NJ; jj += C) {
                    LT val[C][P];
#pragma unroll
                    for (int q4 = 0; q4 < C; q4 += 4) {
                        if (jj + q4 < NJ) {
                            const int4 o = *reinterpret_cast<const int4 *>(tab4 + jj + q4);
                            const int oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                if (jj + q4 + h < NJ) {
                                    const LT *src = reinterpret_cast<const LT *>(planes_t + oo[h]);
#pragma unroll
                                    for (int p = 0; p < P; ++p)
                                        val[q4 + h][p] = gather(src + 32 * p, planes, a.planes_elems, 4);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < C; ++q2) {
                        if (jj + q2 < NJ) {
#pragma unroll
                            for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q2][p], 0u);
                        }
                    }
                }
            } else if constexpr (!LONG) {
                // epochs in batches of C loads in flight, then one at a time
                int jj = 0;
                for (; jj + C <= NJ; jj += C) {
                    LT val[C][P];
                    uint32_t sx[C];
#pragma unroll
                    for (int q2 = 0; q2 < C; q2 += 2) {
                        E t[2];
                        if constexpr (STORAGE == KB_F32) {
                            load_pair(tab + jj + q2, t[0], t[1]);   // one 16-byte shared load
                        } else {
                            t[0] = tab[jj + q2];
                            t[1] = tab[jj + q2 + 1];
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            sx[q2 + h] = entry_sc(t[h]);
                            const LT *src = reinterpret_cast<const LT *>(planes_t + ((t[h].info & wbit) ? t[h].idx : zidx));
#pragma unroll
                            for (int p = 0; p < P; ++p) val[q2 + h][p] = gather(src + 32 * p, planes, a.planes_elems, 2);
                        }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < C; ++q2) {
#pragma unroll
                        for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q2][p], sx[q2]);
                    }
                }
                for (; jj < NJ; ++jj) {
                    const E t = tab[jj];
                    const LT *src = reinterpret_cast<const LT *>(planes_t + ((t.info & wbit) ? t.idx : zidx));
                    LT val[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) val[p] = gather(src + 32 * p, planes, a.planes_elems, 3);
                    const uint32_t sc = entry_sc(t);
#pragma unroll
                    for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[p], sc);
                }
            } else {
                // every batch of C predicated (warp-uniform): the remainder costs one
                // round trip instead of one per epoch, for more registers
                for (int jj = 0; jj < NJ; jj += C) {
                    LT val[C][P];
                    uint32_t sx[C];
#pragma unroll
                    for (int q2 = 0; q2 < C; q2 += 2) {
                        if (jj + q2 < NJ) {
                            E t[2];
                            load_pair(tab + jj + q2, t[0], t[1]);   // the second may be row padding
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                if (jj + q2 + h < NJ) {
                                    sx[q2 + h] = entry_sc(t[h]);
                                    const LT *src = reinterpret_cast<const LT *>(
                                        planes_t + ((t[h].info & wbit) ? t[h].idx : zidx));
#pragma unroll
                                    for (int p = 0; p < P; ++p)
                                        val[q2 + h][p] = gather(src + 32 * p, planes, a.planes_elems, 4);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < C; ++q2) {
                        if (jj + q2 < NJ) {
#pragma unroll
                            for (int p = 0; p < P; ++p) G::acc(acc + p * G::PIX, val[q2][p], sx[q2]);
                        }
                    }
                }
            }
            // scoring, then this velocity's candidates appended to the warp's queue; the
            // lists are updated when 32 or more are pending (the register thresholds stay
            // conservative meanwhile: a stale threshold only admits more candidates)
            float nu[PX];
            uint32_t key[PX];
            bool cand[PX];
            bool any = false;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const float F = acc[p].y;
                nu[p] = acc[p].x * rsqrtf(F);
                if constexpr (KEYS) {
                    key[p] = nu_key(nu[p], v, a.key_bits);
                    cand[p] = (F > 0.0f) && (nu[p] >= a.nu_min) && key[p] > thk[p];
                } else {
                    key[p] = __float_as_uint(nu[p]);
                    cand[p] = (F > 0.0f) && (nu[p] >= a.nu_min) && better(nu[p], v, thn[p], thv[p]);
                }
                any |= cand[p];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const unsigned m = __ballot_sync(0xffffffffu, cand[p]);
                if (cand[p])
                    q[qn + __popc(m & lt_mask)] = make_uint2(key[p], (unsigned)v | ((unsigned)(p * 32 + lane) << 16));
                qn += __popc(m);
            }
            if (qn >= 32) {
                __syncwarp();
                if constexpr (KEYS)
                    flush_keys<PX>(q, qn, s_lk, k, LS, warp, lane, thk);
                else
                    flush_queue<PX, LONG>(q, qn, s_ln, s_lv, k, LS, warp, lane, thn, thv);
                qn = 0;
            }
        }
    }
    if (!active) return;
    if (qn > 0) {
        __syncwarp();
        if constexpr (KEYS)
            flush_keys<PX>(q, qn, s_lk, k, LS, warp, lane, thk);
        else
            flush_queue<PX, LONG>(q, qn, s_ln, s_lv, k, LS, warp, lane, thn, thv);
    }
    __syncwarp();
    if constexpr (KEYS) {
        // candidates for the rescoring, best first, as the keys themselves (4 bytes each,
        // decoded by the rescoring, which recomputes the sums)
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            const int x = xw + (G::PIX == 1 ? lane + 32 * p : 2 * lane + 64 * (p / 2) + (p & 1));
            if (x >= a.W) continue;
            uint32_t *out = reinterpret_cast<uint32_t *>(a.out) + ((long long)y * a.W + x) * k;
            const uint32_t *lk = s_lk + p * THREADS + threadIdx.x;
            for (int i = 0; i < k; ++i) out[i] = lk[i * LS];
        }
        return;
    }

    // epilogue: recompute Psi, Phi (same operation sequence) and nobs of the kept entries;
    // every off-image epoch added a zero in the main loop, so it adds a zero here too.
    // Four epochs at a time: their offsets, then their gathers, then the sums in order.
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        const int x = xw + (G::PIX == 1 ? lane + 32 * p : 2 * lane + 64 * (p / 2) + (p & 1));
        if (x >= a.W) continue;
        Rec *out = a.out + ((long long)y * a.W + x) * k;
        const float *ln = s_ln + p * THREADS + threadIdx.x;
        const uint16_t *lv = s_lv + p * THREADS + threadIdx.x;
        for (int i = 0; i < k; ++i) {
            Rec r;
            const int v = lv[i * LS];
            if (v == kNoV) {
                r.psi = 0.0f;
                r.phi = 0.0f;
                r.nu = -INFINITY;
                r.meta = kEmptyVidx;
            } else if (a.cand_only) {
                r.psi = 0.0f;
                r.phi = 0.0f;
                r.nu = ln[i * LS];
                r.meta = (uint32_t)v;
            } else {
                const int2 *ov = a.offs + (long long)v * N;
                float2 acc = acc0[p];
                int nobs = n0;
                int j = n0;
                for (; j + 4 <= N; j += 4) {
                    T val[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int2 o = __ldg(ov + j + u);
                        const int xx = x + o.x, yy = y + o.y;
                        val[u] = St::zero();
                        if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                            val[u] = St::load(planes + (long long)a.epoch_of[j + u] * a.plane_elems + a.origin +
                                              (long long)yy * a.pitch + xx);
                            ++nobs;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc = St::acc(acc, val[u], s_scale[j + u]);
                }
                for (; j < N; ++j) {
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
                r.nu = ln[i * LS];
                r.meta = (uint32_t)v | ((uint32_t)nobs << 16);
            }
            reinterpret_cast<uint4 *>(out)[i] = *reinterpret_cast<uint4 *>(&r);
        }
    }
}

// Resident CTAs per SM the register allocation is held to (0: no hold), by
// shape.  Lists up to 8 long (plain remainder loop): the narrow shapes (FP32 with
// two pixels per lane, 16-bit with one pixel pair) are held to 5 CTAs (48
// registers; shared memory allows 5 at k = 8); 16-bit with two pixel pairs per
// lane to 3 with 4-epoch batches (80 registers; the k = 8 lists of its 1024-pixel
// CTAs allow 3) and 2 with 8-epoch batches.  Longer lists (predicated remainder,
// shared memory for 2-3 CTAs): 3.  The wide FP32 shapes: 2.  The batch kernel,
// which keeps its search's arguments in shared memory rather than the parameter
// bank and so needs more registers, is held to 3 for the narrow shapes and 2 for
// the others.
template <int STORAGE, int P, int C, bool LONG>
constexpr int min_ctas() {
    constexpr bool narrow = STORAGE == KB_F32 ? P <= 2 : P <= 1;
    if (STORAGE != KB_F32 && P == 2) return (C <= 4 && !LONG) ? 3 : 2;
    if (!narrow) return 2;
    return LONG ? 3 : 5;
}

template <int STORAGE, int P>
constexpr int min_ctas_batch() {
    return (STORAGE == KB_F32 ? P <= 2 : P <= 1) ? 3 : 2;
}

template <int STORAGE, int P, int C, bool LONG, typename I, bool PRUNE, bool KEYS>
__global__ void __launch_bounds__(THREADS, (PRUNE && min_ctas<STORAGE, P, C, LONG>() == 5) ? 4 : min_ctas<STORAGE, P, C, LONG>())
    search_kernel(SearchArgs a) {
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
    search_tile<STORAGE, P, C, LONG, I, PRUNE, KEYS>(a, bx, a.by0 + by, s_scale, s_dyn4);
}

// Persistent batch search: CTAs take (job, tile) work items from an atomic
// counter until the list is exhausted, copying the item's job descriptor into
// shared memory first.  The item list is ordered by cost (largest first), so
// uneven stacks, grids and epoch counts balance across the SMs.
template <int STORAGE, int P, int C, bool LONG, typename I>
__global__ void __launch_bounds__(THREADS, min_ctas_batch<STORAGE, P>())
    search_batch_kernel(const SearchArgs *jobs, const int4 *items, int n_items, int *counter) {
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
        search_tile<STORAGE, P, C, LONG, I, false>(s_job, w.y, w.z, s_scale, s_dyn4);
        __syncthreads();
    }
}

// dynamic shared memory of a CTA with lists of k entries: the table, the lists and the queues
template <int STORAGE, int P, typename I, bool PRUNE = false, bool KEYS = false>
size_t tile_smem(int k) {
    constexpr int PX = P * Gather<STORAGE>::PIX;
    const size_t base = (size_t)table_entries<STORAGE, I, PRUNE>() *
                            (table_entry_bytes<STORAGE, I, PRUNE>() + sizeof(int) + (PRUNE ? sizeof(I) : 0)) +
                        (size_t)k * THREADS * PX * (KEYS ? sizeof(uint32_t) : sizeof(float) + sizeof(uint16_t));
    return (base + 7) / 8 * 8 + (size_t)WARPS * 32 * (PX + 1) * sizeof(uint2);
}

template <int STORAGE, int P, int C, bool LONG, typename I, bool PRUNE, bool KEYS = false>
cudaError_t launch_pt(const SearchArgs &a, cudaStream_t st) {
    constexpr int SPAN = 32 * P * Gather<STORAGE>::PIX;
    static_assert(SPAN <= kSpan, "warp span wider than the zero columns");
    auto kern = search_kernel<STORAGE, P, C, LONG, I, PRUNE, KEYS>;
    dim3 grid((a.W + SPAN - 1) / SPAN, a.nby > 0 ? a.nby : (a.H + WARPS - 1) / WARPS);
    const size_t smem = tile_smem<STORAGE, P, I, PRUNE, KEYS>(a.k);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // Shared-memory carveout: the driver's choice unless the caller sets one
    // (kb_set_search_carveout); it trades resident CTAs against the L1 that the
    // early epochs' gathers reuse across velocities.
    if (err == cudaSuccess && a.carveout >= 0)
        err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, a.carveout);
    if (err != cudaSuccess) return err;
    kern<<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// lists longer than kRankMax take the walking insertion and the predicated remainder
template <int STORAGE, int P, int C, typename I, bool PRUNE>
cudaError_t launch_one(const SearchArgs &a, cudaStream_t st) {
    if (a.k > kRankMax) return launch_pt<STORAGE, P, C, true, I, PRUNE>(a, st);
    return launch_pt<STORAGE, P, C, false, I, PRUNE>(a, st);
}

// the candidate search of the FP64 rescoring in key form (automatic shape, no pruning)
template <int STORAGE, int P, int C>
cudaError_t launch_keys(const SearchArgs &a, cudaStream_t st) {
    const long long span = (STORAGE == KB_F32 ? 1LL : 2LL) * a.N * a.plane_elems;
    if (span < (1LL << 31) - 1) return launch_pt<STORAGE, P, C, false, int, false, true>(a, st);
    return launch_pt<STORAGE, P, C, false, long long, false, true>(a, st);
}

// key form where it keeps at least 11 of nu's 23 fraction bits (up to 4096 velocities)
bool use_keys(const SearchArgs &a) {
    return a.cand_only && !a.snr2 && a.k <= kKeyMax && a.key_bits >= 1 && a.key_bits <= 12;
}

// 32-bit element offsets when every plane of both phases (and the bound planes) fits
template <int STORAGE, int P, int C, bool PRUNE = false>
cudaError_t launch_idx(const SearchArgs &a, cudaStream_t st) {
    const long long span = (STORAGE == KB_F32 ? 1LL : 2LL) * a.N * a.plane_elems;
    const long long rspan = PRUNE ? (long long)a.N * a.H * ((a.W + 31) / 32 + P * Gather<STORAGE>::PIX) : 0;
    if (span < (1LL << 31) - 1 && rspan < (1LL << 31) - 1) return launch_one<STORAGE, P, C, int, PRUNE>(a, st);
    return launch_one<STORAGE, P, C, long long, PRUNE>(a, st);
}

// Shapes: (loads per lane P, epochs per load batch C); a 16-bit load is two pixels.
// Defaults (variant 0), measured on the 12 x 4096^2 stack at k = 8: FP32 (2, 8)
// 88 ms against 89 for (2, 4); 16-bit (2, 4): BF16 80 ms against 91 for (1, 4),
// 96 for (2, 8) and 112 for (1, 8).
template <int STORAGE>
cudaError_t launch_storage(const SearchArgs &a, cudaStream_t st) {
    if constexpr (STORAGE == KB_F32) {
        switch (a.variant) {
            case 1: return launch_idx<STORAGE, 4, 4>(a, st);
            case 2: return launch_idx<STORAGE, 2, 4>(a, st);
            case 3: return launch_idx<STORAGE, 4, 8>(a, st);
            default:
                if (a.snr2) return launch_idx<STORAGE, 2, 8, true>(a, st);
                if (use_keys(a)) return launch_keys<STORAGE, 2, 8>(a, st);
                return launch_idx<STORAGE, 2, 8>(a, st);
        }
    } else {
        switch (a.variant) {
            case 2: return launch_idx<STORAGE, 1, 4>(a, st);
            case 3: return launch_idx<STORAGE, 2, 8>(a, st);
            case 4: return launch_idx<STORAGE, 1, 8>(a, st);
            case 1: return launch_idx<STORAGE, 2, 4>(a, st);
            // automatic: lists longer than kRankMax take the one-pair shape, whose 512-pixel
            // CTAs keep their lists' shared memory within what 3 CTAs per SM can hold
            default:
                if (use_keys(a)) return launch_keys<STORAGE, 2, 4>(a, st);
                if (a.snr2)
                    return a.k > kRankMax ? launch_idx<STORAGE, 1, 4, true>(a, st) : launch_idx<STORAGE, 2, 4, true>(a, st);
                return a.k > kRankMax ? launch_idx<STORAGE, 1, 4>(a, st) : launch_idx<STORAGE, 2, 4>(a, st);
        }
    }
}

template <int STORAGE, int P, int C, bool LONG, typename I>
cudaError_t launch_batch_pt(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int kmax,
                            int carve, int sm_count, cudaStream_t st) {
    const size_t smem = tile_smem<STORAGE, P, I>(kmax);
    auto kern = search_batch_kernel<STORAGE, P, C, LONG, I>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    if (kmax > kRankMax)
        return launch_batch_pt<STORAGE, P, C, true, I>(jobs, items, n_items, counter, kmax, carve, sm_count, st);
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
            case 2: return launch_batch_idx<STORAGE, 1, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 3: return launch_batch_idx<STORAGE, 2, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            case 4: return launch_batch_idx<STORAGE, 1, 8>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
            default: return launch_batch_idx<STORAGE, 2, 4>(jobs, items, n_items, counter, kmax, carve, idx64, sm_count, st);
        }
    }
}

}  // namespace

int search_span(int storage, int variant, int k) {
    // loads per lane P of the shape, times 32 lanes, times pixels per load
    static const int p32[5] = {2, 4, 2, 4, 2}, p16[5] = {2, 2, 1, 2, 1};
    const int v = (variant >= 1 && variant <= 4) ? variant : 0;
    if (storage != KB_F32 && v == 0 && k > kRankMax) return 64;
    return storage == KB_F32 ? 32 * p32[v] : 64 * p16[v];
}

int search_auto_span(int storage, int k) { return search_span(storage, 0, k); }

int default_variant(int storage, int k) {
    if (storage == KB_F32) return 4;       // (2, 8)
    return k > kRankMax ? 2 : 1;           // (1, 4) / (2, 4)
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

bool search_keys(const SearchArgs &a) { return a.variant == 0 && use_keys(a); }

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
    switch (a.storage) {
        case KB_F32: return launch_storage<KB_F32>(a, st);
        case KB_BF16: return launch_storage<KB_BF16>(a, st);
        case KB_F16: return launch_storage<KB_F16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kb
