// Internal declarations of libkb: handle layouts, kernel parameter blocks and
// the launchers each translation unit provides.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/kb.h"

// NVTX ranges around the library's entry points (header-only NVTX3: without a
// tool attached, a push or pop is a check of one function pointer).  Profilers
// attribute the kernels an entry point launches to its range, e.g.
// ncu --nvtx --nvtx-include "kb_search/".
#include <nvtx3/nvToolsExt.h>

namespace kb {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Packed 16-bit (psi, phi) pair: low half psi, high half phi.
typedef uint32_t pair16;

// Plane layout.  Every psi/phi plane row carries pad_x = kSpan zero pixels on
// its left and right, and every plane pad_y = kPadRows zero rows above and
// below; pixel (x, y) of epoch e is element e * plane_elems + origin + y * pitch
// + x with origin = pad_y * pitch + pad_x.  A warp span of up to kSpan pixels
// that overlaps the image only partly therefore reads exactly 0 for its
// off-image pixels ("outside contributes nothing") with no per-lane bounds
// checks, and so does a band of up to kPadRows rows that overlaps the image's
// rows only partly.
constexpr int kSpan = 128;
constexpr int kPadRows = 8;   // >= the rows of a search CTA
struct Layout {
    int pad_x = 0, pad_y = 0, pitch = 0, rows = 0;
    long long plane_elems = 0, origin = 0;
};
inline Layout make_layout(int H, int W) {
    Layout L;
    L.pad_x = kSpan;
    L.pad_y = kPadRows;
    L.pitch = (W + 2 * kSpan + 3) & ~3;
    L.rows = H + 2 * kPadRows;
    L.plane_elems = (long long)L.rows * L.pitch;
    L.origin = (long long)L.pad_y * L.pitch + L.pad_x;
    return L;
}

// Device record of one kept trajectory (16 bytes, one vector store).
struct Rec {
    float psi, phi, nu;
    uint32_t meta;  // vidx (bits 0-15, 0xFFFF = empty) | nobs (bits 16-23) | flags (24-31)
};
constexpr uint32_t kEmptyVidx = 0xFFFFu;
static_assert(sizeof(Rec) == sizeof(kb_result_compact), "the device record is the compact transfer record");

// A candidate of the rescoring's key-form search (one 32-bit key, 0 = empty): with
// b bits for a velocity index, the high 32 - b bits hold nu's order-preserving FP32
// encoding rounded upwards to a multiple of 2^b, the low b bits 2^b - 1 - vidx.
__device__ __forceinline__ float cand_key_nu(uint32_t key, int b) {
    const uint32_t ord = key & ~((1u << b) - 1u);
    return __uint_as_float((ord & 0x80000000u) ? (ord & 0x7FFFFFFFu) : ~ord);
}
__device__ __forceinline__ int cand_key_vidx(uint32_t key, int b) {
    const uint32_t m = (1u << b) - 1u;
    return (int)(m - (key & m));
}

// Device record after FP64 rescoring (32 bytes).
struct Rec64 {
    double psi, phi;
    double nu;
    uint32_t vidx;  // 0xFFFF = empty
    uint32_t nobs;
};

}  // namespace kb

struct kb_ctx {
    int device = 0;
    size_t budget = 0;   // 0 = no cap
    size_t in_use = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    int search_variant = 0;   // 0 = automatic
    int search_carveout = -1; // -1 = automatic
    int search_order = -1;    // velocity processing order: 0 by latest (dy, dx), 1 Hilbert, 2 the caller's
    int search_swizzle = -1;  // register-gather search: tile order in super-columns of this many tiles (0: rows)
    std::string err;
    std::mutex mu;
    // Stream-ordered device memory: a pool that keeps freed blocks for reuse and
    // an internal stream that allocations and frees are ordered on, so creating
    // and freeing stacks and jobs never synchronises the device (cudaMalloc /
    // cudaFree would, stalling every other stream's kernels).
    cudaMemPool_t pool = nullptr;
    cudaStream_t astream = nullptr;
    // pinned host staging blocks returned by freed jobs and stacks, for reuse
    std::vector<std::pair<void *, size_t>> host_cache;
    size_t host_cached = 0;
};

struct kb_stack {
    kb_ctx *ctx = nullptr;
    int N = 0, H = 0, W = 0;
    kb::Layout L;
    int storage = KB_F32;
    float2 *f32 = nullptr;        // [N][plane] (psi, phi), zero border
    kb::pair16 *q16 = nullptr;    // [2][N][plane] packed 16-bit codes: phase 0, and phase 1 shifted by one
                                  // element (phase1[i] = phase0[i + 1]); null for FP32 storage
    float2 *scales = nullptr;     // device [N] (psi scale, phi scale)
    unsigned *maxbits = nullptr;  // device [2N] max |psi|, max phi (float bits) for the scales
    float *taps = nullptr;        // device per-epoch PSF taps (layout in kb_psiphi.cu)
    float *taps_host = nullptr;   // pinned staging of the taps
    size_t taps_host_cap = 0;     // its capacity in bytes
    size_t taps_floats = 0;
    cudaEvent_t taps_done = nullptr;  // taps_host may be rewritten once this has completed
    cudaEvent_t used = nullptr;       // recorded after the last kernel that read the planes
    // likelihood bound planes of the thresholded search (KB_PRUNE), built on first use for
    // one span width and invalidated by kb_make_psi_phi
    float *snr2 = nullptr;        // [N][H][(W + 31) / 32 + snr2_span / 32]
    size_t snr2_bytes = 0;
    int snr2_span = 0;
    bool snr2_valid = false;
    size_t bytes = 0;
    bool filled = false;
    bool zeroed = false;          // the FP32 planes (borders included) were cleared on a stream
};

struct kb_job {
    kb_ctx *ctx = nullptr;
    int H = 0, W = 0, Ncap = 0, Vcap = 0, kcap = 0, flags = 0;
    // last search
    int N = 0, V = 0, k = 0, kkeep = 0;   // kkeep = candidates kept by the search kernel
    int storage = KB_F32;
    bool rescored = false;
    // device tables
    int2 *offs = nullptr;        // [Vcap][Ncap] (dx, dy) in time order of epochs
    int *vorder = nullptr;       // [Vcap] processing order -> caller vidx
    uint32_t *ptab = nullptr;    // [Vcap][Ncap] producer table, processing order
    int *status = nullptr;       // device status word of the last search
    int *hstat = nullptr;        // pinned host copies, written after the last search: [0] status, [1] repaired
    cudaEvent_t done = nullptr;  // recorded after the last search's kernels
    int *epoch_of = nullptr;     // [Ncap] time-order position -> stack epoch
    float2 *vq = nullptr;        // [Vcap] quantised velocity (px/day) for the results
    // pinned staging for the tables
    void *stage = nullptr;
    size_t stage_bytes = 0, stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    // results
    kb::Rec *recs = nullptr;     // [H*W][kkeep_cap]
    kb::Rec64 *recs64 = nullptr; // [H*W][kcap] (rescoring)
    int *ulist = nullptr;        // [H*W] pixels whose rescored top-k was not certified (rescoring)
    int *ucount = nullptr;       // their number (rescoring)
    int kkeep_cap = 0;
    kb_result *expand = nullptr; // device staging for host-bound kb_results (lazy)
    cudaEvent_t rdone = nullptr; // recorded after the last results read (kb_results_async)
    kb_batch *owner = nullptr;   // the batch whose tables this job holds (kb_search refuses it)
    size_t expand_cap = 0;
    size_t bytes = 0;
};

namespace kb {

// ---- stage (a) ---------------------------------------------------------------
struct PsiPhiArgs {
    const float *sci, *var;
    const uint8_t *mask;   // may be null
    float bright_max;
    int N, H, W, pitch, K;
    long long plane_elems, origin;
    bool separable;
    int seg;               // rows per CTA of the streaming separable kernel (set by launch_psi_phi)
    const float *taps;     // device taps (see kb_psiphi.cu)
    float2 *out;           // [N][H][pitch]
    unsigned *maxbits;     // [2N] or null
};
cudaError_t launch_psi_phi(const PsiPhiArgs &a, cudaStream_t st);
cudaError_t launch_quantize(const float2 *f32, pair16 *q16, float2 *scales, const unsigned *maxbits, int N,
                            long long plane_elems, int storage, cudaStream_t st);
// layout helper: floats needed for the taps of N epochs with kernel size K
size_t taps_floats(int N, int K, bool separable);
// rank-1 test and factors of a K x K PSF, T(i, j) = a(i) b(j) (host)
bool factor_psf(const float *T, int K, std::vector<double> &a, std::vector<double> &b);

// ---- stage (b) ---------------------------------------------------------------
struct SearchArgs {
    const void *planes;      // float2 planes, or pair16 planes of both phases
    int storage;             // KB_F32 / KB_BF16 / KB_F16
    long long plane_elems;   // elements per plane (layout)
    long long origin;        // element of pixel (0, 0) within a plane
    long long phase1;        // element offset of the 16-bit phase-1 copy (N * plane_elems)
    long long planes_elems;  // elements (pixels) of the planes' allocation, both phases (KB_DEBUG checks)
    int pad_x;               // zero columns left of every row (layout)
    int pad_y;               // zero rows above every plane (layout)
    int H, W, pitch, N;      // N epochs, in time order through epoch_of
    int n0;                  // leading time-ordered epochs at offset 0 for every velocity
    const int *epoch_of;     // [N]
    const int2 *offs;        // [V][N] time order
    const int *vorder;       // [V]
    int V;
    const float2 *scales;    // [N] stack epochs (16-bit storage), device
    float nu_min;
    int k;                   // results kept per pixel (<= 32)
    Rec *out;                // [H*W][k]
    int variant;             // kernel shape, 0 = automatic
    int carveout;            // preferred shared-memory carveout (percent of the maximum), -1 = automatic
    const uint32_t *ptab;    // [V][N - n0] packed (dx, dy) int16 in processing order (pipelined kernel)
    int *status;             // device status word: KB_ETIMEOUT if a bounded wait gave up
    int by0, nby;            // register-gather kernel: row tiles by0 .. by0 + nby - 1 (nby 0: all)
    int swz;                 // tile order: super-columns of this many tiles (0: row by row)
    int key_bits;            // bits of a velocity index in a candidate key: smallest b with V <= 2^b
    int cand_only;           // candidates for FP64 rescoring: records carry vidx and nu only (the
                             // rescoring recomputes the sums), so the epilogue gathers nothing
    const float *snr2;       // KB_PRUNE: span bound planes [N][H][(W + 31) / 32 + span / 32] (stack epochs), else null
    float nu_min2_slack;     // KB_PRUNE: skip a span when its bound times (1 + 2^-14) is below this (nu_min^2)
};
// register-gather kernel (variant 0 = its default shape, 1..4)
cudaError_t launch_search(const SearchArgs &a, cudaStream_t st);
// KB_DEBUG builds: the first out-of-bounds access the search kernels recorded
// ((site << 56) | offset, 0 if none), then cleared if reset; cudaErrorNotSupported
// in other builds
cudaError_t debug_word(unsigned long long *word, bool reset);
// whether launch_search(a) keeps its candidate lists in key form (a candidate search for
// the FP64 rescoring): the records' nu are then rounded upwards to 32 - key_bits bits
// of their order-preserving FP32 encoding
bool search_keys(const SearchArgs &a);
// the automatic shape's span for lists of k (pixels per warp, the KB_PRUNE window)
int search_auto_span(int storage, int k);

// likelihood bound planes of the thresholded search (kb_prune.cu)
struct SnrArgs {
    const void *planes;      // FP32 planes or 16-bit phase-0 planes of the stack
    int storage;
    const float2 *scales;    // [N] 16-bit scales (device)
    long long plane_elems, origin;
    int N, H, W, pitch, span;
    float *out;              // [N][H][(W + 31) / 32 + span / 32]
};
cudaError_t launch_snr2(const SnrArgs &a, cudaStream_t st);
// TMA-pipelined kernel (variants 5..8)
cudaError_t launch_search_tma(const SearchArgs &a, cudaStream_t st);
// persistent batch kernel over (job, tile) items {job, tile x, tile y, 0}; all jobs of
// one launch share storage, shape (variant 0..4) and index width; lists sized for kmax;
// carve = shared-memory carveout percent (-1: the automatic rule)
cudaError_t launch_search_batch(const SearchArgs *jobs, const int4 *items, int n_items, int *counter, int storage,
                                int variant, int kmax, int carve, bool idx64, int sm_count, cudaStream_t st);
// pixels per CTA row segment of a register-gather shape (tile width) for lists of k
int search_span(int storage, int variant, int k);
// the explicit shape (1..4) that the automatic choice (variant 0) takes for lists of k
int default_variant(int storage, int k);
// rows per CTA tile of the register-gather kernel
constexpr int kTileRows = 8;

struct RescoreArgs {
    const float2 *f32;       // FP32 planes
    long long plane_elems, origin;
    int H, W, pitch, N, V;
    const int *epoch_of;
    const int2 *offs;        // [V][N] time order
    const unsigned *maxbits; // [2N] per-epoch max |psi|, max phi (float bits), for the exact sums
    const Rec *cand;         // [H*W][kc] records, or 32-bit candidate keys when nu_key > 0
    int kc;                  // candidates per pixel
    int k;                   // results per pixel
    double nu_min;
    double unit;             // unit roundoff of the searched storage (0 for FP32)
    int nu_key;              // key bits b of the candidates' nu (search_keys), 0: nu as searched
    Rec64 *out;              // [H*W][k]
    int *ulist;              // uncertain pixels (capacity H*W)
    int *ucount;             // their number
};
// FP64 rescoring of the candidates with the per-pixel certificate; uncertain
// pixels are appended to ulist
cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st);
// exhaustive FP64 re-search of the uncertain pixels (one warp per pixel)
cudaError_t launch_repair(const RescoreArgs &a, cudaStream_t st);

struct ExpandArgs {
    const Rec *recs;         // [H*W][krec] or null
    const Rec64 *recs64;     // [H*W][k] or null
    int krec, k, H, W;
    const float2 *vq;        // [V] quantised velocities
    long long first, count;  // record range [first, first + count) of the H*W*k output
    kb_result *out;          // device
};
cudaError_t launch_expand(const ExpandArgs &a, cudaStream_t st);
// FP64 records of a rescored job to kb_result_compact [H*W][k]
cudaError_t launch_compact(const Rec64 *recs64, long long count, kb_result_compact *out, cudaStream_t st);

// Sec. 3.3 light-curve filter of kept trajectories
struct FilterArgs {
    const float2 *f32;       // FP32 planes (phase 0)
    long long plane_elems, origin;
    int H, W, pitch, N;
    const int *epoch_of;     // [N] time order -> stack epoch
    const int2 *offs;        // [V][N] time order
    const Rec *recs;         // [H*W][krec] or null
    const Rec64 *recs64;     // [H*W][k] or null
    int krec, k;
    double nsigma2;          // nsigma^2
    kb_filtered *out;        // device [H*W][k]
};
cudaError_t launch_filter(const FilterArgs &a, cudaStream_t st);

// Sec. 3.3 postage stamps and moments
struct StampArgs {
    const float *sci;        // [N][H][W]
    const uint8_t *mask;     // [N][H][W] or null
    int N, H, W;
    const int *epoch_of;     // [N] time order -> stack epoch
    const int2 *offs;        // [V][N] time order
    const int4 *cand;        // [n] (x0, y0, vidx, 0)
    int n, r, mode;
    double aperture;         // moments over x^2 + y^2 <= aperture^2 (<= 0: the whole stamp)
    bool cut;
    kb_moment_cuts cuts;
    float *stamps;           // [n][S][S]
    kb_moments *moments;     // [n] or null
};
cudaError_t launch_stamps(const StampArgs &a, cudaStream_t st);

// Sec. 3.3 de-duplication (DBSCAN over start pixel and velocity)
struct ClusterArgs {
    const kb_result *cand;   // [n]
    int n, T;                // candidates, hash slots (a power of two >= 2n)
    double w_pos, w_vel, eps2, inv_side;
    int min_samples;
    int4 *pts, *cells;       // [n] packed (x0, y0, vx bits, vy bits), grid cell
    uint8_t *valid;          // [n] takes part (vidx >= 0, cell in range)
    int *owner, *head;       // [T] first candidate of the slot's cell, list head
    int *next, *parent;      // [n]
    uint8_t *core;           // [n]
    unsigned long long *bestnu;  // [n] per group: ordered bits of the best nu
    int *bestidx;            // [n] per group: lowest index reaching it
    int32_t *label;          // [n] out
    uint8_t *keep;           // [n] out
    uint8_t *core_out;       // [n] out or null
    unsigned *count;         // groups kept
    int *status;             // 1: coordinates out of range, 2: a loop bound was reached
};
cudaError_t launch_cluster(const ClusterArgs &a, int sm_count, cudaStream_t st);

}  // namespace kb
