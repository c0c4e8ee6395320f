// Internal declarations of libkb: handle layouts, kernel parameter blocks and
// the launchers each translation unit provides.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/kb.h"

namespace kb {

// Packed 16-bit (psi, phi) pair: low half psi, high half phi.
typedef uint32_t pair16;

// Device record of one kept trajectory (16 bytes, one vector store).
struct Rec {
    float psi, phi, nu;
    uint32_t meta;  // vidx (bits 0-15, 0xFFFF = empty) | nobs (bits 16-23) | flags (24-31)
};
constexpr uint32_t kEmptyVidx = 0xFFFFu;

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
    std::string err;
    std::mutex mu;
};

struct kb_stack {
    kb_ctx *ctx = nullptr;
    int N = 0, H = 0, W = 0;
    int pitch = 0;         // elements per row (>= W, multiple of 4)
    int storage = KB_F32;
    float2 *f32 = nullptr;        // [N][H][pitch] (psi, phi)
    kb::pair16 *q16 = nullptr;    // [N][H][pitch] packed 16-bit codes, or null
    float2 *scales = nullptr;     // device [N] (psi scale, phi scale)
    unsigned *maxbits = nullptr;  // device [2N] max |psi|, max phi (float bits) for the scales
    float *taps = nullptr;        // device per-epoch PSF taps (layout in kb_psiphi.cu)
    float *taps_host = nullptr;   // pinned staging of the taps
    size_t taps_floats = 0;
    cudaEvent_t taps_done = nullptr;  // taps_host may be rewritten once this has completed
    size_t bytes = 0;
    bool filled = false;
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
    int *epoch_of = nullptr;     // [Ncap] time-order position -> stack epoch
    float2 *vq = nullptr;        // [Vcap] quantised velocity (px/day) for the results
    // pinned staging for the tables
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;
    // results
    kb::Rec *recs = nullptr;     // [H*W][kkeep_cap]
    kb::Rec64 *recs64 = nullptr; // [H*W][kcap] (rescoring)
    int kkeep_cap = 0;
    kb_result *expand = nullptr; // device staging for host-bound kb_results (lazy)
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
    bool separable;
    const float *taps;     // device taps (see kb_psiphi.cu)
    float2 *out;           // [N][H][pitch]
    unsigned *maxbits;     // [2N] or null
};
cudaError_t launch_psi_phi(const PsiPhiArgs &a, cudaStream_t st);
cudaError_t launch_quantize(const float2 *f32, pair16 *q16, float2 *scales, const unsigned *maxbits, int N,
                            int H, int pitch, int storage, cudaStream_t st);
// layout helper: floats needed for the taps of N epochs with kernel size K
size_t taps_floats(int N, int K, bool separable);

// ---- stage (b) ---------------------------------------------------------------
struct SearchArgs {
    const void *planes;      // float2 or pair16 planes [N][H][pitch]
    int storage;             // KB_F32 / KB_BF16 / KB_F16
    long long plane_elems;   // H * pitch
    int H, W, pitch, N;      // N epochs, in time order through epoch_of
    int n0;                  // leading time-ordered epochs at offset 0 for every velocity
    const int *epoch_of;     // [N]
    const int2 *offs;        // [V][N] time order
    const int *vorder;       // [V]
    int V;
    const float2 *scales;    // [N] stack epochs (16-bit storage)
    float nu_min;
    int k;                   // results kept per pixel (<= 16)
    Rec *out;                // [H*W][k]
};
cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, int sm_count);

struct RescoreArgs {
    const float2 *f32;       // FP32 planes [N][H][pitch]
    long long plane_elems;
    int H, W, pitch, N;
    const int *epoch_of;
    const int2 *offs;        // [V][N] time order
    const Rec *cand;         // [H*W][kc]
    int kc;                  // candidates per pixel
    int k;                   // results per pixel
    double nu_min;
    Rec64 *out;              // [H*W][k]
};
cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st);

struct ExpandArgs {
    const Rec *recs;         // [H*W][krec] or null
    const Rec64 *recs64;     // [H*W][k] or null
    int krec, k, H, W;
    const float2 *vq;        // [V] quantised velocities
    long long first, count;  // record range [first, first + count) of the H*W*k output
    kb_result *out;          // device
};
cudaError_t launch_expand(const ExpandArgs &a, cudaStream_t st);

}  // namespace kb
