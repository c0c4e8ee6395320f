// Stage (a): likelihood images of Sec. 2.1.5 on sm_103a.
//
//   psi_t(y) = sum_d nw_t(y + d) T_t(d),   phi_t(y) = sum_d w_t(y + d) T_t(d)^2
//   w = 1/sigma^2 (0 where masked),        nw = n * w (0 where masked, by select)
//
// One CTA produces a TY x TX output tile of one epoch.  It stages the input tile
// plus a halo of r = K/2 pixels in shared memory as (nw, w) pairs (coalesced row
// loads, zero outside the image), then either
//   - separable PSF T(dy, dx) = a(dy) b(dx): a horizontal pass into a second
//     shared tile and a vertical pass to the output (2 K taps per pixel), or
//   - general PSF: a single pass over the K x K taps (the paper's own choice,
//     Sec. 2.3, kept for non-Gaussian PSFs).  For the common sides (K <= 21) a
//     register-blocked form: each thread owns VR consecutive output rows of one
//     column and walks the tap columns, holding a column of taps in registers,
//     so one shared load of the tile feeds up to VR outputs.
// The (psi, phi) pair is carried through both passes as one 64-bit register pair
// and updated with packed fma.rn.f32x2.  The kernel is HBM-bound: it reads 8 B
// (9 B with a mask) and writes 8 B per pixel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "kb_internal.h"

namespace kb {

namespace {

constexpr int TX = 64;
constexpr int TY = 32;
constexpr int THREADS = 256;

__device__ __forceinline__ unsigned long long as_u64(float2 v) {
    return *reinterpret_cast<unsigned long long *>(&v);
}
__device__ __forceinline__ float2 as_f2(unsigned long long u) { return *reinterpret_cast<float2 *>(&u); }

// d = a * b + c on both lanes of a float pair
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
    return as_f2(d);
}

// Sec. 2.1.5 weights with the masking reading: any of mask, non-finite n or
// sigma^2, sigma^2 <= 0, n > bright_max gives (0, 0).  Selects, never 0 * NaN.
__device__ __forceinline__ float2 weighted(float n, float v, uint8_t m, float bright_max) {
    bool bad = (m != 0) || !isfinite(n) || !isfinite(v) || !(v > 0.0f) || (n > bright_max);
    float w = bad ? 0.0f : __frcp_rn(v);   // correctly rounded, the same value as 1.0f / v
    float nw = bad ? 0.0f : n * w;
    return make_float2(nw, w);
}

// Stages the CTA's input tile plus halo as (n w, w) pairs, zero outside the
// image: warps take rows (two at a time), lanes run along a row in chunks of 32
// (coalesced, no index division).  All loads of the two rows are issued before
// any is used, so up to 2 x 4 image/variance pairs per lane are in flight.
__device__ __forceinline__ void stage_tile(const PsiPhiArgs &a, int e, int x0, int y0, int r, int AW, int AH,
                                           float2 *A) {
    constexpr int WARPS = THREADS / 32, CH = 4;     // AW = TX + 2r <= 64 + 62 < 32 * CH
    const size_t npix = (size_t)a.H * a.W;
    const float *sci = a.sci + e * npix;
    const float *var = a.var + e * npix;
    const uint8_t *msk = a.mask ? a.mask + e * npix : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ty0 = warp; ty0 < AH; ty0 += 2 * WARPS) {
        float n[2][CH], v[2][CH];
        uint8_t m[2][CH];
        bool in[2][CH];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ty = ty0 + h * WARPS, y = y0 - r + ty;
            const bool rowin = ty < AH && y >= 0 && y < a.H;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int tx = lane + 32 * c, x = x0 - r + tx;
                in[h][c] = rowin && tx < AW && x >= 0 && x < a.W;
                n[h][c] = 0.0f;
                v[h][c] = 0.0f;
                m[h][c] = 0;
                if (in[h][c]) {
                    const size_t gi = (size_t)y * a.W + x;
                    n[h][c] = __ldg(sci + gi);
                    v[h][c] = __ldg(var + gi);
                    if (msk) m[h][c] = __ldg(msk + gi);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ty = ty0 + h * WARPS;
            if (ty >= AH) continue;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int tx = lane + 32 * c;
                if (tx < AW)
                    A[ty * AW + tx] = in[h][c] ? weighted(n[h][c], v[h][c], m[h][c], a.bright_max)
                                               : make_float2(0.0f, 0.0f);
            }
        }
    }
}

__device__ __forceinline__ void track_max(const PsiPhiArgs &a, float2 o, float &mpsi, float &mphi) {
    mpsi = fmaxf(mpsi, fabsf(o.x));
    mphi = fmaxf(mphi, o.y);
}

// Separable PSF T(dy, dx) = a(dy) b(dx), KT taps (KT = 0: the runtime K).  The
// horizontal pass writes B (AH x TX); the vertical pass gives each thread one
// column and VR consecutive output rows, so one shared load of B feeds up to VR
// outputs.  Every output sums its taps in tap order with one packed FMA each,
// whatever KT, so all instantiations give identical results.
constexpr int VR = 8;
template <int KT>
__global__ void __launch_bounds__(THREADS) psi_phi_sep_kernel(PsiPhiArgs a) {
    extern __shared__ float4 smem_raw[];
    const int K = KT > 0 ? KT : a.K, r = K / 2;
    const int e = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int AW = TX + 2 * r, AH = TY + 2 * r;

    // shared layout: taps (a, a^2)[K] vertical, then (b, b^2)[K] horizontal | A (AH x AW) | B (AH x TX)
    float *s_taps = reinterpret_cast<float *>(smem_raw);
    const int ntaps = 4 * K;
    float2 *A = reinterpret_cast<float2 *>(s_taps + ((ntaps + 3) & ~3));
    float2 *B = A + AH * AW;
    const float *taps = a.taps + (size_t)e * ntaps;
    for (int i = threadIdx.x; i < ntaps; i += THREADS) s_taps[i] = taps[i];
    stage_tile(a, e, x0, y0, r, AW, AH, A);
    __syncthreads();

    const float2 *ta = reinterpret_cast<const float2 *>(s_taps), *tb = ta + K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (KT > 0) {
        // one warp per row, each lane two adjacent outputs c, c + 1 from the K + 1 inputs
        // A[c .. c + K], read as (K + 1) / 2 aligned 16-byte loads (AW and c are even)
        static_assert(TX == 64, "a warp covers one row of TX outputs in pairs");
        for (int ty = warp; ty < AH; ty += THREADS / 32) {
            const int c = 2 * lane;
            const float4 *row = reinterpret_cast<const float4 *>(A + ty * AW + c);
            float2 in[KT + 1];
#pragma unroll
            for (int j = 0; j < (KT + 1) / 2; ++j) {
                const float4 q = row[j];
                in[2 * j] = make_float2(q.x, q.y);
                in[2 * j + 1] = make_float2(q.z, q.w);
            }
            float2 h0 = make_float2(0.0f, 0.0f), h1 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int d = 0; d < KT; ++d) {
                h0 = fma2(in[d], tb[d], h0);
                h1 = fma2(in[d + 1], tb[d], h1);
            }
            reinterpret_cast<float4 *>(B + ty * TX + c)[0] = make_float4(h0.x, h0.y, h1.x, h1.y);
        }
    } else {
        for (int ty = warp; ty < AH; ty += THREADS / 32) {
            for (int c = lane; c < TX; c += 32) {
                const float2 *row = A + ty * AW + c;
                float2 h = make_float2(0.0f, 0.0f);
                for (int d = 0; d < K; ++d) h = fma2(row[d], tb[d], h);
                B[ty * TX + c] = h;
            }
        }
    }
    __syncthreads();

    float2 *out = a.out + e * a.plane_elems + a.origin;
    float mpsi = 0.0f, mphi = 0.0f;
    constexpr int GROUPS = THREADS / TX;            // row groups of VR rows, one column per thread
    const int c = threadIdx.x % TX, g = threadIdx.x / TX;
    const int x = x0 + c;
    for (int row0 = g * VR; row0 < TY; row0 += GROUPS * VR) {
        float2 o[VR];
#pragma unroll
        for (int q = 0; q < VR; ++q) o[q] = make_float2(0.0f, 0.0f);
        if constexpr (KT > 0) {
            // input row row0 + d feeds output q with tap d - q
#pragma unroll
            for (int d = 0; d < KT + VR - 1; ++d) {
                const float2 v = B[(row0 + d) * TX + c];
#pragma unroll
                for (int q = 0; q < VR; ++q)
                    if (d - q >= 0 && d - q < KT) o[q] = fma2(v, ta[d - q], o[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < VR; ++q)
                for (int d = 0; d < K; ++d) o[q] = fma2(B[(row0 + q + d) * TX + c], ta[d], o[q]);
        }
#pragma unroll
        for (int q = 0; q < VR; ++q) {
            const int y = y0 + row0 + q;
            if (y < a.H && x < a.W) {
                out[(long long)y * a.pitch + x] = o[q];
                track_max(a, o[q], mpsi, mphi);
            }
        }
    }
    if (a.maxbits) {
        // non-negative floats order like their bit patterns
        unsigned bp = __reduce_max_sync(0xffffffffu, __float_as_uint(mpsi));
        unsigned bf = __reduce_max_sync(0xffffffffu, __float_as_uint(mphi));
        if ((threadIdx.x & 31) == 0) {
            atomicMax(a.maxbits + 2 * e, bp);
            atomicMax(a.maxbits + 2 * e + 1, bf);
        }
    }
}

// ---- separable PSF, streaming form --------------------------------------------
// One CTA walks a column strip of TX outputs down a segment of a.seg rows of one
// epoch, in batches of SY input rows:
//   1. the batch's raw n, sigma^2 (and mask) rows, TX + 2 R4 columns from x0 - R4
//      (R4 = r rounded up to a multiple of 4), arrive in shared memory by cp.async
//      16-byte copies (4-byte for the mask), zero-filled outside the image; the
//      next batch's copies are issued as soon as this one is converted, so they
//      overlap the two passes;
//   2. they become (n w, w) pairs (Sec. 2.1.5 weights, by select);
//   3. the horizontal pass writes the batch's rows into a ring of RING rows;
//   4. the vertical pass emits the output rows whose K input rows are all in the
//      ring (one batch behind), so no halo row is ever filtered twice.
// Every output sums its taps in tap order with one packed FMA each, as in
// psi_phi_sep_kernel: the two kernels give bit-identical planes.  Requires
// W % 4 == 0 and 16-byte aligned sci/var (4-byte aligned mask): 16-byte chunks
// of a row then never straddle the image edge.
constexpr int SY = 32;           // input rows per batch (= output rows per batch), a multiple of 8
constexpr int RING = 2 * SY;     // ring rows: one batch plus the 2 r rows of the next (2 r <= SY)
constexpr int SVR = SY / (THREADS / TX);   // output rows per thread in the vertical pass

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int KT>
struct StreamGeom {
    static constexpr int R = KT / 2;
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int OFF = R4 - R;               // first tap column within a staged row
    static constexpr int AWS = TX + 2 * R4;          // staged columns (a multiple of 4)
    static constexpr int Q = AWS / 4;                // 16-byte chunks per staged row
    static constexpr int AST = AWS + 2;              // pair-array row stride in float2 (+16 B: rows
    static constexpr int BST = TX + 2;               // one bank group apart, so 8 rows load conflict-free)
    static constexpr int NQ = (OFF + KT + 3 + 1) / 2;   // 16-byte loads for four outputs' inputs
    // shared bytes: taps | raw n, sigma^2 [SY][AWS] | pairs A [SY][AST] | ring [RING][BST] | mask [SY][AWS]
    static constexpr size_t taps_bytes = ((4 * KT + 3) & ~3) * sizeof(float);
    static constexpr size_t raw_bytes = 2 * (size_t)SY * AWS * sizeof(float);
    static constexpr size_t a_bytes = (size_t)SY * AST * sizeof(float2);
    static constexpr size_t ring_bytes = (size_t)RING * BST * sizeof(float2);
    static constexpr size_t mask_bytes = (size_t)SY * AWS;
    static_assert(2 * R <= SY, "the vertical window must fit one batch behind the ring's head");
};

// issue the cp.async copies of input rows [yin0, yin0 + SY) of epoch e (one commit group)
template <int KT>
__device__ __forceinline__ void stream_stage(const PsiPhiArgs &a, int e, int xs, int yin0, float *rn, float *rv,
                                             uint8_t *rm) {
    typedef StreamGeom<KT> G;
    const size_t npix = (size_t)a.H * a.W;
    const float *sci = a.sci + e * npix, *var = a.var + e * npix;
    const uint8_t *msk = a.mask ? a.mask + e * npix : nullptr;
    for (int i = threadIdx.x; i < SY * G::Q; i += THREADS) {
        const int t = i / G::Q, q = i - t * G::Q;
        const int y = yin0 + t, x = xs + 4 * q;   // x is a multiple of 4: a chunk is wholly in or out
        const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
        const size_t gi = in ? (size_t)y * a.W + x : 0;
        cp_async16(rn + t * G::AWS + 4 * q, sci + gi, in);
        cp_async16(rv + t * G::AWS + 4 * q, var + gi, in);
        if (msk) cp_async4(rm + t * G::AWS + 4 * q, msk + gi, in);
    }
    cp_async_commit();
}

template <int KT>
__global__ void __launch_bounds__(THREADS) psi_phi_stream_kernel(PsiPhiArgs a) {
    typedef StreamGeom<KT> G;
    extern __shared__ float4 smem_raw[];
    const int e = blockIdx.z;
    const int x0 = blockIdx.x * TX, xs = x0 - G::R4;
    const int ys = blockIdx.y * a.seg, ye = min(ys + a.seg, a.H);
    const int n_out = (ye - ys + SY - 1) / SY;              // output batches
    const int n_in = (ye - ys + 2 * G::R + SY - 1) / SY;    // input batches (n_in <= n_out + 1)

    float *s_taps = reinterpret_cast<float *>(smem_raw);
    float *rn = s_taps + G::taps_bytes / sizeof(float);
    float *rv = rn + SY * G::AWS;
    float2 *A = reinterpret_cast<float2 *>(rv + SY * G::AWS);
    float2 *ring = A + SY * G::AST;
    uint8_t *rm = reinterpret_cast<uint8_t *>(ring + RING * G::BST);
    const float *taps = a.taps + (size_t)e * 4 * KT;
    for (int i = threadIdx.x; i < 4 * KT; i += THREADS) s_taps[i] = taps[i];
    const float2 *ta = reinterpret_cast<const float2 *>(s_taps), *tb = ta + KT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // input batch i holds image rows ys - R + SY i + t; ring row of image row j: (j - ys + R) mod RING
    stream_stage<KT>(a, e, xs, ys - G::R, rn, rv, rm);
    float2 *out = a.out + e * a.plane_elems + a.origin;
    float mpsi = 0.0f, mphi = 0.0f;
    for (int i = 0; i <= n_out; ++i) {
        cp_async_wait_all();
        __syncthreads();   // batch i staged; the previous vertical pass is done with the ring
        if (i < n_in) {
            for (int j = threadIdx.x; j < SY * G::Q; j += THREADS) {
                const int t = j / G::Q, q = j - t * G::Q;
                const float4 n4 = *reinterpret_cast<const float4 *>(rn + t * G::AWS + 4 * q);
                const float4 v4 = *reinterpret_cast<const float4 *>(rv + t * G::AWS + 4 * q);
                const uchar4 m4 = a.mask ? *reinterpret_cast<const uchar4 *>(rm + t * G::AWS + 4 * q)
                                         : make_uchar4(0, 0, 0, 0);
                const float2 w0 = weighted(n4.x, v4.x, m4.x, a.bright_max);
                const float2 w1 = weighted(n4.y, v4.y, m4.y, a.bright_max);
                const float2 w2 = weighted(n4.z, v4.z, m4.z, a.bright_max);
                const float2 w3 = weighted(n4.w, v4.w, m4.w, a.bright_max);
                float4 *dst = reinterpret_cast<float4 *>(A + t * G::AST + 4 * q);
                dst[0] = make_float4(w0.x, w0.y, w1.x, w1.y);
                dst[1] = make_float4(w2.x, w2.y, w3.x, w3.y);
            }
        }
        __syncthreads();   // pairs ready, raw buffers free
        if (i + 1 < n_in) stream_stage<KT>(a, e, xs, ys - G::R + SY * (i + 1), rn, rv, rm);
        if (i < n_in) {
            // horizontal: a task is four adjacent outputs of one row; a warp takes 8 rows x 16
            // columns, the 8 lanes of a 16-byte load phase 8 different rows (conflict-free
            // with the padded stride)
            for (int s = 0; s < (SY / 8) * (TX / 16) / (THREADS / 32); ++s) {
                const int wt = warp + (THREADS / 32) * s;
                const int t = 8 * (wt % (SY / 8)) + (lane & 7);
                const int c = 16 * (wt / (SY / 8)) + 4 * (lane >> 3);
                const float4 *row = reinterpret_cast<const float4 *>(A + t * G::AST + c);
                float2 in[2 * G::NQ];
#pragma unroll
                for (int j = 0; j < G::NQ; ++j) {
                    const float4 q = row[j];
                    in[2 * j] = make_float2(q.x, q.y);
                    in[2 * j + 1] = make_float2(q.z, q.w);
                }
                float2 h[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) h[u] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int d = 0; d < KT; ++d) {
                    const float2 w = tb[d];
#pragma unroll
                    for (int u = 0; u < 4; ++u) h[u] = fma2(in[G::OFF + u + d], w, h[u]);
                }
                float4 *dst = reinterpret_cast<float4 *>(ring + ((SY * i + t) & (RING - 1)) * G::BST + c);
                dst[0] = make_float4(h[0].x, h[0].y, h[1].x, h[1].y);
                dst[1] = make_float4(h[2].x, h[2].y, h[3].x, h[3].y);
            }
        }
        __syncthreads();   // the batch's ring rows written
        if (i >= 1) {
            // vertical: output batch o = i - 1, rows ys + SY o + [0, SY); output row y reads ring
            // rows of image rows y - R .. y + R, i.e. relative rows SY o + row + d, d < KT
            const int o = i - 1;
            const int c = threadIdx.x % TX, g = threadIdx.x / TX;
            const int x = x0 + c;
#pragma unroll 1
            for (int row0 = g * SVR; row0 < SY; row0 += (THREADS / TX) * SVR) {
                float2 acc[SVR];
#pragma unroll
                for (int q = 0; q < SVR; ++q) acc[q] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int d = 0; d < KT + SVR - 1; ++d) {
                    const float2 v = ring[((SY * o + row0 + d) & (RING - 1)) * G::BST + c];
#pragma unroll
                    for (int q = 0; q < SVR; ++q)
                        if (d - q >= 0 && d - q < KT) acc[q] = fma2(v, ta[d - q], acc[q]);
                }
#pragma unroll
                for (int q = 0; q < SVR; ++q) {
                    const int y = ys + SY * o + row0 + q;
                    if (y < ye && x < a.W) {
                        out[(long long)y * a.pitch + x] = acc[q];
                        track_max(a, acc[q], mpsi, mphi);
                    }
                }
            }
        }
    }
    if (a.maxbits) {
        unsigned bp = __reduce_max_sync(0xffffffffu, __float_as_uint(mpsi));
        unsigned bf = __reduce_max_sync(0xffffffffu, __float_as_uint(mphi));
        if (lane == 0) {
            atomicMax(a.maxbits + 2 * e, bp);
            atomicMax(a.maxbits + 2 * e + 1, bf);
        }
    }
}

// General PSF, register-blocked, K = KT taps per side (3 <= KT <= 21).  Thread
// (column c, strip s) computes rows s*VR .. s*VR+VR-1 of column c.  For each tap
// column dx it keeps T(., dx) in registers and streams the VR + K - 1 tile rows
// of column c + dx through them: every output accumulates its taps with one
// packed FMA each, tap columns outer, tap rows inner.
constexpr int GVR = 16, GTY = (THREADS / TX) * GVR;   // rows per thread, rows per CTA

template <int KT>
__global__ void __launch_bounds__(THREADS) psi_phi_gen_kernel(PsiPhiArgs a) {
    extern __shared__ float4 smem_raw[];
    constexpr int K = KT, r = K / 2, VR = GVR;
    constexpr int AW = TX + 2 * r, AH = GTY + 2 * r;
    const int e = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * GTY;
    float *s_taps = reinterpret_cast<float *>(smem_raw);
    constexpr int ntaps = 2 * K * K;
    float2 *A = reinterpret_cast<float2 *>(s_taps + ((ntaps + 3) & ~3));
    const float *taps = a.taps + (size_t)e * ntaps;
    for (int i = threadIdx.x; i < ntaps; i += THREADS) s_taps[i] = taps[i];
    stage_tile(a, e, x0, y0, r, AW, AH, A);
    __syncthreads();

    const float2 *t = reinterpret_cast<const float2 *>(s_taps);
    const int c = threadIdx.x % TX, oy = (threadIdx.x / TX) * VR;
    float2 o[VR];
#pragma unroll
    for (int i = 0; i < VR; ++i) o[i] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int dx = 0; dx < K; ++dx) {
        float2 tc[K];
#pragma unroll
        for (int dy = 0; dy < K; ++dy) tc[dy] = t[dy * K + dx];
        const float2 *col = A + oy * AW + c + dx;
#pragma unroll
        for (int j = 0; j < VR + K - 1; ++j) {
            const float2 v = col[j * AW];
#pragma unroll
            for (int i = 0; i < VR; ++i)
                if (j - i >= 0 && j - i < K) o[i] = fma2(v, tc[j - i], o[i]);
        }
    }
    float2 *out = a.out + e * a.plane_elems + a.origin;
    float mpsi = 0.0f, mphi = 0.0f;
    const int x = x0 + c;
#pragma unroll
    for (int i = 0; i < VR; ++i) {
        const int y = y0 + oy + i;
        if (y < a.H && x < a.W) {
            out[(long long)y * a.pitch + x] = o[i];
            track_max(a, o[i], mpsi, mphi);
        }
    }
    if (a.maxbits) {
        unsigned bp = __reduce_max_sync(0xffffffffu, __float_as_uint(mpsi));
        unsigned bf = __reduce_max_sync(0xffffffffu, __float_as_uint(mphi));
        if ((threadIdx.x & 31) == 0) {
            atomicMax(a.maxbits + 2 * e, bp);
            atomicMax(a.maxbits + 2 * e + 1, bf);
        }
    }
}

// General PSF: one pass over the K x K taps (the single-pass form of Sec. 2.3).
__global__ void __launch_bounds__(THREADS) psi_phi_kernel(PsiPhiArgs a) {
    extern __shared__ float4 smem_raw[];
    const int K = a.K, r = K / 2;
    const int e = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int AW = TX + 2 * r, AH = TY + 2 * r;
    // shared layout: taps (T, T^2)[K*K] row-major (dy, dx) | A (AH x AW)
    float *s_taps = reinterpret_cast<float *>(smem_raw);
    const int ntaps = 2 * K * K;
    float2 *A = reinterpret_cast<float2 *>(s_taps + ((ntaps + 3) & ~3));
    const float *taps = a.taps + (size_t)e * ntaps;
    for (int i = threadIdx.x; i < ntaps; i += THREADS) s_taps[i] = taps[i];
    stage_tile(a, e, x0, y0, r, AW, AH, A);
    __syncthreads();

    float2 *out = a.out + e * a.plane_elems + a.origin;
    float mpsi = 0.0f, mphi = 0.0f;
    const float2 *t = reinterpret_cast<const float2 *>(s_taps);
    for (int i = threadIdx.x; i < TY * TX; i += THREADS) {
        int ty = i / TX, c = i - ty * TX;
        int y = y0 + ty, x = x0 + c;
        float2 o = make_float2(0.0f, 0.0f);
        for (int dy = 0; dy < K; ++dy) {
            const float2 *row = A + (ty + dy) * AW + c;
            const float2 *k = t + dy * K;
            for (int dx = 0; dx < K; ++dx) o = fma2(row[dx], k[dx], o);
        }
        if (y < a.H && x < a.W) {
            out[(long long)y * a.pitch + x] = o;
            track_max(a, o, mpsi, mphi);
        }
    }
    if (a.maxbits) {
        unsigned bp = __reduce_max_sync(0xffffffffu, __float_as_uint(mpsi));
        unsigned bf = __reduce_max_sync(0xffffffffu, __float_as_uint(mphi));
        if ((threadIdx.x & 31) == 0) {
            atomicMax(a.maxbits + 2 * e, bp);
            atomicMax(a.maxbits + 2 * e + 1, bf);
        }
    }
}

// Power-of-two scale s with max/s in [2^14, 2^15): exact to apply, keeps the
// largest code below the float16 maximum (65504), 1 for an all-zero plane.
__device__ __forceinline__ float pow2_scale(unsigned maxbits) {
    float m = __uint_as_float(maxbits);
    if (!(m > 0.0f)) return 1.0f;
    int ex = (int)((maxbits >> 23) & 0xff) - 127;   // floor(log2 m) for normal m
    int sh = ex + 1 - 15;
    sh = max(-120, min(120, sh));
    return __uint_as_float((unsigned)(sh + 127) << 23);
}

template <int STORAGE>
__device__ __forceinline__ uint32_t quant_pair(float2 v, float ip, float iff) {
    if (STORAGE == KB_BF16) {
        __nv_bfloat162 p = __floats2bfloat162_rn(v.x * ip, v.y * iff);
        return *reinterpret_cast<uint32_t *>(&p);
    } else {
        __half2 p = __floats2half2_rn(v.x * ip, v.y * iff);
        return *reinterpret_cast<uint32_t *>(&p);
    }
}

// Writes both phases of the 16-bit copy of plane e: phase 0 holds the code of
// element i at i, phase 1 holds the code of element i + 1 at i, so that any two
// adjacent pixels are one 8-byte-aligned load in one of the two phases.  The
// element after a plane's last one lies in the zero border of the next plane
// (or past the last plane), whose code is 0 whatever the scale.
template <int STORAGE>
__global__ void quantize_kernel(const float2 *__restrict__ f32, pair16 *__restrict__ q16, float2 *scales,
                                const unsigned *__restrict__ maxbits, int N, long long plane_elems) {
    const int e = blockIdx.y;
    const float sp = pow2_scale(maxbits[2 * e]), sf = pow2_scale(maxbits[2 * e + 1]);
    if (blockIdx.x == 0 && threadIdx.x == 0) scales[e] = make_float2(sp, sf);
    const float ip = 1.0f / sp, iff = 1.0f / sf;   // exact: powers of two
    const float2 *src = f32 + e * plane_elems;
    pair16 *d0 = q16 + e * plane_elems;
    pair16 *d1 = q16 + ((long long)N + e) * plane_elems;
    const long long n2 = plane_elems / 2;   // plane_elems is a multiple of 4
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(src)[i];
        const uint32_t c0 = quant_pair<STORAGE>(make_float2(v.x, v.y), ip, iff);
        const uint32_t c1 = quant_pair<STORAGE>(make_float2(v.z, v.w), ip, iff);
        // the element after the plane's last one is the next plane's first: a border pixel, code 0
        const uint32_t c2 = (2 * i + 2 < plane_elems) ? quant_pair<STORAGE>(src[2 * i + 2], ip, iff) : 0u;
        reinterpret_cast<uint2 *>(d0)[i] = make_uint2(c0, c1);
        reinterpret_cast<uint2 *>(d1)[i] = make_uint2(c1, c2);
    }
}

}  // namespace

size_t taps_floats(int N, int K, bool separable) { return (size_t)N * (separable ? 4 * K : 2 * K * K); }

static size_t psi_phi_smem(int K, bool sep) {
    int r = K / 2;
    int ntaps = sep ? 4 * K : 2 * K * K;
    size_t taps = ((ntaps + 3) & ~3) * sizeof(float);
    size_t A = (size_t)(TY + 2 * r) * (TX + 2 * r) * sizeof(float2);
    size_t B = sep ? (size_t)(TY + 2 * r) * TX * sizeof(float2) : 0;
    return taps + A + B;
}

template <int KT>
cudaError_t launch_sep(const PsiPhiArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    cudaError_t err = cudaFuncSetAttribute(psi_phi_sep_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    psi_phi_sep_kernel<KT><<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int KT>
cudaError_t launch_gen(const PsiPhiArgs &a, dim3, size_t, cudaStream_t st) {
    constexpr int r = KT / 2;
    const dim3 grid((a.W + TX - 1) / TX, (a.H + GTY - 1) / GTY, a.N);
    const size_t smem = ((2 * KT * KT + 3) & ~3) * sizeof(float) + (size_t)(GTY + 2 * r) * (TX + 2 * r) * sizeof(float2);
    cudaError_t err = cudaFuncSetAttribute(psi_phi_gen_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    psi_phi_gen_kernel<KT><<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// streaming separable kernel: segments of up to 512 rows (a 2 r-row warm-up each,
// 3 % of 512 for K = 17), one CTA per (strip, segment, epoch)
template <int KT>
cudaError_t launch_stream(const PsiPhiArgs &a0, cudaStream_t st) {
    typedef StreamGeom<KT> G;
    PsiPhiArgs a = a0;
    a.seg = std::min(512, (a.H + SY - 1) / SY * SY);
    const dim3 grid((a.W + TX - 1) / TX, (a.H + a.seg - 1) / a.seg, a.N);
    const size_t smem = G::taps_bytes + G::raw_bytes + G::a_bytes + G::ring_bytes + (a.mask ? G::mask_bytes : 0);
    cudaError_t err = cudaFuncSetAttribute(psi_phi_stream_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    psi_phi_stream_kernel<KT><<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// the streaming kernel's 16-byte row chunks need W % 4 == 0 and aligned planes; other
// cases take the tile kernel
static bool stream_ok(const PsiPhiArgs &a) {
    return a.separable && a.K >= 3 && a.K <= 21 && (a.K & 1) && a.W % 4 == 0 && ((uintptr_t)a.sci & 15) == 0 &&
           ((uintptr_t)a.var & 15) == 0 && (!a.mask || ((uintptr_t)a.mask & 3) == 0);
}

cudaError_t launch_psi_phi(const PsiPhiArgs &a, cudaStream_t st) {
    dim3 grid((a.W + TX - 1) / TX, (a.H + TY - 1) / TY, a.N);
    size_t smem = psi_phi_smem(a.K, a.separable);
    if (stream_ok(a)) {
        switch (a.K) {
            case 3: return launch_stream<3>(a, st);
            case 5: return launch_stream<5>(a, st);
            case 7: return launch_stream<7>(a, st);
            case 9: return launch_stream<9>(a, st);
            case 11: return launch_stream<11>(a, st);
            case 13: return launch_stream<13>(a, st);
            case 15: return launch_stream<15>(a, st);
            case 17: return launch_stream<17>(a, st);
            case 19: return launch_stream<19>(a, st);
            case 21: return launch_stream<21>(a, st);
            default: break;
        }
    }
    if (a.separable) {
        switch (a.K) {   // the PSF sides of the workloads get fully unrolled taps
            case 3: return launch_sep<3>(a, grid, smem, st);
            case 5: return launch_sep<5>(a, grid, smem, st);
            case 7: return launch_sep<7>(a, grid, smem, st);
            case 9: return launch_sep<9>(a, grid, smem, st);
            case 11: return launch_sep<11>(a, grid, smem, st);
            case 13: return launch_sep<13>(a, grid, smem, st);
            case 15: return launch_sep<15>(a, grid, smem, st);
            case 17: return launch_sep<17>(a, grid, smem, st);
            case 19: return launch_sep<19>(a, grid, smem, st);
            case 21: return launch_sep<21>(a, grid, smem, st);
            default: return launch_sep<0>(a, grid, smem, st);
        }
    }
    switch (a.K) {   // register-blocked single pass for the common sides
        case 3: return launch_gen<3>(a, grid, smem, st);
        case 5: return launch_gen<5>(a, grid, smem, st);
        case 7: return launch_gen<7>(a, grid, smem, st);
        case 9: return launch_gen<9>(a, grid, smem, st);
        case 11: return launch_gen<11>(a, grid, smem, st);
        case 13: return launch_gen<13>(a, grid, smem, st);
        case 15: return launch_gen<15>(a, grid, smem, st);
        case 17: return launch_gen<17>(a, grid, smem, st);
        case 19: return launch_gen<19>(a, grid, smem, st);
        case 21: return launch_gen<21>(a, grid, smem, st);
        default: break;
    }
    cudaError_t err = cudaFuncSetAttribute(psi_phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    psi_phi_kernel<<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float2 *f32, pair16 *q16, float2 *scales, const unsigned *maxbits, int N,
                            long long plane_elems, int storage, cudaStream_t st) {
    long long n2 = plane_elems / 2;
    int blocks = (int)((n2 + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    dim3 grid(blocks, N);
    if (storage == KB_BF16)
        quantize_kernel<KB_BF16><<<grid, 256, 0, st>>>(f32, q16, scales, maxbits, N, plane_elems);
    else
        quantize_kernel<KB_F16><<<grid, 256, 0, st>>>(f32, q16, scales, maxbits, N, plane_elems);
    return cudaGetLastError();
}

}  // namespace kb
