// FP64 rescoring of kept candidates, repair of uncertified pixels, and
// expansion of results into kb_result.
//
// Rescoring: the reduced-precision search keeps kc >= k candidates per start
// pixel.  For each candidate the coadd of Sec. 2.1.5 is recomputed from the
// FP32 psi/phi planes, scored nu = Psi / sqrt(Phi), alpha = Psi / Phi in FP64,
// and the k best by (nu desc, vidx asc) are kept.  A per-pixel certificate
// decides whether a trajectory outside the candidate list could still belong to
// the top-k; the pixels it cannot clear are searched again exhaustively.
//
// The coadds are summed exactly, in 64-bit fixed point on the integer pipe, and
// rounded once to FP64: this GPU's FP64 pipe is a small fraction of its FP32
// and integer pipes, and an FP64 sum of FP32 values spends two FP64 operations
// (a conversion and an add) per value.  Each plane type (psi, phi) of a stack
// gets one binary point 2^L with L = E - 56, where every |value| of the stack is
// below 2^E (from the per-epoch maxima the psi/phi kernel records): a value is
// taken as round(value * 2^-L), exact for every value of magnitude 2^(E-33) or
// more (its last mantissa bit is at least 2^L) and within 2^(L-1) below that, and
// a sum of up to 128 such integers stays below 2^63.  The error of a coadd is
// therefore at most N * 2^(E-57), below the N * 2^-53 * 2^(E+7) bound of FP64
// summation, and it does not depend on the order of the epochs.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "kb_internal.h"

namespace kb {

namespace {

// Binary points of the exact coadd sums (see above): the exponent shifts that
// take a value to units of 2^L and the double factors back (2^L).
struct FixedPoint {
    int sh_p, sh_f;          // -150 - L: a float's exponent field plus this is its shift to units of 2^L
    int L_p, L_f;            // the binary points
};

// one plane type: every |value| < 2^E, E from the largest per-epoch maximum (bits of
// a non-negative float order like the float); E kept in [-60, 100] so that 2^-L and
// 2^L stay normal floats and doubles
__device__ __forceinline__ void fixed_point_of(unsigned maxbits, int &sh, int &L) {
    int E = maxbits == 0u ? -60 : (int)((maxbits >> 23) & 0xff) - 126;   // floor(log2 m) + 1
    E = max(-60, min(100, E));
    L = E - 56;
    sh = -150 - L;
}

// A fixed-point sum s in units of 2^L, rounded once to FP64: (double)s * 2^L, the
// power-of-two scaling done by adding L to the exponent field (exact: |s| >= 1 and
// L in [-116, 44] keep the result normal) on the integer pipe, not by an FP64 multiply.
__device__ __forceinline__ double scaled(long long s, int L) {
    const double d = (double)s;
    return s == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(d) + ((long long)L << 52));
}

// round(x 2^-L) (ties away from zero) for |x| < 2^(L+56), on the integer pipe: with
// exponent field e and significand m (the implicit bit included when e > 0),
// |x| = m 2^(max(e, 1) - 150), so |x| 2^-L = m 2^s with s = max(e, 1) + sh <= 32.
// A shift left is exact; a shift right by r adds 2^(r-1) first (r is clamped at 31,
// where m + 2^30 < 2^31 shifts to 0, as every |x| 2^-L < 1/2 must).  The float to
// 64-bit integer conversion instruction would run on the FP64 pipe, which this
// GPU keeps narrow.
__device__ __forceinline__ long long fixed_of(float x, int sh) {
    const uint32_t u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xffu);
    const uint32_t m = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int s = max(e, 1) + sh;
    const int r = min(max(-s, 0), 31);
    const unsigned long long left = (unsigned long long)m << max(s, 0);
    const uint32_t right = (m + ((1u << r) >> 1)) >> r;
    const long long v = s >= 0 ? (long long)left : (long long)right;
    return (u >> 31) ? -v : v;
}

// The binary points of a stack, from its 2N per-epoch maxima [max |psi|, max phi]
// (every thread of the block calls it; uses one barrier)
__device__ __forceinline__ FixedPoint stack_fixed_point(const RescoreArgs &a) {
    __shared__ unsigned s_m[2];
    if (threadIdx.x < 2) s_m[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * a.N; i += blockDim.x) atomicMax(&s_m[i & 1], a.maxbits[i]);
    __syncthreads();
    FixedPoint fp;
    fixed_point_of(s_m[0], fp.sh_p, fp.L_p);
    fixed_point_of(s_m[1], fp.sh_f, fp.L_f);
    return fp;
}

// Exact coadd of one trajectory from the FP32 planes: the fixed-point sums p, f in
// units of 2^L_p, 2^L_f (see above; scaled() rounds them once to FP64) and the
// count of in-image epochs.  Four epochs at a time: their offsets, then their four
// plane gathers, then the sums, so that the scattered loads overlap instead of
// forming one dependent chain.
__device__ __forceinline__ void traj_exact(const RescoreArgs &a, const FixedPoint &fp, int x, int y, int v,
                                           long long &p, long long &f, int &nobs) {
    const int2 *ov = a.offs + (long long)v * a.N;
    const float2 *base = a.f32 + a.origin;
    p = 0;
    f = 0;
    nobs = 0;
    int j = 0;
    for (; j + 4 <= a.N; j += 4) {
        int2 o[4];
        float2 pp[4];
        bool in[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = __ldg(ov + j + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int xx = x + o[q].x, yy = y + o[q].y;
            in[q] = (unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H;
            pp[q] = in[q] ? __ldg(base + (long long)a.epoch_of[j + q] * a.plane_elems + (long long)yy * a.pitch + xx)
                          : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p += fixed_of(pp[q].x, fp.sh_p);
            f += fixed_of(pp[q].y, fp.sh_f);
            nobs += in[q] ? 1 : 0;
        }
    }
    for (; j < a.N; ++j) {
        const int2 o = __ldg(ov + j);
        const int xx = x + o.x, yy = y + o.y;
        if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
            const float2 pp = __ldg(base + (long long)a.epoch_of[j] * a.plane_elems + (long long)yy * a.pitch + xx);
            p += fixed_of(pp.x, fp.sh_p);
            f += fixed_of(pp.y, fp.sh_f);
            ++nobs;
        }
    }
}


// FP64 nu of a coadd, Psi / sqrt(Phi) as Psi * rsqrt(Phi) (CUDA's double rsqrt):
// one reciprocal square root instead of a correctly rounded square root and a
// division, which on this GPU's narrow FP64 pipe cost several times more.  Equal
// sums still give equal nu, so exact ties keep breaking by velocity index.
__device__ __forceinline__ double nu64(double P, double F) { return P * rsqrt(F); }

// Order-preserving integer key of a double (-inf < ... < +inf; NaN never occurs
// here): comparisons of the running lists run on the integer pipe, not the FP64 one.
__device__ __forceinline__ unsigned long long okey(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double okey_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k));
}
// (key desc, vidx asc): the order (nu desc, vidx asc) of the doubles the keys encode
__device__ __forceinline__ bool betterk(unsigned long long ak, int av, unsigned long long bk, int bv) {
    return ak > bk || (ak == bk && av < bv);
}

// Upper bound on |nu - nu16| for a candidate of FP64 score nu whose reduced-
// precision score nu16 lies in (lo, hi]: in key form (b > 0) hi is its key's value
// (an order-preserving FP32 encoding that is a multiple of 2^b) and lo the value 2^b
// below it in that encoding; in value form (b = 0) nu16 = hi = lo.  The bound is
// max(|nu - lo|, |nu - hi|), formed in FP32 on the FP32 pipe: nf, nu rounded to FP32,
// is within 2^-24 |nf| of nu (twice that is added, and 2^-126 for the subnormal
// range), and every difference and sum rounds upwards.  Infinite where lo, hi or nf
// is not finite (such a pixel is never certified).
__device__ __forceinline__ float cand_error(double nu, float hi, int b) {
    const float nf = __double2float_rn(nu);
    if (!(fabsf(hi) < INFINITY) || !(fabsf(nf) < INFINITY)) return INFINITY;
    float lo = hi;
    if (b > 0) {
        const uint32_t u = __float_as_uint(hi);
        const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        if (ord < 0x00800000u + (1u << b)) return INFINITY;
        const uint32_t lo_ord = ord - (1u << b);
        lo = __uint_as_float((lo_ord & 0x80000000u) ? (lo_ord & 0x7FFFFFFFu) : ~lo_ord);
    }
    const float d = fmaxf(__fsub_ru(fmaxf(nf, hi), fminf(nf, hi)), __fsub_ru(fmaxf(nf, lo), fminf(nf, lo)));
    return __fadd_ru(__fadd_ru(d, __fmul_ru(fabsf(nf), 0x1p-23f)), 0x1p-126f);
}

// Pixel order of the rescoring: one 32 x 4 tile per CTA of 128 threads, tiles
// walked down strips kStrip pixels wide, strip after strip.  The pixels in flight
// at one time then form a compact region (about 256 x 300 pixels on a full GPU),
// and the gathers of their trajectories, which reach up to the largest offset of
// the velocity grid away, share the L2; in row order they would spread over the
// image's full width.
constexpr int kStrip = 256;

long long rescore_tiles(int H, int W) { return (long long)((W + kStrip - 1) / kStrip) * (kStrip / 32) * ((H + 3) / 4); }

// pixel (x, y) of thread t of tile `tile`, and its index y * W + x (-1 outside the image)
__device__ __forceinline__ long long rescore_pixel(int H, int W, long long tile, int t, int &x, int &y) {
    const long long per_strip = (long long)(kStrip / 32) * ((H + 3) / 4);
    const int strip = (int)(tile / per_strip);
    const long long r = tile - (long long)strip * per_strip;
    x = strip * kStrip + (int)(r % (kStrip / 32)) * 32 + (t & 31);
    y = (int)(r / (kStrip / 32)) * 4 + (t >> 5);
    return (x < W && y < H) ? (long long)y * W + x : -1;
}

// One thread per start pixel: FP64 sums of the kc candidates, re-ranking, and the
// certificate.  A trajectory outside the candidate list had a 16-bit score at
// most nu16 of the last candidate; the pixel is certified when the k-th
// rescored nu (or nu_min, if fewer than k pass it) exceeds that score by more
// than twice the largest 16-bit error seen among the pixel's own candidates
// plus unit * (1 + |nu|).  Pixels whose candidate list was not full hold every
// valid trajectory and are certified.  The others go to the repair list.
// Key-form candidates (a.nu_key) carry nu16 rounded upwards, still an upper bound for
// the trajectories left out; each candidate's error is then taken over the rounding
// interval of its key.
// The running top-K list lives in registers (K >= k, a compile-time bound).
template <int K>
__global__ void __launch_bounds__(128) rescore_kernel(RescoreArgs a) {
    const FixedPoint fp = stack_fixed_point(a);
    int x, y;
    const long long pix = rescore_pixel(a.H, a.W, blockIdx.x, threadIdx.x, x, y);
    if (pix >= 0) {
        double lp[K], lf[K];
        unsigned long long lk[K];   // nu as its order key
        int lv[K], lo[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            lk[i] = okey(-INFINITY);
            lp[i] = 0.0;
            lf[i] = 0.0;
            lv[i] = INT_MAX;
            lo[i] = 0;
        }
        int ncand = 0, n = 0;
        float emax = 0.0f;   // largest bound on a candidate's own |nu - nu16|
        float nu16_last = -INFINITY;
        const Rec *cand = a.cand + pix * a.kc;
        const uint32_t *ckey = reinterpret_cast<const uint32_t *>(a.cand) + pix * a.kc;
        for (int c = 0; c < a.kc; ++c) {
            uint32_t v;
            float nu16;
            if (a.nu_key) {   // key form: 0 is an empty slot
                const uint32_t kk = ckey[c];
                if (kk == 0u) break;
                v = (uint32_t)cand_key_vidx(kk, a.nu_key);
                nu16 = cand_key_nu(kk, a.nu_key);
            } else {
                const Rec rc = cand[c];
                v = rc.meta & 0xffffu;
                if (v == kEmptyVidx) break;
                nu16 = rc.nu;
            }
            ++ncand;
            nu16_last = nu16;
            long long ps, fs;
            int nobs;
            traj_exact(a, fp, x, y, (int)v, ps, fs, nobs);
            if (fs <= 0) continue;   // Phi = 0: no valid trajectory
            const double P = scaled(ps, fp.L_p), F = scaled(fs, fp.L_f);
            const double nu = nu64(P, F);
            // a key-form nu16 is rounded upwards: the unrounded score lies in (lo, hi]
            emax = fmaxf(emax, cand_error(nu, nu16, a.nu_key));
            if (!(nu >= a.nu_min)) continue;
            ++n;
            // bubble the candidate down the sorted register list (nu desc, vidx asc),
            // comparing integer keys; skipped when it does not beat the last entry
            unsigned long long ck = okey(nu);
            int cv = (int)v, co = nobs;
            if (!betterk(ck, cv, lk[K - 1], lv[K - 1])) continue;
            double cp = P, cf = F;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const bool sw = betterk(ck, cv, lk[i], lv[i]);
                const double tp = lp[i], tf = lf[i];
                const unsigned long long tk = lk[i];
                const int tv = lv[i], to = lo[i];
                lk[i] = sw ? ck : tk;
                lp[i] = sw ? cp : tp;
                lf[i] = sw ? cf : tf;
                lv[i] = sw ? cv : tv;
                lo[i] = sw ? co : to;
                ck = sw ? tk : ck;
                cp = sw ? tp : cp;
                cf = sw ? tf : cf;
                cv = sw ? tv : cv;
                co = sw ? to : co;
            }
        }
        Rec64 *out = a.out + pix * a.k;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i >= a.k) break;
            Rec64 r;
            if (lv[i] != INT_MAX) {
                r.psi = lp[i];
                r.phi = lf[i];
                r.nu = okey_value(lk[i]);
                r.vidx = (uint32_t)lv[i];
                r.nobs = (uint32_t)lo[i];
            } else {
                r.psi = 0.0;
                r.phi = 0.0;
                r.nu = -INFINITY;
                r.vidx = kEmptyVidx;
                r.nobs = 0;
            }
            out[i] = r;
        }
        if (ncand == a.kc && a.ucount) {
            double bar = a.nu_min;
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (i == a.k - 1 && n >= a.k) bar = okey_value(lk[i]);
            const double margin = 2.0 * (double)emax + a.unit * (1.0 + fabs((double)nu16_last));
            if (!((double)nu16_last + margin < bar)) {
                const int slot = atomicAdd(a.ucount, 1);
                a.ulist[slot] = (int)pix;
            }
        }
    }
}

// One CTA of kRepairThreads per uncertain pixel: every velocity's exact sums from
// the FP32 planes (thread t takes velocities t, t + 256, ...), a sorted top-k per
// thread, k rounds of a warp-shuffle arg-max merge (nu desc, vidx asc) per warp
// into shared memory, then the same merge of the 8 warps' lists by warp 0.  A CTA
// per pixel, rather than a warp, keeps the pixels in flight few (about 900 on a full
// GPU) and, in the rescoring's strip order of the list, close together: their
// trajectories' gathers then share the L2, where thousands of pixels a strip apart
// would not.
constexpr int kRepairThreads = 256;
constexpr int kRepairWarps = kRepairThreads / 32;

__global__ void __launch_bounds__(kRepairThreads) repair_kernel(RescoreArgs a) {
    const FixedPoint fp = stack_fixed_point(a);
    __shared__ Rec64 s_best[kRepairWarps][KB_MAX_TOPK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int count = *a.ucount;
    for (int u = blockIdx.x; u < count; u += gridDim.x) {
        const int pix = a.ulist[u];
        const int y = pix / a.W, x = pix - y * a.W;
        // nu as its order key: the list's compares and the merge's shuffles on the integer pipe
        unsigned long long lk[KB_MAX_TOPK];
        double lp[KB_MAX_TOPK], lf[KB_MAX_TOPK];
        int lv[KB_MAX_TOPK], lo[KB_MAX_TOPK];
        int n = 0;
        for (int v = threadIdx.x; v < a.V; v += kRepairThreads) {
            long long ps, fs;
            int nobs;
            traj_exact(a, fp, x, y, v, ps, fs, nobs);
            if (fs <= 0) continue;   // Phi = 0: no valid trajectory
            const double P = scaled(ps, fp.L_p), F = scaled(fs, fp.L_f);
            const double nu = nu64(P, F);
            if (!(nu >= a.nu_min)) continue;
            const unsigned long long key = okey(nu);
            if (n == a.k && !betterk(key, v, lk[n - 1], lv[n - 1])) continue;
            int i = (n < a.k) ? n++ : a.k - 1;
            while (i > 0 && betterk(key, v, lk[i - 1], lv[i - 1])) {
                lk[i] = lk[i - 1];
                lp[i] = lp[i - 1];
                lf[i] = lf[i - 1];
                lv[i] = lv[i - 1];
                lo[i] = lo[i - 1];
                --i;
            }
            lk[i] = key;
            lp[i] = P;
            lf[i] = F;
            lv[i] = v;
            lo[i] = nobs;
        }
        // per warp: each round the best head among the lanes goes to s_best[warp][r]
        int head = 0;
        for (int r = 0; r < a.k; ++r) {
            // key 0 is below the key of every score, -inf included
            unsigned long long bk = head < n ? lk[head] : 0ull;
            int bv = head < n ? lv[head] : INT_MAX;
            int bl = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                if (betterk(ok, ov, bk, bv)) {
                    bk = ok;
                    bv = ov;
                    bl = ol;
                }
            }
            if (bl == lane && bv != INT_MAX) {
                Rec64 q;
                q.psi = lp[head];
                q.phi = lf[head];
                q.nu = okey_value(lk[head]);
                q.vidx = (uint32_t)lv[head];
                q.nobs = (uint32_t)lo[head];
                s_best[warp][r] = q;
                ++head;
            } else if (lane == 0 && bv == INT_MAX) {
                Rec64 q;
                q.psi = 0.0;
                q.phi = 0.0;
                q.nu = -INFINITY;
                q.vidx = kEmptyVidx;
                q.nobs = 0;
                s_best[warp][r] = q;
            }
            __syncwarp();
        }
        __syncthreads();
        // warp 0: lane w < kRepairWarps walks warp w's sorted list
        if (warp == 0) {
            int h = 0;
            Rec64 *out = a.out + (long long)pix * a.k;
            for (int r = 0; r < a.k; ++r) {
                const bool has = lane < kRepairWarps && h < a.k && s_best[lane][h].vidx != kEmptyVidx;
                unsigned long long bk = has ? okey(s_best[lane][h].nu) : 0ull;
                int bv = has ? (int)s_best[lane][h].vidx : INT_MAX;
                int bl = lane;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                    const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                    if (betterk(ok, ov, bk, bv)) {
                        bk = ok;
                        bv = ov;
                        bl = ol;
                    }
                }
                if (bv == INT_MAX) {
                    if (lane == 0) {   // fewer than k valid trajectories
                        Rec64 q;
                        q.psi = 0.0;
                        q.phi = 0.0;
                        q.nu = -INFINITY;
                        q.vidx = kEmptyVidx;
                        q.nobs = 0;
                        out[r] = q;
                    }
                } else if (bl == lane) {
                    out[r] = s_best[lane][h];
                    ++h;
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

__global__ void expand_kernel(ExpandArgs a) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < a.count;
         r += (long long)gridDim.x * blockDim.x) {
        const long long g = a.first + r;
        const long long pix = g / a.k;
        const int i = (int)(g - pix * a.k);
        kb_result o;
        o.y0 = (int)(pix / a.W);
        o.x0 = (int)(pix - (long long)o.y0 * a.W);
        uint32_t v;
        if (a.recs64) {
            const Rec64 &q = a.recs64[pix * a.k + i];
            v = q.vidx;
            o.nobs = (int)q.nobs;
            o.psi = (float)q.psi;
            o.phi = (float)q.phi;
            o.nu = q.nu;
            o.alpha = (v == kEmptyVidx) ? 0.0 : q.psi / q.phi;
        } else {
            const Rec &q = a.recs[pix * a.krec + i];
            v = q.meta & 0xffffu;
            o.nobs = (int)((q.meta >> 16) & 0xffu);
            o.psi = q.psi;
            o.phi = q.phi;
            o.nu = (double)q.nu;
            o.alpha = (v == kEmptyVidx) ? 0.0 : (double)(q.psi / q.phi);
        }
        if (v == kEmptyVidx) {
            o.vidx = -1;
            o.vx = 0.0f;
            o.vy = 0.0f;
            o.nobs = 0;
        } else {
            o.vidx = (int)v;
            float2 q = a.vq[v];
            o.vx = q.x;
            o.vy = q.y;
        }
        a.out[r] = o;
    }
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st) {
    const long long blocks = rescore_tiles(a.H, a.W);
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a.k <= 4)
        rescore_kernel<4><<<(int)blocks, 128, 0, st>>>(a);
    else if (a.k <= 8)
        rescore_kernel<8><<<(int)blocks, 128, 0, st>>>(a);
    else
        rescore_kernel<16><<<(int)blocks, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_repair(const RescoreArgs &a, cudaStream_t st) {
    repair_kernel<<<152 * 6, kRepairThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// Sec. 3.3 light-curve filter, one thread per kept trajectory: pass 1 sums the
// coadd in FP64 (epochs in time order), pass 2 re-gathers each in-image epoch
// and rejects it when its flux psi_e / phi_e differs from the other epochs'
// weighted mean (Psi - psi_e) / (Phi - phi_e) by more than nsigma sigma, with
// sigma^2 = 1 / phi_e + 1 / (Phi - phi_e).  Multiplying through by
// phi_e (Phi - phi_e) > 0 gives the division-free test
//     (psi_e Phi - Psi phi_e)^2 > nsigma^2 Phi phi_e (Phi - phi_e),
// which spares the narrow FP64 pipe two divisions and a square root per epoch.
__global__ void filter_kernel(FilterArgs a) {
    const long long total = (long long)a.H * a.W * a.k;
    const float2 *base = a.f32 + a.origin;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long pix = g / a.k;
        const int slot = (int)(g - pix * a.k);
        const int y = (int)(pix / a.W), x = (int)(pix - (long long)y * a.W);
        const uint32_t v = a.recs64 ? a.recs64[pix * a.k + slot].vidx : (a.recs[pix * a.krec + slot].meta & 0xffffu);
        kb_filtered o;
        o.x0 = x;
        o.y0 = y;
        o.reserved = 0;
        o.rejected[0] = o.rejected[1] = o.rejected[2] = o.rejected[3] = 0u;
        if (v == kEmptyVidx) {
            o.vidx = -1;
            o.nobs = 0;
            o.nrejected = 0;
            o.psi = o.phi = 0.0;
            o.nu = -INFINITY;
            o.alpha = 0.0;
            a.out[g] = o;
            continue;
        }
        const int2 *ov = a.offs + (long long)v * a.N;
        double P = 0.0, F = 0.0;
        for (int j = 0; j < a.N; ++j) {
            const int2 d = __ldg(ov + j);
            const int xx = x + d.x, yy = y + d.y;
            if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                const float2 q = __ldg(base + (long long)a.epoch_of[j] * a.plane_elems + (long long)yy * a.pitch + xx);
                P += (double)q.x;
                F += (double)q.y;
            }
        }
        double Pk = 0.0, Fk = 0.0;
        int kept = 0, rej = 0;
        for (int j = 0; j < a.N; ++j) {
            const int2 d = __ldg(ov + j);
            const int xx = x + d.x, yy = y + d.y;
            if (!((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H)) continue;
            const int e = a.epoch_of[j];
            const float2 q = __ldg(base + (long long)e * a.plane_elems + (long long)yy * a.pitch + xx);
            const double pe = (double)q.x, fe = (double)q.y, rest = F - fe;
            bool out = false;
            if (fe > 0.0 && rest > 0.0) {
                const double dev = pe * F - P * fe;
                out = dev * dev > a.nsigma2 * F * fe * rest;
            }
            if (out) {
                o.rejected[e >> 5] |= 1u << (e & 31);
                ++rej;
            } else {
                Pk += pe;
                Fk += fe;
                ++kept;
            }
        }
        o.vidx = (int)v;
        o.nobs = kept;
        o.nrejected = rej;
        o.psi = Pk;
        o.phi = Fk;
        o.nu = Fk > 0.0 ? Pk / sqrt(Fk) : -INFINITY;
        o.alpha = Fk > 0.0 ? Pk / Fk : 0.0;
        a.out[g] = o;
    }
}

cudaError_t launch_filter(const FilterArgs &a, cudaStream_t st) {
    const long long total = (long long)a.H * a.W * a.k;
    if (total <= 0) return cudaSuccess;
    long long blocks = (total + 127) / 128;
    if (blocks > 152 * 64) blocks = 152 * 64;
    filter_kernel<<<(int)blocks, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// Sec. 3.3 postage stamps: one CTA per candidate, one thread per stamp pixel.
// A thread gathers its pixel's science values over the epochs along the search's
// trajectory offsets (finite, unmasked, in the image), then takes their mean
// (FP64 sum) or median (insertion sort of at most N values in local memory).
// The CTA then reduces the stamp's central moments in FP64 and applies the cuts.
__global__ void stamp_kernel(StampArgs a) {
    __shared__ double red[6][32];
    const int S = 2 * a.r + 1, npx = S * S;
    const size_t plane = (size_t)a.H * a.W;
    for (int c = blockIdx.x; c < a.n; c += gridDim.x) {
        const int4 q = a.cand[c];
        const int2 *ov = a.offs + (long long)q.z * a.N;
        const int t = threadIdx.x;
        float val = 0.0f;
        if (t < npx) {
            const int sy = t / S - a.r, sx = t % S - a.r;
            float vals[KB_MAX_EPOCHS];
            int m = 0;
            double sum = 0.0;
            for (int j = 0; j < a.N; ++j) {
                const int2 d = __ldg(ov + j);
                const int x = q.x + d.x + sx, y = q.y + d.y + sy;
                if ((unsigned)x >= (unsigned)a.W || (unsigned)y >= (unsigned)a.H) continue;
                const size_t i = (size_t)a.epoch_of[j] * plane + (size_t)y * a.W + x;
                const float v = __ldg(a.sci + i);
                if (!isfinite(v) || (a.mask && __ldg(a.mask + i))) continue;
                if (a.mode == KB_STAMP_MEAN) {
                    sum += (double)v;
                } else {
                    int k = m;                           // insertion into the sorted prefix
                    while (k > 0 && vals[k - 1] > v) {
                        vals[k] = vals[k - 1];
                        --k;
                    }
                    vals[k] = v;
                }
                ++m;
            }
            if (m > 0)
                val = a.mode == KB_STAMP_MEAN ? (float)(sum / m)
                      : ((m & 1) ? vals[m / 2] : (float)(0.5 * ((double)vals[m / 2 - 1] + (double)vals[m / 2])));
            a.stamps[(size_t)c * npx + t] = val;
        }
        if (!a.moments) continue;
        // moments: sums of v, x v, y v, then (after the centroid) the central ones
        // over the central aperture x^2 + y^2 <= aperture^2 (the whole stamp when aperture <= 0)
        const double x = t < npx ? (double)(t % S - a.r) : 0.0, y = t < npx ? (double)(t / S - a.r) : 0.0;
        const bool in_ap = t < npx && (a.aperture <= 0.0 || x * x + y * y <= a.aperture * a.aperture);
        const double v = in_ap ? (double)val : 0.0;
        double s[6] = {v, x * v, y * v, 0.0, 0.0, 0.0};
        const int lane = t & 31, w = t >> 5, nw = (blockDim.x + 31) >> 5;
        for (int pass = 0; pass < 2; ++pass) {
            const int lo = pass == 0 ? 0 : 3;
            for (int i = lo; i < lo + 3; ++i) {
                double u = s[i];
                for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                if (lane == 0) red[i][w] = u;
            }
            __syncthreads();
            if (t < 32)
                for (int i = lo; i < lo + 3; ++i) {
                    double u = t < nw ? red[i][t] : 0.0;
                    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                    if (t == 0) red[i][0] = u;
                }
            __syncthreads();
            if (pass == 0) {
                const double m00 = red[0][0];
                const double cx = m00 != 0.0 ? red[1][0] / m00 : 0.0, cy = m00 != 0.0 ? red[2][0] / m00 : 0.0;
                s[3] = (x - cx) * (x - cx) * v;
                s[4] = (y - cy) * (y - cy) * v;
                s[5] = (x - cx) * (y - cy) * v;
            }
        }
        if (t == 0) {
            kb_moments mo;
            mo.m00 = red[0][0];
            const bool any = mo.m00 != 0.0;
            mo.mx = any ? red[1][0] / mo.m00 : 0.0;
            mo.my = any ? red[2][0] / mo.m00 : 0.0;
            mo.mu20 = any ? red[3][0] / mo.m00 : 0.0;
            mo.mu02 = any ? red[4][0] / mo.m00 : 0.0;
            mo.mu11 = any ? red[5][0] / mo.m00 : 0.0;
            mo.reserved = 0;
            mo.passed = !a.cut || (mo.m00 > 0.0 && fabs(mo.mx) <= a.cuts.max_offset &&
                                   fabs(mo.my) <= a.cuts.max_offset && mo.mu20 >= a.cuts.min_var &&
                                   mo.mu20 <= a.cuts.max_var && mo.mu02 >= a.cuts.min_var &&
                                   mo.mu02 <= a.cuts.max_var && fabs(mo.mu11) <= a.cuts.max_mu11);
            a.moments[c] = mo;
        }
        __syncthreads();
    }
}

cudaError_t launch_stamps(const StampArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const int S = 2 * a.r + 1;
    const int threads = ((S * S + 31) / 32) * 32;
    const int blocks = a.n < 152 * 16 ? a.n : 152 * 16;
    stamp_kernel<<<blocks, threads, 0, st>>>(a);
    return cudaGetLastError();
}

namespace {
__global__ void compact_kernel(const Rec64 *recs64, long long count, kb_result_compact *out) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < count;
         r += (long long)gridDim.x * blockDim.x) {
        const Rec64 q = recs64[r];
        kb_result_compact o;
        const bool empty = q.vidx == kEmptyVidx;
        o.psi = empty ? 0.0f : (float)q.psi;
        o.phi = empty ? 0.0f : (float)q.phi;
        o.nu = empty ? -INFINITY : (float)q.nu;
        o.vidx = (uint16_t)q.vidx;
        o.nobs = empty ? 0 : (uint8_t)q.nobs;
        o.reserved = 0;
        out[r] = o;
    }
}
}  // namespace

cudaError_t launch_compact(const Rec64 *recs64, long long count, kb_result_compact *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    compact_kernel<<<(int)blocks, 256, 0, st>>>(recs64, count, out);
    return cudaGetLastError();
}

cudaError_t launch_expand(const ExpandArgs &a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    expand_kernel<<<(int)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace kb
