// FP64 rescoring of kept candidates and expansion of results into kb_result.
//
// Rescoring: the reduced-precision search keeps kc >= k candidates per start
// pixel.  For each candidate the coadd of Sec. 2.1.5 is recomputed from the
// FP32 psi/phi planes with FP64 accumulation (epochs in time order), scored
// nu = Psi / sqrt(Phi), alpha = Psi / Phi in FP64, and the k best by
// (nu desc, vidx asc) are kept.  One thread per start pixel; the candidates'
// FP32 plane reads are gathers (k_c * N per pixel).
#include <cuda_runtime.h>
#include <math.h>

#include "kb_internal.h"

namespace kb {

namespace {

__global__ void rescore_kernel(RescoreArgs a) {
    const long long npix = (long long)a.H * a.W;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < npix;
         pix += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(pix / a.W), x = (int)(pix - (long long)y * a.W);
        double ln[32], lp[32], lf[32];
        int lv[32], lo[32];
        int n = 0;
        const Rec *cand = a.cand + pix * a.kc;
        for (int c = 0; c < a.kc; ++c) {
            uint32_t v = cand[c].meta & 0xffffu;
            if (v == kEmptyVidx) break;
            const int2 *ov = a.offs + (long long)v * a.N;
            double P = 0.0, F = 0.0;
            int nobs = 0;
            for (int j = 0; j < a.N; ++j) {
                int2 o = __ldg(ov + j);
                int xx = x + o.x, yy = y + o.y;
                if ((unsigned)xx < (unsigned)a.W && (unsigned)yy < (unsigned)a.H) {
                    float2 pp = __ldg(a.f32 + (long long)a.epoch_of[j] * a.plane_elems + (long long)yy * a.pitch + xx);
                    P += (double)pp.x;
                    F += (double)pp.y;
                    ++nobs;
                }
            }
            if (!(F > 0.0)) continue;
            double nu = P / sqrt(F);
            if (!(nu >= a.nu_min)) continue;
            // insertion by (nu desc, vidx asc)
            int i = n;
            while (i > 0 && (nu > ln[i - 1] || (nu == ln[i - 1] && (int)v < lv[i - 1]))) {
                ln[i] = ln[i - 1];
                lp[i] = lp[i - 1];
                lf[i] = lf[i - 1];
                lv[i] = lv[i - 1];
                lo[i] = lo[i - 1];
                --i;
            }
            ln[i] = nu;
            lp[i] = P;
            lf[i] = F;
            lv[i] = (int)v;
            lo[i] = nobs;
            ++n;
        }
        Rec64 *out = a.out + pix * a.k;
        for (int i = 0; i < a.k; ++i) {
            Rec64 r;
            if (i < n) {
                r.psi = lp[i];
                r.phi = lf[i];
                r.nu = ln[i];
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
    long long npix = (long long)a.H * a.W;
    long long blocks = (npix + 127) / 128;
    if (blocks > 152 * 64) blocks = 152 * 64;
    rescore_kernel<<<(int)blocks, 128, 0, st>>>(a);
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
