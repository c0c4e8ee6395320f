// Sec. 3.3 de-duplication of candidate trajectories: DBSCAN over (x0, y0, vx, vy).
//
// Distance, core points, clusters, border and noise points are as documented at
// kb_cluster in include/kb.h.  The GPU form:
//   - a first pass packs each candidate into 16 bytes (x0, y0, vx, vy) and
//     computes its cell of a 4-D uniform grid of cells a little wider than eps
//     (in the weighted coordinates), so that every neighbour of a point lies in
//     the 3^4 cells around its own; the cells live in an open-addressing hash
//     table whose slots hold a linked list of their points (built with atomics);
//   - neighbour counts (stopping at min_samples) give the core points;
//   - a lock-free union-find over the core points, always hooking the larger
//     root under the smaller, so every cluster ends rooted at its lowest core
//     index whatever the order of the unions;
//   - border points take the root of their nearest core neighbour (smallest d2,
//     then lowest index), noise points their own index;
//   - per group, an atomic maximum of the ordered nu bits, then an atomic
//     minimum of the index among the members that reach it.
// The squared distance is evaluated with explicitly rounded FP64 operations in a
// fixed order (no contraction into FMA), so neighbour decisions are exact and
// deterministic.  Every loop is bounded; a bound that is reached sets the status
// word instead of spinning.
#include <algorithm>

#include "kb_internal.h"

namespace kb {
namespace {

constexpr int kThreads = 256;

// Points are packed as (x0, y0, bits of vx, bits of vy).
__device__ __forceinline__ double dist2(int4 a, int4 b, double w_pos, double w_vel) {
    const double ax = __dmul_rn((double)((long long)a.x - (long long)b.x), w_pos);
    const double ay = __dmul_rn((double)((long long)a.y - (long long)b.y), w_pos);
    const double au = __dmul_rn(__dsub_rn((double)__int_as_float(a.z), (double)__int_as_float(b.z)), w_vel);
    const double av = __dmul_rn(__dsub_rn((double)__int_as_float(a.w), (double)__int_as_float(b.w)), w_vel);
    return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(au, au)),
                     __dmul_rn(av, av));
}

// Grid cell of a candidate; false when a coordinate is too far from the origin
// in units of the cell width (the caller's weights and eps are unusable then).
__device__ __forceinline__ bool cell_of(const kb_result &r, const ClusterArgs &a, int4 &c) {
    const double f0 = (double)r.x0 * a.w_pos * a.inv_side, f1 = (double)r.y0 * a.w_pos * a.inv_side;
    const double f2 = (double)r.vx * a.w_vel * a.inv_side, f3 = (double)r.vy * a.w_vel * a.inv_side;
    const double lim = 1073741824.0;   // 2^30
    if (!(fabs(f0) < lim && fabs(f1) < lim && fabs(f2) < lim && fabs(f3) < lim)) return false;
    c = make_int4((int)floor(f0), (int)floor(f1), (int)floor(f2), (int)floor(f3));
    return true;
}

__device__ __forceinline__ unsigned hash4(int4 c, unsigned mask) {
    unsigned long long h = (unsigned long long)(unsigned)c.x * 0x9E3779B97F4A7C15ull;
    h ^= (unsigned long long)(unsigned)c.y * 0xC2B2AE3D27D4EB4Full;
    h ^= (unsigned long long)(unsigned)c.z * 0x165667B19E3779F9ull;
    h ^= (unsigned long long)(unsigned)c.w * 0xD6E8FEB86659FD93ull;
    h ^= h >> 31;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 29;
    return (unsigned)h & mask;
}

__device__ __forceinline__ bool same_cell(const ClusterArgs &a, int o, int4 c) {
    const int4 d = a.cells[o];
    return d.x == c.x && d.y == c.y && d.z == c.z && d.w == c.w;
}

// Slot of cell c in the finished table, or -1.
__device__ int find_slot(const ClusterArgs &a, int4 c) {
    unsigned s = hash4(c, a.T - 1);
    for (int probe = 0; probe < a.T; ++probe) {
        const int o = a.owner[s];
        if (o < 0) return -1;
        if (same_cell(a, o, c)) return (int)s;
        s = (s + 1) & (a.T - 1);
    }
    return -1;
}

__device__ __forceinline__ unsigned long long nu_key(double nu) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(nu);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ int find_root(volatile int *parent, int x, int n, int *status) {
    for (int it = 0; it <= n; ++it) {
        const int p = parent[x];
        if (p == x) return x;
        const int g = parent[p];
        if (g != p) parent[x] = g;   // path halving: g is an ancestor of x
        x = p;
    }
    atomicExch(status, 2);
    return x;
}

__global__ void init_kernel(ClusterArgs a) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.T; s += stride) {
        a.owner[s] = -1;
        a.head[s] = -1;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        a.parent[i] = i;
        a.next[i] = -1;
        a.bestnu[i] = 0ull;
        a.bestidx[i] = 0x7fffffff;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.count = 0u;
        *a.status = 0;
    }
}

__global__ void prep_kernel(ClusterArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const kb_result r = a.cand[i];
        int4 c = make_int4(0, 0, 0, 0);
        bool ok = r.vidx >= 0;
        if (ok && !cell_of(r, a, c)) {
            atomicExch(a.status, 1);
            ok = false;
        }
        a.pts[i] = make_int4(r.x0, r.y0, __float_as_int(r.vx), __float_as_int(r.vy));
        a.cells[i] = c;
        a.valid[i] = ok ? 1 : 0;
    }
}

__global__ void insert_kernel(ClusterArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        if (!a.valid[i]) continue;
        const int4 c = a.cells[i];
        unsigned s = hash4(c, a.T - 1);
        bool placed = false;
        for (int probe = 0; probe < a.T && !placed; ++probe) {
            const int o = atomicCAS(&a.owner[s], -1, i);
            if (o == -1 || same_cell(a, o, c)) {
                a.next[i] = atomicExch(&a.head[s], i);
                placed = true;
            } else {
                s = (s + 1) & (a.T - 1);
            }
        }
        if (!placed) atomicExch(a.status, 2);
    }
}

// Visits every candidate j in the 3^4 cells around i's cell; f(j) returns false to stop.
template <class F>
__device__ void for_neighbours(const ClusterArgs &a, int i, F f) {
    const int4 c = a.cells[i];
    for (int d = 0; d < 81; ++d) {
        const int4 q = make_int4(c.x + d % 3 - 1, c.y + (d / 3) % 3 - 1, c.z + (d / 9) % 3 - 1, c.w + d / 27 - 1);
        const int s = find_slot(a, q);
        if (s < 0) continue;
        int j = a.head[s];
        for (int walk = 0; j >= 0 && walk < a.n; ++walk) {
            if (!f(j)) return;
            j = a.next[j];
        }
    }
}

__global__ void core_kernel(ClusterArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const bool ok = a.valid[i];
        int cnt = 0;
        if (ok) {
            const int4 p = a.pts[i];
            for_neighbours(a, i, [&](int j) {
                if (dist2(p, a.pts[j], a.w_pos, a.w_vel) <= a.eps2) ++cnt;
                return cnt < a.min_samples;
            });
        }
        a.core[i] = (ok && cnt >= a.min_samples) ? 1 : 0;
    }
}

__global__ void union_kernel(ClusterArgs a) {
    volatile int *parent = a.parent;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        if (!a.core[i]) continue;
        const int4 p = a.pts[i];
        for_neighbours(a, i, [&](int j) {
            if (j < i && a.core[j] && dist2(p, a.pts[j], a.w_pos, a.w_vel) <= a.eps2) {
                int u = i, v = j;
                for (int it = 0; it <= 2 * a.n + 2; ++it) {
                    u = find_root(parent, u, a.n, a.status);
                    v = find_root(parent, v, a.n, a.status);
                    if (u == v) break;
                    if (u < v) {
                        const int t = u;
                        u = v;
                        v = t;
                    }
                    // u > v: hook the larger root under the smaller
                    if (atomicCAS(&a.parent[u], u, v) == u) break;
                    if (it == 2 * a.n + 2) atomicExch(a.status, 2);
                }
            }
            return true;
        });
    }
}

__global__ void label_kernel(ClusterArgs a) {
    volatile int *parent = a.parent;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        int lab = -1;
        if (a.valid[i]) {
            if (a.core[i]) {
                lab = find_root(parent, i, a.n, a.status);
            } else {
                const int4 p = a.pts[i];
                int best = -1;
                double bd = 0.0;
                for_neighbours(a, i, [&](int j) {
                    if (a.core[j]) {
                        const double d2 = dist2(p, a.pts[j], a.w_pos, a.w_vel);
                        if (d2 <= a.eps2 && (best < 0 || d2 < bd || (d2 == bd && j < best))) {
                            best = j;
                            bd = d2;
                        }
                    }
                    return true;
                });
                lab = best >= 0 ? find_root(parent, best, a.n, a.status) : i;
            }
            atomicMax(&a.bestnu[lab], nu_key(a.cand[i].nu));
        }
        a.label[i] = lab;
        if (a.core_out) a.core_out[i] = a.core[i];
    }
}

__global__ void pick_kernel(ClusterArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int lab = a.label[i];
        if (lab >= 0 && nu_key(a.cand[i].nu) == a.bestnu[lab]) atomicMin(&a.bestidx[lab], i);
    }
}

__global__ void keep_kernel(ClusterArgs a) {
    unsigned mine = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int lab = a.label[i];
        const bool k = lab >= 0 && a.bestidx[lab] == i;
        a.keep[i] = k ? 1 : 0;
        mine += k;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.count, mine);
}

}  // namespace

cudaError_t launch_cluster(const ClusterArgs &a, int sm_count, cudaStream_t st) {
    const int cap = 8 * (sm_count > 0 ? sm_count : 152);
    auto grid = [&](long long m) { return (int)std::max(1LL, std::min<long long>((m + kThreads - 1) / kThreads, cap)); };
    init_kernel<<<grid(std::max<long long>(a.T, a.n)), kThreads, 0, st>>>(a);
    if (a.n > 0) {
        prep_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        insert_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        core_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        union_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        label_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        pick_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
        keep_kernel<<<grid(a.n), kThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace kb
