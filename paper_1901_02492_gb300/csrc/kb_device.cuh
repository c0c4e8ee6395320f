// Device helpers shared by the search kernels: packed f32x2 arithmetic, the
// storage traits of the psi/phi planes, the (nu desc, vidx asc) order, and the
// mbarrier / TMA inline-PTX wrappers of the pipelined search.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kb_internal.h"

namespace kb {
namespace dev {

__device__ __forceinline__ unsigned long long as_u64(float2 v) { return *reinterpret_cast<unsigned long long *>(&v); }
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

// storage traits: element type, load, accumulate (16-bit codes are scaled by the
// epoch's power-of-two scales, exact, then added in FP32)
template <int STORAGE>
struct Store;

template <>
struct Store<KB_F32> {
    typedef float2 T;
    static constexpr int kAlign = 2;   // elements per 16 bytes (TMA box starts)
    __device__ __forceinline__ static T load(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static T zero() { return make_float2(0.0f, 0.0f); }
    __device__ __forceinline__ static float2 acc(float2 a, T v, float2) { return add2(a, v); }
};

template <>
struct Store<KB_BF16> {
    typedef pair16 T;
    static constexpr int kAlign = 4;
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
    static constexpr int kAlign = 4;
    __device__ __forceinline__ static T load(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static T zero() { return 0u; }
    __device__ __forceinline__ static float2 acc(float2 a, T v, float2 s) {
        __half2 h = *reinterpret_cast<__half2 *>(&v);
        return fma2(__half22float2(h), s, a);
    }
};

// (nu desc, vidx asc)
__device__ __forceinline__ bool better(float an, int av, float bn, int bv) {
    return an > bn || (an == bn && av < bv);
}

// ---- mbarrier / TMA ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Wait for the phase `parity` of `bar` to complete.  Gives up after `limit`
// SM cycles (or as soon as another thread of the CTA has given up): it then
// raises the CTA's abort flag and the job's status word and returns false, so
// that no wait of the kernel can spin forever.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status,
                                          long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicExch(status, KB_ETIMEOUT);
            return false;
        }
    }
}

}  // namespace dev
}  // namespace kb
