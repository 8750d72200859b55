// Tensor-memory-accelerator (TMA) staging: bulk tensor copies from global to
// shared memory completed on an mbarrier, outside the LSU/L1 data path.
//
// Every wait is bounded in time (%globaltimer): on expiry the kernel records
// TC_ERR_TIMEOUT in a device flag that the host reads at its next
// synchronising call, and returns instead of spinning on.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "common.cuh"

// 1 s: far above any copy of the few tens of KB staged here
#define TC_WAIT_LIMIT_NS 1000000000ull

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Box at coordinates (x, y, z) of a 3D tensor map into shared memory (the
// destination 128-byte aligned); completion is counted on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Wait for phase `parity` of bar to complete, for at most limit_ns.  Returns
// false (and records TC_ERR_TIMEOUT in *err) when the limit expires.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int *err,
                                         unsigned long long limit_ns = TC_WAIT_LIMIT_NS) {
    const unsigned a = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) {
            if (err) atomicExch(err, TC_ERR_TIMEOUT);
            return false;
        }
    }
}

// Host: encode a tiled map of a float32 volume [d2][d1][d0] (d0 innermost,
// rows of d0 floats) with boxes of b0 x b1 x 1 elements.  b0 * 4 must be a
// multiple of 16 bytes and base 16-byte aligned.  Returns TC_OK or an error.
int tma_encode_f32_3d(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
                      uint32_t b1);
