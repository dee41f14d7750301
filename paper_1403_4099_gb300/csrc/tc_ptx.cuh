// tc_ptx.cuh -- inline-PTX helpers of the tcgen05 kernels (sm_103a): shared
// addresses, bounded mbarrier waits, the 128-byte-swizzled K-major operand
// descriptor, the BF16 MMA with FP32 accumulation in tensor memory, and 16-byte
// cp.async. Written against the PTX ISA; nothing here is part of the ABI.
#pragma once

#include "gpga_internal.cuh"

namespace gpga {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\n"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait: false once `budget` SM cycles have passed since the
// wait began (the budget is checked before each try, so budget 0 gives up at
// once); the default bound, 2^32 cycles, is about 2 s at the SM clock
constexpr long long WAIT_BOUND = 1ll << 32;
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity,
                                          long long budget = WAIT_BOUND)
{
    const long long t0 = clock64();
    for (;;) {
        if (clock64() - t0 >= budget) return false;
        if (mbar_try_wait(a, parity)) return true;
    }
}

// 128-byte-swizzled, K-major shared-memory operand descriptor (rows of 128
// bytes, 8-row groups 1024 bytes apart; start address 16-byte granular)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :
                 : "r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(bytes)
                 : "memory");
}


// barrier init / commit / TMEM management (one warp allocates and frees)
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
        : "memory");
}

} // namespace gpga
