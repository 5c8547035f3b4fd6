// Inline-PTX helpers shared by the tcgen05 kernels (h2_umma.cu, h2nn_tc.cu)
// and the bulk-copy pipeline of the symmetric-storage kernel (h2_sym.cu):
// mbarriers with bounded waits, bulk asynchronous copies, shared-memory
// matrix descriptors of the canonical no-swizzle K-major layout, the bf16
// instruction descriptor, the single-CTA MMA and its commit.
#pragma once

#include <cstdint>

namespace h2 {
namespace tc {

// polls of the waits that let copies (and MMAs) in flight finish after a
// bounded wait ran out, before a CTA releases its shared memory
constexpr uint32_t kDrainLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// plain arrival (release at CTA scope): one of the barrier's expected arrivals
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// barrier over the first `count` threads of the CTA (a multiple of 32) on
// hardware barrier `id` (1..15; 0 is __syncthreads)
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for the phase with the given parity; false when `limit` polls ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor of the matrix operand: K-major, no swizzle,
// N rows of 16-byte chunks: 8-row core matrices 128 B apart, chunks 16 N B apart
__device__ __forceinline__ uint64_t bdesc(uint32_t saddr, int n)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)((16 * n) >> 4) << 16;             // leading byte offset: next chunk along K
    d |= (uint64_t)(128 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // layout type 0: no swizzle
}

// shared-memory matrix descriptor: K-major, no swizzle, 128 rows of 16-byte
// chunks: 8-row core matrices 128 B apart (stride), consecutive K chunks
// `lbo` bytes apart (leading)
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;       // leading byte offset: next chunk along K
    d |= (uint64_t)(128 >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // layout type 0: no swizzle
}

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}


}  // namespace tc
}  // namespace h2
