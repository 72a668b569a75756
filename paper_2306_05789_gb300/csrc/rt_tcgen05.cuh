// rt_tcgen05.cuh -- inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators) used by the streamed multi-right-hand-
// side apply: shared-memory matrix descriptors with 128-byte swizzling,
// kind::f16 instruction descriptors, TMEM allocation and loads, commits.
//
// Operand layouts (16-bit elements, one 128-byte row = 64 elements):
//   * K-major, 128-byte swizzle: M rows of 128 bytes (64 K values each), 8-row
//     atoms of 1024 bytes at stride SBO = 1024; the 16-byte chunk c of row r
//     sits at chunk position c ^ (r mod 8).  The k-th group of 16 K values
//     starts 32 k bytes into the rows.
//   * MN-major, 128-byte swizzle: K rows of 128 bytes (64 M/N values each),
//     8-row atoms at SBO = 1024 along K, same chunk permutation; the k-th group
//     of 16 K rows starts 2048 k bytes in.
// Every atom is 1024-byte aligned in shared memory, so the swizzle phase of a
// row is its row index mod 8 within the tile.
#pragma once

#include <cstdint>

namespace rt {
namespace t5 {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading and stride byte offsets (16-byte
// units), descriptor version 1 (bit 46), layout type 2 = 128-byte swizzle (bits 61-63)
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16 (bf16 = 1) or F16,
// A / B MN-major when mn_a / mn_b, M and N
__device__ __forceinline__ uint32_t idesc(int bf16, int mn_a, int mn_b, int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;
    d |= (uint32_t)bf16 << 7;
    d |= (uint32_t)bf16 << 10;
    d |= (uint32_t)mn_a << 15;
    d |= (uint32_t)mn_b << 16;
    d |= (uint32_t)(N >> 3) << 17;
    d |= (uint32_t)(M >> 4) << 24;
    return d;
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accum)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(accum));
}

// arrive on the mbarrier once every MMA this thread issued so far has completed
__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the async proxy (tensor cores, bulk copies)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate ncols TMEM columns (power of two >= 32), address to *dst (shared)
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// whole warp: 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace t5
}  // namespace rt
