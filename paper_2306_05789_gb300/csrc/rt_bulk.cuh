// rt_bulk.cuh -- bulk global->shared copies completed on mbarriers, for the
// streamed kernels: one producer warp copies contiguous operator pieces into a
// ring of shared-memory stages (cp.async.bulk, byte-counted completion on the
// stage's "full" mbarrier) and the consumer warps release a stage by arriving
// on its "empty" mbarrier.  Every wait is bounded by a clock budget; a wait
// that gives up returns false and the caller reports it through a flag.
#pragma once

#include <cstdint>

namespace rt {
namespace bulk {

constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// makes the initialised mbarriers visible to the async proxy (the bulk copies)
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also raises the expected transaction bytes of the phase
__device__ __forceinline__ void arrive_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// raise the expected transaction bytes of the current phase without arriving
__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bytes (a multiple of 16) from a 16-byte aligned global address to a
// 16-byte aligned shared address; completion counted on bar
__device__ __forceinline__ void copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// wait for the completion of the phase with the given parity; false when the
// clock budget runs out first.  Each probe may suspend the thread for up to
// kSuspendNs (it resumes as soon as the phase completes), so waiting warps
// leave the issue slots to the working ones.
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done = 0;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// barrier over the first `count` threads (whole warps) on hardware barrier
// `id` (1..15); returns whether any of them passed pred = true
__device__ __forceinline__ bool bar_or(int id, int count, bool pred)
{
    uint32_t r = 0;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace bulk
}  // namespace rt
