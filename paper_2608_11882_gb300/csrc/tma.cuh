// Inline-PTX helpers for tiled TMA loads (cp.async.bulk.tensor) completing on
// shared-memory mbarriers, with bounded waits, and the host-side tensor-map
// encoder (driver entry point looked up through the runtime).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hcg {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes the mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; gives up once max_cycles SM
// clock cycles have passed since `start` and returns false.
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity, long long start,
                                                long long max_cycles)
{
    while (!mbar_try_wait(bar, parity))
        if (clock64() - start > max_cycles) return false;
    return true;
}

// Bounded wait of its own: about one second at GB300 clocks.
constexpr long long kWaitCycles = 2000000000ll;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    return mbar_wait_until(bar, parity, clock64(), kWaitCycles);
}

// 3-D tiled TMA load of one box into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Host: encode a 3-D tiled tensor map over a padded field buffer
// (dims: pitch x (ny+2) x (nz+2) elements).  Returns a cudaError_t-style code
// (0 on success) and fills *out.
int encode_field_map(CUtensorMap* out, void* base, CUtensorMapDataType dt, size_t elem,
                     uint64_t pitch, uint64_t rows, uint64_t planes, uint32_t box_x, uint32_t box_y);

}  // namespace hcg
