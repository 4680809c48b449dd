// ws_tma.cuh -- Tensor Memory Accelerator (TMA) staging helpers for sm_100+:
// mbarrier set-up, arrive/expect-tx, bounded waits, and tiled
// cp.async.bulk.tensor loads of 3D boxes into shared memory; plus the host
// side that encodes CUtensorMap descriptors through the driver entry point
// (no link against libcuda).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_device.cuh"

namespace ws {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `phase` of `bar`.  Returns false (and records
// DEV_TIMEOUT) if the copy did not land within the time limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase, DevStatus *status)
{
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > 2000000000ull) {  // 2 s
            record_error(status, DEV_TIMEOUT, 101);
            return false;
        }
    }
}

// Tiled 3D TMA load of the box at element coordinates (c0, c1, c2) into dst
// (16-byte aligned shared memory); completion is signalled on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Host: encodes a rank-3 tiled tensor map over a dense (W, H, D) array of
// `elem` bytes per element.  Returns false when the layout breaks a TMA rule
// (base not 16-byte aligned, row pitch not a multiple of 16 bytes, box too
// large) so that the caller can use its plain-load path instead.
bool make_tmap_3d(CUtensorMap *map, const void *base, int elem, uint64_t W, uint64_t H, uint64_t D, uint32_t bx,
                  uint32_t by, uint32_t bz);

}  // namespace ws
