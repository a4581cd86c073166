// vdi_tma.cuh -- the tensor memory accelerator (TMA) and mbarrier primitives
// of the render kernels, as inline PTX for sm_103a: tiled tensor loads of a
// VDI tile into shared memory (completion counted in bytes on an mbarrier),
// bounded waits on that barrier, and bulk stores from shared memory to global
// memory.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vdi {

// Tensor maps over a VDI's arrays, built once per VDI on the host
// (vdi_api.cu): the list ranges as a 2-D tensor of 32-bit words (2 w x h),
// the depth slot pairs and the colour records as 3-D tensors
// (4 w x h x planes: one 16-byte record per list and plane), and the VDI's
// device status word (kStatus* bits, read by vdi_stats).  Passed to a kernel
// as a __grid_constant__ parameter.
struct TileMaps {
    CUtensorMap range, depth, colour;
    uint32_t *status;
};

// A wait on a staged tile gives up after kWaitNs nanoseconds of the global
// timer or kWaitLimit attempts, whichever comes first: both far above any
// copy's latency (a tile lands in microseconds).
constexpr uint64_t kWaitNs = 200000000ull;
constexpr uint32_t kWaitLimit = 1u << 24;

// device status word bits (TileMaps::status)
constexpr uint32_t kStatusStageTimeout = 1u;  // a staged-tile wait ran out; the rays used global loads

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barrier visible to the async proxy (the TMA unit)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also announces `bytes` of transactions still to land
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the barrier's phase `parity` to complete, within kWaitNs and
// kWaitLimit attempts; false when either ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (i == 0)
            t0 = global_ns();
        else if (global_ns() - t0 > kWaitNs)
            return false;
    }
    return false;
}

// tiled tensor loads into this CTA's shared memory, completing on `bar`; the
// innermost coordinate times 4 bytes must be a multiple of 16
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *m, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// order this thread's earlier shared-memory writes before later async-proxy
// reads of them (a bulk store's source)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// shared to global memory, then wait until it is complete
__device__ __forceinline__ void bulk_store_wait(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(reinterpret_cast<uint64_t>(gdst)),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace vdi
