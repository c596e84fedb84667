// Tensor-memory-accelerator (TMA) staging for the pass kernels (sm_90 and later; written for
// sm_103a): shared-memory barriers with transaction counts, tiled bulk tensor copies from
// global to shared memory, and bounded waits.
//
// Every wait on a barrier is bounded by a cycle budget. A wait that runs out reports it to the
// caller, which records LBM_ERR_TIMEOUT in the context's device error word and leaves the
// kernel (after waiting, again bounded, for the copies it still has in flight), so a copy that
// never lands cannot hang the GPU.
#pragma once
#include <cuda.h>  // CUtensorMap (type only: the library calls no driver function directly)
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// barrier with one expected arrival per phase (the issuing thread's arrive.expect_tx)
__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void fence_bar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses (and those it observed
// through a CTA barrier) before later async-proxy writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// 2D tiled copy of the box at element coordinates (x, y) of `map` into shared memory at dst,
// completing `bytes` of the barrier's transaction count when it lands
__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// waits for the barrier's phase `parity` to complete; false if `budget` clock cycles pass first
__device__ __forceinline__ bool bar_wait_bounded(uint64_t *bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!bar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// device error word bits
constexpr int kErrTimeout = 1;

}  // namespace tma
}  // namespace lbm
