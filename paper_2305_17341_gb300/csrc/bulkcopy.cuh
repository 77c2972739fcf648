// bulkcopy.cuh -- mbarrier and bulk asynchronous copy primitives (inline PTX,
// sm_90 and later) shared by the kernels that stage global memory in shared
// memory through the copy engine.
#pragma once
#include <cuda.h>   // CUtensorMap

#include "modarith.cuh"

namespace he {

// Iteration limit of every mbarrier wait: a wait that runs out reports an
// error instead of spinning forever.
constexpr int BC_WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ u32 bc_smem(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bc_bar_init(u64 *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bc_smem(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the copy engine; then a CTA barrier.
__device__ __forceinline__ void bc_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bc_arrive(u64 *bar) {
    [[maybe_unused]] u64 state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(bc_smem(bar)) : "memory");
}

__device__ __forceinline__ void bc_expect_tx(u64 *bar, u32 bytes) {
    [[maybe_unused]] u64 state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(bc_smem(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bc_try_wait(u64 *bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bc_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of the phase of `parity`.
__device__ __forceinline__ bool bc_wait(u64 *bar, u32 parity) {
    for (int it = 0; it < BC_WAIT_LIMIT; it++)
        if (bc_try_wait(bar, parity)) return true;
    return false;
}

// `bytes` (a multiple of 16) from global `src` to shared `dst` (both 16-byte
// aligned), completing on bar's transaction count.
__device__ __forceinline__ void bc_bulk(void *dst, const void *src, u32 bytes, u64 *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            bc_smem(dst)),
        "l"(src), "r"(bytes), "r"(bc_smem(bar))
        : "memory");
}

// Asks the copy engine to bring `bytes` (a multiple of 16, 16-byte aligned)
// of global memory into L2; nothing waits for it.
__device__ __forceinline__ void bc_prefetch_l2(const void *src, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// One box of a 2-D tensor map (coordinates x innermost, y) into shared `dst`.
__device__ __forceinline__ void bc_tensor2d(void *dst, const CUtensorMap *map, int x, int y, u64 *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(bc_smem(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bc_smem(bar))
        : "memory");
}

}  // namespace he
