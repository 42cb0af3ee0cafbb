// Tensor-memory-access (TMA) and mbarrier helpers shared by the fused kernels: 4D tiled
// copies global -> shared completing on an mbarrier, and bounded waits that give up after
// about a second instead of hanging.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace lks {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// One 4D tiled tensor copy {0, x, y, z} into shared memory, completing `bytes` on `bar`.
__device__ __forceinline__ void tma_load_box(uint32_t dst, const CUtensorMap* map, int x, int y,
                                             int z, uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Bounded wait on an mbarrier phase: about a second of spinning, then give up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

// A wait that first polls once (the common case: the copy has landed), then falls back to the
// bounded wait.
__device__ __forceinline__ bool mbar_wait_once(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
        " selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done ? true : mbar_wait(bar, parity);
}

struct Geom;
// Host: tensor map over a float4-per-node state {4, nx, ny, nz} with box {4, bx, by, 1}.
bool encode_state_map(CUtensorMap* map, const void* base, const Geom& g, int bx, int by);

}  // namespace lks
