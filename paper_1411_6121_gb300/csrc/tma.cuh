// tma.cuh -- tensor-memory-accelerator loads of state planes into shared memory (sm_103a):
// the mbarrier and cp.async.bulk.tensor instructions as inline PTX, and the host-side
// encoding of the tensor map of a state buffer.
//
// A state buffer is the 4D array [Q][nz][ny][px] (x fastest, rows padded to px elements,
// px a multiple of 8, so every row starts on a 16-byte boundary). One copy moves a box of
// BX x RY cells of one z plane for all Q velocities into shared memory as [Q][RY][BX].
// Rules of the unit: the box's starting x times the element size must be a multiple of 16
// bytes (callers round x down to 4 floats / 8 16-bit values and index from the remainder);
// the shared-memory destination must be 128-byte aligned; out-of-range rows and columns
// read as zero.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dugks {

// Set by a kernel whose wait on a copy gave up (the copy never completed); read and cleared
// by the host (tma_wait_failures in step3d_q19.cu, the translation unit whose kernels use
// these copies; each translation unit has its own flag).
static __device__ int g_tma_wait_failed = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the copy unit before the first copy uses them.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 4D tiled copy global -> shared, completing `bytes` on `bar` (coordinates in elements).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until phase `parity` of `bar` has completed. Gives up after about two seconds
// (a copy that never lands): returns false after raising g_tma_wait_failed. The caller
// makes the whole CTA leave together (__syncthreads_or on the result).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    uint32_t done = 0;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > 2000000000ull) {
            atomicExch(&g_tma_wait_failed, 1);
            return false;
        }
    }
}

// Host: tensor map of one state buffer [Q][nz][ny][px] of `esize`-byte elements (4: FP32,
// 2: BF16 or F16) with the box BX x RY x 1 x Q. Returns cudaSuccess or an error.
cudaError_t encode_state_map(CUtensorMap *map, const void *base, int esize, bool bf16, int64_t px, int64_t ny,
                             int64_t nz, int q, int bx, int ry);

}  // namespace dugks
