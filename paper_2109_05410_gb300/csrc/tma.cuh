// tma.cuh -- TMA tensor copies into shared memory with mbarrier completion,
// and bounded mbarrier waits, shared by the TMA-staged stencil kernels
// (heat_tma.cu, wave_tma.cu).
#pragma once
#include <cuda.h>

#include "stencil_common.cuh"

namespace ooc {
namespace sten {

// A bounded mbarrier wait gives up after kMbarTries polls, each suspending
// the thread for up to about a microsecond.
constexpr int kMbarTries = 1 << 20;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// true once the phase with parity `parity` has completed; false after
// kMbarTries polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (int it = 0; it < kMbarTries; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(1000u)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

// TMA copy of the box at (x, y, slot) of the ring's tensor map into `dst`,
// completing `bar`'s transaction count
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}


}  // namespace sten

// Tensor map of a ring of nslot planes of nx x ny floats (dims x, y, slot)
// for boxes of box_x x box_y x 1 floats; out-of-range x and y read as zero
// (the zero ghosts of the boundary).  Maps are encoded once per (ring, box)
// and cached.  box_x * 4 must be a multiple of 16 bytes, nx a multiple of 4,
// base 16-byte aligned.
cudaError_t ring_tensor_map(const float *base, int64_t nx, int64_t ny, int64_t nslot, int box_x, int box_y,
                            CUtensorMap *out);
// Reads and clears the device fault word of the TMA-staged wave kernel.
cudaError_t take_wave_fault(unsigned *fault);

}  // namespace ooc
