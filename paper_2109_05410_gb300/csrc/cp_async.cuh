// cp_async.cuh -- cp.async helpers and the x-neighbour pick of the wave25
// kernels (stencil.cu: one step per launch; wave_fused.cu: two).
#pragma once
#include "stencil_common.cuh"

namespace ooc {
namespace sten {

// x-neighbour at offset idx in [-4, 7] from the thread's first point, given
// its own 4 points c and the 4-point groups to its left (l) and right (rr).
__device__ __forceinline__ float pick(const float (&l)[4], const float (&c)[4], const float (&rr)[4], int idx)
{
    return idx < 0 ? l[idx + 4] : (idx < 4 ? c[idx] : rr[idx - 4]);
}

// cp.async (16-byte global -> shared copies that bypass the registers; a
// source size of 0 fills zeros) and its group waits.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace sten
}  // namespace ooc
