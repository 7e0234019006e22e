// pack.cu -- BF16 slab storage (FP32 <-> BF16, round to nearest even).
//
// BF16 is the cheapest lossy storage format of the precision study: 2 bytes
// per value on the host link instead of 4.  Packing rounds to nearest even
// by integer arithmetic on the float's bits (NaN stays a quiet NaN); the
// widening back is exact.  HBM-bound: 6 bytes per value moved.
#include "common.cuh"

namespace ooc {
namespace {

__device__ __forceinline__ uint32_t bf16_rne(uint32_t u)
{
    if ((u & 0x7FFFFFFFu) > 0x7F800000u)
        return (u >> 16) | 0x40u;
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

// Planes [z0, z1) of a ring, 4 values per thread (nx*ny is a multiple of 4).
__global__ void bf16_pack_ring_kernel(ConstRing in, int64_t plane, int64_t z0, int64_t nquads, uint16_t *out)
{
    const int64_t qpp = plane >> 2;  // quads per plane
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nquads;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t zl = i / qpp, r = i - zl * qpp;
        const int64_t slot = ring_slot(z0 + zl, in.zbase, in.nslot);
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in.base + slot * plane) + r);
        uint2 o;
        o.x = bf16_rne(v.x) | (bf16_rne(v.y) << 16);
        o.y = bf16_rne(v.z) | (bf16_rne(v.w) << 16);
        reinterpret_cast<uint2 *>(out)[i] = o;
    }
}

__global__ void bf16_unpack_ring_kernel(const uint16_t *in, int64_t plane, int64_t z0, int64_t nquads, Ring out)
{
    const int64_t qpp = plane >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nquads;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t zl = i / qpp, r = i - zl * qpp;
        const int64_t slot = ring_slot(z0 + zl, out.zbase, out.nslot);
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(in) + i);
        uint4 o;
        o.x = v.x << 16;
        o.y = v.x & 0xFFFF0000u;
        o.z = v.y << 16;
        o.w = v.y & 0xFFFF0000u;
        reinterpret_cast<uint4 *>(out.base + slot * plane)[r] = o;
    }
}

unsigned grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    const int64_t cap = 152 * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_bf16_pack_ring(ConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, uint16_t *out,
                                  cudaStream_t st)
{
    const int64_t plane = nx * ny, nquads = plane * (z1 - z0) / 4;
    if (nquads <= 0)
        return cudaSuccess;
    bf16_pack_ring_kernel<<<grid_for(nquads), 256, 0, st>>>(in, plane, z0, nquads, out);
    return cudaGetLastError();
}

cudaError_t launch_bf16_unpack_ring(const uint16_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, Ring out,
                                    cudaStream_t st)
{
    const int64_t plane = nx * ny, nquads = plane * (z1 - z0) / 4;
    if (nquads <= 0)
        return cudaSuccess;
    bf16_unpack_ring_kernel<<<grid_for(nquads), 256, 0, st>>>(in, plane, z0, nquads, out);
    return cudaGetLastError();
}

}  // namespace ooc
