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

// Planes [z0, z1) of a ring: blockIdx.y is the plane, and each thread moves
// up to four quads of 4 values of it (16-byte FP32 / 8-byte BF16 accesses),
// all loads first, so that several are in flight (nx*ny is a multiple of 4).
constexpr int kQuadsPerThread = 4;

__global__ void bf16_pack_ring_kernel(ConstRing in, int64_t plane, int64_t z0, uint16_t *out)
{
    const int64_t qpp = plane >> 2;  // quads per plane
    const int64_t zl = blockIdx.y;
    const uint4 *src = reinterpret_cast<const uint4 *>(in.base + ring_slot(z0 + zl, in.zbase, in.nslot) * plane);
    uint2 *dst = reinterpret_cast<uint2 *>(out) + zl * qpp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < qpp; i += kQuadsPerThread * stride) {
        uint4 v[kQuadsPerThread];
#pragma unroll
        for (int k = 0; k < kQuadsPerThread; ++k)
            if (i + k * stride < qpp)
                v[k] = __ldg(src + i + k * stride);
#pragma unroll
        for (int k = 0; k < kQuadsPerThread; ++k)
            if (i + k * stride < qpp)
                dst[i + k * stride] = make_uint2(bf16_rne(v[k].x) | (bf16_rne(v[k].y) << 16),
                                                 bf16_rne(v[k].z) | (bf16_rne(v[k].w) << 16));
    }
}

__global__ void bf16_unpack_ring_kernel(const uint16_t *in, int64_t plane, int64_t z0, Ring out)
{
    const int64_t qpp = plane >> 2;
    const int64_t zl = blockIdx.y;
    const uint2 *src = reinterpret_cast<const uint2 *>(in) + zl * qpp;
    uint4 *dst = reinterpret_cast<uint4 *>(out.base + ring_slot(z0 + zl, out.zbase, out.nslot) * plane);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < qpp; i += kQuadsPerThread * stride) {
        uint2 v[kQuadsPerThread];
#pragma unroll
        for (int k = 0; k < kQuadsPerThread; ++k)
            if (i + k * stride < qpp)
                v[k] = __ldg(src + i + k * stride);
#pragma unroll
        for (int k = 0; k < kQuadsPerThread; ++k)
            if (i + k * stride < qpp)
                dst[i + k * stride] =
                    make_uint4(v[k].x << 16, v[k].x & 0xFFFF0000u, v[k].y << 16, v[k].y & 0xFFFF0000u);
    }
}

// CTAs of 256 threads per plane: enough for each thread to move
// kQuadsPerThread quads once.
dim3 plane_grid(int64_t plane, int64_t nplanes)
{
    const int64_t qpp = plane >> 2;
    int64_t bx = (qpp + 256 * kQuadsPerThread - 1) / (256 * kQuadsPerThread);
    bx = bx < 1 ? 1 : (bx > 65535 ? 65535 : bx);
    return dim3((unsigned)bx, (unsigned)nplanes);
}

}  // namespace

cudaError_t launch_bf16_pack_ring(ConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, uint16_t *out,
                                  cudaStream_t st)
{
    const int64_t plane = nx * ny;
    if (z1 <= z0 || plane <= 0)
        return cudaSuccess;
    for (int64_t z = z0; z < z1; z += 65535) {  // gridDim.y limit
        const int64_t n = z1 - z < 65535 ? z1 - z : 65535;
        bf16_pack_ring_kernel<<<plane_grid(plane, n), 256, 0, st>>>(in, plane, z, out + (z - z0) * plane);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bf16_unpack_ring(const uint16_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, Ring out,
                                    cudaStream_t st)
{
    const int64_t plane = nx * ny;
    if (z1 <= z0 || plane <= 0)
        return cudaSuccess;
    for (int64_t z = z0; z < z1; z += 65535) {  // gridDim.y limit
        const int64_t n = z1 - z < 65535 ? z1 - z : 65535;
        bf16_unpack_ring_kernel<<<plane_grid(plane, n), 256, 0, st>>>(in + (z - z0) * plane, plane, z, out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace ooc
