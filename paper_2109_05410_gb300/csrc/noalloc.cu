// noalloc.cu -- ooc_heat7_steps_noalloc: the in-core heat7 steps of
// ooc_heat7_steps without the caller-supplied scratch field.
//
// Some callers cannot hand this library a scratch buffer.  A host
// application or framework that owns every device allocation (a fixed pool,
// a custom allocator that must not grow) may have no memory to spare for a
// second full field, and a caller in a time-critical step loop may not want
// to allocate at all, because an allocation can fail or stall there.  This
// entry point keeps its ping-pong field in a fixed device array that is part
// of the library image instead, so the caller passes only the field itself.
//
// The array holds kNoAllocMaxPoints floats (16 MiB).  Every GPU that loads
// the library keeps it until the process exits.  Grids larger than that are
// refused with OOC_E_INVALID.  All calls share the one array: calls that
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.  A step writes every point of its
// output before any point is read, so nothing left in the array by an
// earlier call is ever used and nothing has to be cleared between calls.
#include <mutex>

#include "common.cuh"

using namespace ooc;

namespace {

constexpr int64_t kNoAllocMaxPoints = OOC_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_heat_scratch[kNoAllocMaxPoints];

// Device address of g_heat_scratch per device, looked up once per device
// (with that device current) on the first call made on it.
float *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

ooc_status scratch_for_current_device(float **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return OOC_E_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_heat_scratch) != cudaSuccess || p == nullptr)
            return OOC_E_CUDA;
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return OOC_OK;
}

}  // namespace

extern "C" ooc_status ooc_heat7_steps_noalloc(float *d_u, int64_t nx, int64_t ny, int64_t nz, double r,
                                              int64_t nsteps, void *stream)
{
    if (!d_u || nx <= 0 || ny <= 0 || nz <= 0 || nx % 4 || ny % 4 || nz % 4 || nsteps < 0 ||
        ((uintptr_t)d_u % 16))
        return OOC_E_INVALID;
    if (nx > kNoAllocMaxPoints || ny > kNoAllocMaxPoints || nz > kNoAllocMaxPoints ||
        nx * ny > kNoAllocMaxPoints || nx * ny * nz > kNoAllocMaxPoints)
        return OOC_E_INVALID;  // grid does not fit the fixed scratch array
    float *tmp = nullptr;
    const ooc_status s = scratch_for_current_device(&tmp);
    if (s != OOC_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *a = d_u, *b = tmp;
    for (int64_t i = 0; i < nsteps; ++i) {
        if (launch_heat7(ConstRing{a, nz, 0}, Ring{b, nz, 0}, nx, ny, nz, 0, nz, (float)r, st) != cudaSuccess)
            return OOC_E_CUDA;
        float *t = a;
        a = b;
        b = t;
    }
    if (a != d_u && cudaMemcpyAsync(d_u, a, sizeof(float) * nx * ny * nz, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return OOC_E_CUDA;
    return OOC_OK;
}
