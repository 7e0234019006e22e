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
#include <cuda.h>

#include <mutex>

#include "common.cuh"

using namespace ooc;

namespace {

constexpr int64_t kNoAllocMaxPoints = OOC_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_heat_scratch[kNoAllocMaxPoints];

// Device address of g_heat_scratch per device, with the unique ID of the
// context it was looked up in.  The address belongs to the module loaded
// in that context: if the context is destroyed and another one made (a
// cudaDeviceReset, for one), the module is loaded again and the array may
// move, so a call whose current context has another ID looks it up again.
struct ScratchEntry {
    unsigned long long ctx_id;
    float *addr;
};
ScratchEntry g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique ID of the calling thread's current context (0 when there is none
// yet).  The driver functions come through the runtime's entry-point query,
// so the library does not link the driver library itself.
ooc_status current_ctx_id(unsigned long long *id)
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return OOC_E_CUDA;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS)
        return OOC_E_CUDA;
    *id = 0;
    if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS)
        return OOC_E_CUDA;
    return OOC_OK;
}

ooc_status scratch_for_current_device(float **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return OOC_E_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    if (current_ctx_id(&id) != OOC_OK)
        return OOC_E_CUDA;
    if (id == 0 || g_scratch[dev].addr == nullptr || g_scratch[dev].ctx_id != id) {
        // the lookup also makes the device's primary context current when
        // no context is yet
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_heat_scratch) != cudaSuccess || p == nullptr)
            return OOC_E_CUDA;
        if (current_ctx_id(&id) != OOC_OK || id == 0)
            return OOC_E_CUDA;
        g_scratch[dev] = ScratchEntry{id, static_cast<float *>(p)};
    }
    *out = g_scratch[dev].addr;
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
