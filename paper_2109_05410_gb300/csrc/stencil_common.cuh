// stencil_common.cuh -- device helpers and launch geometry shared by the
// stencil kernels (stencil.cu: heat7, wave25, FP64 heat7, the register-
// loading fused heat7 pairs; heat_tma.cu: the TMA-staged fused heat7 pairs).
#pragma once
#include "common.cuh"
#include "f32x2.cuh"

#define OOC_PRAGMA_(x) _Pragma(#x)
#define OOC_PRAGMA(x) OOC_PRAGMA_(x)
// fused heat7 pairs: 3: heat7x2t_kernel (TMA-staged), 2: heat7x2r_kernel,
// 1: heat7x2_kernel
#ifndef OOC_HEATX2_ROWS
#define OOC_HEATX2_ROWS 3
#endif
// wave25: 0 = cp.async-staged kernel (stencil.cu), 1 = TMA-staged kernel
// (wave_tma.cu).  The TMA kernel passes the same tests but measured slower:
// 0.393 against 0.369 ms per step at 512^3, and 188 against 209 Gpts/s for
// the 1024^3 code-4 pipeline on one box.
#ifndef OOC_WAVE_TMA
#define OOC_WAVE_TMA 0
#endif

namespace ooc {
namespace sten {

constexpr int kTX = 32;  // threads per row segment (4 points each: 128 x)
constexpr int kSeg = 4 * kTX;

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

struct Grid3 {
    int64_t nx, ny, nz, plane;
};

// All rings of one launch share the slot geometry (Z, zbase), so one 32-bit
// slot counter per z-step addresses every field; it advances with wrap-around.
__device__ __forceinline__ int wrap_add(int s, int d, int nslot)
{
    s += d;
    return s >= nslot ? s - nslot : s;
}

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// One heat7 point in a fixed operation order, written with rounding
// intrinsics so that the compiler cannot contract or reorder it: every heat
// kernel uses it, and a fused two-step launch reproduces two single-step
// launches bit for bit.
//   u' = u + r * (((x- + x+) + (y- + y+)) + (z- + z+) - 6 u)
__device__ __forceinline__ float heat_pt(float c, float xl, float xr, float up, float dn, float zm, float zp, float r)
{
    const float t = __fadd_rn(__fadd_rn(__fadd_rn(xl, xr), __fadd_rn(up, dn)), __fadd_rn(zm, zp));
    return __fmaf_rn(r, __fmaf_rn(-6.0f, c, t), c);
}

// Four consecutive x points; xl / xr are the neighbours left of c.x and
// right of c.w.
__device__ __forceinline__ float4 heat_pt4(float4 c, float xl, float xr, float4 up, float4 dn, float4 zm, float4 zp,
                                           float r)
{
    float4 o;
    o.x = heat_pt(c.x, xl, c.y, up.x, dn.x, zm.x, zp.x, r);
    o.y = heat_pt(c.y, c.x, c.z, up.y, dn.y, zm.y, zp.y, r);
    o.z = heat_pt(c.z, c.y, c.w, up.z, dn.z, zm.z, zp.z, r);
    o.w = heat_pt(c.w, c.z, xr, up.w, dn.w, zm.w, zp.w, r);
    return o;
}

// heat_pt4 with points (0, 1) and (2, 3) in packed FP32 pairs (f32x2.cuh):
// the same operations in the same order, so the same bits, with half the
// floating-point instructions.
__device__ __forceinline__ float4 heat_pt4x2(float4 c, float xl, float xr, float4 up, float4 dn, float4 zm, float4 zp,
                                             float r)
{
    const F2 c01 = pk2(c.x, c.y), c23 = pk2(c.z, c.w);
    const F2 mid = pk2(c.y, c.z);  // right neighbours of (0, 1), left neighbours of (2, 3)
    const F2 t01 = add2(add2(add2(pk2(xl, c.x), mid), add2(pk2(up.x, up.y), pk2(dn.x, dn.y))),
                        add2(pk2(zm.x, zm.y), pk2(zp.x, zp.y)));
    const F2 t23 = add2(add2(add2(mid, pk2(c.w, xr)), add2(pk2(up.z, up.w), pk2(dn.z, dn.w))),
                        add2(pk2(zm.z, zm.w), pk2(zp.z, zp.w)));
    const F2 m6 = dup2(-6.0f), r2 = dup2(r);
    float4 o;
    unpk2(fma2(r2, fma2(m6, c01, t01), c01), o.x, o.y);
    unpk2(fma2(r2, fma2(m6, c23, t23), c23), o.z, o.w);
    return o;
}

// z-chunk so that the grid fills whole waves: pick the chunk count (1..8,
// chunks of at least min_chunk planes) minimising waves x (chunk + overhead).
inline int64_t choose_chunk(int64_t ntiles, int64_t height, int64_t min_chunk, int64_t overhead, int resident_ctas)
{
    int64_t best_n = 1;
    double best_cost = 1e300;
    for (int64_t n = 1; n <= 8; ++n) {
        const int64_t chunk = (height + n - 1) / n;
        if (n > 1 && chunk < min_chunk)
            break;
        const int64_t ctas = ntiles * n;
        const int64_t waves = (ctas + resident_ctas - 1) / resident_ctas;
        const double cost = (double)waves * (double)(chunk + overhead);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best_n = n;
        }
    }
    return (height + best_n - 1) / best_n;
}

inline int resident(const void *fn, int threads, size_t dyn_smem = 0)
{
    static const int sms = [] {  // once, thread-safe
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 152;
    }();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn_smem) != cudaSuccess || per_sm <= 0)
        per_sm = 1;
    return per_sm * sms;
}

// Grid of a fused-pair launch: whole waves of whole tiles, then the remaining
// tiles cut into z-chunks that fill the last wave, when the model (waves x
// (planes + 5)) says it beats one chunk size (`chunk`) for all tiles.  CTAs
// below nfull march whole tiles; the others chunks of zch planes.
struct FusedGrid {
    int64_t nfull, zch, ncta;
};

inline FusedGrid fused_grid(int64_t ntiles, int64_t H, int64_t chunk, int res)
{
    const int64_t gz = (H + chunk - 1) / chunk;
    FusedGrid fg{0, chunk, ntiles * gz};
    double best = (double)((fg.ncta + res - 1) / res) * (double)(chunk + 5);
    const int64_t full = ntiles / res * res, rest = ntiles - full;
    if (full > 0 && rest > 0) {
        for (int64_t m = 1; m <= 16; ++m) {
            const int64_t c = (H + m - 1) / m;
            if (m > 1 && c < 8)
                break;
            const double cost = (double)(full / res) * (double)(H + 5) +
                                (double)((rest * m + res - 1) / res) * (double)(c + 5);
            if (cost < best * 0.999) {
                best = cost;
                fg = FusedGrid{full, c, full + rest * ((H + c - 1) / c)};
            }
        }
    }
    return fg;
}

}  // namespace sten

cudaError_t launch_heat7x2_regs(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                                int64_t lo, int64_t hi, const float *band_in, int64_t bin_lo, float *band_out,
                                int64_t bout_lo, float r, cudaStream_t st);

}  // namespace ooc
