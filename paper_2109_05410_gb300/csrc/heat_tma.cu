// heat_tma.cu -- the fused heat7 pairs of the pipeline (two heat7 steps per
// launch, Section III's neighbour average with temporal blocking inside the
// kernel), with each plane of level s-1 staged in shared memory by a TMA
// tensor copy.
#include <mutex>

#include "tma.cuh"

// the pair's point updates in packed FP32 pairs (heat_pt4x2, the same bits
// as heat_pt4, which -DOOC_HEAT_F32X2=0 selects)
#ifndef OOC_HEAT_F32X2
#define OOC_HEAT_F32X2 1
#endif
#if OOC_HEAT_F32X2
#define OOC_HEATX2T_PT heat_pt4x2
#else
#define OOC_HEATX2T_PT heat_pt4
#endif

namespace ooc {

using namespace sten;

// Set by a kernel whose bounded wait gave up (see heat7x2t_kernel); read and
// cleared by take_stencil_fault().
__device__ unsigned g_stencil_fault = 0u;

namespace {

// ---- fused heat7 pairs with TMA-staged planes ---------------------------------
// Same tiles, planes, bands and per-point arithmetic as heat7x2r_kernel (so
// the results are bit-identical), but level s-1 reaches the CTA as whole
// planes of its tile: one thread issues a TMA tensor copy per plane
// (cp.async.bulk.tensor, 136 x 18 floats: the 128 level-s columns with 4 on
// each side, the 16 level-s rows with 1 above and below) into a ring of NS
// shared-memory stages, each guarded by an mbarrier that the copy completes.
// The tensor map's zero fill of out-of-range x and y is the zero ghost of
// the boundary, so no thread tests or loads halos; the threads only read
// shared memory, compute and store.  Level s goes to a 3-plane shared ring
// for the y-neighbours of level s+1.  One CTA barrier per plane orders the
// level-s ring and frees the stage the next copy lands in.
//
// Every wait on an mbarrier is bounded: after kMbarTries polls (each
// suspending up to ~1 us) the CTA agrees, through the plane barrier, to stop;
// thread 0 then waits (bounded again) for the copies it issued, sets
// g_stencil_fault and the CTA returns without writing further planes.
// Tile shape: NW warps, R level-s rows per warp (R = 2: the tiles of
// heat7x2r_kernel), so R NW level-s rows and R NW - 2 output rows.  Three
// or four rows per thread (fewer instructions per point, fewer warps) gave
// the same time on the pipeline's 56-plane windows (112-116 us per launch)
// and 7 % more on 512-plane fields; two rows keep 72 registers.
#ifndef OOC_HEATX2T_R
#define OOC_HEATX2T_R 2
#endif
#ifndef OOC_HEATX2T_NW
#define OOC_HEATX2T_NW 8
#endif
template <int R, int NW>
struct X2tShape {
    static constexpr int rows = R * NW;                                  // level-s rows of a tile
    static constexpr int tyo = rows - 2;                                 // level s+1 (output) rows
    static constexpr int srows = rows + 2;                               // level s-1 rows staged
    static constexpr int scols = 4 * kTX + 8;                            // level s-1 columns staged (136)
    static constexpr int stage_floats = (srows * scols + 31) / 32 * 32;  // 128-byte aligned stages
    static constexpr int copy_bytes = srows * scols * 4;
    static constexpr int l1_float4 = rows * kTX;                         // one level-s plane of the tile
};
constexpr int kX2tR = OOC_HEATX2T_R;
constexpr int kX2tNW = OOC_HEATX2T_NW;
using X2t = X2tShape<kX2tR, kX2tNW>;
// 5 stages and 3 CTAs per SM (72 KB of shared memory and at most 85
// registers each), loop unrolled 3 times (the z-queues rotate without
// copies).  In the 1024^3 FR4-16 pipeline (56-plane windows), per launch:
// 110.4 us; 112.4 us not unrolled; 6 stages and 2 CTAs per SM 128.6 us
// (120.6 us unrolled); heat7x2r_kernel 146.2 us.
#ifndef OOC_HEATX2T_NS
#define OOC_HEATX2T_NS 5
#endif
#ifndef OOC_HEATX2T_MINB
#define OOC_HEATX2T_MINB 3
#endif
#ifndef OOC_HEATX2T_UNROLL
#define OOC_HEATX2T_UNROLL 3
#endif
constexpr int kX2tNS = OOC_HEATX2T_NS;
size_t heat7x2t_smem_bytes()
{
    return (size_t)kX2tNS * X2t::stage_floats * 4 + 3 * (size_t)X2t::l1_float4 * 16 + kX2tNS * 8;
}

template <int NS, int R, int NW>
__global__ void __launch_bounds__(kTX *NW, OOC_HEATX2T_MINB)
    heat7x2t_kernel(const __grid_constant__ CUtensorMap tin, float *__restrict__ out, int nslot, int64_t zbase,
                    Grid3 g, int64_t z0, int64_t z1, int64_t ntiles, int64_t nfull, int64_t zchunk, int64_t lo64,
                    int64_t hi64, const float *__restrict__ band_in, int64_t bin_lo64, float *__restrict__ band_out,
                    int64_t bout_lo64, float r)
{
    using S = X2tShape<R, NW>;
    constexpr int TYO = S::tyo;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);
    float4 *l1 = reinterpret_cast<float4 *>(smem_raw + (size_t)NS * S::stage_floats * 4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + (size_t)NS * S::stage_floats * 4 +
                                                 3 * (size_t)S::l1_float4 * 16);
    const int lane = threadIdx.x, w = threadIdx.y;
    const bool leader = lane == 0 && w == 0;
    int64_t tile, zs64, ze64;
    if ((int64_t)blockIdx.x < nfull) {
        tile = blockIdx.x;
        zs64 = z0;
        ze64 = z1;
    } else {
        const int64_t j = (int64_t)blockIdx.x - nfull, rest = ntiles - nfull;
        tile = nfull + j % rest;
        zs64 = z0 + (j / rest) * zchunk;
        ze64 = min(zs64 + zchunk, z1);
    }
    const int64_t gx = (g.nx + kSeg - 9) / (kSeg - 8);  // x tiles; tile = by * gx + bx
    const int64_t xs = (tile % gx) * (kSeg - 8) - 4;     // first level-s column
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (tile / gx) * TYO;
    const int L0 = R * w;  // this warp's first level-s row in the tile (row y0 - 1 + L0)
    // plane indices fit 32 bits (nz <= 2^30)
    const int nz = (int)g.nz, lo = (int)lo64, hi = (int)hi64, bin_lo = (int)bin_lo64, bout_lo = (int)bout_lo64;
    const int zs = (int)zs64, ze = (int)ze64;
    const int64_t plane = g.plane;
    const bool xin = x4 >= 0 && x4 < g.nx;
    const bool lin = lane >= 1 && lane <= kTX - 2;
    bool in[R], own[R];
    int64_t off[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int64_t y = y0 - 1 + L0 + j;
        in[j] = xin && y >= 0 && y < g.ny;
        off[j] = in[j] ? y * g.nx + x4 : 0;
        own[j] = in[j] && lin && L0 + j >= 1 && L0 + j <= S::rows - 2;  // level s+1 stored here
    }
    const float4 z4 = zero4();

    // staged planes zs-2 .. ze+1: stage index i holds plane zs - 2 + i in
    // slot i mod NS, completing phase (i / NS) of that slot's mbarrier
    const int zfirst = zs - 2, nplanes = ze - zs + 4;
    const int tx = (int)(xs - 4), ty = (int)(y0 - 2);
    // ring slot of the next plane the leader copies (advanced one plane per
    // copy, so no division in the loop)
    int islot = (int)ring_slot(zfirst, zbase, nslot);
    auto issue = [&](int i) {  // copies plane zfirst + i; i advances by one per call
        const int zp = zfirst + i, sl = i % NS;
        if (zp >= 0 && zp < nz) {
            mbar_arrive_tx(&bar[sl], (unsigned)S::copy_bytes);
            tma_load_3d(stages + sl * S::stage_floats, &tin, tx, ty, islot, &bar[sl]);
        } else {
            mbar_arrive(&bar[sl]);  // a plane outside the grid: nothing to copy, the phase completes at once
        }
        islot = wrap_add(islot, 1, nslot);
    };
    if (leader) {
        for (int j = 0; j < NS; ++j)
            mbar_init(&bar[j], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    int issued = 0;  // stage indices issued so far (tracked by every thread)
    if (leader)
        for (int i = 0; i < NS && i < nplanes; ++i)
            issue(i);
    issued = NS < nplanes ? NS : nplanes;
    // staged row `row` (row 0 = y0 - 2); this thread's float4 is at column
    // 4 lane + 4, the halo floats of lanes 0 and 31 at columns 3 and 4 kTX + 4
    auto srow = [&](int sl, int row) -> const float * { return stages + sl * S::stage_floats + row * S::scols; };
    auto s4 = [&](int sl, int row) -> float4 { return reinterpret_cast<const float4 *>(srow(sl, row))[lane + 1]; };

    unsigned fail = 0;
    fail |= mbar_wait(&bar[0], 0) ? 0u : 1u;
    fail |= mbar_wait(&bar[1 % NS], (1 / NS) & 1) ? 0u : 1u;
    // level s-1 queue z-1, z, z+1 of the thread's rows (zero outside the
    // grid: the copies fill zeros there, and planes outside are not read)
    float4 pq[R], cq[R], s2[R], s1[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        pq[j] = (!fail && zfirst >= 0) ? s4(0, L0 + j + 1) : z4;
        cq[j] = (!fail && zfirst + 1 >= 0 && zfirst + 1 < nz) ? s4(1 % NS, L0 + j + 1) : z4;
        s2[j] = z4;  // level s at planes z-2, z-1
        s1[j] = z4;
    }
    int sc = 1 % NS, sn = 2 % NS;                      // stages of planes z and z+1
    int l1c = 0;                                       // level-s ring plane of z
    int oslot = (int)ring_slot(zs - 2, zbase, nslot);  // output ring slot of plane z-1
OOC_PRAGMA(unroll OOC_HEATX2T_UNROLL)
    for (int z = zs - 1, i = 1; z <= ze; ++z, ++i) {
        // level s-1 plane z+1 (stage index i + 1)
        if (!mbar_wait(&bar[sn], (unsigned)(((i + 1) / NS) & 1)))
            fail = 1u;
        float4 nq[R], sv[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            nq[j] = z + 1 < nz ? s4(sn, L0 + j + 1) : z4;
            sv[j] = z4;
        }
        // level s at plane z (z is uniform over the CTA); a row's neighbours
        // on the thread's other rows come from registers
        if (z >= lo && z < hi) {
            const float4 upo = s4(sc, L0);          // the row above the thread's first
            const float4 dno = s4(sc, L0 + R + 1);  // the row below its last
#pragma unroll
            for (int j = 0; j < R; ++j) {
                float xl = __shfl_up_sync(0xffffffffu, cq[j].w, 1), xr = __shfl_down_sync(0xffffffffu, cq[j].x, 1);
                if (lane == 0)
                    xl = srow(sc, L0 + j + 1)[3];
                if (lane == kTX - 1)
                    xr = srow(sc, L0 + j + 1)[4 * kTX + 4];
                const float4 o = OOC_HEATX2T_PT(cq[j], xl, xr, j == 0 ? upo : cq[j - 1], j == R - 1 ? dno : cq[j + 1],
                                          pq[j], nq[j], r);
                sv[j] = in[j] ? o : z4;
            }
        } else if (band_in != nullptr && z >= bin_lo && z < bin_lo + 2) {
            const float *bp = band_in + (int64_t)(z - bin_lo) * plane;
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (in[j])
                    sv[j] = ldg4(bp + off[j]);
        }
        if (band_out != nullptr && z >= bout_lo && z < bout_lo + 2) {
            float *bp = band_out + (int64_t)(z - bout_lo) * plane;
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (own[j])
                    *reinterpret_cast<float4 *>(bp + off[j]) = sv[j];
        }
#pragma unroll
        for (int j = 0; j < R; ++j)
            l1[l1c * S::l1_float4 + (L0 + j) * kTX + lane] = sv[j];
        // all threads have read stage z-1 and written level s of plane z;
        // the plane read next (level s of z-1) was written before this
        // barrier in the previous iteration
        if (__syncthreads_or((int)fail)) {
            if (leader) {
                // the last copy issued into each slot may still be in flight
                for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                    mbar_wait(&bar[j % NS], (unsigned)((j / NS) & 1));
                atomicOr(&g_stencil_fault, 1u);
            }
            return;
        }
        if (i - 1 + NS < nplanes) {
            if (leader)
                issue(i - 1 + NS);  // into the slot of plane z-1
            ++issued;
        }
        // level s+1 at plane z-1 from level s at planes z-2, z-1, z
        if (z - 1 >= zs) {
            const int lp = l1c == 0 ? 2 : l1c - 1;
            const float4 upo = w >= 1 ? l1[lp * S::l1_float4 + (L0 - 1) * kTX + lane] : z4;
            const float4 dno = w <= NW - 2 ? l1[lp * S::l1_float4 + (L0 + R) * kTX + lane] : z4;
            float *op = out + (int64_t)oslot * plane;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float yl = __shfl_up_sync(0xffffffffu, s1[j].w, 1);
                const float yr = __shfl_down_sync(0xffffffffu, s1[j].x, 1);
                const float4 o = OOC_HEATX2T_PT(s1[j], yl, yr, j == 0 ? upo : s1[j - 1], j == R - 1 ? dno : s1[j + 1],
                                          s2[j], sv[j], r);
                if (own[j])
                    *reinterpret_cast<float4 *>(op + off[j]) = o;
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            s2[j] = s1[j];
            s1[j] = sv[j];
            pq[j] = cq[j];
            cq[j] = nq[j];
        }
        sc = sn;
        sn = sn + 1 == NS ? 0 : sn + 1;
        l1c = l1c == 2 ? 0 : l1c + 1;
        oslot = wrap_add(oslot, 1, nslot);
    }
}

// Tensor maps of the rings the TMA kernels read, keyed by (base, nx, ny,
// slots, box); the pipelines use a few rings, so a few entries cover them
// and a map is encoded once per ring and box.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
struct MapEntry {
    const void *base;
    int64_t nx, ny, nslot;
    int box_x, box_y, dev;
    CUtensorMap map;
};
constexpr int kMapCache = 16;
MapEntry g_maps[kMapCache];
int g_maps_used = 0, g_maps_next = 0;
std::mutex g_maps_mutex;

}  // namespace

cudaError_t ring_tensor_map(const float *base, int64_t nx, int64_t ny, int64_t nslot, int box_x, int box_y,
                            CUtensorMap *out)
{
    static EncodeTiledFn encode = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_maps_mutex);
    for (int i = 0; i < g_maps_used; ++i)
        if (g_maps[i].base == base && g_maps[i].nx == nx && g_maps[i].ny == ny && g_maps[i].nslot == nslot &&
            g_maps[i].box_x == box_x && g_maps[i].box_y == box_y && g_maps[i].dev == dev) {
            *out = g_maps[i].map;
            return cudaSuccess;
        }
    if (!encode) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f)
            return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeTiledFn>(f);
    }
    // dims x, y, slot; out-of-range x and y read as zero (the boundary's
    // zero ghosts)
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nslot};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    MapEntry e{base, nx, ny, nslot, box_x, box_y, dev, {}};
    if (encode(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (g_maps_used < kMapCache)
        g_maps[g_maps_used++] = e;
    else {
        g_maps[g_maps_next] = e;
        g_maps_next = (g_maps_next + 1) % kMapCache;
    }
    *out = e.map;
    return cudaSuccess;
}

cudaError_t take_stencil_fault(unsigned *fault)
{
    unsigned v = 0u;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_stencil_fault, sizeof(v));
    if (e == cudaSuccess && v != 0u) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_stencil_fault, &zero, sizeof(zero));
    }
    unsigned vw = 0u;
    if (e == cudaSuccess)
        e = take_wave_fault(&vw);
    *fault = v | vw;
    return e;
}

cudaError_t launch_heat7x2(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                           int64_t lo, int64_t hi, const float *band_in, int64_t bin_lo, float *band_out,
                           int64_t bout_lo, float r, cudaStream_t st)
{
#if OOC_HEATX2_ROWS != 3
    return launch_heat7x2_regs(in, out, nx, ny, nz, z0, z1, lo, hi, band_in, bin_lo, band_out, bout_lo, r, st);
#else
    if (z1 <= z0)
        return cudaSuccess;
    constexpr int NW = kX2tNW;
    constexpr int TYO = X2t::tyo;
    const size_t smem = heat7x2t_smem_bytes();
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = [smem]() -> int {
        if (cudaFuncSetAttribute(heat7x2t_kernel<kX2tNS, kX2tR, kX2tNW>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 0;
        return resident((const void *)heat7x2t_kernel<kX2tNS, kX2tR, kX2tNW>, kTX * NW, smem);
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kSeg - 9) / (kSeg - 8), gy = (ny + TYO - 1) / TYO;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 8, 5, res);
    if (in.nslot != out.nslot || in.zbase != out.zbase || in.nslot > (1ll << 30) || in.base == out.base ||
        gx * gy > 0x7fffffffll || nz > (1ll << 30))
        return cudaErrorInvalidValue;
    const FusedGrid fg = fused_grid(gx * gy, z1 - z0, chunk, res);
    if (fg.ncta > 0x7fffffffll)
        return cudaErrorInvalidValue;
    // the TMA x coordinate (first column - 8) is a multiple of 4 floats:
    // tiles start at multiples of 120; ring strides are multiples of 16 bytes
    if (nx % 4 || ((uintptr_t)in.base % 16) || nx > 0x7fffffffll || ny > 0x7fffffffll)
        return cudaErrorInvalidValue;
    CUtensorMap map;
    cudaError_t e = ring_tensor_map(in.base, nx, ny, in.nslot, X2t::scols, X2t::srows, &map);
    if (e != cudaSuccess)
        return e;
    heat7x2t_kernel<kX2tNS, kX2tR, kX2tNW><<<(unsigned)fg.ncta, dim3(kTX, NW), smem, st>>>(
        map, out.base, (int)in.nslot, in.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, gx * gy, fg.nfull, fg.zch, lo, hi,
        band_in, bin_lo, band_out, bout_lo, r);
    return cudaGetLastError();
#endif
}

}  // namespace ooc
