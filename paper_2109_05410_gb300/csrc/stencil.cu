// stencil.cu -- heat7 and wave25 window kernels on sm_103a.
//
// Both kernels update the planes [z0, z1) of a slab window held in ring
// buffers (plane z at slot (z + zbase) mod Z).  Values outside the grid are
// zero ghosts.  They are HBM-bound (no tensor cores: nothing here is a
// dense contraction), so the design is about bytes in flight:
//   - a warp owns a 128-wide row segment, 4 points per thread, moved with
//     128-bit loads and stores;
//   - x-neighbours come from the adjacent lanes by warp shuffles (only lanes
//     0 and 31 touch the tile's x-halo in memory);
//   - y-neighbours come from a shared-memory copy of the current plane
//     (double buffered, one barrier per plane), whose halo rows are loaded by
//     the edge warps;
//   - z-neighbours live in a register queue.  heat7 loads the planes two
//     ahead of their use; wave25 stages each plane (tile, halos, p_prev,
//     kappa) in shared memory with cp.async eight planes ahead and fills
//     its 9-plane queue from there; its z-loop runs in rounds of 9 planes,
//     so that the queue and the stage rings are indexed by constants.
// Each CTA marches a chunk of z; the chunk count is chosen from the
// occupancy so that the grid fills whole waves of the 152 SMs.
// Also here: the register-loading fused heat7 pairs (two steps per launch,
// the intermediate level on chip), heat7x2r_kernel (two rows per thread)
// and heat7x2_kernel (one row), built in with OOC_HEATX2_ROWS = 2 or 1 (the
// default build runs the TMA-staged pairs of heat_tma.cu).  The FP64
// kernels are in stencil64.cu.
//
// heat7 (Section III's neighbour average, 3D):
//   u' = u + r (u[x-1] + u[x+1] + u[y-1] + u[y+1] + u[z-1] + u[z+1] - 6u)
// wave25 (Section VI's 25-point propagator, HALO = 4, Table I), leapfrog:
//   p' = 2p - p_prev + kappa * sum_axes[c0 p + sum_m c_m (p[+m] + p[-m])]
// p' overwrites p_prev in place (or goes to a separate array): each point's
// p_prev is read only by the thread that writes p' there.
#include <type_traits>

#include "cp_async.cuh"
#include "f32x2.cuh"
#include "stencil_common.cuh"

namespace ooc {

using namespace sten;

namespace {

constexpr int kHeatTY = 2;  // rows per CTA: small CTAs balance the waves of short windows
// rows per CTA of the cp.async wave kernel: 8 (2 CTAs per SM) or 16 (one
// CTA of 16 warps, a third fewer staged halo rows per output row): 16
// measured slower, 0.380 against 0.367 ms per 512^3 step, with the same bits
#ifndef OOC_WAVE_TY
#define OOC_WAVE_TY 8
#endif
[[maybe_unused]] constexpr int kWaveTY = OOC_WAVE_TY;
// the wave Laplacian in packed FP32 pairs (f32x2.cuh): the same bits as the
// scalar form with half the floating-point instructions, but measured
// slower (0.368 against 0.365 ms per 512^3 step, 118 against 114
// registers): the step is not bound by instruction issue
#ifndef OOC_WAVE_F32X2
#define OOC_WAVE_F32X2 0
#endif
#ifndef OOC_HEAT_UNROLL
#define OOC_HEAT_UNROLL 8
#endif
#ifndef OOC_HEATX2_UNROLL
#define OOC_HEATX2_UNROLL 1
#endif
#ifndef OOC_WAVE_UNROLL
#define OOC_WAVE_UNROLL 1
#endif
#ifndef OOC_HEATX2_MINB
#define OOC_HEATX2_MINB 2  // heat7x2 CTAs per SM (16 warps each): 64 registers, no loop unrolling
#endif
#ifndef OOC_HEATX2_TY
#define OOC_HEATX2_TY 14
#endif
[[maybe_unused]] constexpr int kHeatX2TY = OOC_HEATX2_TY;  // level s+1 rows per CTA of heat7x2_kernel
#ifndef OOC_HEATX2_NW
#define OOC_HEATX2_NW 8
#endif
constexpr int kHeatX2NW = OOC_HEATX2_NW;  // warps of heat7x2r_kernel (2 NW - 2 output rows)
__global__ void __launch_bounds__(kTX *kHeatTY)
    heat7_kernel(const float *__restrict__ in, float *__restrict__ out, int nslot, int64_t zbase, Grid3 g,
                 int64_t z0, int64_t z1, int64_t zchunk, float r)
{
    __shared__ float4 tile[2][kHeatTY + 2][kTX];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t gx = (g.nx + kSeg - 1) / kSeg;  // x tiles; blockIdx.x = by * gx + bx
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kHeatTY;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int64_t nz = g.nz, plane = g.plane;
    // loop-invariant in-grid flags and in-plane offsets
    const bool inside = x4 < g.nx && y < g.ny;
    const int64_t off = inside ? y * g.nx + x4 : 0;
    const int64_t yh = ty == 0 ? y0 - 1 : y0 + kHeatTY;  // halo row of the edge warps
    const bool hrow = (ty == 0 || ty == kHeatTY - 1) && yh >= 0 && yh < g.ny && x4 < g.nx;
    const int64_t hoff = hrow ? yh * g.nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 1 : xs + kSeg;  // halo column of the edge lanes
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx && y < g.ny;
    const int64_t xoff = hcol ? y * g.nx + xh : 0;
    const float4 z4 = zero4();

    int s = (int)ring_slot(za, zbase, nslot);  // slot of plane z
    const float *pm = in + (int64_t)wrap_add(s, nslot - 1, nslot) * plane;
    const float *p0 = in + (int64_t)s * plane;
    const float *p1 = in + (int64_t)wrap_add(s, 1, nslot) * plane;
    const float *p2 = in + (int64_t)wrap_add(s, 2, nslot) * plane;
    // register queue z-1 .. z+2 and the halos of planes z, z+1: loads run
    // two planes ahead of their use
    float4 prev = (inside && za >= 1) ? ldg4(pm + off) : z4;
    float4 cur = (inside && za < nz) ? ldg4(p0 + off) : z4;
    float4 nxt = (inside && za + 1 < nz) ? ldg4(p1 + off) : z4;
    float4 nn = (inside && za + 2 < nz) ? ldg4(p2 + off) : z4;
    float4 hyv = (hrow && za < nz) ? ldg4(p0 + hoff) : z4;
    float4 hyv1 = (hrow && za + 1 < nz) ? ldg4(p1 + hoff) : z4;
    float hx = (hcol && za < nz) ? __ldg(p0 + xoff) : 0.f;
    float hx1 = (hcol && za + 1 < nz) ? __ldg(p1 + xoff) : 0.f;
    int64_t z = za;
    // unrolled twice so that the register queue rotates by renaming
OOC_PRAGMA(unroll OOC_HEAT_UNROLL)
    for (int i = 0; i < cnt; ++i, ++z) {
        const int s2 = wrap_add(s, 2, nslot), s3 = wrap_add(s, 3, nslot);
        const float *q2 = in + (int64_t)s2 * plane;
        const float *q3 = in + (int64_t)s3 * plane;
        const float4 pfv = (inside && z + 3 < nz) ? ldg4(q3 + off) : z4;
        const bool v2 = z + 2 < nz;
        const float4 hyv2 = (hrow && v2) ? ldg4(q2 + hoff) : z4;
        const float hx2 = (hcol && v2) ? __ldg(q2 + xoff) : 0.f;

        const int b = i & 1;
        tile[b][ty + 1][lane] = cur;
        if (ty == 0)
            tile[b][0][lane] = hyv;
        if (ty == kHeatTY - 1)
            tile[b][kHeatTY + 1][lane] = hyv;
        float xl = __shfl_up_sync(0xffffffffu, cur.w, 1);
        float xr = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (lane == 0)
            xl = hx;
        if (lane == kTX - 1)
            xr = hx;
        __syncthreads();
        const float4 up = tile[b][ty][lane];
        const float4 dn = tile[b][ty + 2][lane];
        const float4 o = heat_pt4(cur, xl, xr, up, dn, prev, nxt, r);
        if (inside)
            *reinterpret_cast<float4 *>(out + (int64_t)s * plane + off) = o;
        prev = cur;
        cur = nxt;
        nxt = nn;
        nn = pfv;
        hyv = hyv1;
        hyv1 = hyv2;
        hx = hx1;
        hx1 = hx2;
        s = wrap_add(s, 1, nslot);
    }
}


// Two heat7 steps per launch: levels s and s+1 of a pair, with level s kept
// on chip (temporal blocking inside the kernel, so HBM carries 8 bytes per
// point for two steps instead of 16).
//
// A CTA owns an output tile of 120 x TYO points of level s+1 and marches z.
// Warp w holds row y0 - 1 + w of level s (rows y0-1 .. y0+TYO) over 128 x
// (the tile and 4 points on each side), computed from level s-1 with the
// register queue, shuffles and shared-memory rows of heat7_kernel.  Level s
// of plane z goes to a shared-memory row; level s+1 of plane z-1 is then
// formed on the inner warps and lanes from the level-s rows of planes
// z-2..z.  One barrier per plane: both shared arrays are double buffered.
//
// Level s is computed on the planes [lo, hi) only.  Its two planes below
// lo come from band_in (planes bin_lo, bin_lo+1: left by the previous slab
// of the pipeline), and the two planes [bout_lo, bout_lo+2) are saved to
// band_out for the next slab.  Outside the grid every level is zero.
template <int TYO>
__global__ void __launch_bounds__(kTX *(TYO + 2), OOC_HEATX2_MINB)
    heat7x2_kernel(const float *__restrict__ in, float *__restrict__ out, int nslot, int64_t zbase, Grid3 g,
                   int64_t z0, int64_t z1, int64_t zchunk, int64_t lo, int64_t hi, const float *__restrict__ band_in,
                   int64_t bin_lo, float *__restrict__ band_out, int64_t bout_lo, float r)
{
    constexpr int NW = TYO + 2;
    __shared__ float4 ta[2][TYO + 4][kTX];  // level s-1, rows y0-2 .. y0+TYO+1
    __shared__ float4 tb[2][TYO + 2][kTX];  // level s, rows y0-1 .. y0+TYO
    const int lane = threadIdx.x, w = threadIdx.y;
    const int64_t gx = (g.nx + kSeg - 9) / (kSeg - 8);  // x tiles; blockIdx.x = by * gx + bx
    const int64_t xs = (int64_t)(blockIdx.x % gx) * (kSeg - 8) - 4;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * TYO;
    const int64_t y = y0 - 1 + w;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int64_t nz = g.nz, plane = g.plane;
    const bool xin = x4 >= 0 && x4 < g.nx;
    const bool yin = y >= 0 && y < g.ny;
    const bool inside = xin && yin;
    const int64_t off = inside ? y * g.nx + x4 : 0;
    const int64_t yh = w == 0 ? y0 - 2 : y0 + TYO + 1;  // halo row of the edge warps
    const bool hrow = (w == 0 || w == NW - 1) && yh >= 0 && yh < g.ny && xin;
    const int64_t hoff = hrow ? yh * g.nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 1 : xs + kSeg;  // halo column of the edge lanes
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx && yin;
    const int64_t xoff = hcol ? y * g.nx + xh : 0;
    const bool mid = w >= 1 && w <= TYO;                        // warp produces level s+1
    const bool own = inside && mid && lane >= 1 && lane <= kTX - 2;  // and this thread stores it
    const float4 z4 = zero4();

    int64_t z = za - 1;  // plane of level s produced in the current iteration
    int s = (int)ring_slot(z, zbase, nslot);
    const float *pm = in + (int64_t)wrap_add(s, nslot - 1, nslot) * plane;
    const float *p0 = in + (int64_t)s * plane;
    const float *p1 = in + (int64_t)wrap_add(s, 1, nslot) * plane;
    const float *p2 = in + (int64_t)wrap_add(s, 2, nslot) * plane;
    // level s-1 queue z-1 .. z+2 and the halos of planes z, z+1
    float4 prev = (inside && z >= 1) ? ldg4(pm + off) : z4;
    float4 cur = (inside && z >= 0) ? ldg4(p0 + off) : z4;
    float4 nxt = (inside && z + 1 < nz) ? ldg4(p1 + off) : z4;
    float4 nn = (inside && z + 2 < nz) ? ldg4(p2 + off) : z4;
    float4 hyv = (hrow && z >= 0) ? ldg4(p0 + hoff) : z4;
    float4 hyv1 = (hrow && z + 1 < nz) ? ldg4(p1 + hoff) : z4;
    float hx = (hcol && z >= 0) ? __ldg(p0 + xoff) : 0.f;
    float hx1 = (hcol && z + 1 < nz) ? __ldg(p1 + xoff) : 0.f;
    float4 sm2 = z4, sm1 = z4;  // level s at planes z-2, z-1
OOC_PRAGMA(unroll OOC_HEATX2_UNROLL)
    for (int i = 0; i < cnt + 2; ++i, ++z) {
        const int s2 = wrap_add(s, 2, nslot), s3 = wrap_add(s, 3, nslot);
        const float4 pfv = (inside && z + 3 < nz) ? ldg4(in + (int64_t)s3 * plane + off) : z4;
        const bool v2 = z + 2 >= 0 && z + 2 < nz;
        const float4 hyv2 = (hrow && v2) ? ldg4(in + (int64_t)s2 * plane + hoff) : z4;
        const float hx2 = (hcol && v2) ? __ldg(in + (int64_t)s2 * plane + xoff) : 0.f;

        const int b = i & 1;
        ta[b][w + 1][lane] = cur;
        if (w == 0)
            ta[b][0][lane] = hyv;
        if (w == NW - 1)
            ta[b][TYO + 3][lane] = hyv;
        float xl = __shfl_up_sync(0xffffffffu, cur.w, 1);
        float xr = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (lane == 0)
            xl = hx;
        if (lane == kTX - 1)
            xr = hx;
        __syncthreads();
        // level s at plane z (z is uniform over the CTA)
        float4 sv = z4;
        if (z >= lo && z < hi) {
            const float4 up = ta[b][w][lane];
            const float4 dn = ta[b][w + 2][lane];
            const float4 o = heat_pt4(cur, xl, xr, up, dn, prev, nxt, r);
            sv = inside ? o : z4;
        } else if (band_in != nullptr && z >= bin_lo && z < bin_lo + 2 && inside) {
            sv = ldg4(band_in + (z - bin_lo) * plane + off);
        }
        if (band_out != nullptr && own && z >= bout_lo && z < bout_lo + 2)
            *reinterpret_cast<float4 *>(band_out + (z - bout_lo) * plane + off) = sv;
        tb[b][w][lane] = sv;
        // level s+1 at plane z-1 from the level-s rows of plane z-1 (written
        // in the previous iteration) and planes z-2, z in registers
        if (i >= 2 && mid) {
            const float4 up = tb[b ^ 1][w - 1][lane];
            const float4 dn = tb[b ^ 1][w + 1][lane];
            const float yl = __shfl_up_sync(0xffffffffu, sm1.w, 1);
            const float yr = __shfl_down_sync(0xffffffffu, sm1.x, 1);
            const float4 o = heat_pt4(sm1, yl, yr, up, dn, sm2, sv, r);
            if (own)
                *reinterpret_cast<float4 *>(out + (int64_t)wrap_add(s, nslot - 1, nslot) * plane + off) = o;
        }
        sm2 = sm1;
        sm1 = sv;
        prev = cur;
        cur = nxt;
        nxt = nn;
        nn = pfv;
        hyv = hyv1;
        hyv1 = hyv2;
        hx = hx1;
        hx1 = hx2;
        s = wrap_add(s, 1, nslot);
    }
}

// Two heat7 steps per launch, two rows per thread.  Warp w of NW holds the
// level-s rows a = y0 - 1 + 2w and b = y0 + 2w (rows y0-1 .. y0+TYO of the
// tile, TYO = 2 NW - 2 outputs) over 128 x.  Each row's neighbour on the
// warp's other row comes from registers and only the outer neighbour from
// shared memory; the per-plane address, predicate and barrier work is shared
// by 8 points per thread instead of 4.  Same planes, bands and arithmetic
// (heat_pt4 with the operands in the same slots) as heat7x2_kernel.
template <int NW>
__global__ void __launch_bounds__(kTX *NW, 2)
    heat7x2r_kernel(const float *__restrict__ in, float *__restrict__ out, int nslot, int64_t zbase, Grid3 g,
                    int64_t z0, int64_t z1, int64_t ntiles, int64_t nfull, int64_t zchunk, int64_t lo64,
                    int64_t hi64, const float *__restrict__ band_in, int64_t bin_lo64, float *__restrict__ band_out,
                    int64_t bout_lo64, float r)
{
    constexpr int TYO = 2 * NW - 2;
    __shared__ float4 ta[2][2 * NW + 2][kTX];  // level s-1, row y at index y - y0 + 2
    __shared__ float4 tb[2][2 * NW][kTX];      // level s, row y at index y - y0 + 1
    const int lane = threadIdx.x, w = threadIdx.y;
    // CTAs below nfull march tiles 0 .. nfull-1 over [z0, z1); the others
    // march z-chunks of zchunk planes of the remaining tiles, chunk-major
    // (the tiles of one chunk side by side, so neighbouring tiles run
    // together and share their halo rows through L2).
    int64_t tile, zs, ze;
    if ((int64_t)blockIdx.x < nfull) {
        tile = blockIdx.x;
        zs = z0;
        ze = z1;
    } else {
        const int64_t j = (int64_t)blockIdx.x - nfull, rest = ntiles - nfull;
        tile = nfull + j % rest;
        zs = z0 + (j / rest) * zchunk;
        ze = min(zs + zchunk, z1);
    }
    const int cnt = (int)(ze - zs);
    const int64_t gx = (g.nx + kSeg - 9) / (kSeg - 8);  // x tiles; tile = by * gx + bx
    const int64_t xs = (tile % gx) * (kSeg - 8) - 4;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (tile / gx) * TYO;
    const int64_t ya = y0 - 1 + 2 * w, yb = ya + 1;
    // plane indices fit 32 bits (nz <= 2^20)
    const int nz = (int)g.nz, lo = (int)lo64, hi = (int)hi64, bin_lo = (int)bin_lo64, bout_lo = (int)bout_lo64;
    const int64_t plane = g.plane;
    const bool xin = x4 >= 0 && x4 < g.nx;
    const bool ina = xin && ya >= 0 && ya < g.ny, inb = xin && yb >= 0 && yb < g.ny;
    const int64_t offa = ina ? ya * g.nx + x4 : 0, offb = inb ? yb * g.nx + x4 : 0;
    const int64_t yh = w == 0 ? y0 - 2 : y0 + TYO + 1;  // halo row of the edge warps
    const bool hrow = (w == 0 || w == NW - 1) && yh >= 0 && yh < g.ny && xin;
    const int64_t hoff = hrow ? yh * g.nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 1 : xs + kSeg;  // halo column of the edge lanes
    const bool xhin = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx;
    const bool hca = xhin && ya >= 0 && ya < g.ny, hcb = xhin && yb >= 0 && yb < g.ny;
    const int64_t xoffa = hca ? ya * g.nx + xh : 0, xoffb = hcb ? yb * g.nx + xh : 0;
    // level s+1 is stored on rows y0 .. y0+TYO-1 and the inner lanes
    const bool lin = lane >= 1 && lane <= kTX - 2;
    const bool owna = ina && lin && w >= 1, ownb = inb && lin && w <= NW - 2;
    const float4 z4 = zero4();

    int z = (int)zs - 1;  // plane of level s produced in the current iteration
    int s = (int)ring_slot(z, zbase, nslot);
    const float *pm = in + (int64_t)wrap_add(s, nslot - 1, nslot) * plane;
    const float *p0 = in + (int64_t)s * plane;
    const float *p1 = in + (int64_t)wrap_add(s, 1, nslot) * plane;
    const float *p2 = in + (int64_t)wrap_add(s, 2, nslot) * plane;
    // level s-1 queues z-1 .. z+2 of rows a and b, halos of planes z, z+1
    float4 pa = (ina && z >= 1) ? ldg4(pm + offa) : z4, pb = (inb && z >= 1) ? ldg4(pm + offb) : z4;
    float4 ca = (ina && z >= 0) ? ldg4(p0 + offa) : z4, cb = (inb && z >= 0) ? ldg4(p0 + offb) : z4;
    float4 na = (ina && z + 1 < nz) ? ldg4(p1 + offa) : z4, nb = (inb && z + 1 < nz) ? ldg4(p1 + offb) : z4;
    float4 nna = (ina && z + 2 < nz) ? ldg4(p2 + offa) : z4, nnb = (inb && z + 2 < nz) ? ldg4(p2 + offb) : z4;
    float4 hyv = (hrow && z >= 0) ? ldg4(p0 + hoff) : z4;
    float4 hyv1 = (hrow && z + 1 < nz) ? ldg4(p1 + hoff) : z4;
    float hxa = (hca && z >= 0) ? __ldg(p0 + xoffa) : 0.f, hxb = (hcb && z >= 0) ? __ldg(p0 + xoffb) : 0.f;
    float hxa1 = (hca && z + 1 < nz) ? __ldg(p1 + xoffa) : 0.f, hxb1 = (hcb && z + 1 < nz) ? __ldg(p1 + xoffb) : 0.f;
    float4 s2a = z4, s1a = z4, s2b = z4, s1b = z4;  // level s at planes z-2, z-1
OOC_PRAGMA(unroll OOC_HEATX2_UNROLL)
    for (int i = 0; i < cnt + 2; ++i, ++z) {
        const int s2 = wrap_add(s, 2, nslot), s3 = wrap_add(s, 3, nslot);
        const float *q2 = in + (int64_t)s2 * plane;
        const float *q3 = in + (int64_t)s3 * plane;
        const bool v3 = z + 3 < nz, v2 = z + 2 < nz;  // z >= -1
        const float4 pfa = (ina && v3) ? ldg4(q3 + offa) : z4;
        const float4 pfb = (inb && v3) ? ldg4(q3 + offb) : z4;
        const float4 hyv2 = (hrow && v2) ? ldg4(q2 + hoff) : z4;
        const float hxa2 = (hca && v2) ? __ldg(q2 + xoffa) : 0.f;
        const float hxb2 = (hcb && v2) ? __ldg(q2 + xoffb) : 0.f;

        const int bb = i & 1;
        ta[bb][2 * w + 1][lane] = ca;
        ta[bb][2 * w + 2][lane] = cb;
        if (w == 0)
            ta[bb][0][lane] = hyv;
        if (w == NW - 1)
            ta[bb][2 * NW + 1][lane] = hyv;
        float xla = __shfl_up_sync(0xffffffffu, ca.w, 1), xra = __shfl_down_sync(0xffffffffu, ca.x, 1);
        float xlb = __shfl_up_sync(0xffffffffu, cb.w, 1), xrb = __shfl_down_sync(0xffffffffu, cb.x, 1);
        if (lane == 0) {
            xla = hxa;
            xlb = hxb;
        }
        if (lane == kTX - 1) {
            xra = hxa;
            xrb = hxb;
        }
        __syncthreads();
        // level s at plane z (z is uniform over the CTA)
        float4 sva = z4, svb = z4;
        if (z >= lo && z < hi) {
            const float4 upa = ta[bb][2 * w][lane];
            const float4 dnb = ta[bb][2 * w + 3][lane];
            const float4 oa = heat_pt4(ca, xla, xra, upa, cb, pa, na, r);
            const float4 ob = heat_pt4(cb, xlb, xrb, ca, dnb, pb, nb, r);
            sva = ina ? oa : z4;
            svb = inb ? ob : z4;
        } else if (band_in != nullptr && z >= bin_lo && z < bin_lo + 2) {
            const float *bp = band_in + (int64_t)(z - bin_lo) * plane;
            if (ina)
                sva = ldg4(bp + offa);
            if (inb)
                svb = ldg4(bp + offb);
        }
        if (band_out != nullptr && z >= bout_lo && z < bout_lo + 2) {
            float *bp = band_out + (int64_t)(z - bout_lo) * plane;
            if (owna)
                *reinterpret_cast<float4 *>(bp + offa) = sva;
            if (ownb)
                *reinterpret_cast<float4 *>(bp + offb) = svb;
        }
        tb[bb][2 * w][lane] = sva;
        tb[bb][2 * w + 1][lane] = svb;
        // level s+1 at plane z-1 from level s at planes z-2, z-1 (registers and
        // the neighbouring warps' rows, written in the previous iteration) and z
        if (i >= 2) {
            const float4 upa = w >= 1 ? tb[bb ^ 1][2 * w - 1][lane] : z4;
            const float4 dnb = w <= NW - 2 ? tb[bb ^ 1][2 * w + 2][lane] : z4;
            const float yla = __shfl_up_sync(0xffffffffu, s1a.w, 1), yra = __shfl_down_sync(0xffffffffu, s1a.x, 1);
            const float ylb = __shfl_up_sync(0xffffffffu, s1b.w, 1), yrb = __shfl_down_sync(0xffffffffu, s1b.x, 1);
            const float4 oa = heat_pt4(s1a, yla, yra, upa, s1b, s2a, sva, r);
            const float4 ob = heat_pt4(s1b, ylb, yrb, s1a, dnb, s2b, svb, r);
            float *op = out + (int64_t)wrap_add(s, nslot - 1, nslot) * plane;
            if (owna)
                *reinterpret_cast<float4 *>(op + offa) = oa;
            if (ownb)
                *reinterpret_cast<float4 *>(op + offb) = ob;
        }
        s2a = s1a;
        s1a = sva;
        s2b = s1b;
        s1b = svb;
        pa = ca;
        ca = na;
        na = nna;
        nna = pfa;
        pb = cb;
        cb = nb;
        nb = nnb;
        nnb = pfb;
        hyv = hyv1;
        hyv1 = hyv2;
        hxa = hxa1;
        hxa1 = hxa2;
        hxb = hxb1;
        hxb1 = hxb2;
        s = wrap_add(s, 1, nslot);
    }
}

#if !OOC_WAVE_TMA
// wave25 staging: the p tile of every plane (8 own rows and 4 halo rows on
// each side, plus the 4-point groups beyond the own rows' ends) in kWavePS
// stages, and p_prev / kappa of the own rows in kWaveKS stages.  The copy
// group of plane g, issued kWaveLead planes before g is the centre, carries
// the p tile of g and p_prev / kappa of plane g - kWaveLead + 2.  The z-loop
// runs in rounds of 9 planes, so that the 9-plane z-queue and both stage
// rings are indexed by constants: the queue rotates by renaming, not by
// register copies.
constexpr int kWaveR = 4;
constexpr int kWavePS = 9;
constexpr int kWaveKS = 3;
constexpr int kWaveLead = 8;
struct WaveSmem {
    float4 p[kWavePS][kWaveTY + 2 * kWaveR][kTX];
    float4 xh[kWavePS][kWaveTY][2];
    float4 pp[kWaveKS][kWaveTY][kTX];
    float4 kk[kWaveKS][kWaveTY][kTX];
};

template <int V>
using IC = std::integral_constant<int, V>;

// MODE 0: the leapfrog step above.  MODE 1 (gradient of the adjoint run):
// gsum[own] += (double) pprev * (double) L(pin) in FP64, with `pprev` the
// adjoint field and kappa, pout and the source unused.  MODE 2: the same
// term accumulated in FP32, gacc[own] = fma(pprev, L(pin), gacc[own]) (the
// adjoint run's short in-segment sums, added to an FP64 total per segment).
// The arithmetic is written with rounding intrinsics in a fixed order:
//   L = 3 c0 p + sum_m c_m (((x-m + x+m) + (y-m + y+m)) + (z-m + z+m))
//   p' = kappa L + (2 p - p_prev)
template <int MODE>
__global__ void __launch_bounds__(kTX *kWaveTY, kWaveTY <= 8 ? 2 : 1)
    wave25_kernel(const float *__restrict__ pin, const float *pprev, float *pout, const float *__restrict__ kap, int nslot,
                  int64_t zbase, Grid3 g, int64_t z0, int64_t z1, int64_t zchunk, int64_t sx, int64_t sy, int64_t sz,
                  float w, double *__restrict__ gsum, WaveSrcTable tab, float *__restrict__ gacc = nullptr)
{
    constexpr int R = kWaveR;
    static_assert(kWavePS == 2 * R + 1 && kWavePS % kWaveKS == 0 && kWaveLead == kWavePS - 1, "stage geometry");
    extern __shared__ __align__(16) unsigned char wave_smem[];
    WaveSmem &sm = *reinterpret_cast<WaveSmem *>(wave_smem);
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t gx = (g.nx + kSeg - 1) / kSeg;  // x tiles; blockIdx.x = by * gx + bx
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kWaveTY;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int64_t zend = za + cnt;
    const int64_t nz = g.nz, plane = g.plane;
    const bool xin = x4 < g.nx;
    const bool inside = xin && y < g.ny;
    const int64_t off = inside ? y * g.nx + x4 : 0;
    // copies of this thread: tile rows ty and ty + 8 (y0 - 4 + row), its own
    // p_prev / kappa group, and (lanes 0, 31) the group beyond its row end;
    // an invalid copy reads nothing and fills zeros (its address stays in
    // the ring)
    const int64_t ya = y0 - R + ty, yb = y0 - R + ty + kWaveTY;
    // the tile has kWaveTY + 8 rows: every thread copies row ty, threads
    // ty < 8 also row ty + kWaveTY
    const bool has_b = ty < 2 * R;
    const bool va = xin && ya >= 0 && ya < g.ny, vb = has_b && xin && yb >= 0 && yb < g.ny;
    const int64_t offa = va ? ya * g.nx + x4 : 0, offb = vb ? yb * g.nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 4 : xs + kSeg;
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx && y < g.ny;
    const int64_t xoff = hcol ? y * g.nx + xh : 0;
    const bool src_here = inside && y == sy && sx >= x4 && sx < x4 + 4;
    const float4 z4 = zero4();

    // Copy group of plane gz into p stage ST and, with K, p_prev / kappa of
    // plane gz - kWaveLead + 2 into stage KST.  Copies past the chunk's last
    // use are skipped (the group stays, empty, so that the counts hold).
    // The p slot advances with every group, the p_prev / kappa slot with
    // every group that carries them.
    int ps = (int)ring_slot(za, zbase, nslot), ks = ps, os = ps;
    auto issue = [&](auto st_c, auto kst_c, int64_t gz, bool with_k) {
        constexpr int ST = decltype(st_c)::value, KST = decltype(kst_c)::value;
        if (gz < zend + R) {
            const bool vz = gz < nz;
            const float *pl = pin + (int64_t)ps * plane;
            cp_async16(&sm.p[ST][ty][lane], pl + offa, vz && va);
            if (has_b)
                cp_async16(&sm.p[ST][ty + kWaveTY][lane], pl + offb, vz && vb);
            if (lane == 0 || lane == kTX - 1)
                cp_async16(&sm.xh[ST][ty][lane == 0 ? 0 : 1], pl + xoff, vz && hcol);
        }
        ps = wrap_add(ps, 1, nslot);
        if (with_k) {
            if (gz - kWaveLead + 2 < zend) {
                const int64_t kb = (int64_t)ks * plane;
                cp_async16(&sm.pp[KST][ty][lane], pprev + kb + off, inside);
                if (MODE == 0)
                    cp_async16(&sm.kk[KST][ty][lane], kap + kb + off, inside);
            }
            ks = wrap_add(ks, 1, nslot);
        }
        cp_async_commit();
    };

    // q[(phase + j) mod 9] = p at plane z - 4 + j of this thread's 4 points;
    // planes za - 4 .. za + 3 are read directly, later ones come from the
    // staged tiles
    float4 q[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        const int64_t zj = za - R + j;
        const float *pj = pin + (int64_t)wrap_add(os, nslot - R + j >= nslot ? j - R : nslot - R + j, nslot) * plane;
        q[j] = (inside && zj >= 0 && zj < nz) ? ldg4(pj + off) : z4;
    }
    issue(IC<0>{}, IC<0>{}, za + 0, false);
    issue(IC<1>{}, IC<0>{}, za + 1, false);
    issue(IC<2>{}, IC<0>{}, za + 2, false);
    issue(IC<3>{}, IC<0>{}, za + 3, false);
    issue(IC<4>{}, IC<0>{}, za + 4, false);
    issue(IC<5>{}, IC<0>{}, za + 5, false);
    issue(IC<6>{}, IC<0>{}, za + 6, true);
    issue(IC<7>{}, IC<1>{}, za + 7, true);

    int64_t z = za;
    int base = 0;  // first iteration of the current round
    auto step = [&](auto ph_c) {
        constexpr int PH = decltype(ph_c)::value;  // iteration mod 9: stage of plane z
        if (base + PH >= cnt)
            return;
        cp_async_wait<1>();  // groups up to plane z + 6 have landed (p tile of z + 4, p_prev / kappa of z)
        __syncthreads();     // ... for every thread; the stages of plane z - 1 are free
        issue(IC<(PH + kWaveLead) % kWavePS>{}, IC<(PH + 2) % kWaveKS>{}, z + kWaveLead, true);
        q[(PH + 2 * R) % kWavePS] = sm.p[(PH + R) % kWavePS][ty + R][lane];
        const float4 c = q[(PH + R) % kWavePS];
        float4 lf, rt;
        lf.x = __shfl_up_sync(0xffffffffu, c.x, 1);
        lf.y = __shfl_up_sync(0xffffffffu, c.y, 1);
        lf.z = __shfl_up_sync(0xffffffffu, c.z, 1);
        lf.w = __shfl_up_sync(0xffffffffu, c.w, 1);
        rt.x = __shfl_down_sync(0xffffffffu, c.x, 1);
        rt.y = __shfl_down_sync(0xffffffffu, c.y, 1);
        rt.z = __shfl_down_sync(0xffffffffu, c.z, 1);
        rt.w = __shfl_down_sync(0xffffffffu, c.w, 1);
        if (lane == 0)
            lf = sm.xh[PH][ty][0];
        if (lane == kTX - 1)
            rt = sm.xh[PH][ty][1];
        const float4 ppv = sm.pp[PH % kWaveKS][ty][lane];
        const float4 kv = MODE == 0 ? sm.kk[PH % kWaveKS][ty][lane] : z4;
        const float L[4] = {lf.x, lf.y, lf.z, lf.w};
        const float C[4] = {c.x, c.y, c.z, c.w};
        const float Rt[4] = {rt.x, rt.y, rt.z, rt.w};
        const float PP[4] = {ppv.x, ppv.y, ppv.z, ppv.w};
        const float KV[4] = {kv.x, kv.y, kv.z, kv.w};
        const float cf[R] = {kC1, kC2, kC3, kC4};
        float lap[4];
#if OOC_WAVE_F32X2
        // points (0, 1) and (2, 3) in packed pairs: the same operations in the
        // same order as the scalar form below, two points per instruction
        F2 lp[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            lp[h] = mul2(dup2(3.0f * kC0), pk2(C[2 * h], C[2 * h + 1]));
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const float4 ym = sm.p[PH][ty + R - m][lane];
            const float4 yp = sm.p[PH][ty + R + m][lane];
            const float4 zm = q[(PH + R - m) % kWavePS];
            const float4 zp = q[(PH + R + m) % kWavePS];
            const F2 ys[2] = {add2(pk2(ym.x, ym.y), pk2(yp.x, yp.y)), add2(pk2(ym.z, ym.w), pk2(yp.z, yp.w))};
            const F2 zs[2] = {add2(pk2(zm.x, zm.y), pk2(zp.x, zp.y)), add2(pk2(zm.z, zm.w), pk2(zp.z, zp.w))};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * h;
                const F2 xsum = add2(pk2(pick(L, C, Rt, j - m), pick(L, C, Rt, j + 1 - m)),
                                     pk2(pick(L, C, Rt, j + m), pick(L, C, Rt, j + 1 + m)));
                lp[h] = fma2(dup2(cf[m - 1]), add2(add2(xsum, ys[h]), zs[h]), lp[h]);
            }
        }
        unpk2(lp[0], lap[0], lap[1]);
        unpk2(lp[1], lap[2], lap[3]);
#else
#pragma unroll
        for (int j = 0; j < 4; ++j)
            lap[j] = __fmul_rn(3.0f * kC0, C[j]);
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const float4 ym = sm.p[PH][ty + R - m][lane];
            const float4 yp = sm.p[PH][ty + R + m][lane];
            const float4 zm = q[(PH + R - m) % kWavePS];
            const float4 zp = q[(PH + R + m) % kWavePS];
            const float YM[4] = {ym.x, ym.y, ym.z, ym.w};
            const float YP[4] = {yp.x, yp.y, yp.z, yp.w};
            const float ZM[4] = {zm.x, zm.y, zm.z, zm.w};
            const float ZP[4] = {zp.x, zp.y, zp.z, zp.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float xsum = __fadd_rn(pick(L, C, Rt, j - m), pick(L, C, Rt, j + m));
                const float s = __fadd_rn(__fadd_rn(xsum, __fadd_rn(YM[j], YP[j])), __fadd_rn(ZM[j], ZP[j]));
                lap[j] = __fmaf_rn(cf[m - 1], s, lap[j]);
            }
        }
#endif
        if (MODE == 0) {
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = __fmaf_rn(KV[j], lap[j], __fmaf_rn(2.0f, C[j], -PP[j]));
            if (src_here && z == sz) {
                float ws = w;
                if (tab.w) {  // amplitude of step n = plan time + n_off, from the device table
                    const int64_t n = *tab.t + tab.n_off;
                    ws = n >= 0 && n < tab.nw ? tab.w[n] : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sx == x4 + j)
                        o[j] += ws;
            }
            if (inside)
                *reinterpret_cast<float4 *>(pout + (int64_t)os * plane + off) = make_float4(o[0], o[1], o[2], o[3]);
        } else if (MODE == 2 && inside) {
            float4 *ap = reinterpret_cast<float4 *>(gacc + (int64_t)os * plane + off);
            float4 a = *ap;
            a.x = __fmaf_rn(PP[0], lap[0], a.x);
            a.y = __fmaf_rn(PP[1], lap[1], a.y);
            a.z = __fmaf_rn(PP[2], lap[2], a.z);
            a.w = __fmaf_rn(PP[3], lap[3], a.w);
            *ap = a;
        } else if (MODE == 1 && inside) {
            double2 *gp = reinterpret_cast<double2 *>(gsum + (int64_t)os * plane + off);
            double2 g0 = gp[0], g1 = gp[1];
            g0.x += (double)PP[0] * (double)lap[0];
            g0.y += (double)PP[1] * (double)lap[1];
            g1.x += (double)PP[2] * (double)lap[2];
            g1.y += (double)PP[3] * (double)lap[3];
            gp[0] = g0;
            gp[1] = g1;
        }
        os = wrap_add(os, 1, nslot);
        ++z;
    };
#pragma unroll 1
    for (; base < cnt; base += kWavePS) {
        step(IC<0>{});
        step(IC<1>{});
        step(IC<2>{});
        step(IC<3>{});
        step(IC<4>{});
        step(IC<5>{});
        step(IC<6>{});
        step(IC<7>{});
        step(IC<8>{});
    }
    cp_async_wait<0>();  // no copy may outlive the CTA's shared memory
}

#endif

__global__ void add_time_kernel(int64_t *t, int64_t n) { *t += n; }

__global__ void swap_kernel(float *a, float *b, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float t = a[i];
        a[i] = b[i];
        b[i] = t;
    }
}

}  // namespace

cudaError_t launch_heat7(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                         float r, cudaStream_t st)
{
    if (z1 <= z0)
        return cudaSuccess;
    static const int res = resident((const void *)heat7_kernel, kTX * kHeatTY);  // once, thread-safe
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kHeatTY - 1) / kHeatTY;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 8, 3, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    if (in.nslot != out.nslot || in.zbase != out.zbase || in.nslot > (1ll << 30) || gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    heat7_kernel<<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kHeatTY), 0, st>>>(
        in.base, out.base, (int)in.nslot, in.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, r);
    return cudaGetLastError();
}

// The fused pairs of the register-loading kernels (build option
// OOC_HEATX2_ROWS = 2: heat7x2r_kernel, 1: heat7x2_kernel); the default
// build launches the TMA-staged kernel (heat_tma.cu).
cudaError_t launch_heat7x2_regs(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                                int64_t lo, int64_t hi, const float *band_in, int64_t bin_lo, float *band_out,
                                int64_t bout_lo, float r, cudaStream_t st)
{
    if (z1 <= z0)
        return cudaSuccess;
#if OOC_HEATX2_ROWS != 1
    constexpr int NW = kHeatX2NW;
    constexpr int TYO = 2 * NW - 2;
    static const int res = resident((const void *)heat7x2r_kernel<NW>, kTX * NW);  // once, thread-safe
#else
    constexpr int TYO = kHeatX2TY;
    static const int res = resident((const void *)heat7x2_kernel<TYO>, kTX * (TYO + 2));  // once, thread-safe
#endif
    const int64_t gx = (nx + kSeg - 9) / (kSeg - 8), gy = (ny + TYO - 1) / TYO;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 8, 5, res);
    if (in.nslot != out.nslot || in.zbase != out.zbase || in.nslot > (1ll << 30) || in.base == out.base ||
        gx * gy > 0x7fffffffll || nz > (1ll << 30))
        return cudaErrorInvalidValue;
#if OOC_HEATX2_ROWS != 1
    const FusedGrid fg = fused_grid(gx * gy, z1 - z0, chunk, res);
    if (fg.ncta > 0x7fffffffll)
        return cudaErrorInvalidValue;
    heat7x2r_kernel<NW><<<(unsigned)fg.ncta, dim3(kTX, NW), 0, st>>>(
        in.base, out.base, (int)in.nslot, in.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, gx * gy, fg.nfull, fg.zch, lo,
        hi, band_in, bin_lo, band_out, bout_lo, r);
#else
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    heat7x2_kernel<TYO><<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, TYO + 2), 0, st>>>(
        in.base, out.base, (int)in.nslot, in.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, lo, hi, band_in, bin_lo,
        band_out, bout_lo, r);
#endif
    return cudaGetLastError();
}


#if !OOC_WAVE_TMA
cudaError_t launch_wave25_to(ConstRing p, ConstRing pprev, Ring pnew, ConstRing kappa, int64_t nx, int64_t ny,
                             int64_t nz, int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w,
                             cudaStream_t st, WaveSrcTable tab)
{
    if (z1 <= z0)
        return cudaSuccess;
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = []() -> int {
        if (cudaFuncSetAttribute(wave25_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(WaveSmem)) != cudaSuccess)
            return 0;
        return resident((const void *)wave25_kernel<0>, kTX * kWaveTY, sizeof(WaveSmem));
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kWaveTY - 1) / kWaveTY;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 16, 9, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    if (p.nslot != pnew.nslot || p.zbase != pnew.zbase || p.nslot != kappa.nslot || p.zbase != kappa.zbase ||
        p.nslot != pprev.nslot || p.zbase != pprev.zbase || p.nslot > (1ll << 30) || gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    wave25_kernel<0><<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kWaveTY), sizeof(WaveSmem), st>>>(
        p.base, pprev.base, pnew.base, kappa.base, (int)p.nslot, p.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk,
        sx, sy, sz, w, nullptr, tab);
    return cudaGetLastError();
}

cudaError_t launch_wave25_grad(const float *p, const float *mu, double *g, int64_t nx, int64_t ny, int64_t nz,
                               cudaStream_t st)
{
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = []() -> int {
        if (cudaFuncSetAttribute(wave25_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(WaveSmem)) != cudaSuccess)
            return 0;
        return resident((const void *)wave25_kernel<1>, kTX * kWaveTY, sizeof(WaveSmem));
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kWaveTY - 1) / kWaveTY;
    const int64_t chunk = choose_chunk(gx * gy, nz, 16, 9, res);
    const int64_t gz = (nz + chunk - 1) / chunk;
    if (gx * gy > 0x7fffffffll || nz > (1ll << 30))
        return cudaErrorInvalidValue;
    wave25_kernel<1><<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kWaveTY), sizeof(WaveSmem), st>>>(
        p, mu, nullptr, nullptr, (int)nz, 0, Grid3{nx, ny, nz, nx * ny}, 0, nz, chunk, -1, -1, -1, 0.0f, g,
        WaveSrcTable{});
    return cudaGetLastError();
}

cudaError_t launch_wave25_grad32(const float *p, const float *mu, float *gacc, int64_t nx, int64_t ny, int64_t nz,
                                 cudaStream_t st)
{
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = []() -> int {
        if (cudaFuncSetAttribute(wave25_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(WaveSmem)) != cudaSuccess)
            return 0;
        return resident((const void *)wave25_kernel<2>, kTX * kWaveTY, sizeof(WaveSmem));
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kWaveTY - 1) / kWaveTY;
    const int64_t chunk = choose_chunk(gx * gy, nz, 16, 9, res);
    const int64_t gz = (nz + chunk - 1) / chunk;
    if (gx * gy > 0x7fffffffll || nz > (1ll << 30))
        return cudaErrorInvalidValue;
    wave25_kernel<2><<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kWaveTY), sizeof(WaveSmem), st>>>(
        p, mu, nullptr, nullptr, (int)nz, 0, Grid3{nx, ny, nz, nx * ny}, 0, nz, chunk, -1, -1, -1, 0.0f, nullptr,
        WaveSrcTable{}, gacc);
    return cudaGetLastError();
}

cudaError_t launch_wave25(ConstRing p, Ring pprev_out, ConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                          int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w, cudaStream_t st,
                          WaveSrcTable tab)
{
    return launch_wave25_to(p, ConstRing{pprev_out.base, pprev_out.nslot, pprev_out.zbase}, pprev_out, kappa, nx, ny,
                            nz, z0, z1, sx, sy, sz, w, st, tab);
}

#endif

cudaError_t launch_add_time(int64_t *t, int64_t n, cudaStream_t st)
{
    add_time_kernel<<<1, 1, 0, st>>>(t, n);
    return cudaGetLastError();
}

cudaError_t launch_swap(float *a, float *b, int64_t n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    swap_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace ooc
