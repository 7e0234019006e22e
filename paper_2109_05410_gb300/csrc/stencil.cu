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
//   - z-neighbours live in a register queue; the next input plane and every
//     halo value are prefetched one plane ahead so that a load is always in
//     flight while the current plane is computed.
// Each CTA marches a chunk of z; the chunk count is chosen from the
// occupancy so that the grid fills whole waves of the 152 SMs.
//
// heat7 (Section III's neighbour average, 3D):
//   u' = u + r (u[x-1] + u[x+1] + u[y-1] + u[y+1] + u[z-1] + u[z+1] - 6u)
// wave25 (Section VI's 25-point propagator, HALO = 4, Table I), leapfrog:
//   p' = 2p - p_prev + kappa * sum_axes[c0 p + sum_m c_m (p[+m] + p[-m])]
// p' overwrites p_prev in place: each point's p_prev is read only by the
// thread that writes p' there.
#include "common.cuh"

namespace ooc {
namespace {

constexpr int kTX = 32;  // threads per row segment (4 points each: 128 x)
constexpr int kHeatTY = 8;
constexpr int kWaveTY = 8;
constexpr int kSeg = 4 * kTX;

__device__ __forceinline__ int64_t next_slot(int64_t s, int64_t nslot) { return s + 1 == nslot ? 0 : s + 1; }

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

struct Grid3 {
    int64_t nx, ny, nz, plane;
};

// 128-bit load of the 4 points at (x4..x4+3, y, z) or zeros outside the grid.
__device__ __forceinline__ float4 ld4(const float *base, const Grid3 &g, int64_t z, int64_t slot, int64_t x4,
                                      int64_t y)
{
    if (z < 0 || z >= g.nz || y < 0 || y >= g.ny || x4 < 0 || x4 >= g.nx)
        return zero4();
    return __ldg(reinterpret_cast<const float4 *>(base + slot * g.plane + y * g.nx + x4));
}

__device__ __forceinline__ float ld1(const float *base, const Grid3 &g, int64_t z, int64_t slot, int64_t x, int64_t y)
{
    if (z < 0 || z >= g.nz || y < 0 || y >= g.ny || x < 0 || x >= g.nx)
        return 0.0f;
    return __ldg(base + slot * g.plane + y * g.nx + x);
}

__global__ void __launch_bounds__(kTX *kHeatTY)
    heat7_kernel(ConstRing in, Ring out, Grid3 g, int64_t z0, int64_t z1, int64_t zchunk, float r)
{
    __shared__ float4 tile[2][kHeatTY + 2][kTX];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t xs = (int64_t)blockIdx.x * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)blockIdx.y * kHeatTY;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.z * zchunk;
    const int64_t zb = min(za + zchunk, z1);
    const bool inside = x4 < g.nx && y < g.ny;
    // halo duties: edge warps load one y-halo row, edge lanes one x value
    const int64_t yh = ty == 0 ? y0 - 1 : (ty == kHeatTY - 1 ? y0 + kHeatTY : -1);
    const bool row_halo = ty == 0 || ty == kHeatTY - 1;
    const int64_t xh = lane == 0 ? xs - 1 : xs + kSeg;
    const bool col_halo = lane == 0 || lane == kTX - 1;

    int64_t s = ring_slot(za - 1, in.zbase, in.nslot);  // slot of plane za - 1
    float4 prev = ld4(in.base, g, za - 1, s, x4, y);
    s = next_slot(s, in.nslot);
    float4 cur = ld4(in.base, g, za, s, x4, y);
    float4 hyv = row_halo ? ld4(in.base, g, za, s, x4, yh) : zero4();
    float hx = col_halo ? ld1(in.base, g, za, s, xh, y) : 0.f;
    s = next_slot(s, in.nslot);
    float4 nxt = ld4(in.base, g, za + 1, s, x4, y);
    int64_t s_next = s;  // slot of plane z + 1
    int64_t s_out = ring_slot(za, out.zbase, out.nslot);
    for (int64_t z = za; z < zb; ++z) {
        // prefetch plane z + 2 and the halo of plane z + 1
        const int64_t s_pf = next_slot(s_next, in.nslot);
        const float4 pf = ld4(in.base, g, z + 2, s_pf, x4, y);
        const float4 hyv_n = row_halo ? ld4(in.base, g, z + 1, s_next, x4, yh) : zero4();
        const float hx_n = col_halo ? ld1(in.base, g, z + 1, s_next, xh, y) : 0.f;

        const int b = (int)((z - za) & 1);
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
        float4 o;
        o.x = cur.x + r * (((xl + cur.y) + (up.x + dn.x)) + (prev.x + nxt.x) - 6.0f * cur.x);
        o.y = cur.y + r * (((cur.x + cur.z) + (up.y + dn.y)) + (prev.y + nxt.y) - 6.0f * cur.y);
        o.z = cur.z + r * (((cur.y + cur.w) + (up.z + dn.z)) + (prev.z + nxt.z) - 6.0f * cur.z);
        o.w = cur.w + r * (((cur.z + xr) + (up.w + dn.w)) + (prev.w + nxt.w) - 6.0f * cur.w);
        if (inside)
            *reinterpret_cast<float4 *>(out.base + s_out * g.plane + y * g.nx + x4) = o;
        prev = cur;
        cur = nxt;
        nxt = pf;
        hyv = hyv_n;
        hx = hx_n;
        s_next = s_pf;
        s_out = next_slot(s_out, out.nslot);
    }
}

// x-neighbour m (1..4) to the left / right of point j (0..3) of the thread,
// given its own 4 points c and the 4-point groups to the left (l) and right (rr).
__device__ __forceinline__ float pick(const float (&l)[4], const float (&c)[4], const float (&rr)[4], int idx)
{
    // idx in [-4, 7]: -4..-1 -> l[idx+4], 0..3 -> c[idx], 4..7 -> rr[idx-4]
    return idx < 0 ? l[idx + 4] : (idx < 4 ? c[idx] : rr[idx - 4]);
}

__global__ void __launch_bounds__(kTX *kWaveTY)
    wave25_kernel(ConstRing pin, Ring pout, ConstRing kap, Grid3 g, int64_t z0, int64_t z1, int64_t zchunk,
                  int64_t sx, int64_t sy, int64_t sz, float w)
{
    constexpr int R = 4;
    __shared__ float4 tile[2][kWaveTY + 2 * R][kTX];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t xs = (int64_t)blockIdx.x * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)blockIdx.y * kWaveTY;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.z * zchunk;
    const int64_t zb = min(za + zchunk, z1);
    const bool inside = x4 < g.nx && y < g.ny;
    // warp ty loads y-halo row: 4 above (ty < 4) or 4 below (ty >= 4)
    const int hrow = ty < R ? ty : kWaveTY + ty;  // tile row it fills
    const int64_t yh = ty < R ? y0 - R + ty : y0 + kWaveTY + (ty - R);
    const int64_t xh = lane == 0 ? xs - 4 : xs + kSeg;  // x-halo group (lanes 0, 31)
    const bool col_halo = lane == 0 || lane == kTX - 1;

    // q[j] = p at plane z - 4 + j of this thread's 4 points
    float4 q[2 * R + 1];
    int64_t sq = ring_slot(za - R, pin.zbase, pin.nslot);
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) {
        q[j] = ld4(pin.base, g, za - R + j, sq, x4, y);
        if (j < 2 * R)
            sq = next_slot(sq, pin.nslot);
    }
    // sq: slot of plane za + 4
    int64_t s_c = ring_slot(za, pin.zbase, pin.nslot);
    int64_t s_o = ring_slot(za, pout.zbase, pout.nslot);
    int64_t s_k = ring_slot(za, kap.zbase, kap.nslot);
    float4 hyv = ld4(pin.base, g, za, s_c, x4, yh);
    float4 hxv = col_halo ? ld4(pin.base, g, za, s_c, xh, y) : zero4();
    float4 ppv = inside && za < zb ? *reinterpret_cast<const float4 *>(pout.base + s_o * g.plane + y * g.nx + x4)
                                   : zero4();
    float4 kv = inside && za < zb ? __ldg(reinterpret_cast<const float4 *>(kap.base + s_k * g.plane + y * g.nx + x4))
                                  : zero4();
    for (int64_t z = za; z < zb; ++z) {
        // prefetch for plane z + 1: its p at z + 5 (queue head), halos, p_prev, kappa
        const int64_t sq_n = next_slot(sq, pin.nslot);
        const int64_t s_c1 = next_slot(s_c, pin.nslot);
        const int64_t s_o1 = next_slot(s_o, pout.nslot);
        const int64_t s_k1 = next_slot(s_k, kap.nslot);
        const bool more = z + 1 < zb;
        const float4 pf = ld4(pin.base, g, z + R + 1, sq_n, x4, y);
        const float4 hyv_n = more ? ld4(pin.base, g, z + 1, s_c1, x4, yh) : zero4();
        const float4 hxv_n = (more && col_halo) ? ld4(pin.base, g, z + 1, s_c1, xh, y) : zero4();
        const float4 ppv_n = (more && inside)
                                 ? *reinterpret_cast<const float4 *>(pout.base + s_o1 * g.plane + y * g.nx + x4)
                                 : zero4();
        const float4 kv_n = (more && inside)
                                ? __ldg(reinterpret_cast<const float4 *>(kap.base + s_k1 * g.plane + y * g.nx + x4))
                                : zero4();

        const int b = (int)((z - za) & 1);
        const float4 c = q[R];
        tile[b][ty + R][lane] = c;
        tile[b][hrow][lane] = hyv;
        // x-neighbour groups from the adjacent lanes (edge lanes: the halo)
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
            lf = hxv;
        if (lane == kTX - 1)
            rt = hxv;
        __syncthreads();
        float4 ym[R], yp[R];
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            ym[m - 1] = tile[b][ty + R - m][lane];
            yp[m - 1] = tile[b][ty + R + m][lane];
        }
        const float L[4] = {lf.x, lf.y, lf.z, lf.w};
        const float C[4] = {c.x, c.y, c.z, c.w};
        const float Rt[4] = {rt.x, rt.y, rt.z, rt.w};
        const float cf[R] = {kC1, kC2, kC3, kC4};
        float o[4];
        const float PP[4] = {ppv.x, ppv.y, ppv.z, ppv.w};
        const float KV[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float lap = (3.0f * kC0) * C[j];
#pragma unroll
            for (int m = 1; m <= R; ++m) {
                const float xsum = pick(L, C, Rt, j - m) + pick(L, C, Rt, j + m);
                const float ysum = (&ym[m - 1].x)[j] + (&yp[m - 1].x)[j];
                const float zsum = (&q[R - m].x)[j] + (&q[R + m].x)[j];
                lap += cf[m - 1] * ((xsum + ysum) + zsum);
            }
            o[j] = 2.0f * C[j] - PP[j] + KV[j] * lap;
        }
        if (inside) {
            if (z == sz && y == sy) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sx == x4 + j)
                        o[j] += w;
            }
            *reinterpret_cast<float4 *>(pout.base + s_o * g.plane + y * g.nx + x4) = make_float4(o[0], o[1], o[2], o[3]);
        }
#pragma unroll
        for (int j = 0; j < 2 * R; ++j)
            q[j] = q[j + 1];
        q[2 * R] = pf;
        hyv = hyv_n;
        hxv = hxv_n;
        ppv = ppv_n;
        kv = kv_n;
        sq = sq_n;
        s_c = s_c1;
        s_o = s_o1;
        s_k = s_k1;
    }
}

// z-chunk so that the grid fills whole waves: pick the chunk count (1..8,
// chunks of at least min_chunk planes) minimising waves x (chunk + overhead).
int64_t choose_chunk(int64_t ntiles, int64_t height, int64_t min_chunk, int64_t overhead, int resident_ctas)
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

int resident(const void *fn, int threads)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 152;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm <= 0)
        per_sm = 1;
    return per_sm * sms;
}

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
    static int res = 0;
    if (res == 0)
        res = resident((const void *)heat7_kernel, kTX * kHeatTY);
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kHeatTY - 1) / kHeatTY;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 8, 3, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    heat7_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(kTX, kHeatTY), 0, st>>>(
        in, out, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, r);
    return cudaGetLastError();
}

cudaError_t launch_wave25(ConstRing p, Ring pprev_out, ConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                          int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w, cudaStream_t st)
{
    if (z1 <= z0)
        return cudaSuccess;
    static int res = 0;
    if (res == 0)
        res = resident((const void *)wave25_kernel, kTX * kWaveTY);
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kWaveTY - 1) / kWaveTY;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 16, 9, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    wave25_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(kTX, kWaveTY), 0, st>>>(
        p, pprev_out, kappa, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, sx, sy, sz, w);
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
