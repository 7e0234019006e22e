// stencil64.cu -- FP64 heat7 and wave25 window kernels on sm_103a.
//
// The paper ran its fields in double precision (Section VI).  These kernels
// update the planes [z0, z1) of FP64 ring windows (plane z in slot
// (z + zbase) mod nslot; a dense field is the ring with nslot = nz, zbase =
// 0) with zero ghosts outside the grid, one step per launch.  GB300's FP64
// pipe, not HBM, bounds them (about 7 FP64 operations per heat7 point and
// 27 per wave25 point), so the design is simple: a warp owns a 64-point row
// segment, two points per thread (16-byte double2 accesses); x-neighbours
// come from warp shuffles (heat7) or a shared-memory copy of the row
// (wave25), y-neighbours from a shared-memory copy of the plane (double
// buffered, one barrier per plane) and z-neighbours from a register queue,
// each load issued one plane ahead of its use.  The arithmetic is written
// with rounding intrinsics in a fixed order:
//   heat7:  u' = u + r (((x- + x+) + (y- + y+)) + (z- + z+) - 6u)
//   wave25: L = 3 c0 p + sum_m c_m (((x-m + x+m) + (y-m + y+m)) + (z-m + z+m)),
//           p' = kappa L + (2p - p_prev)  (+ the source amplitude)
#include "stencil_common.cuh"

namespace ooc {

using namespace sten;

namespace {

constexpr int kTY64 = 2;  // heat7 rows per CTA
constexpr int kSeg64 = 2 * kTX;
constexpr int kWTY64 = 8;  // wave25 rows per CTA
constexpr int kWR = 4;
constexpr double kD0 = -205.0 / 72.0, kD1 = 8.0 / 5.0, kD2 = -1.0 / 5.0, kD3 = 8.0 / 315.0, kD4 = -1.0 / 560.0;

__device__ __forceinline__ double heat_pt64(double c, double xl, double xr, double up, double dn, double zm,
                                            double zp, double r)
{
    const double t = __dadd_rn(__dadd_rn(__dadd_rn(xl, xr), __dadd_rn(up, dn)), __dadd_rn(zm, zp));
    return __fma_rn(r, __fma_rn(-6.0, c, t), c);
}

__device__ __forceinline__ double2 ldg2(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }

// Plane z of a ring (its slot pointer), or nullptr outside [0, nz).
__device__ __forceinline__ const double *plane_at(const double *base, int64_t z, int64_t nz, int64_t zbase, int nslot,
                                                  int64_t plane)
{
    return (z >= 0 && z < nz) ? base + ring_slot(z, zbase, nslot) * plane : nullptr;
}

__global__ void __launch_bounds__(kTX *kTY64)
    heat7_f64_kernel(const double *__restrict__ in, double *__restrict__ out, int nslot, int64_t zbase, Grid3 g,
                     int64_t z0, int64_t z1, int64_t zchunk, double r)
{
    __shared__ double2 tile[2][kTY64 + 2][kTX];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t gx = (g.nx + kSeg64 - 1) / kSeg64;
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg64;
    const int64_t x2 = xs + 2 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kTY64;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int64_t nz = g.nz, plane = g.plane;
    const bool inside = x2 < g.nx && y < g.ny;
    const int64_t off = inside ? y * g.nx + x2 : 0;
    const int64_t yh = ty == 0 ? y0 - 1 : y0 + kTY64;
    const bool hrow = (ty == 0 || ty == kTY64 - 1) && yh >= 0 && yh < g.ny && x2 < g.nx;
    const int64_t hoff = hrow ? yh * g.nx + x2 : 0;
    const int64_t xh = lane == 0 ? xs - 1 : xs + kSeg64;
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx && y < g.ny;
    const int64_t xoff = hcol ? y * g.nx + xh : 0;
    const double2 z2 = make_double2(0.0, 0.0);
    const double *pm1 = plane_at(in, za - 1, nz, zbase, nslot, plane);
    const double *p0 = plane_at(in, za, nz, zbase, nslot, plane);
    const double *p1 = plane_at(in, za + 1, nz, zbase, nslot, plane);
    double2 prev = (inside && pm1) ? ldg2(pm1 + off) : z2;
    double2 cur = (inside && p0) ? ldg2(p0 + off) : z2;
    double2 nxt = (inside && p1) ? ldg2(p1 + off) : z2;
    double2 hyv = (hrow && p0) ? ldg2(p0 + hoff) : z2;
    double hx = (hcol && p0) ? __ldg(p0 + xoff) : 0.0;
    for (int i = 0; i < cnt; ++i) {
        const int64_t z = za + i;
        const double *q1 = plane_at(in, z + 1, nz, zbase, nslot, plane);
        const double *q2 = plane_at(in, z + 2, nz, zbase, nslot, plane);
        const double2 pfv = (inside && q2) ? ldg2(q2 + off) : z2;
        const double2 hyv1 = (hrow && q1) ? ldg2(q1 + hoff) : z2;
        const double hx1 = (hcol && q1) ? __ldg(q1 + xoff) : 0.0;
        const int b = i & 1;
        tile[b][ty + 1][lane] = cur;
        if (ty == 0)
            tile[b][0][lane] = hyv;
        if (ty == kTY64 - 1)
            tile[b][kTY64 + 1][lane] = hyv;
        double xl = __shfl_up_sync(0xffffffffu, cur.y, 1);
        double xr = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (lane == 0)
            xl = hx;
        if (lane == kTX - 1)
            xr = hx;
        __syncthreads();
        const double2 up = tile[b][ty][lane];
        const double2 dn = tile[b][ty + 2][lane];
        double2 o;
        o.x = heat_pt64(cur.x, xl, cur.y, up.x, dn.x, prev.x, nxt.x, r);
        o.y = heat_pt64(cur.y, cur.x, xr, up.y, dn.y, prev.y, nxt.y, r);
        if (inside)
            *reinterpret_cast<double2 *>(out + ring_slot(z, zbase, nslot) * plane + off) = o;
        prev = cur;
        cur = nxt;
        nxt = pfv;
        hyv = hyv1;
        hx = hx1;
    }
}

// One wave25 point: its x-neighbours xm/xp[m-1] at +-m, y and z likewise.
__device__ __forceinline__ double wave_lap64(double c, const double (&xm)[kWR], const double (&xp)[kWR],
                                             const double (&ym)[kWR], const double (&yp)[kWR], const double (&zm)[kWR],
                                             const double (&zp)[kWR])
{
    const double cf[kWR] = {kD1, kD2, kD3, kD4};
    double lap = __dmul_rn(3.0 * kD0, c);
#pragma unroll
    for (int m = 0; m < kWR; ++m) {
        const double s = __dadd_rn(__dadd_rn(__dadd_rn(xm[m], xp[m]), __dadd_rn(ym[m], yp[m])),
                                   __dadd_rn(zm[m], zp[m]));
        lap = __fma_rn(cf[m], s, lap);
    }
    return lap;
}

// Leapfrog on FP64 rings: p' = kappa L(p) + (2p - p_prev) written over
// p_prev in place (each point's p_prev is read only by its own thread).
// Row tile of a plane in shared memory: 4 + 8 + 4 rows of 2 + 32 + 2
// double2 (the 4 x-neighbours beyond each row end in the outer columns).
__global__ void __launch_bounds__(kTX *kWTY64)
    wave25_f64_kernel(const double *__restrict__ pin, double *pout, const double *__restrict__ kap, int nslot,
                      int64_t zbase, Grid3 g, int64_t z0, int64_t z1, int64_t zchunk, int64_t sx, int64_t sy,
                      int64_t sz, double w, WaveSrcTable tab)
{
    __shared__ double2 tile[2][kWTY64 + 2 * kWR][kTX + 4];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t gx = (g.nx + kSeg64 - 1) / kSeg64;
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg64;
    const int64_t x2 = xs + 2 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kWTY64;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int64_t nz = g.nz, plane = g.plane;
    const bool inside = x2 < g.nx && y < g.ny;
    const int64_t off = inside ? y * g.nx + x2 : 0;
    // this thread's halo row (rows y0-4 .. y0-1 and y0+8 .. y0+11)
    const int64_t yh = ty < kWR ? y0 - kWR + ty : y0 + kWTY64 + (ty - kWR);
    const int hrow_t = ty < kWR ? ty : ty + kWTY64;
    const bool hrow = x2 < g.nx && yh >= 0 && yh < g.ny;
    const int64_t hoff = hrow ? yh * g.nx + x2 : 0;
    // lanes 0, 1 and 30, 31 also load the two double2 beyond their row's ends
    const bool xl_lane = lane < 2, xr_lane = lane >= kTX - 2;
    const int64_t xe = xl_lane ? xs - 4 + 2 * lane : xs + kSeg64 + 2 * (lane - (kTX - 2));
    const bool xhalo = (xl_lane || xr_lane) && xe >= 0 && xe < g.nx && y < g.ny;
    const int64_t xoff = xhalo ? y * g.nx + xe : 0;
    const int xcol = xl_lane ? lane : lane + 4;
    const bool src_here = inside && y == sy && (sx == x2 || sx == x2 + 1);
    const double2 z2 = make_double2(0.0, 0.0);

    // q[j] = p at plane z - 4 + j of this thread's two points
    double2 q[2 * kWR + 1];
#pragma unroll
    for (int j = 0; j <= 2 * kWR; ++j) {
        const double *pj = plane_at(pin, za - kWR + j, nz, zbase, nslot, plane);
        q[j] = (inside && pj) ? ldg2(pj + off) : z2;
    }
    const double *c0 = plane_at(pin, za, nz, zbase, nslot, plane);
    double2 hv = (hrow && c0) ? ldg2(c0 + hoff) : z2;
    double2 xv = (xhalo && c0) ? ldg2(c0 + xoff) : z2;
    const double *k0 = plane_at(kap, za, nz, zbase, nslot, plane);
    const double *pp0 = plane_at(pout, za, nz, zbase, nslot, plane);
    double2 kv = (inside && k0) ? ldg2(k0 + off) : z2;
    // p_prev is overwritten by this kernel: plain loads, not the read-only path
    double2 ppv = (inside && pp0) ? *reinterpret_cast<const double2 *>(pp0 + off) : z2;
    for (int i = 0; i < cnt; ++i) {
        const int64_t z = za + i;
        // next plane's loads, issued before this plane's work
        const double *n5 = plane_at(pin, z + kWR + 1, nz, zbase, nslot, plane);
        const double *n1 = plane_at(pin, z + 1, nz, zbase, nslot, plane);
        const bool more = i + 1 < cnt;
        const double2 q_next = (inside && n5 && more) ? ldg2(n5 + off) : z2;
        const double2 hv_next = (hrow && n1 && more) ? ldg2(n1 + hoff) : z2;
        const double2 xv_next = (xhalo && n1 && more) ? ldg2(n1 + xoff) : z2;
        const double *k1 = plane_at(kap, z + 1, nz, zbase, nslot, plane);
        const double *pp1 = plane_at(pout, z + 1, nz, zbase, nslot, plane);
        const double2 kv_next = (inside && k1 && more) ? ldg2(k1 + off) : z2;
        const double2 ppv_next = (inside && pp1 && more) ? *reinterpret_cast<const double2 *>(pp1 + off) : z2;

        const int b = i & 1;
        const double2 c = q[kWR];
        tile[b][ty + kWR][lane + 2] = c;
        tile[b][hrow_t][lane + 2] = hv;
        if (xl_lane || xr_lane)
            tile[b][ty + kWR][xcol] = xv;
        __syncthreads();
        // x-neighbours: the row's double2 e-2 .. e+2 around this thread's e
        const int e = lane + 2;
        const double2 a2 = tile[b][ty + kWR][e - 2], a1 = tile[b][ty + kWR][e - 1];
        const double2 b1 = tile[b][ty + kWR][e + 1], b2 = tile[b][ty + kWR][e + 2];
        double ymx[kWR], ypx[kWR], ymy[kWR], ypy[kWR], zmx[kWR], zpx[kWR], zmy[kWR], zpy[kWR];
#pragma unroll
        for (int m = 1; m <= kWR; ++m) {
            const double2 um = tile[b][ty + kWR - m][e], up = tile[b][ty + kWR + m][e];
            ymx[m - 1] = um.x;
            ypx[m - 1] = up.x;
            ymy[m - 1] = um.y;
            ypy[m - 1] = up.y;
            zmx[m - 1] = q[kWR - m].x;
            zpx[m - 1] = q[kWR + m].x;
            zmy[m - 1] = q[kWR - m].y;
            zpy[m - 1] = q[kWR + m].y;
        }
        // point x2 (c.x): x-1 = a1.y, x+1 = c.y, x-+2 = a1.x / b1.x, x-+3 = a2.y / b1.y, x-+4 = a2.x / b2.x
        const double xmx[kWR] = {a1.y, a1.x, a2.y, a2.x}, xpx[kWR] = {c.y, b1.x, b1.y, b2.x};
        // point x2 + 1 (c.y): x-1 = c.x, x+1 = b1.x, x-+2 = a1.y / b1.y, x-+3 = a1.x / b2.x, x-+4 = a2.y / b2.y
        const double xmy[kWR] = {c.x, a1.y, a1.x, a2.y}, xpy[kWR] = {b1.x, b1.y, b2.x, b2.y};
        const double lx = wave_lap64(c.x, xmx, xpx, ymx, ypx, zmx, zpx);
        const double ly = wave_lap64(c.y, xmy, xpy, ymy, ypy, zmy, zpy);
        double2 o;
        o.x = __fma_rn(kv.x, lx, __fma_rn(2.0, c.x, -ppv.x));
        o.y = __fma_rn(kv.y, ly, __fma_rn(2.0, c.y, -ppv.y));
        if (src_here && z == sz) {
            double ws = w;
            if (tab.w) {  // amplitude of step n = plan time + n_off, from the device table
                const int64_t n = *tab.t + tab.n_off;
                ws = n >= 0 && n < tab.nw ? (double)tab.w[n] : 0.0;
            }
            if (sx == x2)
                o.x = __dadd_rn(o.x, ws);
            else
                o.y = __dadd_rn(o.y, ws);
        }
        if (inside)
            *reinterpret_cast<double2 *>(pout + ring_slot(z, zbase, nslot) * plane + off) = o;
#pragma unroll
        for (int j = 0; j < 2 * kWR; ++j)
            q[j] = q[j + 1];
        q[2 * kWR] = q_next;
        hv = hv_next;
        xv = xv_next;
        kv = kv_next;
        ppv = ppv_next;
    }
}

}  // namespace

cudaError_t launch_heat7_f64_ring(DConstRing in, DRing out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                                  double r, cudaStream_t st)
{
    if (z1 <= z0)
        return cudaSuccess;
    static const int res = resident((const void *)heat7_f64_kernel, kTX * kTY64);  // once, thread-safe
    const int64_t gx = (nx + kSeg64 - 1) / kSeg64, gy = (ny + kTY64 - 1) / kTY64;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 8, 2, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    if (in.nslot != out.nslot || in.zbase != out.zbase || in.base == out.base || in.nslot > (1ll << 30) ||
        gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    heat7_f64_kernel<<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kTY64), 0, st>>>(
        in.base, out.base, (int)in.nslot, in.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, r);
    return cudaGetLastError();
}

cudaError_t launch_heat7_f64(const double *in, double *out, int64_t nx, int64_t ny, int64_t nz, double r,
                             cudaStream_t st)
{
    return launch_heat7_f64_ring(DConstRing{in, nz, 0}, DRing{out, nz, 0}, nx, ny, nz, 0, nz, r, st);
}

cudaError_t launch_wave25_f64(DConstRing p, DRing pprev_out, DConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                              int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, double w, cudaStream_t st,
                              WaveSrcTable tab)
{
    if (z1 <= z0)
        return cudaSuccess;
    static const int res = resident((const void *)wave25_f64_kernel, kTX * kWTY64);  // once, thread-safe
    const int64_t gx = (nx + kSeg64 - 1) / kSeg64, gy = (ny + kWTY64 - 1) / kWTY64;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 16, 9, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    if (p.nslot != pprev_out.nslot || p.zbase != pprev_out.zbase || p.nslot != kappa.nslot ||
        p.zbase != kappa.zbase || p.base == pprev_out.base || p.nslot > (1ll << 30) || gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    wave25_f64_kernel<<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kWTY64), 0, st>>>(
        p.base, pprev_out.base, kappa.base, (int)p.nslot, p.zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, sx, sy,
        sz, w, tab);
    return cudaGetLastError();
}

}  // namespace ooc
