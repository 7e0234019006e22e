// wave_tma.cu -- the 25-point acoustic wave step (Section VI, Table I:
// 8th-order Laplacian, HALO = 4, leapfrog in time) with its input planes
// staged in shared memory by TMA tensor copies, and its gradient modes for
// the adjoint run.  Built with OOC_WAVE_TMA = 1; the default build runs the
// cp.async-staged kernel of stencil.cu, which measured faster (0.369 against
// 0.393 ms per 512^3 step).
//
//   p' = 2p - p_prev + kappa * sum_axes[c0 p + sum_m c_m (p[+m] + p[-m])]
//
// A CTA owns a 128 x 8 tile (a warp per row, 4 points per thread) and
// marches a chunk of z.  For each plane one thread issues three TMA copies,
// each completing one mbarrier: the p tile with its 4-wide x and y halos
// (136 x 16 floats, zero outside the grid) into a ring of 7 stages, and the
// p_prev and kappa tiles (128 x 8) of the plane 4 below into a ring of 3.
// The copies run 6 planes ahead of the plane they serve as the centre.  The
// z-neighbours come from a 9-plane register queue of the thread's own
// points, filled from the staged tiles; the x-neighbours (the 4-point
// groups on each side) and y-neighbours are read from the centre plane's
// tile.  One CTA barrier per plane frees the stages the next copies land
// in.  p' overwrites p_prev in place (or goes to a separate array): each
// point's p_prev is read only by the CTA that writes p' there, and its copy
// has landed before that write.
//
// MODE 0: the leapfrog step.  MODE 1 (gradient of the adjoint run):
// gsum[own] += (double) pprev * (double) L(pin) in FP64, with `pprev` the
// adjoint field and kappa, pout and the source unused.  MODE 2: the same
// term in FP32, gacc[own] = fma(pprev, L(pin), gacc[own]).
//
// Every mbarrier wait is bounded; a CTA that gives up agrees to stop
// through its plane barrier, waits (bounded again) for its own copies, sets
// g_wave_fault and returns.
#include "tma.cuh"

namespace ooc {

using namespace sten;

// Set by a wave CTA whose bounded wait gave up; read and cleared by
// take_wave_fault().
__device__ unsigned g_wave_fault = 0u;

#if OOC_WAVE_TMA
namespace {

constexpr int kWTY = 8;                 // rows per CTA (one per warp)
constexpr int kWR = 4;                  // stencil radius
constexpr int kWPD = 2;                 // planes of copies in flight beyond the queue
constexpr int kWPS = 2 * kWR - 3 + kWPD;  // p-tile stages: planes z .. z + 4 + kWPD
constexpr int kWKS = kWPD + 1;          // p_prev / kappa stages
constexpr int kWCols = 4 * kTX + 2 * kWR;      // staged p columns (136)
constexpr int kWRows = kWTY + 2 * kWR;         // staged p rows (16)
constexpr int kWPFloats = kWCols * kWRows;     // 2176 floats = 8704 bytes (a multiple of 128)
constexpr int kWKFloats = 4 * kTX * kWTY;      // 1024 floats per p_prev or kappa tile
constexpr unsigned kWPBytes = kWPFloats * 4;
constexpr int kWaveTmaBlocksPerSM = 2;

size_t wave_tma_smem_bytes() { return (size_t)kWPS * kWPFloats * 4 + (size_t)kWKS * 2 * kWKFloats * 4 + (kWPS + kWKS) * 8; }

__device__ __forceinline__ float pickx(const float (&l)[4], const float (&c)[4], const float (&rr)[4], int idx)
{
    return idx < 0 ? l[idx + 4] : (idx < 4 ? c[idx] : rr[idx - 4]);
}

template <int MODE>
__global__ void __launch_bounds__(kTX *kWTY, kWaveTmaBlocksPerSM)
    wave25t_kernel(const __grid_constant__ CUtensorMap tp, const __grid_constant__ CUtensorMap tpp,
                   const __grid_constant__ CUtensorMap tk, const float *__restrict__ pin, float *pout, int nslot,
                   int64_t zbase, Grid3 g, int64_t z0,
                   int64_t z1, int64_t zchunk, int64_t sx, int64_t sy, int64_t sz, float w, double *__restrict__ gsum,
                   float *__restrict__ gacc, WaveSrcTable tab)
{
    constexpr int R = kWR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ps = reinterpret_cast<float *>(smem_raw);                          // kWPS p tiles
    float *ks = ps + kWPS * kWPFloats;                                        // kWKS (p_prev, kappa) pairs
    uint64_t *barP = reinterpret_cast<uint64_t *>(ks + kWKS * 2 * kWKFloats);  // one per p stage
    uint64_t *barK = barP + kWPS;                                             // one per p_prev/kappa stage
    const int lane = threadIdx.x, ty = threadIdx.y;
    const bool leader = lane == 0 && ty == 0;
    const int64_t gx = (g.nx + kSeg - 1) / kSeg;  // x tiles; blockIdx.x = by * gx + bx
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kWTY;
    const int64_t y = y0 + ty;
    const int64_t za = z0 + (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, z1) - za);
    const int nz = (int)g.nz;
    const int64_t plane = g.plane;
    const bool inside = x4 < g.nx && y < g.ny;
    const int64_t off = inside ? y * g.nx + x4 : 0;
    const bool src_here = inside && y == sy && sx >= x4 && sx < x4 + 4;
    const float4 z4 = zero4();
    const int tx = (int)(xs - R), tyc = (int)(y0 - R), kx = (int)xs, ky = (int)y0;

    // Copy group gi (plane za + gi): the p tile into p stage gi mod kWPS, and,
    // from gi = R on, p_prev and kappa of plane za + gi - R into stage
    // (gi - R) mod kWKS.  Planes past the grid copy nothing; their barrier
    // phase completes at once.  Ring slots advance by one plane per group.
    int gslot = (int)ring_slot(za, zbase, nslot), kslot = gslot;
    auto issue = [&](int gi) {
        const int gz = (int)za + gi;
        const int sp = gi % kWPS;
        if (gz < nz) {
            mbar_arrive_tx(&barP[sp], kWPBytes);
            tma_load_3d(ps + sp * kWPFloats, &tp, tx, tyc, gslot, &barP[sp]);
        } else {
            mbar_arrive(&barP[sp]);
        }
        gslot = wrap_add(gslot, 1, nslot);
        if (gi >= R) {
            const int sk = (gi - R) % kWKS;
            const unsigned bytes = MODE == 0 ? 2u * kWKFloats * 4 : (unsigned)kWKFloats * 4;
            if (gz - R < nz) {
                mbar_arrive_tx(&barK[sk], bytes);
                tma_load_3d(ks + sk * 2 * kWKFloats, &tpp, kx, ky, kslot, &barK[sk]);
                if (MODE == 0)
                    tma_load_3d(ks + sk * 2 * kWKFloats + kWKFloats, &tk, kx, ky, kslot, &barK[sk]);
            } else {
                mbar_arrive(&barK[sk]);
            }
            kslot = wrap_add(kslot, 1, nslot);
        }
    };
    if (leader) {
        for (int j = 0; j < kWPS; ++j)
            mbar_init(&barP[j], 1);
        for (int j = 0; j < kWKS; ++j)
            mbar_init(&barK[j], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    const int ngroups = cnt + R;  // planes za .. za + cnt - 1 + R
    if (leader)
        for (int gi = 0; gi < R + kWPD && gi < ngroups; ++gi)
            issue(gi);
    int issued = R + kWPD < ngroups ? R + kWPD : ngroups;

    // q[j] = p at plane z - 4 + j of this thread's 4 points; planes za - 4 ..
    // za + 3 are read directly, later ones come from the staged tiles
    int s = (int)ring_slot(za, zbase, nslot);  // slot of plane z
    float4 q[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
        const int64_t zj = za - R + j;
        const float *pj = pin + (int64_t)wrap_add(s, nslot - R + j >= nslot ? j - R : nslot - R + j, nslot) * plane;
        q[j] = (inside && zj >= 0 && zj < nz) ? ldg4(pj + off) : z4;
    }
    q[2 * R] = z4;
    unsigned fail = 0;
    int64_t z = za;
    for (int i = 0; i < cnt; ++i, ++z) {
        // the p tiles of planes z (group i) and z + 4 (group i + R), and
        // p_prev / kappa of plane z (group i + R); group i was already
        // waited for as plane z + 4 four planes ago, except in the first four
        if (!mbar_wait(&barP[i % kWPS], (unsigned)((i / kWPS) & 1)))
            fail = 1u;
        if (!mbar_wait(&barP[(i + R) % kWPS], (unsigned)(((i + R) / kWPS) & 1)))
            fail = 1u;
        if (!mbar_wait(&barK[i % kWKS], (unsigned)((i / kWKS) & 1)))
            fail = 1u;
        // every thread is done with the stages of plane z - 1; they take the
        // next copies
        if (__syncthreads_or((int)fail)) {
            if (leader) {
                for (int j = issued > kWPS ? issued - kWPS : 0; j < issued; ++j)
                    mbar_wait(&barP[j % kWPS], (unsigned)((j / kWPS) & 1));
                for (int j = issued - R > kWKS ? issued - R - kWKS : 0; j < issued - R; ++j)
                    mbar_wait(&barK[j % kWKS], (unsigned)((j / kWKS) & 1));
                atomicOr(&g_wave_fault, 1u);
            }
            return;
        }
        if (issued < ngroups) {
            if (leader)
                issue(issued);
            ++issued;
        }
        const float *tc = ps + (i % kWPS) * kWPFloats;   // p tile of plane z
        const float *t4 = ps + ((i + R) % kWPS) * kWPFloats;  // p tile of plane z + 4
        q[2 * R] = z + R < nz ? reinterpret_cast<const float4 *>(t4 + (ty + R) * kWCols)[lane + 1] : z4;
        const float4 c = q[R];
        const float4 lf = reinterpret_cast<const float4 *>(tc + (ty + R) * kWCols)[lane];
        const float4 rt = reinterpret_cast<const float4 *>(tc + (ty + R) * kWCols)[lane + 2];
        const float *kt = ks + (i % kWKS) * 2 * kWKFloats;
        const float4 ppv = reinterpret_cast<const float4 *>(kt)[ty * kTX + lane];
        const float4 kv = MODE == 0 ? reinterpret_cast<const float4 *>(kt + kWKFloats)[ty * kTX + lane] : z4;
        const float L[4] = {lf.x, lf.y, lf.z, lf.w};
        const float C[4] = {c.x, c.y, c.z, c.w};
        const float Rt[4] = {rt.x, rt.y, rt.z, rt.w};
        const float PP[4] = {ppv.x, ppv.y, ppv.z, ppv.w};
        const float KV[4] = {kv.x, kv.y, kv.z, kv.w};
        const float cf[R] = {kC1, kC2, kC3, kC4};
        float lap[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            lap[j] = (3.0f * kC0) * C[j];
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const float4 ym = reinterpret_cast<const float4 *>(tc + (ty + R - m) * kWCols)[lane + 1];
            const float4 yp = reinterpret_cast<const float4 *>(tc + (ty + R + m) * kWCols)[lane + 1];
            const float YM[4] = {ym.x, ym.y, ym.z, ym.w};
            const float YP[4] = {yp.x, yp.y, yp.z, yp.w};
            const float ZM[4] = {q[R - m].x, q[R - m].y, q[R - m].z, q[R - m].w};
            const float ZP[4] = {q[R + m].x, q[R + m].y, q[R + m].z, q[R + m].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float xsum = pickx(L, C, Rt, j - m) + pickx(L, C, Rt, j + m);
                lap[j] += cf[m - 1] * ((xsum + (YM[j] + YP[j])) + (ZM[j] + ZP[j]));
            }
        }
        if (MODE == 0) {
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = 2.0f * C[j] - PP[j] + KV[j] * lap[j];
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
                *reinterpret_cast<float4 *>(pout + (int64_t)s * plane + off) = make_float4(o[0], o[1], o[2], o[3]);
        } else if (MODE == 2 && inside) {
            float4 *ap = reinterpret_cast<float4 *>(gacc + (int64_t)s * plane + off);
            float4 a = *ap;
            a.x = __fmaf_rn(PP[0], lap[0], a.x);
            a.y = __fmaf_rn(PP[1], lap[1], a.y);
            a.z = __fmaf_rn(PP[2], lap[2], a.z);
            a.w = __fmaf_rn(PP[3], lap[3], a.w);
            *ap = a;
        } else if (MODE == 1 && inside) {
            double2 *gp = reinterpret_cast<double2 *>(gsum + (int64_t)s * plane + off);
            double2 g0 = gp[0], g1 = gp[1];
            g0.x += (double)PP[0] * (double)lap[0];
            g0.y += (double)PP[1] * (double)lap[1];
            g1.x += (double)PP[2] * (double)lap[2];
            g1.y += (double)PP[3] * (double)lap[3];
            gp[0] = g0;
            gp[1] = g1;
        }
#pragma unroll
        for (int j = 0; j < 2 * R; ++j)
            q[j] = q[j + 1];
        s = wrap_add(s, 1, nslot);
    }
}

cudaError_t wave_maps(const float *p, const float *pp, const float *k, int64_t nx, int64_t ny, int64_t nslot,
                      CUtensorMap *mp, CUtensorMap *mpp, CUtensorMap *mk)
{
    if (nx % 4 || ((uintptr_t)p % 16) || ((uintptr_t)pp % 16) || (k && ((uintptr_t)k % 16)) || nx > 0x7fffffffll ||
        ny > 0x7fffffffll)
        return cudaErrorInvalidValue;
    cudaError_t e = ring_tensor_map(p, nx, ny, nslot, kWCols, kWRows, mp);
    if (e == cudaSuccess)
        e = ring_tensor_map(pp, nx, ny, nslot, 4 * kTX, kWTY, mpp);
    if (e == cudaSuccess)
        e = k ? ring_tensor_map(k, nx, ny, nslot, 4 * kTX, kWTY, mk) : ring_tensor_map(pp, nx, ny, nslot, 4 * kTX, kWTY, mk);
    return e;
}

template <int MODE>
cudaError_t launch_wave25t(const float *p, const float *pprev, float *pout, const float *kappa, int64_t nslot,
                           int64_t zbase, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1, int64_t sx,
                           int64_t sy, int64_t sz, float w, double *gsum, float *gacc, WaveSrcTable tab,
                           cudaStream_t st)
{
    if (z1 <= z0)
        return cudaSuccess;
    const size_t smem = wave_tma_smem_bytes();
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = [smem]() -> int {
        if (cudaFuncSetAttribute(wave25t_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem) != cudaSuccess)
            return 0;
        return resident((const void *)wave25t_kernel<MODE>, kTX * kWTY, smem);
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kWTY - 1) / kWTY;
    const int64_t chunk = choose_chunk(gx * gy, z1 - z0, 16, 9, res);
    const int64_t gz = (z1 - z0 + chunk - 1) / chunk;
    if (nslot > (1ll << 30) || nz > (1ll << 30) || gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    CUtensorMap mp, mpp, mk;
    cudaError_t e = wave_maps(p, pprev, MODE == 0 ? kappa : nullptr, nx, ny, nslot, &mp, &mpp, &mk);
    if (e != cudaSuccess)
        return e;
    wave25t_kernel<MODE><<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kWTY), smem, st>>>(
        mp, mpp, mk, p, pout, (int)nslot, zbase, Grid3{nx, ny, nz, nx * ny}, z0, z1, chunk, sx, sy, sz, w, gsum, gacc,
        tab);
    return cudaGetLastError();
}

}  // namespace
#endif

cudaError_t take_wave_fault(unsigned *fault)
{
    unsigned v = 0u;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_wave_fault, sizeof(v));
    if (e == cudaSuccess && v != 0u) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_wave_fault, &zero, sizeof(zero));
    }
    *fault = v;
    return e;
}

#if OOC_WAVE_TMA
// the wave launchers (the default build has them in stencil.cu)
cudaError_t launch_wave25_to(ConstRing p, ConstRing pprev, Ring pnew, ConstRing kappa, int64_t nx, int64_t ny,
                             int64_t nz, int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w,
                             cudaStream_t st, WaveSrcTable tab)
{
    if (p.nslot != pnew.nslot || p.zbase != pnew.zbase || p.nslot != kappa.nslot || p.zbase != kappa.zbase ||
        p.nslot != pprev.nslot || p.zbase != pprev.zbase)
        return cudaErrorInvalidValue;
    return launch_wave25t<0>(p.base, pprev.base, pnew.base, kappa.base, p.nslot, p.zbase, nx, ny, nz, z0, z1, sx, sy,
                             sz, w, nullptr, nullptr, tab, st);
}

cudaError_t launch_wave25(ConstRing p, Ring pprev_out, ConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                          int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w, cudaStream_t st,
                          WaveSrcTable tab)
{
    return launch_wave25_to(p, ConstRing{pprev_out.base, pprev_out.nslot, pprev_out.zbase}, pprev_out, kappa, nx, ny,
                            nz, z0, z1, sx, sy, sz, w, st, tab);
}

cudaError_t launch_wave25_grad(const float *p, const float *mu, double *g, int64_t nx, int64_t ny, int64_t nz,
                               cudaStream_t st)
{
    return launch_wave25t<1>(p, mu, nullptr, nullptr, nz, 0, nx, ny, nz, 0, nz, -1, -1, -1, 0.0f, g, nullptr,
                             WaveSrcTable{}, st);
}

cudaError_t launch_wave25_grad32(const float *p, const float *mu, float *gacc, int64_t nx, int64_t ny, int64_t nz,
                                 cudaStream_t st)
{
    return launch_wave25t<2>(p, mu, nullptr, nullptr, nz, 0, nx, ny, nz, 0, nz, -1, -1, -1, 0.0f, nullptr, gacc,
                             WaveSrcTable{}, st);
}
#endif

}  // namespace ooc
