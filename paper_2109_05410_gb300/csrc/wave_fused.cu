// wave_fused.cu -- two wave25 leapfrog steps per launch (in-core, dense
// fields), the intermediate level kept on chip.
//
// Temporal blocking inside the kernel (Section III's idea applied within a
// launch, Section VII's "better orchestration"): from p^{n-1}, p^n and kappa
// the launch writes p^{n+1} and p^{n+2}, 20 B per point per two steps
// against 32 B for two single steps.  The 25-point stencil has a halo of 4
// (HALO = 4, Table I), so level n+1 is computed on the output tile plus 4
// on every side:
//   - a CTA of 16 warps computes level n+1 on 16 rows (one per warp) and
//     128 columns (4 per lane), and level n+2 on the middle 8 rows and the
//     middle 120 columns; tiles overlap by 8 rows and 8 columns;
//   - a CTA marches z over its chunk, level n+1 four planes ahead of level
//     n+2; level n+1 stays in a 9-plane shared-memory ring, which gives
//     level n+2 its x-, y- and z-neighbours;
//   - p^n arrives as staged tiles (24 rows: the 16 level-(n+1) rows and 4
//     above and below) by cp.async, 8 stages, with p^{n-1} and kappa of the
//     level-(n+1) rows in 3 stages; each thread keeps its own column's 9-
//     plane queue of p^n in registers (z-neighbours, and p^n as level n+2's
//     p_prev).
// Every point of both levels goes through the arithmetic of the single-step
// kernel in the same order, so the pair is bit-identical to two single
// steps.  The recomputed halo (16 level-(n+1) rows per 8 output rows, plus
// 4 planes at each end of a chunk) and the shared-memory neighbour reads of
// both levels cost more than the 12 B per point the pair saves: the single
// step already runs near the HBM bound, and on GB300 this pair runs at about
// 0.36 of its speed (it is kept as the measured answer, and for its bit
// identity, not as the fast path).
#include "cp_async.cuh"
#include "stencil_common.cuh"

namespace ooc {

using namespace sten;

namespace {

constexpr int kFR = 4;          // stencil radius
constexpr int kFW = 16;         // warps: level-(n+1) rows per CTA
constexpr int kFO = 8;          // level-(n+2) rows per CTA (warps 4 .. 11)
constexpr int kFT = kFW + 2 * kFR;  // staged p^n rows
constexpr int kFS = 8;          // p^n tile stages (planes z .. z + 7)
constexpr int kFK = 3;          // p^{n-1} / kappa stages
constexpr int kFQ = 2 * kFR + 1;  // z-queue and level ring depth
constexpr int kFSeg = kSeg - 2 * kFR;  // output columns per CTA (120)

struct FusedSmem {
    float4 p[kFS][kFT][kTX];
    float4 xh[kFS][kFW][2];
    float4 pp[kFK][kFW][kTX];
    float4 kk[kFK][kFW][kTX];
    float4 lv[kFQ][kFW][kTX];  // level n+1, planes z - 8 .. z
};

// One leapfrog update of 4 points in the single-step kernel's order:
//   L = 3 c0 p + sum_m c_m (((x-m + x+m) + (y-m + y+m)) + (z-m + z+m)),
//   p' = kappa L + (2p - p_prev).
__device__ __forceinline__ void wave_pt4(const float (&L)[4], const float (&C)[4], const float (&Rt)[4],
                                         const float4 (&ym)[kFR], const float4 (&yp)[kFR], const float4 (&zm)[kFR],
                                         const float4 (&zp)[kFR], const float (&PP)[4], const float (&KV)[4],
                                         float (&o)[4])
{
    const float cf[kFR] = {kC1, kC2, kC3, kC4};
    float lap[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        lap[j] = __fmul_rn(3.0f * kC0, C[j]);
#pragma unroll
    for (int m = 1; m <= kFR; ++m) {
        const float YM[4] = {ym[m - 1].x, ym[m - 1].y, ym[m - 1].z, ym[m - 1].w};
        const float YP[4] = {yp[m - 1].x, yp[m - 1].y, yp[m - 1].z, yp[m - 1].w};
        const float ZM[4] = {zm[m - 1].x, zm[m - 1].y, zm[m - 1].z, zm[m - 1].w};
        const float ZP[4] = {zp[m - 1].x, zp[m - 1].y, zp[m - 1].z, zp[m - 1].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float xsum = __fadd_rn(pick(L, C, Rt, j - m), pick(L, C, Rt, j + m));
            const float s = __fadd_rn(__fadd_rn(xsum, __fadd_rn(YM[j], YP[j])), __fadd_rn(ZM[j], ZP[j]));
            lap[j] = __fmaf_rn(cf[m - 1], s, lap[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        o[j] = __fmaf_rn(KV[j], lap[j], __fmaf_rn(2.0f, C[j], -PP[j]));
}

__device__ __forceinline__ void shuffles(const float4 c, float4 &lf, float4 &rt)
{
    lf.x = __shfl_up_sync(0xffffffffu, c.x, 1);
    lf.y = __shfl_up_sync(0xffffffffu, c.y, 1);
    lf.z = __shfl_up_sync(0xffffffffu, c.z, 1);
    lf.w = __shfl_up_sync(0xffffffffu, c.w, 1);
    rt.x = __shfl_down_sync(0xffffffffu, c.x, 1);
    rt.y = __shfl_down_sync(0xffffffffu, c.y, 1);
    rt.z = __shfl_down_sync(0xffffffffu, c.z, 1);
    rt.w = __shfl_down_sync(0xffffffffu, c.w, 1);
}

// Levels n+1 (into c_out) and n+2 (into d_out) of the output tile (columns
// [120 bx, 120 bx + 120), rows [8 by, 8 by + 8), planes [za, za + cnt)) from
// p^n (a), p^{n-1} (b) and kappa; w1 / w2 are the source amplitudes of the
// two steps.
__global__ void __launch_bounds__(kTX *kFW, 1)
    wave25x2_kernel(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ kap,
                    float *__restrict__ c_out, float *__restrict__ d_out, Grid3 g, int64_t zchunk, int64_t sx,
                    int64_t sy, int64_t sz, float w1, float w2)
{
    extern __shared__ __align__(16) unsigned char fused_smem[];
    FusedSmem &sm = *reinterpret_cast<FusedSmem *>(fused_smem);
    const int lane = threadIdx.x, wp = threadIdx.y;
    const int64_t gx = (g.nx + kFSeg - 1) / kFSeg;
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kFSeg - kFR;  // first level-(n+1) column
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kFO;          // first output row
    const int64_t y = y0 - kFR + wp;                                 // this warp's level-(n+1) row
    const int64_t za = (int64_t)blockIdx.y * zchunk;
    const int64_t nz = g.nz, plane = g.plane;
    const int64_t zend = min(za + zchunk, nz);
    const bool xin = x4 >= 0 && x4 < g.nx;
    const bool inside = xin && y >= 0 && y < g.ny;
    const int64_t off = inside ? y * g.nx + x4 : 0;
    // output points: the middle 8 rows (warps 4 .. 11) and 30 lanes
    const bool orow = wp >= kFR && wp < kFR + kFO;
    const bool own = inside && orow && lane >= 1 && lane <= kTX - 2;
    // staged rows: row r of the tile is y0 - 8 + r; warp wp copies row wp and,
    // for wp < 8, row wp + 16
    const int64_t ya = y0 - 2 * kFR + wp, yb = ya + kFW;
    const bool va = xin && ya >= 0 && ya < g.ny, vb = wp < 2 * kFR && xin && yb >= 0 && yb < g.ny;
    const int64_t offa = va ? ya * g.nx + x4 : 0, offb = vb ? yb * g.nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 4 : xs + kSeg;
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < g.nx && y >= 0 && y < g.ny;
    const int64_t xoff = hcol ? y * g.nx + xh : 0;
    const bool src1 = inside && y == sy && sx >= x4 && sx < x4 + 4;
    const float4 z4 = zero4();

    // level n+1 runs over planes zs in [za - 4, zend + 4) (clipped to the
    // grid: outside it the level is the zero ghost); level n+2 at zs - 4
    const int64_t z1lo = za - kFR, z1hi = zend + kFR;
    // copy group of p^n plane gz (stage (gz - z1lo) mod kFS) and of p^{n-1}
    // and kappa of plane gz - 5 (their stage (gz - 5 - z1lo) mod kFK)
    int st_issue = 0, kst_issue = 0;
    auto issue = [&](int64_t gz) {
        if (gz - kFR < z1hi) {  // the queue needs p^n up to z1hi + 3
            const bool vz = gz >= 0 && gz < nz;
            const float *pl = a + (vz ? gz : 0) * plane;
            cp_async16(&sm.p[st_issue][wp][lane], pl + offa, vz && va);
            if (wp < 2 * kFR)
                cp_async16(&sm.p[st_issue][wp + kFW][lane], pl + offb, vz && vb);
            if (lane == 0 || lane == kTX - 1)
                cp_async16(&sm.xh[st_issue][wp][lane == 0 ? 0 : 1], pl + xoff, vz && hcol);
        }
        st_issue = st_issue + 1 == kFS ? 0 : st_issue + 1;
        const int64_t kz = gz - (kFS - 3);
        if (kz >= z1lo) {
            if (kz < z1hi) {
                const bool vk = inside && kz >= 0 && kz < nz;
                const int64_t kb = (vk ? kz : 0) * plane;
                cp_async16(&sm.pp[kst_issue][wp][lane], b + kb + off, vk);
                cp_async16(&sm.kk[kst_issue][wp][lane], kap + kb + off, vk);
            }
            kst_issue = kst_issue + 1 == kFK ? 0 : kst_issue + 1;
        }
        cp_async_commit();
    };

    // q[j] = p^n at plane zs - 4 + j of this thread's points
    float4 q[kFQ];
#pragma unroll
    for (int j = 0; j < 2 * kFR; ++j) {
        const int64_t zj = z1lo - kFR + j;
        q[j] = (inside && zj >= 0 && zj < nz) ? ldg4(a + zj * plane + off) : z4;
    }
    // groups for planes z1lo .. z1lo + 6 before the loop; iteration zs issues
    // group zs + 7.  The queue's plane zs + 4 comes from group zs + 4 (issued
    // three iterations earlier), p^{n-1} / kappa of zs from group zs + 5 (two)
    for (int i = 0; i < kFS - 1; ++i)
        issue(z1lo + i);
    int st = 0, kst = 0, lv = 0;  // stages of plane zs; level ring slot of zs
    for (int64_t zs = z1lo; zs < z1hi; ++zs) {
        cp_async_wait<1>();  // groups up to zs + 5 have landed (tile zs + 4; p^{n-1}, kappa of zs)
        __syncthreads();     // ... for all threads; the stages of zs - 1 and the ring slot of zs - 9 are free
        issue(zs + kFS - 1);
        const int st4 = st + kFR >= kFS ? st + kFR - kFS : st + kFR;
        q[2 * kFR] = sm.p[st4][wp + kFR][lane];
        // ---- level n+1 at plane zs (zero outside the grid) ----
        float4 v = z4;
        if (zs >= 0 && zs < nz) {
            const float4 c = q[kFR];
            float4 lf, rt;
            shuffles(c, lf, rt);
            if (lane == 0)
                lf = sm.xh[st][wp][0];
            if (lane == kTX - 1)
                rt = sm.xh[st][wp][1];
            float4 ym[kFR], yp[kFR], zm[kFR], zp[kFR];
#pragma unroll
            for (int m = 1; m <= kFR; ++m) {
                ym[m - 1] = sm.p[st][wp + kFR - m][lane];
                yp[m - 1] = sm.p[st][wp + kFR + m][lane];
                zm[m - 1] = q[kFR - m];
                zp[m - 1] = q[kFR + m];
            }
            const float4 ppv = sm.pp[kst][wp][lane], kv = sm.kk[kst][wp][lane];
            const float L[4] = {lf.x, lf.y, lf.z, lf.w}, C[4] = {c.x, c.y, c.z, c.w}, R[4] = {rt.x, rt.y, rt.z, rt.w};
            const float PP[4] = {ppv.x, ppv.y, ppv.z, ppv.w}, KV[4] = {kv.x, kv.y, kv.z, kv.w};
            float o[4];
            wave_pt4(L, C, R, ym, yp, zm, zp, PP, KV, o);
            if (src1 && zs == sz) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sx == x4 + j)
                        o[j] += w1;
            }
            if (inside) {
                v = make_float4(o[0], o[1], o[2], o[3]);
                if (own && zs >= za && zs < zend)
                    *reinterpret_cast<float4 *>(c_out + zs * plane + off) = v;
            }
        }
        sm.lv[lv][wp][lane] = v;
        __syncthreads();  // level n+1 of plane zs is in the ring
        // ---- level n+2 at plane zo = zs - 4 ----
        const int64_t zo = zs - kFR;
        if (orow && zo >= za && zo < zend) {
            const int lo = lv >= kFR ? lv - kFR : lv + kFQ - kFR;  // ring slot of zo
            const float4 c = sm.lv[lo][wp][lane];
            float4 lf, rt;
            shuffles(c, lf, rt);  // lanes 0 and 31 compute nothing that is stored
            float4 ym[kFR], yp[kFR], zm[kFR], zp[kFR];
#pragma unroll
            for (int m = 1; m <= kFR; ++m) {
                ym[m - 1] = sm.lv[lo][wp - m][lane];
                yp[m - 1] = sm.lv[lo][wp + m][lane];
                const int sm_ = lo >= m ? lo - m : lo + kFQ - m, sp = lo + m >= kFQ ? lo + m - kFQ : lo + m;
                zm[m - 1] = sm.lv[sm_][wp][lane];
                zp[m - 1] = sm.lv[sp][wp][lane];
            }
            const float4 ppv = q[0];  // p^n at zo: level n+2's p_prev
            const float4 kv = own ? ldg4(kap + zo * plane + off) : z4;
            const float L[4] = {lf.x, lf.y, lf.z, lf.w}, C[4] = {c.x, c.y, c.z, c.w}, R[4] = {rt.x, rt.y, rt.z, rt.w};
            const float PP[4] = {ppv.x, ppv.y, ppv.z, ppv.w}, KV[4] = {kv.x, kv.y, kv.z, kv.w};
            float o[4];
            wave_pt4(L, C, R, ym, yp, zm, zp, PP, KV, o);
            if (own && y == sy && zo == sz && sx >= x4 && sx < x4 + 4) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sx == x4 + j)
                        o[j] += w2;
            }
            if (own)
                *reinterpret_cast<float4 *>(d_out + zo * plane + off) = make_float4(o[0], o[1], o[2], o[3]);
        }
#pragma unroll
        for (int j = 0; j < 2 * kFR; ++j)
            q[j] = q[j + 1];
        st = st + 1 == kFS ? 0 : st + 1;
        kst = kst + 1 == kFK ? 0 : kst + 1;
        lv = lv + 1 == kFQ ? 0 : lv + 1;
    }
    cp_async_wait<0>();  // no copy may outlive the CTA's shared memory
}

}  // namespace

// Two leapfrog steps of the whole field: p^{n+1} into c_out, p^{n+2} into
// d_out (both distinct from a, b and each other).
cudaError_t launch_wave25x2(const float *a, const float *b, const float *kap, float *c_out, float *d_out, int64_t nx,
                            int64_t ny, int64_t nz, int64_t sx, int64_t sy, int64_t sz, float w1, float w2,
                            cudaStream_t st)
{
    // set once (thread-safe); 0 if the attribute could not be set
    static const int res = []() -> int {
        if (cudaFuncSetAttribute(wave25x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FusedSmem)) != cudaSuccess)
            return 0;
        return resident((const void *)wave25x2_kernel, kTX * kFW, sizeof(FusedSmem));
    }();
    if (res <= 0)
        return cudaErrorInvalidValue;
    const int64_t gx = (nx + kFSeg - 1) / kFSeg, gy = (ny + kFO - 1) / kFO;
    const int64_t chunk = choose_chunk(gx * gy, nz, 24, 17, res);
    const int64_t gz = (nz + chunk - 1) / chunk;
    if (gx * gy > 0x7fffffffll || a == c_out || a == d_out || b == c_out || b == d_out || c_out == d_out)
        return cudaErrorInvalidValue;
    wave25x2_kernel<<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kFW), sizeof(FusedSmem), st>>>(
        a, b, kap, c_out, d_out, Grid3{nx, ny, nz, nx * ny}, chunk, sx, sy, sz, w1, w2);
    return cudaGetLastError();
}

}  // namespace ooc
