// adjoint.cu -- gradient of a receiver misfit with respect to the wave25
// velocity model: forward run with compressed checkpoints, then the discrete
// adjoint run backward segment by segment, replaying each segment's
// forward wavefield from its checkpoint.  (Not in the paper: an added
// differentiation workload on top of its 25-point propagator.)
//
// Forward, n = 0 .. N-1, p^0 = p^{-1} = 0:
//   p^{n+1} = 2 p^n - p^{n-1} + kappa L(p^n) + w[n] delta_src,  tr[n] = p^{n+1}(rec)
// Adjoint of that map for dJ/dtr = res (mu^{N+1} = mu^{N+2} = 0):
//   mu^m = 2 mu^{m+1} - mu^{m+2} + L(kappa mu^{m+1}) + S^T res[m-1],  m = N .. 1
//   dJ/dkappa = sum_{n=0}^{N-1} mu^{n+1} L(p^n)          (accumulated in FP64)
// and with kappa = (v dt/dx)^2, dJ/dv = dJ/dkappa * 2 v (dt/dx)^2.
//
// Checkpoints hold (p^{kK}, p^{k K - 1}) every K steps in pinned host memory,
// FR4-compressed at `rate` bits/value (or FP32 with rate 0).  The backward
// pass replays K steps from a checkpoint into a device history, so its
// device footprint is K + 6 fields whatever the number of steps.
//
// The backward pass carries w = kappa mu instead of mu.  Multiplying the
// adjoint recurrence by kappa gives
//   w^m = 2 w^{m+1} - w^{m+2} + kappa L(w^{m+1}) + kappa S^T res[m-1],
// the forward propagator's own form, so the adjoint step runs on the
// forward wave25 kernel; and dJ/dkappa = (sum_n w^{n+1} L(p^n)) / kappa,
// the sum accumulated in FP64 and divided once at the end (kappa > 0).
// Within a K-step segment the products and their sum are FP32 (at most K
// terms, in a device field); each segment's sum is then added to the FP64
// total.  GB300's FP64 pipe made a per-step FP64 update (two conversions, a
// multiply and an add per point) the slowest kernel of the backward pass.
#include <chrono>
#include <cstring>
#include <thread>

#include "common.cuh"

using namespace ooc;

namespace ooc {
// Set by a gather or scatter kernel that skipped an index outside its field;
// read and cleared by take_index_fault().
__device__ unsigned g_index_fault = 0u;

cudaError_t take_index_fault(unsigned *fault)
{
    unsigned v = 0u;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_index_fault, sizeof(v));
    if (e == cudaSuccess && v != 0u) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_index_fault, &zero, sizeof(zero));
    }
    *fault = v;
    return e;
}
}  // namespace ooc

namespace {

// Set by check_indices_kernel (receiver indices of the checkpointed calls).
__device__ unsigned g_receivers_bad = 0u;

constexpr int kTX = 32, kTY = 8, kSeg = 4 * kTX, kR = 4;

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 mul4(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }

// Adjoint step in its mu form on dense fields (plane z at z * nx * ny):
// out = 2 a - b + L(kappa * a); out may alias b.  The tiling follows the
// forward kernel: a warp owns 128 x-points, the y-neighbours come from a
// shared-memory plane, the z-neighbours from a register queue of kappa * a.
__global__ void __launch_bounds__(kTX *kTY, 2)
    wave25_adjoint_kernel(const float *__restrict__ a, const float *__restrict__ kap, const float *b, float *out,
                          int64_t nx, int64_t ny, int64_t nz, int64_t zchunk)
{
    __shared__ float4 tile[2][kTY + 2 * kR][kTX];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t gx = (nx + kSeg - 1) / kSeg;  // x tiles; blockIdx.x = by * gx + bx
    const int64_t xs = (int64_t)(blockIdx.x % gx) * kSeg;
    const int64_t x4 = xs + 4 * lane;
    const int64_t y0 = (int64_t)(blockIdx.x / gx) * kTY;
    const int64_t y = y0 + ty;
    const int64_t za = (int64_t)blockIdx.y * zchunk;
    const int cnt = (int)(min(za + zchunk, nz) - za);
    const int64_t plane = nx * ny;
    const bool inside = x4 < nx && y < ny;
    const int64_t off = inside ? y * nx + x4 : 0;
    const int hr = ty < kR ? ty : kTY + ty;
    const int64_t yh = ty < kR ? y0 - kR + ty : y0 + kTY + (ty - kR);
    const bool hrow = yh >= 0 && yh < ny && x4 < nx;
    const int64_t hoff = hrow ? yh * nx + x4 : 0;
    const int64_t xh = lane == 0 ? xs - 4 : xs + kSeg;
    const bool hcol = (lane == 0 || lane == kTX - 1) && xh >= 0 && xh < nx && y < ny;
    const int64_t xoff = hcol ? y * nx + xh : 0;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // operand of L at flat index i: kappa * a
    auto opnd = [&](int64_t i) -> float4 { return mul4(ldg4(a + i), ldg4(kap + i)); };

    float4 q[2 * kR + 1];
#pragma unroll
    for (int j = 0; j < 2 * kR + 1; ++j) {
        const int64_t zj = za - kR + j;
        q[j] = (inside && zj >= 0 && zj < nz) ? opnd(zj * plane + off) : z4;
    }
    float4 hyv = hrow ? opnd(za * plane + hoff) : z4;
    float4 hxv = hcol ? opnd(za * plane + xoff) : z4;
    float4 e1 = inside ? ldg4(a + za * plane + off) : z4;
    float4 e2 = inside ? *reinterpret_cast<const float4 *>(b + za * plane + off) : z4;
    int64_t z = za;
    for (int i = 0; i < cnt; ++i, ++z) {
        const bool more = i + 1 < cnt;
        const int64_t b1 = (z + 1) * plane;
        const float4 pfv = (inside && z + kR + 1 < nz) ? opnd((z + kR + 1) * plane + off) : z4;
        const float4 hyv_n = (more && hrow) ? opnd(b1 + hoff) : z4;
        const float4 hxv_n = (more && hcol) ? opnd(b1 + xoff) : z4;
        const float4 e1_n = (more && inside) ? ldg4(a + b1 + off) : z4;
        const float4 e2_n = (more && inside) ? *reinterpret_cast<const float4 *>(b + b1 + off) : z4;

        const int bb = i & 1;
        const float4 c = q[kR];
        tile[bb][ty + kR][lane] = c;
        tile[bb][hr][lane] = hyv;
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
        const float X[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w, rt.x, rt.y, rt.z, rt.w};
        float lap[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            lap[j] = (3.0f * kC0) * X[4 + j];
        const float cf[kR] = {kC1, kC2, kC3, kC4};
#pragma unroll
        for (int m = 1; m <= kR; ++m) {
            const float4 ym = tile[bb][ty + kR - m][lane];
            const float4 yp = tile[bb][ty + kR + m][lane];
            const float YM[4] = {ym.x, ym.y, ym.z, ym.w}, YP[4] = {yp.x, yp.y, yp.z, yp.w};
            const float ZM[4] = {q[kR - m].x, q[kR - m].y, q[kR - m].z, q[kR - m].w};
            const float ZP[4] = {q[kR + m].x, q[kR + m].y, q[kR + m].z, q[kR + m].w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                lap[j] += cf[m - 1] * (((X[4 + j - m] + X[4 + j + m]) + (YM[j] + YP[j])) + (ZM[j] + ZP[j]));
        }
        if (inside) {
            const float A[4] = {e1.x, e1.y, e1.z, e1.w}, B[4] = {e2.x, e2.y, e2.z, e2.w};
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = 2.0f * A[j] - B[j] + lap[j];
            *reinterpret_cast<float4 *>(out + z * plane + off) = make_float4(o[0], o[1], o[2], o[3]);
        }
#pragma unroll
        for (int j = 0; j < 2 * kR; ++j)
            q[j] = q[j + 1];
        q[2 * kR] = pfv;
        hyv = hyv_n;
        hxv = hxv_n;
        e1 = e1_n;
        e2 = e2_n;
    }
}

// Gather and scatter skip an index outside the field [0, size) (a gather
// writes 0 there) and set g_index_fault, so no index reaches memory beyond
// the field.
__global__ void gather_kernel(const float *__restrict__ f, int64_t size, const int64_t *__restrict__ idx, int64_t n,
                              float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int64_t j = idx[i];
        if (j >= 0 && j < size) {
            out[i] = f[j];
        } else {
            out[i] = 0.0f;
            atomicOr(&g_index_fault, 1u);
        }
    }
}

// Receiver indices are distinct, so every point has one writer.
__global__ void scatter_add_kernel(float *f, int64_t size, const int64_t *__restrict__ idx, int64_t n,
                                   const float *__restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int64_t j = idx[i];
        if (j >= 0 && j < size)
            f[j] += v[i];
        else
            atomicOr(&g_index_fault, 1u);
    }
}

// f[idx[i]] += v[i] * kap[idx[i]] (receiver residual injected into w = kappa mu).
__global__ void scatter_add_scaled_kernel(float *f, int64_t size, const int64_t *__restrict__ idx, int64_t n,
                                          const float *__restrict__ v, const float *__restrict__ kap)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int64_t j = idx[i];
        if (j >= 0 && j < size)
            f[j] += v[i] * kap[j];
        else
            atomicOr(&g_index_fault, 1u);
    }
}

// Sets g_receivers_bad when an index lies outside [0, size).
__global__ void check_indices_kernel(const int64_t *__restrict__ idx, int64_t n, int64_t size)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (idx[i] < 0 || idx[i] >= size))
        atomicOr(&g_receivers_bad, 1u);
}

// g[i] += (double) a[i]; a[i] = 0: a segment's FP32 gradient sum into the
// FP64 total.
__global__ void flush_segment_kernel(double *__restrict__ g, float *__restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        g[i] += (double)a[i];
        a[i] = 0.0f;
    }
}

__global__ void divide_by_kappa_kernel(double *g, const float *__restrict__ kap, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] /= (double)kap[i];
}

__global__ void kappa_kernel(const float *__restrict__ v, float *__restrict__ kappa, int64_t n, float c)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float s = v[i] * c;
        kappa[i] = s * s;
    }
}

__global__ void grad_v_kernel(const double *__restrict__ gk, const float *__restrict__ v, float *__restrict__ gv,
                              int64_t n, double c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gv[i] = (float)(gk[i] * 2.0 * (double)v[i] * c2);
}

unsigned grid1d(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

bool dims_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx > 0 && ny > 0 && nz > 0 && nx % 4 == 0 && ny % 4 == 0 && nz % 4 == 0;
}

cudaError_t launch_adjoint_step(const float *a, const float *kap, const float *b, float *out, int64_t nx, int64_t ny,
                                int64_t nz, cudaStream_t st)
{
    const int64_t gx = (nx + kSeg - 1) / kSeg, gy = (ny + kTY - 1) / kTY;
    int64_t nchunk = (152 * 4 + gx * gy - 1) / (gx * gy);
    if (nchunk > nz / 16)
        nchunk = nz / 16 > 0 ? nz / 16 : 1;
    const int64_t chunk = (nz + nchunk - 1) / nchunk;
    const int64_t gz = (nz + chunk - 1) / chunk;
    if (gx * gy > 0x7fffffffll)
        return cudaErrorInvalidValue;
    wave25_adjoint_kernel<<<dim3((unsigned)(gx * gy), (unsigned)gz), dim3(kTX, kTY), 0, st>>>(a, kap, b, out, nx, ny,
                                                                                              nz, chunk);
    return cudaGetLastError();
}

size_t field_bytes(int64_t n, int rate) { return rate > 0 ? (size_t)n * rate / 8 : (size_t)n * 4; }
size_t a256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
    size_t p, pp, stage[2][2];   // forward
    size_t mu1, mu2, gacc, hist0;  // backward (hist: K + 1 fields from hist0)
    size_t total;
};

Layout make_layout(int64_t n, int64_t every, int rate)
{
    Layout L{};
    const size_t fb = a256((size_t)n * 4), cb = a256(field_bytes(n, rate));
    size_t off = 0;
    for (int i = 0; i < 2; ++i)
        for (int f = 0; f < 2; ++f) {
            L.stage[i][f] = off;
            off += cb;
        }
    const size_t common = off;
    L.p = common;
    L.pp = common + fb;
    const size_t fwd_end = common + 2 * fb;
    L.mu1 = common;
    L.mu2 = common + fb;
    L.gacc = common + 2 * fb;
    L.hist0 = common + 3 * fb;
    const size_t bwd_end = L.hist0 + (size_t)(every + 1) * fb;
    L.total = fwd_end > bwd_end ? fwd_end : bwd_end;
    return L;
}

ooc_status wait_ev(cudaEvent_t ev, int64_t timeout_ms)
{
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess)
            return OOC_OK;
        if (e != cudaErrorNotReady)
            return OOC_E_CUDA;
        if (std::chrono::steady_clock::now() > deadline)
            return OOC_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

struct Events {
    cudaEvent_t e[8];
    int made = 0;
    cudaError_t make()
    {
        for (; made < 8; ++made) {
            cudaError_t r = cudaEventCreateWithFlags(&e[made], cudaEventDisableTiming);
            if (r != cudaSuccess)
                return r;
        }
        return cudaSuccess;
    }
    ~Events()
    {
        for (int i = 0; i < made; ++i)
            cudaEventDestroy(e[i]);
    }
};

// The checkpointed calls check their receiver indices once, before any
// kernel reads or writes through them: OOC_E_INVALID if one lies outside
// the field.  The wait is bounded like the calls' other waits.
ooc_status check_receivers(const int64_t *d_rec, int64_t nrec, int64_t size, cudaStream_t st, cudaEvent_t ev)
{
    if (nrec == 0)
        return OOC_OK;
    const unsigned zero = 0u;
    if (cudaMemcpyToSymbolAsync(g_receivers_bad, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return OOC_E_CUDA;
    check_indices_kernel<<<(unsigned)((nrec + 255) / 256), 256, 0, st>>>(d_rec, nrec, size);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess)
        return OOC_E_CUDA;
    const ooc_status w = wait_ev(ev, 600000);
    if (w != OOC_OK)
        return w;
    unsigned bad = 0u;
    if (cudaMemcpyFromSymbolAsync(&bad, g_receivers_bad, sizeof(bad), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(ev, st) != cudaSuccess)
        return OOC_E_CUDA;
    const ooc_status w2 = wait_ev(ev, 600000);
    if (w2 != OOC_OK)
        return w2;
    return bad ? OOC_E_INVALID : OOC_OK;
}

#define TRY_CUDA(x)                  \
    do {                             \
        if ((x) != cudaSuccess)      \
            return OOC_E_CUDA;       \
    } while (0)

}  // namespace

extern "C" {

ooc_status ooc_gather(const float *d_field, int64_t field_size, const int64_t *d_idx, int64_t n, float *d_out,
                      void *stream)
{
    if (n < 0 || field_size < 0 || (n > 0 && (!d_field || !d_idx || !d_out)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_field, field_size, d_idx, n,
                                                                                 d_out);
    return cudaGetLastError() == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

ooc_status ooc_scatter_add(float *d_field, int64_t field_size, const int64_t *d_idx, int64_t n, const float *d_val,
                           void *stream)
{
    if (n < 0 || field_size < 0 || (n > 0 && (!d_field || !d_idx || !d_val)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    scatter_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_field, field_size, d_idx, n,
                                                                                      d_val);
    return cudaGetLastError() == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

ooc_status ooc_wave25_adjoint_step(const float *d_mu, const float *d_mu_prev, float *d_out, const float *d_kappa,
                                   int64_t nx, int64_t ny, int64_t nz, void *stream)
{
    if (!d_mu || !d_mu_prev || !d_out || !d_kappa || !dims_ok(nx, ny, nz))
        return OOC_E_INVALID;
    return launch_adjoint_step(d_mu, d_kappa, d_mu_prev, d_out, nx, ny, nz, (cudaStream_t)stream) == cudaSuccess
               ? OOC_OK
               : OOC_E_CUDA;
}

ooc_status ooc_wave25_grad_accum(double *d_grad, const float *d_mu, const float *d_p, int64_t nx, int64_t ny,
                                 int64_t nz, void *stream)
{
    if (!d_grad || !d_mu || !d_p || !dims_ok(nx, ny, nz) || ((uintptr_t)d_grad % 32))
        return OOC_E_INVALID;
    return launch_wave25_grad(d_p, d_mu, d_grad, nx, ny, nz, (cudaStream_t)stream) == cudaSuccess ? OOC_OK
                                                                                                : OOC_E_CUDA;
}

ooc_status ooc_kappa_from_velocity(const float *d_v, float *d_kappa, int64_t n, double dt_over_dx, void *stream)
{
    if (n < 0 || (n > 0 && (!d_v || !d_kappa)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    kappa_kernel<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(d_v, d_kappa, n, (float)dt_over_dx);
    return cudaGetLastError() == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

ooc_status ooc_velocity_grad(const double *d_grad_kappa, const float *d_v, float *d_grad_v, int64_t n,
                             double dt_over_dx, void *stream)
{
    if (n < 0 || (n > 0 && (!d_grad_kappa || !d_v || !d_grad_v)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    grad_v_kernel<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(d_grad_kappa, d_v, d_grad_v, n,
                                                                   dt_over_dx * dt_over_dx);
    return cudaGetLastError() == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

size_t ooc_wave25_ckpt_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t nsteps, int64_t every, int rate)
{
    if (!dims_ok(nx, ny, nz) || nsteps < 1 || every < 1 || rate < 0 || rate > 64)
        return 0;
    const int64_t nseg = (nsteps + every - 1) / every;
    return (size_t)nseg * 2 * a256(field_bytes(nx * ny * nz, rate));
}

size_t ooc_wave25_adjoint_work_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t every, int rate)
{
    if (!dims_ok(nx, ny, nz) || every < 1 || rate < 0 || rate > 64)
        return 0;
    return make_layout(nx * ny * nz, every, rate).total;
}

ooc_status ooc_wave25_forward_ckpt(const float *d_kappa, int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy,
                                   int64_t sz, const float *h_w, int64_t nsteps, const int64_t *d_rec, int64_t nrec,
                                   float *d_traces, int64_t every, int rate, void *h_ckpt, size_t ckpt_bytes,
                                   void *d_work, size_t work_bytes, void *const streams[2])
{
    const int64_t n = nx * ny * nz;
    if (!d_kappa || !dims_ok(nx, ny, nz) || nsteps < 1 || every < 1 || rate < 0 || rate > 64 || !h_ckpt ||
        !d_work || !streams || (nrec > 0 && (!d_rec || !d_traces)) || nrec < 0 ||
        ckpt_bytes < ooc_wave25_ckpt_bytes(nx, ny, nz, nsteps, every, rate) ||
        work_bytes < ooc_wave25_adjoint_work_bytes(nx, ny, nz, every, rate) || ((uintptr_t)d_work % 256))
        return OOC_E_INVALID;
    cudaStream_t sC = (cudaStream_t)streams[0], sD = (cudaStream_t)streams[1];
    const Layout L = make_layout(n, every, rate);
    char *w = (char *)d_work;
    float *p = (float *)(w + L.p), *pp = (float *)(w + L.pp);
    const size_t cb = a256(field_bytes(n, rate));
    Events ev;
    TRY_CUDA(ev.make());  // e[0..1]: staging filled, e[2..3]: staging drained
    {
        const ooc_status rc = check_receivers(d_rec, nrec, n, sC, ev.e[4]);
        if (rc != OOC_OK)
            return rc;
    }
    TRY_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * n, sC));
    TRY_CUDA(cudaMemsetAsync(pp, 0, sizeof(float) * n, sC));
    const bool src = sx >= 0 && h_w != nullptr;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (s % every == 0) {
            const int64_t k = s / every;
            const int bi = (int)(k & 1);
            if (k >= 2)
                TRY_CUDA(cudaStreamWaitEvent(sC, ev.e[2 + bi], 0));
            const float *fld[2] = {p, pp};
            for (int f = 0; f < 2; ++f) {
                char *stg = w + L.stage[bi][f];
                if (rate > 0)
                    TRY_CUDA(launch_fr4_encode(ConstRing{fld[f], nz, 0}, nx, ny, 0, nz, rate, (uint32_t *)stg, sC));
                else
                    TRY_CUDA(cudaMemcpyAsync(stg, fld[f], sizeof(float) * n, cudaMemcpyDeviceToDevice, sC));
            }
            TRY_CUDA(cudaEventRecord(ev.e[bi], sC));
            TRY_CUDA(cudaStreamWaitEvent(sD, ev.e[bi], 0));
            for (int f = 0; f < 2; ++f)
                TRY_CUDA(cudaMemcpyAsync((char *)h_ckpt + ((size_t)k * 2 + f) * cb, w + L.stage[bi][f],
                                         field_bytes(n, rate), cudaMemcpyDeviceToHost, sD));
            TRY_CUDA(cudaEventRecord(ev.e[2 + bi], sD));
        }
        TRY_CUDA(launch_wave25(ConstRing{p, nz, 0}, Ring{pp, nz, 0}, ConstRing{d_kappa, nz, 0}, nx, ny, nz, 0, nz,
                               src ? sx : -1, sy, sz, src ? h_w[s] : 0.0f, sC));
        float *t = p;  // pp now holds p^{s+1}
        p = pp;
        pp = t;
        if (nrec > 0)
            TRY_CUDA(ooc_gather(p, n, d_rec, nrec, d_traces + s * nrec, sC) == OOC_OK ? cudaSuccess
                                                                                     : cudaErrorUnknown);
    }
    TRY_CUDA(cudaEventRecord(ev.e[4], sC));
    TRY_CUDA(cudaEventRecord(ev.e[5], sD));
    ooc_status st = wait_ev(ev.e[4], 600000);
    if (st == OOC_OK)
        st = wait_ev(ev.e[5], 600000);
    return st;
}

ooc_status ooc_wave25_backward_ckpt(const float *d_kappa, int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy,
                                    int64_t sz, const float *h_w, int64_t nsteps, const int64_t *d_rec, int64_t nrec,
                                    const float *d_res, int64_t every, int rate, const void *h_ckpt,
                                    size_t ckpt_bytes, double *d_grad, void *d_work, size_t work_bytes,
                                    void *const streams[2])
{
    const int64_t n = nx * ny * nz;
    if (!d_kappa || !dims_ok(nx, ny, nz) || nsteps < 1 || every < 1 || rate < 0 || rate > 64 || !h_ckpt ||
        !d_work || !d_grad || !streams || nrec < 0 || (nrec > 0 && (!d_rec || !d_res)) ||
        ckpt_bytes < ooc_wave25_ckpt_bytes(nx, ny, nz, nsteps, every, rate) ||
        work_bytes < ooc_wave25_adjoint_work_bytes(nx, ny, nz, every, rate) || ((uintptr_t)d_work % 256) ||
        ((uintptr_t)d_grad % 32))
        return OOC_E_INVALID;
    cudaStream_t sC = (cudaStream_t)streams[0], sD = (cudaStream_t)streams[1];
    const Layout L = make_layout(n, every, rate);
    char *w = (char *)d_work;
    const size_t fb = a256((size_t)n * 4), cb = a256(field_bytes(n, rate));
    float *mu1 = (float *)(w + L.mu1), *mu2 = (float *)(w + L.mu2), *gacc = (float *)(w + L.gacc);
    auto hist = [&](int64_t j) { return (float *)(w + L.hist0 + (size_t)j * fb); };
    Events ev;
    TRY_CUDA(ev.make());  // e[0..1]: staging loaded (sD), e[2..3]: staging consumed (sC)
    {
        const ooc_status rc = check_receivers(d_rec, nrec, n, sC, ev.e[4]);
        if (rc != OOC_OK)
            return rc;
    }
    TRY_CUDA(cudaMemsetAsync(mu1, 0, sizeof(float) * n, sC));
    TRY_CUDA(cudaMemsetAsync(mu2, 0, sizeof(float) * n, sC));
    TRY_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(double) * n, sC));
    TRY_CUDA(cudaMemsetAsync(gacc, 0, sizeof(float) * n, sC));
    const bool src = sx >= 0 && h_w != nullptr;
    const int64_t nseg = (nsteps + every - 1) / every;
    auto load = [&](int64_t k) -> cudaError_t {  // checkpoint k -> staging (k & 1), on sD
        const int bi = (int)(k & 1);
        for (int f = 0; f < 2; ++f) {
            cudaError_t e = cudaMemcpyAsync(w + L.stage[bi][f], (const char *)h_ckpt + ((size_t)k * 2 + f) * cb,
                                            field_bytes(n, rate), cudaMemcpyHostToDevice, sD);
            if (e != cudaSuccess)
                return e;
        }
        return cudaEventRecord(ev.e[bi], sD);
    };
    TRY_CUDA(load(nseg - 1));
    for (int64_t k = nseg - 1; k >= 0; --k) {
        const int bi = (int)(k & 1);
        const int64_t n0 = k * every, n1 = n0 + every < nsteps ? n0 + every : nsteps, len = n1 - n0;
        // checkpoint k -> hist[0] = p^{n0-1}, hist[1] = p^{n0}
        TRY_CUDA(cudaStreamWaitEvent(sC, ev.e[bi], 0));
        float *dst[2] = {hist(1), hist(0)};  // staging order: (p^{n0}, p^{n0-1})
        for (int f = 0; f < 2; ++f) {
            const char *stg = w + L.stage[bi][f];
            if (rate > 0)
                TRY_CUDA(launch_fr4_decode((const uint32_t *)stg, nx, ny, 0, nz, rate, Ring{dst[f], nz, 0}, sC));
            else
                TRY_CUDA(cudaMemcpyAsync(dst[f], stg, sizeof(float) * n, cudaMemcpyDeviceToDevice, sC));
        }
        TRY_CUDA(cudaEventRecord(ev.e[2 + bi], sC));
        if (k >= 1) {  // prefetch the previous checkpoint into the other buffer
            TRY_CUDA(cudaStreamWaitEvent(sD, ev.e[2 + (1 - bi)], 0));
            TRY_CUDA(load(k - 1));
        }
        // replay: hist[j + 1] = p^{n0 + j}, j = 1 .. len - 1
        for (int64_t j = 1; j < len; ++j) {
            const int64_t s = n0 + j - 1;
            TRY_CUDA(launch_wave25_to(ConstRing{hist(j), nz, 0}, ConstRing{hist(j - 1), nz, 0}, Ring{hist(j + 1), nz, 0},
                                      ConstRing{d_kappa, nz, 0}, nx, ny, nz, 0, nz, src ? sx : -1, sy, sz,
                                      src ? h_w[s] : 0.0f, sC));
        }
        // adjoint through the segment, on w = kappa mu (mu1 / mu2 hold w)
        for (int64_t m = n1; m >= n0 + 1; --m) {
            TRY_CUDA(launch_wave25_to(ConstRing{mu1, nz, 0}, ConstRing{mu2, nz, 0}, Ring{mu2, nz, 0},
                                      ConstRing{d_kappa, nz, 0}, nx, ny, nz, 0, nz, -1, -1, -1, 0.0f, sC));
            if (nrec > 0) {  // + kappa S^T res[m-1]
                scatter_add_scaled_kernel<<<(unsigned)((nrec + 255) / 256), 256, 0, sC>>>(
                    mu2, n, d_rec, nrec, d_res + (m - 1) * nrec, d_kappa);
                TRY_CUDA(cudaGetLastError());
            }
            // += w^m L(p^{m-1}), in FP32 within the segment
            TRY_CUDA(launch_wave25_grad32(hist(m - n0), mu2, gacc, nx, ny, nz, sC));
            float *t = mu1;
            mu1 = mu2;
            mu2 = t;
        }
        // the segment's sum (at most `every` terms) into the FP64 total
        flush_segment_kernel<<<grid1d(n, 256), 256, 0, sC>>>(d_grad, gacc, n);
        TRY_CUDA(cudaGetLastError());
    }
    divide_by_kappa_kernel<<<grid1d(n, 256), 256, 0, sC>>>(d_grad, d_kappa, n);
    TRY_CUDA(cudaGetLastError());
    TRY_CUDA(cudaEventRecord(ev.e[4], sC));
    TRY_CUDA(cudaEventRecord(ev.e[5], sD));
    ooc_status st = wait_ev(ev.e[4], 600000);
    if (st == OOC_OK)
        st = wait_ev(ev.e[5], 600000);
    return st;
}

}  // extern "C"
