// api.cu -- stand-alone entry points of the C ABI: codec, BF16, in-core
// stencil runs and status strings.  See include/ooc.h for the contract.
#include <chrono>
#include <cmath>
#include <thread>

#include "common.cuh"

using namespace ooc;

namespace {

bool dims_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx > 0 && ny > 0 && nz > 0 && nx % 4 == 0 && ny % 4 == 0 && nz % 4 == 0 && nx <= (1ll << 30) &&
           ny <= (1ll << 30) && nz <= (1ll << 30);
}

// Deadline of the host waits inside stand-alone calls (ooc_compress_var).
constexpr int64_t kCallWaitMs = 600000;

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

ooc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? OOC_OK : OOC_E_CUDA; }

// Waits until the work enqueued so far on `st` has run, polling an event
// against a deadline (OOC_E_TIMEOUT past it; the work still runs).
ooc_status wait_stream(cudaStream_t st, int64_t timeout_ms)
{
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return OOC_E_CUDA;
    ooc_status s = cudaEventRecord(ev, st) == cudaSuccess ? OOC_OK : OOC_E_CUDA;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (s == OOC_OK) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess)
            break;
        if (e != cudaErrorNotReady)
            s = OOC_E_CUDA;
        else if (std::chrono::steady_clock::now() > deadline)
            s = OOC_E_TIMEOUT;
        else
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaEventDestroy(ev);
    return s;
}

// Flat BF16 conversion.  Quads of 4 values move as 16-byte (FP32) and
// 8-byte (BF16) accesses, four quads per thread per round so that several
// loads are in flight; a tail of n mod 4 values is done by thread 0.
__device__ __forceinline__ uint32_t bf16_rne_bits(uint32_t u)
{
    if ((u & 0x7FFFFFFFu) > 0x7F800000u)
        return (u >> 16) | 0x40u;  // NaN stays a quiet NaN
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

__global__ void bf16_pack_flat(const float *in, uint16_t *out, int64_t n)
{
    const int64_t nq = n >> 2, stride = (int64_t)gridDim.x * blockDim.x;
    const uint4 *in4 = reinterpret_cast<const uint4 *>(in);
    uint2 *out2 = reinterpret_cast<uint2 *>(out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i + k * stride < nq)
                v[k] = __ldg(in4 + i + k * stride);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i + k * stride < nq)
                out2[i + k * stride] = make_uint2(bf16_rne_bits(v[k].x) | (bf16_rne_bits(v[k].y) << 16),
                                                  bf16_rne_bits(v[k].z) | (bf16_rne_bits(v[k].w) << 16));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t j = nq << 2; j < n; ++j)
            out[j] = (uint16_t)bf16_rne_bits(__float_as_uint(in[j]));
}

__global__ void bf16_unpack_flat(const uint16_t *in, float *out, int64_t n)
{
    const int64_t nq = n >> 2, stride = (int64_t)gridDim.x * blockDim.x;
    const uint2 *in2 = reinterpret_cast<const uint2 *>(in);
    uint4 *out4 = reinterpret_cast<uint4 *>(out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += 4 * stride) {
        uint2 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i + k * stride < nq)
                v[k] = __ldg(in2 + i + k * stride);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i + k * stride < nq)
                out4[i + k * stride] = make_uint4(v[k].x << 16, v[k].x & 0xFFFF0000u, v[k].y << 16,
                                                  v[k].y & 0xFFFF0000u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t j = nq << 2; j < n; ++j)
            out[j] = __uint_as_float((uint32_t)in[j] << 16);
}

unsigned flat_grid(int64_t n)
{
    int64_t b = (n / 4 + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

extern "C" {

const char *ooc_status_string(ooc_status s)
{
    switch (s) {
    case OOC_OK: return "ok";
    case OOC_E_INVALID: return "invalid argument";
    case OOC_E_BUDGET: return "device budget too small";
    case OOC_E_ALLOC: return "host allocation failed";
    case OOC_E_CUDA: return "CUDA error";
    case OOC_E_TIMEOUT: return "timed out waiting for the GPU";
    case OOC_E_CORRUPT: return "corrupt stored data";
    default: return "unknown status";
    }
}

size_t ooc_compressed_bytes(int64_t nx, int64_t ny, int64_t nz, int rate)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || rate < 1 || rate > 64 || nx > (1ll << 40) || ny > (1ll << 40) ||
        nz > (1ll << 40))
        return 0;
    return (size_t)fr4_blocks(nx, ny, nz) * 8 * (size_t)rate;
}

ooc_status ooc_compress(const float *d_in, int64_t nx, int64_t ny, int64_t nz, int rate, void *d_out, size_t out_cap,
                        void *stream)
{
    const size_t need = ooc_compressed_bytes(nx, ny, nz, rate);
    if (!d_in || !d_out || need == 0 || !aligned(d_out, 4) || out_cap < need)
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (dims_ok(nx, ny, nz)) {  // whole blocks: 128-bit loads
        if (!aligned(d_in, 16))
            return OOC_E_INVALID;
        return cuda_status(launch_fr4_encode(ConstRing{d_in, nz, 0}, nx, ny, 0, nz, rate, (uint32_t *)d_out, st));
    }
    if (!aligned(d_in, 4))
        return OOC_E_INVALID;
    return cuda_status(
        launch_fr4_encode_dense(d_in, nx, ny, nz, 2 * rate, (uint32_t *)d_out, st));
}

ooc_status ooc_decompress(const void *d_in, size_t in_bytes, int64_t nx, int64_t ny, int64_t nz, int rate,
                          float *d_out, void *stream)
{
    const size_t need = ooc_compressed_bytes(nx, ny, nz, rate);
    if (!d_in || !d_out || need == 0 || !aligned(d_in, 4) || in_bytes < need)
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (dims_ok(nx, ny, nz)) {
        if (!aligned(d_out, 16))
            return OOC_E_INVALID;
        return cuda_status(launch_fr4_decode((const uint32_t *)d_in, nx, ny, 0, nz, rate, Ring{d_out, nz, 0}, st));
    }
    if (!aligned(d_out, 4))
        return OOC_E_INVALID;
    return cuda_status(launch_fr4_decode_dense((const uint32_t *)d_in, (int64_t)(in_bytes / 4), nullptr, nx, ny, nz,
                                               2 * rate, OOC_FR4_RATE, 0, d_out, st));
}

ooc_status ooc_compress64(const double *d_in, int64_t nx, int64_t ny, int64_t nz, int rate, void *d_out,
                          size_t out_cap, void *stream)
{
    const size_t need = ooc_compressed_bytes(nx, ny, nz, rate);
    if (!d_in || !d_out || need == 0 || !dims_ok(nx, ny, nz) || !aligned(d_in, 16) || !aligned(d_out, 4) ||
        out_cap < need)
        return OOC_E_INVALID;
    return cuda_status(launch_fr4d_encode(DConstRing{d_in, nz, 0}, nx, ny, 0, nz, rate, (uint32_t *)d_out,
                                          (cudaStream_t)stream));
}

ooc_status ooc_decompress64(const void *d_in, size_t in_bytes, int64_t nx, int64_t ny, int64_t nz, int rate,
                            double *d_out, void *stream)
{
    const size_t need = ooc_compressed_bytes(nx, ny, nz, rate);
    if (!d_in || !d_out || need == 0 || !dims_ok(nx, ny, nz) || !aligned(d_in, 4) || !aligned(d_out, 16) ||
        in_bytes < need)
        return OOC_E_INVALID;
    return cuda_status(launch_fr4d_decode((const uint32_t *)d_in, nx, ny, 0, nz, rate, DRing{d_out, nz, 0},
                                          (cudaStream_t)stream));
}

namespace {

constexpr int64_t kVarBlockWords = 130;

// Mode parameter for the kernels: P, or L = floor(log2 tol).  False if the
// mode or its parameter is invalid.
bool var_mparam(int mode, double param, int *mparam)
{
    if (mode == OOC_FR4_PRECISION) {
        if (!(param >= 1.0 && param <= 32.0) || param != std::floor(param))
            return false;
        *mparam = (int)param;
        return true;
    }
    if (mode == OOC_FR4_ACCURACY) {
        if (!(param > 0.0) || !std::isfinite(param))
            return false;
        int e = 0;
        std::frexp(param, &e);  // param = m 2^e, m in [0.5, 1)
        *mparam = e - 1;
        return true;
    }
    return false;
}

bool shape_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx > 0 && ny > 0 && nz > 0 && nx <= (1ll << 40) && ny <= (1ll << 40) && nz <= (1ll << 40);
}

}  // namespace

size_t ooc_compress_var_bound(int64_t nx, int64_t ny, int64_t nz)
{
    return shape_ok(nx, ny, nz) ? (size_t)fr4_blocks(nx, ny, nz) * kVarBlockWords * 4 : 0;
}

size_t ooc_var_scratch_bytes(int64_t nx, int64_t ny, int64_t nz)
{
    return shape_ok(nx, ny, nz) ? var_scratch_bytes(fr4_blocks(nx, ny, nz)) : 0;
}

ooc_status ooc_compress_var(const float *d_in, int64_t nx, int64_t ny, int64_t nz, int mode, double param,
                            void *d_out, size_t out_cap, uint64_t *d_index, void *d_scratch, size_t scratch_bytes,
                            size_t *out_bytes, void *stream)
{
    int mparam = 0;
    if (!d_in || !d_out || !d_index || !d_scratch || !out_bytes || !shape_ok(nx, ny, nz) ||
        !var_mparam(mode, param, &mparam) || !aligned(d_in, 4) || !aligned(d_out, 4) || !aligned(d_index, 8) ||
        !aligned(d_scratch, 8) || scratch_bytes < ooc_var_scratch_bytes(nx, ny, nz))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nblk = fr4_blocks(nx, ny, nz);
    *out_bytes = 0;
    // one pass: every block's size, offset and words (a block is written
    // only if it ends within out_cap)
    if (launch_fr4_encode_var(d_in, nx, ny, nz, mode, mparam, (uint32_t *)d_out, (uint64_t)(out_cap / 4), d_index,
                              d_scratch, st) != cudaSuccess)
        return OOC_E_CUDA;
    // the total is read once the pass has run; the wait is bounded
    const ooc_status ws = wait_stream(st, kCallWaitMs);
    if (ws != OOC_OK)
        return ws;
    unsigned fault = 0u;
    if (take_codec_fault(&fault) != cudaSuccess)
        return OOC_E_CUDA;
    if (fault)
        return OOC_E_TIMEOUT;
    uint64_t total = 0;
    if (cudaMemcpy(&total, d_index + nblk, sizeof(total), cudaMemcpyDeviceToHost) != cudaSuccess)
        return OOC_E_CUDA;
    *out_bytes = (size_t)total * 4;
    return *out_bytes > out_cap ? OOC_E_INVALID : OOC_OK;
}

ooc_status ooc_decompress_var(const void *d_in, size_t in_bytes, const uint64_t *d_index, int64_t nx, int64_t ny,
                              int64_t nz, int mode, double param, float *d_out, void *stream)
{
    int mparam = 0;
    if (!d_in || !d_index || !d_out || !shape_ok(nx, ny, nz) || !var_mparam(mode, param, &mparam) ||
        !aligned(d_in, 4) || !aligned(d_index, 8) || !aligned(d_out, 4))
        return OOC_E_INVALID;
    return cuda_status(launch_fr4_decode_dense((const uint32_t *)d_in, (int64_t)(in_bytes / 4), d_index, nx, ny, nz,
                                               (int)kVarBlockWords, mode, mparam, d_out, (cudaStream_t)stream));
}

ooc_status ooc_bf16_pack(const float *d_in, uint16_t *d_out, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!d_in || !d_out)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    if (!aligned(d_in, 16) || !aligned(d_out, 8))
        return OOC_E_INVALID;
    bf16_pack_flat<<<flat_grid(n), 256, 0, (cudaStream_t)stream>>>(d_in, d_out, n);
    return cuda_status(cudaGetLastError());
}

ooc_status ooc_bf16_unpack(const uint16_t *d_in, float *d_out, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!d_in || !d_out)))
        return OOC_E_INVALID;
    if (n == 0)
        return OOC_OK;
    if (!aligned(d_in, 8) || !aligned(d_out, 16))
        return OOC_E_INVALID;
    bf16_unpack_flat<<<flat_grid(n), 256, 0, (cudaStream_t)stream>>>(d_in, d_out, n);
    return cuda_status(cudaGetLastError());
}

ooc_status ooc_heat7_steps(float *d_u, float *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r, int64_t nsteps,
                           void *stream)
{
    if (!d_u || !d_tmp || d_u == d_tmp || !dims_ok(nx, ny, nz) || nsteps < 0 || !aligned(d_u, 16) ||
        !aligned(d_tmp, 16))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    float *a = d_u, *b = d_tmp;
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e = launch_heat7(ConstRing{a, nz, 0}, Ring{b, nz, 0}, nx, ny, nz, 0, nz, (float)r, st);
        if (e != cudaSuccess)
            return OOC_E_CUDA;
        float *t = a;
        a = b;
        b = t;
    }
    if (a != d_u)
        return cuda_status(cudaMemcpyAsync(d_u, a, sizeof(float) * nx * ny * nz, cudaMemcpyDeviceToDevice, st));
    return OOC_OK;
}

ooc_status ooc_heat7_steps_f64(double *d_u, double *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r,
                               int64_t nsteps, void *stream)
{
    if (!d_u || !d_tmp || d_u == d_tmp || !dims_ok(nx, ny, nz) || nsteps < 0 || !aligned(d_u, 16) ||
        !aligned(d_tmp, 16))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    double *a = d_u, *b = d_tmp;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (launch_heat7_f64(a, b, nx, ny, nz, r, st) != cudaSuccess)
            return OOC_E_CUDA;
        double *t = a;
        a = b;
        b = t;
    }
    if (a != d_u)
        return cuda_status(cudaMemcpyAsync(d_u, a, sizeof(double) * nx * ny * nz, cudaMemcpyDeviceToDevice, st));
    return OOC_OK;
}

ooc_status ooc_heat7_steps_fused(float *d_u, float *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r,
                                 int64_t nsteps, void *stream)
{
    if (!d_u || !d_tmp || !dims_ok(nx, ny, nz) || nsteps < 0 || d_u == d_tmp || !aligned(d_u, 16) ||
        !aligned(d_tmp, 16))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    float *a = d_u, *b = d_tmp;
    for (int64_t s = 0; s < nsteps; s += 2) {
        cudaError_t e = s + 2 <= nsteps
                            ? launch_heat7x2(ConstRing{a, nz, 0}, Ring{b, nz, 0}, nx, ny, nz, 0, nz, 0, nz, nullptr, 0,
                                             nullptr, 0, (float)r, st)
                            : launch_heat7(ConstRing{a, nz, 0}, Ring{b, nz, 0}, nx, ny, nz, 0, nz, (float)r, st);
        if (e != cudaSuccess)
            return OOC_E_CUDA;
        float *t = a;
        a = b;
        b = t;
    }
    if (a != d_u)
        return cuda_status(cudaMemcpyAsync(d_u, a, sizeof(float) * nx * ny * nz, cudaMemcpyDeviceToDevice, st));
    return OOC_OK;
}

ooc_status ooc_wave25_steps(float *d_p, float *d_pprev, const float *d_kappa, int64_t nx, int64_t ny, int64_t nz,
                            int64_t sx, int64_t sy, int64_t sz, const float *h_w, int64_t t, int64_t nsteps,
                            void *stream)
{
    if (!d_p || !d_pprev || !d_kappa || d_p == d_pprev || !dims_ok(nx, ny, nz) || nsteps < 0 || t < 0 ||
        !aligned(d_p, 16) || !aligned(d_pprev, 16) || !aligned(d_kappa, 16))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    float *a = d_p, *b = d_pprev;  // a holds p^n, b holds p^{n-1}
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool src = sx >= 0 && h_w != nullptr;
        const float w = src ? h_w[t + s] : 0.0f;
        cudaError_t e = launch_wave25(ConstRing{a, nz, 0}, Ring{b, nz, 0}, ConstRing{d_kappa, nz, 0}, nx, ny, nz, 0,
                                      nz, src ? sx : -1, sy, sz, w, st);
        if (e != cudaSuccess)
            return OOC_E_CUDA;
        float *tmp = a;  // b now holds p^{n+1}
        a = b;
        b = tmp;
    }
    if (a != d_p)
        return cuda_status(launch_swap(d_p, d_pprev, nx * ny * nz, st));
    return OOC_OK;
}

ooc_status ooc_wave25_steps_fused(float *d_p, float *d_pprev, const float *d_kappa, float *d_t1, float *d_t2,
                                  int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy, int64_t sz,
                                  const float *h_w, int64_t t, int64_t nsteps, void *stream)
{
    float *buf[4] = {d_p, d_pprev, d_t1, d_t2};
    for (int i = 0; i < 4; ++i) {
        if (!buf[i] || !aligned(buf[i], 16))
            return OOC_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (buf[i] == buf[j])
                return OOC_E_INVALID;
    }
    if (!d_kappa || !aligned(d_kappa, 16) || !dims_ok(nx, ny, nz) || nsteps < 0 || t < 0)
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const bool src = sx >= 0 && h_w != nullptr;
    // a = p^n, b = p^{n-1}; each pair writes p^{n+1}, p^{n+2} into the two
    // free buffers (c, d), and the next pair writes into (b, a): outputs
    // alternate between (t1, t2) and (pprev, p), so an even number of pairs
    // ends in place and (a, b) is always both fields or both scratch buffers
    float *a = d_p, *b = d_pprev, *c = d_t1, *d = d_t2;
    int64_t s = 0;
    for (; s + 2 <= nsteps; s += 2) {
        const float w1 = src ? h_w[t + s] : 0.0f, w2 = src ? h_w[t + s + 1] : 0.0f;
        if (launch_wave25x2(a, b, d_kappa, c, d, nx, ny, nz, src ? sx : -1, sy, sz, w1, w2, st) != cudaSuccess)
            return OOC_E_CUDA;
        float *oa = a, *ob = b;
        a = d;
        b = c;
        c = ob;
        d = oa;
    }
    if (s < nsteps) {  // an odd last step, p^{n+1} over p^{n-1} in place
        const float w = src ? h_w[t + s] : 0.0f;
        if (launch_wave25(ConstRing{a, nz, 0}, Ring{b, nz, 0}, ConstRing{d_kappa, nz, 0}, nx, ny, nz, 0, nz,
                          src ? sx : -1, sy, sz, w, st) != cudaSuccess)
            return OOC_E_CUDA;
        float *tmp = a;
        a = b;
        b = tmp;
    }
    // the results are in (a, b): in place, swapped, or in the scratch fields
    if (a == d_pprev && b == d_p)
        return cuda_status(launch_swap(d_p, d_pprev, nx * ny * nz, st));
    const size_t bytes = sizeof(float) * (size_t)(nx * ny * nz);
    if (a != d_p && cudaMemcpyAsync(d_p, a, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return OOC_E_CUDA;
    if (b != d_pprev && cudaMemcpyAsync(d_pprev, b, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return OOC_E_CUDA;
    return OOC_OK;
}

ooc_status ooc_wave25_steps_f64(double *d_p, double *d_pprev, const double *d_kappa, int64_t nx, int64_t ny,
                                int64_t nz, int64_t sx, int64_t sy, int64_t sz, const double *h_w, int64_t t,
                                int64_t nsteps, void *stream)
{
    if (!d_p || !d_pprev || !d_kappa || d_p == d_pprev || !dims_ok(nx, ny, nz) || nsteps < 0 || t < 0 ||
        !aligned(d_p, 16) || !aligned(d_pprev, 16) || !aligned(d_kappa, 16))
        return OOC_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    double *a = d_p, *b = d_pprev;  // a holds p^n, b holds p^{n-1}
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool src = sx >= 0 && h_w != nullptr;
        const double w = src ? h_w[t + s] : 0.0;
        cudaError_t e = launch_wave25_f64(DConstRing{a, nz, 0}, DRing{b, nz, 0}, DConstRing{d_kappa, nz, 0}, nx, ny,
                                          nz, 0, nz, src ? sx : -1, sy, sz, w, st);
        if (e != cudaSuccess)
            return OOC_E_CUDA;
        double *tmp = a;  // b now holds p^{n+1}
        a = b;
        b = tmp;
    }
    if (a != d_p)  // swap the two buffers' contents (as 32-bit words)
        return cuda_status(launch_swap((float *)d_p, (float *)d_pprev, 2 * nx * ny * nz, st));
    return OOC_OK;
}

}  // extern "C"

extern "C" ooc_status ooc_take_device_fault(int *fault)
{
    if (!fault)
        return OOC_E_INVALID;
    unsigned v = 0u, vc = 0u, vi = 0u;
    if (take_stencil_fault(&v) != cudaSuccess || take_codec_fault(&vc) != cudaSuccess ||
        take_index_fault(&vi) != cudaSuccess)
        return OOC_E_CUDA;
    *fault = (v != 0u || vc != 0u ? 1 : 0) | (vi != 0u ? 2 : 0);
    return OOC_OK;
}
