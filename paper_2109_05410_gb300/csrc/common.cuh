// common.cuh -- shared definitions of the CUDA library (product path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ooc.h"

namespace ooc {

// A "ring" holds a window of z-planes of one field on the device.  Plane z
// (global index, 0 <= z < nz) lives in slot (z + zbase) mod nslot.  With
// nslot = nz and zbase = 0 a ring is an ordinary dense field.
struct Ring {
    float *base;      // nslot planes of nx*ny floats
    int64_t nslot;    // Z
    int64_t zbase;    // in [0, Z)
};

struct ConstRing {
    const float *base;
    int64_t nslot;
    int64_t zbase;
};

// The same window of an FP64 field.
struct DRing {
    double *base;
    int64_t nslot;
    int64_t zbase;
};

struct DConstRing {
    const double *base;
    int64_t nslot;
    int64_t zbase;
};

__host__ __device__ inline int64_t ring_slot(int64_t z, int64_t zbase, int64_t nslot)
{
    int64_t s = z + zbase;
    s %= nslot;
    return s < 0 ? s + nslot : s;
}

// Stencil coefficients of the 8th-order central second difference.
constexpr float kC0 = -205.0f / 72.0f;
constexpr float kC1 = 8.0f / 5.0f;
constexpr float kC2 = -1.0f / 5.0f;
constexpr float kC3 = 8.0f / 315.0f;
constexpr float kC4 = -1.0f / 560.0f;

// Source amplitudes of a wave plan kept on the device: step n adds w[n]
// (n < nw) with n = *t + n_off, *t being the plan's time on the device.  With
// w == nullptr the launch's own amplitude argument is used.
struct WaveSrcTable {
    const float *w = nullptr;
    const int64_t *t = nullptr;
    int64_t n_off = 0, nw = 0;
};

// Kernel launchers (stream-ordered, no synchronisation).  All return
// cudaGetLastError() of the launch.
cudaError_t launch_heat7(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                         float r, cudaStream_t st);
// g[i] += (double) mu[i] * (double) L(p)[i] over whole dense fields (the
// 25-point Laplacian without kappa); g 32-byte aligned.
cudaError_t launch_wave25_grad(const float *p, const float *mu, double *g, int64_t nx, int64_t ny, int64_t nz,
                               cudaStream_t st);
// gacc[i] = fma(mu[i], L(p)[i], gacc[i]) in FP32 over whole dense fields
// (gacc 16-byte aligned): the adjoint run's in-segment gradient sums.
cudaError_t launch_wave25_grad32(const float *p, const float *mu, float *gacc, int64_t nx, int64_t ny, int64_t nz,
                                 cudaStream_t st);
// Two heat7 steps in one launch: level s on [lo, hi) computed on chip from
// ring `in` (level s-1), level s+1 written to ring `out` on [z0, z1).  The
// two level-s planes below lo are read from band_in (planes bin_lo,
// bin_lo+1, nx*ny floats each; NULL when lo has no planes below it), and
// level s on [bout_lo, bout_lo+2) is written to band_out (NULL: not saved).
// `in` and `out` must be different buffers.
cudaError_t launch_heat7x2(ConstRing in, Ring out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                           int64_t lo, int64_t hi, const float *band_in, int64_t bin_lo, float *band_out,
                           int64_t bout_lo, float r, cudaStream_t st);
// FP64 heat7 step over a whole dense field (nx even, in != out).
cudaError_t launch_heat7_f64(const double *in, double *out, int64_t nx, int64_t ny, int64_t nz, double r,
                             cudaStream_t st);
// FP64 rings (stencil64.cu): heat7 one step on [z0, z1) from `in` into
// `out`; wave25 one leapfrog step with p_prev overwritten in place.
// Two wave25 steps per launch on dense fields (wave_fused.cu): p^{n+1}
// into c_out and p^{n+2} into d_out, all five buffers distinct.
cudaError_t launch_wave25x2(const float *a, const float *b, const float *kap, float *c_out, float *d_out, int64_t nx,
                            int64_t ny, int64_t nz, int64_t sx, int64_t sy, int64_t sz, float w1, float w2,
                            cudaStream_t st);
cudaError_t launch_heat7_f64_ring(DConstRing in, DRing out, int64_t nx, int64_t ny, int64_t nz, int64_t z0, int64_t z1,
                                  double r, cudaStream_t st);
cudaError_t launch_wave25_f64(DConstRing p, DRing pprev_out, DConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                              int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, double w, cudaStream_t st,
                              WaveSrcTable tab = WaveSrcTable{});
cudaError_t launch_wave25(ConstRing p, Ring pprev_out, ConstRing kappa, int64_t nx, int64_t ny, int64_t nz,
                          int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w, cudaStream_t st,
                          WaveSrcTable tab = WaveSrcTable{});
// Same step with p_prev read from `pprev` and p' written to `pnew` (may alias).
cudaError_t launch_wave25_to(ConstRing p, ConstRing pprev, Ring pnew, ConstRing kappa, int64_t nx, int64_t ny,
                             int64_t nz, int64_t z0, int64_t z1, int64_t sx, int64_t sy, int64_t sz, float w,
                             cudaStream_t st, WaveSrcTable tab = WaveSrcTable{});
// Reads and clears the device word that a stencil kernel sets when one of
// its bounded waits gives up (nonzero: that launch left planes unwritten).
cudaError_t take_stencil_fault(unsigned *fault);
// Reads and clears the word set by gather / scatter kernels that skipped an
// index outside their field.
cudaError_t take_index_fault(unsigned *fault);
// plan time on the device: *t += n (one thread)
cudaError_t launch_add_time(int64_t *t, int64_t n, cudaStream_t st);
// Codec over the 4-aligned plane range [z0, z1) of a ring; the stream part
// for those planes is contiguous (2*rate words per block).
cudaError_t launch_fr4_encode(ConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                              uint32_t *out, cudaStream_t st);
cudaError_t launch_fr4_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                              Ring out, cudaStream_t st);
// FR4D (FP64 fields, rate 1..64): planes [z0, z1) of an FP64 ring, whole
// 4^3 blocks (nx, ny, z1 - z0 multiples of 4), the stream of plane z0 first.
cudaError_t launch_fr4d_encode(DConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                               uint32_t *out, cudaStream_t st);
cudaError_t launch_fr4d_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                               DRing out, cudaStream_t st);
// Dense fields of any shape (partial blocks edge-padded).  Fixed rate:
// mode OOC_FR4_RATE, `words` = 2R per block.  Variable-size modes
// (OOC_FR4_PRECISION / OOC_FR4_ACCURACY, mparam = P or floor(log2 tol)):
// `words` = 130; encode phase 0 writes block word counts to index[b], phase 1
// writes the blocks at the offsets then in index.
int64_t fr4_blocks(int64_t nx, int64_t ny, int64_t nz);
cudaError_t launch_fr4_encode_dense(const float *in, int64_t nx, int64_t ny, int64_t nz, int words, uint32_t *out,
                                    cudaStream_t st);
// Variable-size modes in one pass: block b's words at out + index[b]
// (index[nblk] = total); blocks ending past out_words are not written.
// scratch: var_scratch_bytes(nblk) device bytes.
cudaError_t launch_fr4_encode_var(const float *in, int64_t nx, int64_t ny, int64_t nz, int mode, int mparam,
                                  uint32_t *out, uint64_t out_words, uint64_t *index, void *scratch, cudaStream_t st);
size_t var_scratch_bytes(int64_t nblk);
// Reads and clears the word set when the variable-size encoder's bounded
// look-back gave up.
cudaError_t take_codec_fault(unsigned *fault);
cudaError_t launch_fr4_decode_dense(const uint32_t *in, int64_t in_words, const uint64_t *index, int64_t nx,
                                    int64_t ny, int64_t nz, int words, int mode, int mparam, float *out,
                                    cudaStream_t st);
// Exclusive prefix sum of v[0..n) in place, v[n] = total; scratch of
// scan_scratch_bytes(n) bytes.
// BF16 storage over plane ranges of a ring.
cudaError_t launch_bf16_pack_ring(ConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, uint16_t *out,
                                  cudaStream_t st);
cudaError_t launch_bf16_unpack_ring(const uint16_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, Ring out,
                                    cudaStream_t st);
cudaError_t launch_swap(float *a, float *b, int64_t n, cudaStream_t st);

}  // namespace ooc
