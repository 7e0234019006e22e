/*
 * ooc.h -- C ABI of the out-of-core stencil library with on-the-fly
 * fixed-rate compression (libooc.so, CUDA sm_103a).
 *
 * The method (Shen, Wu, Okita, Ino, "Accelerating GPU-Based Out-of-Core
 * Stencil Computation with On-the-Fly Compression"):
 *   - Section III: a grid larger than device memory is cut into blocks
 *     (here z-slabs) that stream to and from the GPU with their halo;
 *     contiguous blocks share the common region on the GPU instead of
 *     re-sending it (region sharing, Fig. 2), and each block is advanced
 *     several time steps per transfer (temporal blocking, Section VI setup).
 *   - Section IV: the fixed-rate lossy codec stores R bits per value, so
 *     compressed sizes are known and device buffers are preallocated.
 *   - Section V-A: separate compression -- each slab's output is written
 *     back as two independently compressed units, the remainder R_i and the
 *     common region C_{i-1} (Fig. 4).
 *   - Section V-B: copies and kernels overlap on three CUDA streams (Fig. 5).
 *
 * Conventions for every entry point:
 *   - Grids are [z][y][x], x fastest; nx, ny, nz are multiples of 4.
 *   - Pointers are plain host or device addresses as stated; the library
 *     never frees memory it did not allocate, and no call allocates device
 *     memory: the caller passes a device arena (its size *is* the device
 *     budget) and a pinned host arena.  The one piece of device memory the
 *     library holds itself is the fixed 16 MiB array of
 *     ooc_heat7_steps_noalloc, part of the loaded library image on every
 *     GPU that loads it, outside any plan's budget.
 *   - Every function returns an ooc_status and never aborts the process.
 *   - Streams are cudaStream_t passed as void* (0 = legacy default stream).
 *   - Threads: different plans, and in-core calls on distinct buffers, may
 *     run at the same time from different host threads; the library's
 *     process-wide state (launch constants, the tensor-map cache) is set up
 *     once, thread-safely.  Calls on one plan must not overlap.  The device
 *     fault words (ooc_take_device_fault) are per process.
 */
#ifndef OOC_H
#define OOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ooc_status;
#define OOC_OK 0
#define OOC_E_INVALID 1  /* bad argument, shape, rate or call order */
#define OOC_E_BUDGET 2   /* device arena too small for any slab plan */
#define OOC_E_ALLOC 3    /* host-side bookkeeping allocation failed */
#define OOC_E_CUDA 4     /* a CUDA runtime call or kernel launch failed */
#define OOC_E_TIMEOUT 5  /* a bounded wait on the GPU ran past its deadline */
#define OOC_E_CORRUPT 6  /* inconsistent stored data, or a failed debug check (debug_checks) */

/* Stencils (Section III's neighbour average; Section VI's 25-point
 * acoustic propagator with HALO = 4, Table I). */
#define OOC_HEAT7 1
#define OOC_WAVE25 2

/* Storage formats of a field in host memory and on the wire.  FP32 plans
 * take FP32, BF16 or FR4; FP64 plans take FP64 or FR4 (which is then the
 * FP64 codec FR4D, ooc_compress64). */
#define OOC_FMT_FP32 0  /* 4 bytes per value, uncompressed */
#define OOC_FMT_BF16 1  /* 2 bytes per value, round to nearest even */
#define OOC_FMT_FR4 2   /* fixed-rate 4^3-block codec, `rate` bits per value */
#define OOC_FMT_FP64 3  /* 8 bytes per value, uncompressed (FP64 plans) */

/* Precision of a plan's fields and arithmetic.  The paper's runs are in
 * double precision (Section VI); FP64 plans compute in FP64 on the GPU,
 * run heat7 one step per launch, and exchange whole fields with
 * ooc_set_field64 / ooc_get_field64.  Wave source amplitudes stay FP32
 * values (ooc_set_source) in both precisions. */
#define OOC_PREC_FP32 0
#define OOC_PREC_FP64 1

/* Field indices.  HEAT7: 0 = u.  WAVE25: 0 = p^t, 1 = p^{t-1} (both
 * read-write, Section VI), 2 = kappa = (v dt / dx)^2 (read-only). */
#define OOC_FIELD_U 0
#define OOC_FIELD_P 0
#define OOC_FIELD_P_PREV 1
#define OOC_FIELD_KAPPA 2

typedef struct {
    int64_t nx, ny, nz;          /* grid, multiples of 4 */
    int32_t stencil;             /* OOC_HEAT7 or OOC_WAVE25 */
    int32_t k;                   /* temporal block: steps per transfer, >= 1 */
    double r;                    /* heat7 coefficient (1/6 = neighbour average) */
    int32_t rw_format, rw_rate;  /* read-write fields: format and bits/value */
    int32_t ro_format, ro_rate;  /* wave25 kappa: format and bits/value */
    int64_t device_budget_bytes; /* device arena size the plan must fit in */
    int32_t slab_planes;         /* slab thickness T (multiple of 4); 0 = largest that fits */
    int32_t profile;             /* 1 = time every launch and copy with CUDA events */
    int64_t wait_timeout_ms;     /* deadline for host waits on the GPU; 0 = 600000 */
    int32_t heat_steps_per_launch; /* heat7: 2 = each pair of the k steps in one launch with the
                                      intermediate level kept on chip; 1 = one step per launch; 0 =
                                      default = 2 when k >= 2, else 1.  Results are bit-identical.
                                      wave25: 0 or 1. */
    int32_t graph_mode;          /* 0 = calls without profiling are captured once per distinct nsteps
                                    as a CUDA graph and replayed (heat7 always; wave25 when its
                                    source series fits the device table of 16384 amplitudes, or
                                    it has no source); 1 = always launch directly */
    int32_t debug_checks;        /* 1 = guard words after every region of the device arena, checked on
                                    the device after each ooc_step / ooc_set_field / ooc_get_field
                                    (a failure returns OOC_E_CORRUPT), and ooc_set_field checks
                                    that every input value is finite (OOC_E_INVALID otherwise; the
                                    field's stored contents are then unspecified).  The host checks
                                    of every launch's plane window and every copy's byte range run
                                    in every plan (OOC_E_CORRUPT).  0 = off */
    int32_t precision;           /* OOC_PREC_FP32 (0) or OOC_PREC_FP64 */
} ooc_config;

typedef struct ooc_plan ooc_plan;

typedef struct {
    int64_t steps_done;        /* time steps completed since bind */
    int64_t passes;            /* temporal-block passes executed */
    int64_t slabs;             /* slab visits executed */
    int64_t h2d_bytes, d2h_bytes;
    int64_t kernel_launches;   /* launches of this library's kernels in ooc_step */
    /* Filled only with profile = 1 (summed CUDA-event durations, ms, and the
     * launches or copies they cover).  The stencil launches of a slab share
     * one event pair, so ms_stencil / n_stencil is their mean duration
     * including the gaps between them. */
    double ms_decode, ms_stencil, ms_encode, ms_h2d, ms_d2h;
    int64_t n_decode, n_stencil, n_encode, n_h2d, n_d2h;
    double ms_last_step;       /* wall time of the last ooc_step call (host clock) */
} ooc_stats;

/* Geometry of a plan, for inspection and host-side checks. */
typedef struct {
    int64_t slab_planes, nslab, common_planes /* W */, halo /* h */;
    int64_t ring_planes /* Z */, nrings;
    int64_t device_bytes, host_bytes;
    int64_t staging_in_bytes, staging_out_bytes; /* per buffer, per field */
} ooc_plan_info;

/* Static string for a status code. */
const char *ooc_status_string(ooc_status s);

/* Bytes of an nx*ny*nz field stored by the fixed-rate codec at `rate` bits
 * per value, FR4 (FP32) or FR4D (FP64) alike (Section IV: R bits per value,
 * a size fixed in advance):
 * ceil(nx/4)*ceil(ny/4)*ceil(nz/4) blocks of 8*rate bytes, i.e.
 * nx*ny*nz*rate/8 when the sides are multiples of 4.  Returns 0 for invalid
 * arguments. */
size_t ooc_compressed_bytes(int64_t nx, int64_t ny, int64_t nz, int rate);

/* Compress an FP32 device field d_in[nz][ny][nx] into d_out (device,
 * ooc_compressed_bytes(...) bytes, 4-byte aligned) on `stream`,
 * asynchronously.  Rate 1..64 bits/value.  Inputs must be finite.  The
 * stream layout is 4^3 blocks, bx fastest, each exactly 2*rate 32-bit
 * words, so any 4-aligned z range is a contiguous byte range (Section V-A's
 * separately compressed units).  Sides need not be multiples of 4: a block
 * reaching past the field is padded with the value of the nearest point
 * inside it.  d_in must be 16-byte aligned when nx is a multiple of 4, and
 * 4-byte aligned otherwise.  Returns OOC_E_INVALID on bad shapes, rates,
 * alignment or out_cap < required; OOC_E_CUDA if the launch fails. */
ooc_status ooc_compress(const float *d_in, int64_t nx, int64_t ny, int64_t nz, int rate,
                        void *d_out, size_t out_cap, void *stream);

/* Inverse of ooc_compress: d_in holds in_bytes >= ooc_compressed_bytes(...)
 * bytes of codec stream (device); writes d_out[nz][ny][nx] (device, only
 * the points inside the field).  Any word content decodes without
 * faulting. */
ooc_status ooc_decompress(const void *d_in, size_t in_bytes, int64_t nx, int64_t ny, int64_t nz,
                          int rate, float *d_out, void *stream);

/* FR4D: the fixed-rate codec for FP64 fields (Section VI ran its double
 * fields at 32 and 24 of every 64 bits).  The same 4^3 blocks, stream layout
 * and bit-plane coder as FR4, with 58-bit block floating point (emax
 * clamped at -1022, 11 header bits), the lifting in 64-bit integers and 64
 * bit planes.  Compresses d_in[nz][ny][nx] (device FP64, 16-byte aligned,
 * finite values; nx, ny, nz multiples of 4) into d_out (device, 4-byte
 * aligned, ooc_compressed_bytes(nx, ny, nz, rate) bytes: R bits per value
 * as for FR4) on `stream`, asynchronously; rate 1..64.  Returns
 * OOC_E_INVALID on bad shapes, rates, alignment or out_cap < required;
 * OOC_E_CUDA if the launch fails. */
ooc_status ooc_compress64(const double *d_in, int64_t nx, int64_t ny, int64_t nz, int rate,
                          void *d_out, size_t out_cap, void *stream);

/* Inverse of ooc_compress64 into d_out (device FP64, 16-byte aligned).  Any
 * word content decodes without faulting. */
ooc_status ooc_decompress64(const void *d_in, size_t in_bytes, int64_t nx, int64_t ny, int64_t nz,
                            int rate, double *d_out, void *stream);

/* ---- Codec variants with variable-size blocks ------------------------------
 * Not used by the paper, which needs a size known in advance (Section IV);
 * it names comparing other compressors as future work.  The same block
 * coder codes bit planes 31 .. pmin with no bit budget:
 *   OOC_FR4_PRECISION, param = P in 1..32:  pmin = 32 - P;
 *   OOC_FR4_ACCURACY,  param = tol > 0:     pmin = L - (emax - 26) - 4
 *     clamped to [0, 32], L = floor(log2 tol), emax the block's exponent;
 *     |x - x'| <= tol for every value unless pmin clamps to 0 (the block
 *     is then kept to full precision).
 * Block b occupies the 32-bit words [index[b], index[b+1]) of the stream
 * (index[0] = 0, index[nblocks] = total words); a block is at most 130
 * words.  Partial blocks as in ooc_compress. */
#define OOC_FR4_RATE 0
#define OOC_FR4_PRECISION 1
#define OOC_FR4_ACCURACY 2

/* Worst-case stream bytes (130 words per block) and the device scratch
 * ooc_compress_var needs, for an nx*ny*nz field. */
size_t ooc_compress_var_bound(int64_t nx, int64_t ny, int64_t nz);
size_t ooc_var_scratch_bytes(int64_t nx, int64_t ny, int64_t nz);

/* Compress d_in (device, 4-byte aligned) in a variable-size mode into d_out
 * (device, out_cap bytes) and d_index (device, nblocks + 1 uint64).
 * d_scratch: ooc_var_scratch_bytes(...) device bytes.  Runs on `stream`
 * and returns when the size is known: *out_bytes (host) = 4 * total words.
 * One pass: each CTA codes its blocks, learns its offset from the CTAs
 * before it (a decoupled look-back over per-tile sums in d_scratch, every
 * wait bounded) and writes its blocks and their offsets.  If the stream
 * exceeds out_cap, returns OOC_E_INVALID with *out_bytes the size it
 * needs; d_index then holds every offset, and d_out only the blocks that
 * end within out_cap (nothing is written past it).  The host waits for
 * the pass by polling an event against a 10-minute deadline (OOC_E_TIMEOUT
 * past it, with the pass still enqueued); a look-back that gave up also
 * returns OOC_E_TIMEOUT. */
ooc_status ooc_compress_var(const float *d_in, int64_t nx, int64_t ny, int64_t nz, int mode, double param,
                            void *d_out, size_t out_cap, uint64_t *d_index, void *d_scratch,
                            size_t scratch_bytes, size_t *out_bytes, void *stream);

/* Decode a variable-size stream (in_bytes bytes at d_in, offsets d_index;
 * device) into d_out[nz][ny][nx] (device), asynchronously on `stream`.
 * Offsets are clamped to the stream and each block to 130 words, so any
 * content decodes without faulting. */
ooc_status ooc_decompress_var(const void *d_in, size_t in_bytes, const uint64_t *d_index, int64_t nx,
                              int64_t ny, int64_t nz, int mode, double param, float *d_out, void *stream);

/* BF16 storage: d_out[i] = bfloat16 of d_in[i], round to nearest even, NaN
 * kept quiet; and the exact widening back.  Device pointers, n values; the
 * FP32 side 16-byte and the BF16 side 8-byte aligned (OOC_E_INVALID
 * otherwise). */
ooc_status ooc_bf16_pack(const float *d_in, uint16_t *d_out, int64_t n, void *stream);
ooc_status ooc_bf16_unpack(const uint16_t *d_in, float *d_out, int64_t n, void *stream);

/* In-core reference runs of the same stencil kernels the pipeline uses
 * (whole grid as one window), for parity checks.  heat7: nsteps Jacobi steps
 * of u (device) with scratch d_tmp (device, same size); result in d_u.
 * wave25: from (d_p, d_pprev) = (p^t, p^{t-1}) to (p^{t+n}, p^{t+n-1}),
 * adding h_w[t + s] (host array, may be NULL) at (sx, sy, sz) in step s
 * (0-based); pass sx < 0 for no source.  Device buffers 16-byte aligned and
 * distinct; OOC_E_INVALID otherwise. */
ooc_status ooc_heat7_steps(float *d_u, float *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r,
                           int64_t nsteps, void *stream);
ooc_status ooc_wave25_steps(float *d_p, float *d_pprev, const float *d_kappa, int64_t nx, int64_t ny,
                            int64_t nz, int64_t sx, int64_t sy, int64_t sz, const float *h_w, int64_t t,
                            int64_t nsteps, void *stream);

/* heat7 in double precision, as the paper's runs (Section VI): nsteps steps
 * of d_u (device, FP64, result in place) with scratch d_tmp (device, same
 * size, distinct).  nx, ny, nz multiples of 4, buffers 16-byte aligned.
 * Same update and zero ghosts as ooc_heat7_steps, computed in FP64. */
ooc_status ooc_heat7_steps_f64(double *d_u, double *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r,
                               int64_t nsteps, void *stream);

/* The nsteps wave25 steps of ooc_wave25_steps with each pair of steps in
 * one kernel launch (temporal blocking inside the kernel: level n+1 of the
 * pair stays in shared memory, so HBM carries p^n, p^{n-1} and kappa once
 * and p^{n+1}, p^{n+2} once per two steps).  d_t1, d_t2: scratch fields of
 * the same size; all four fields distinct and 16-byte aligned.  Results,
 * in d_p and d_pprev, are bit-identical to ooc_wave25_steps.  An odd last
 * step runs alone. */
ooc_status ooc_wave25_steps_fused(float *d_p, float *d_pprev, const float *d_kappa, float *d_t1, float *d_t2,
                                  int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy, int64_t sz,
                                  const float *h_w, int64_t t, int64_t nsteps, void *stream);

/* wave25 in double precision: as ooc_wave25_steps with FP64 device fields
 * (16-byte aligned) and an FP64 source series h_w (host). */
ooc_status ooc_wave25_steps_f64(double *d_p, double *d_pprev, const double *d_kappa, int64_t nx, int64_t ny,
                                int64_t nz, int64_t sx, int64_t sy, int64_t sz, const double *h_w, int64_t t,
                                int64_t nsteps, void *stream);

/* The nsteps heat7 steps of ooc_heat7_steps with each pair of steps in one
 * kernel launch (temporal blocking inside the kernel, Section III: the
 * intermediate level stays in shared memory and registers, so HBM carries
 * one read and one write of the field per two steps).  An odd last step
 * runs alone.  Same arguments and errors as ooc_heat7_steps; results are
 * bit-identical to it. */
ooc_status ooc_heat7_steps_fused(float *d_u, float *d_tmp, int64_t nx, int64_t ny, int64_t nz, double r,
                                 int64_t nsteps, void *stream);

/* Reads and clears the library's device fault words on the current device.
 * *fault is a bit set, 0 when nothing went wrong: 1 if a kernel launched
 * since the last read gave up one of its bounded waits (a shared-memory
 * copy, or the variable-size encoder's look-back at an earlier tile, that
 * did not complete within about a second) and returned without writing the
 * rest of its output; 2 if ooc_gather or ooc_scatter_add met an
 * index outside its field and skipped it.  ooc_step checks the first
 * itself and returns OOC_E_TIMEOUT; callers of the in-core entry points
 * read it after synchronising their stream.  Kernels never trap, spin
 * without bound or access memory through an unchecked index. */
ooc_status ooc_take_device_fault(int *fault);

/* Largest grid, in points, that ooc_heat7_steps_noalloc accepts: the size of
 * its fixed scratch array (4 Mi floats, 16 MiB). */
#define OOC_NOALLOC_MAX_POINTS (4ll * 1024 * 1024)

/* The paper has no counterpart to this call.  It runs the same nsteps heat7
 * steps as ooc_heat7_steps on d_u (device, result in place) but takes no
 * scratch field, for callers that cannot provide one: code whose device
 * memory is owned by a host application or framework allocator with nothing
 * to spare, or a time-critical loop that must not allocate because an
 * allocation there can fail or stall.  The second field lives in a fixed
 * array inside the library (OOC_NOALLOC_MAX_POINTS floats, kept on every GPU
 * that loads the library until the process exits); no call allocates
 * anything.  Grids with more points return OOC_E_INVALID.  The first call
 * on a device looks up the array's device address for that device, so make
 * that first call before any stream capture begins.  The address is kept
 * with the ID of the context it was looked up in; a call made in another
 * context of the device (after a cudaDeviceReset, say) looks it up again,
 * so make the first call after such a reset outside stream capture too.
 * All calls share the
 * array: calls that overlap on the GPU race on it, so the caller must order
 * them.  Results are bit-identical to ooc_heat7_steps. */
ooc_status ooc_heat7_steps_noalloc(float *d_u, int64_t nx, int64_t ny, int64_t nz, double r, int64_t nsteps,
                                   void *stream);

/* ---- Adjoint (gradient of a receiver misfit w.r.t. velocity) -------------
 * Not in the paper: a differentiation workload on its 25-point propagator.
 * Forward, n = 0..N-1, from rest (p^0 = p^{-1} = 0):
 *   p^{n+1} = 2 p^n - p^{n-1} + kappa L(p^n) + w[n] delta_src,  tr[n] = p^{n+1}(rec)
 * Adjoint for dJ/dtr = res:  mu^m = 2 mu^{m+1} - mu^{m+2} + L(kappa mu^{m+1})
 * + S^T res[m-1], m = N..1;  dJ/dkappa = sum_n mu^{n+1} L(p^n) (FP64).
 * Receivers are flat indices (int64, device, distinct) in [0, nx ny nz):
 * both checkpointed calls check them before any kernel uses them and
 * return OOC_E_INVALID if one lies outside the field. */

/* d_out[i] = d_field[d_idx[i]], i < n (device pointers; d_field holds
 * field_size values).  An index outside [0, field_size) is skipped (d_out[i]
 * = 0) and sets bit 2 of the device fault word (ooc_take_device_fault). */
ooc_status ooc_gather(const float *d_field, int64_t field_size, const int64_t *d_idx, int64_t n, float *d_out,
                      void *stream);
/* d_field[d_idx[i]] += d_val[i]; indices must be distinct.  An index
 * outside [0, field_size) is skipped and sets bit 2 of the fault word. */
ooc_status ooc_scatter_add(float *d_field, int64_t field_size, const int64_t *d_idx, int64_t n, const float *d_val,
                           void *stream);
/* One adjoint step on dense fields: d_out = 2 mu - mu_prev + L(kappa * mu);
 * d_out may alias d_mu_prev (then it is updated in place). */
ooc_status ooc_wave25_adjoint_step(const float *d_mu, const float *d_mu_prev, float *d_out, const float *d_kappa,
                                   int64_t nx, int64_t ny, int64_t nz, void *stream);
/* d_grad[i] += (double)mu[i] * (double)L(p)[i]; d_grad 32-byte aligned. */
ooc_status ooc_wave25_grad_accum(double *d_grad, const float *d_mu, const float *d_p, int64_t nx, int64_t ny,
                                 int64_t nz, void *stream);
/* kappa = (v * dt/dx)^2 and dJ/dv = dJ/dkappa * 2 v (dt/dx)^2, n values. */
ooc_status ooc_kappa_from_velocity(const float *d_v, float *d_kappa, int64_t n, double dt_over_dx, void *stream);
ooc_status ooc_velocity_grad(const double *d_grad_kappa, const float *d_v, float *d_grad_v, int64_t n,
                             double dt_over_dx, void *stream);
/* Pinned host bytes for checkpoints every `every` steps at `rate` bits/value
 * (0 = FP32): ceil(N/every) checkpoints of (p^{kK}, p^{kK-1}).  Device work
 * bytes for the forward and backward runs (K + 6 fields at most). */
size_t ooc_wave25_ckpt_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t nsteps, int64_t every, int rate);
size_t ooc_wave25_adjoint_work_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t every, int rate);
/* Forward run from rest writing d_traces[nsteps][nrec] and the checkpoints
 * (h_ckpt pinned).  streams[0] computes, streams[1] copies checkpoints.
 * Blocks until done (OOC_E_TIMEOUT after 10 minutes). */
ooc_status ooc_wave25_forward_ckpt(const float *d_kappa, int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy,
                                   int64_t sz, const float *h_w, int64_t nsteps, const int64_t *d_rec, int64_t nrec,
                                   float *d_traces, int64_t every, int rate, void *h_ckpt, size_t ckpt_bytes,
                                   void *d_work, size_t work_bytes, void *const streams[2]);
/* Backward run: d_grad = dJ/dkappa (FP64, device, overwritten) for the
 * residual d_res[nsteps][nrec], replaying each segment from its checkpoint.
 * Within a segment of `every` steps the gradient terms are summed in FP32;
 * each segment's sum is added to the FP64 total.
 * The adjoint state is carried as kappa * mu (the forward propagator's
 * form) and the gradient divided by kappa at the end, so kappa must be
 * positive everywhere (as (v dt/dx)^2 of a positive velocity is). */
ooc_status ooc_wave25_backward_ckpt(const float *d_kappa, int64_t nx, int64_t ny, int64_t nz, int64_t sx, int64_t sy,
                                    int64_t sz, const float *h_w, int64_t nsteps, const int64_t *d_rec, int64_t nrec,
                                    const float *d_res, int64_t every, int rate, const void *h_ckpt,
                                    size_t ckpt_bytes, double *d_grad, void *d_work, size_t work_bytes,
                                    void *const streams[2]);

/* Plan an out-of-core run (Section III decomposition with Section V-A
 * units).  Validates `cfg`, chooses the slab thickness T (largest multiple of
 * 4 that fits device_budget_bytes unless cfg->slab_planes is set) and
 * reports the device arena and pinned host arena sizes needed.  No CUDA call
 * is made.  Errors: OOC_E_INVALID (shape not a multiple of 4, k < 1, rate
 * outside 1..64, unknown format/stencil, T not a multiple of 4),
 * OOC_E_BUDGET (no T fits), OOC_E_ALLOC. */
ooc_status ooc_plan_create(const ooc_config *cfg, ooc_plan **out, size_t *device_bytes, size_t *host_bytes);

ooc_status ooc_plan_get_info(const ooc_plan *plan, ooc_plan_info *info);

/* Bind caller-owned memory and streams.  device_arena: >= device_bytes,
 * 256-byte aligned.  host_arena: >= host_bytes, pinned (cudaHostAlloc or
 * torch pin_memory), 16-byte aligned; it holds every field in its storage
 * format and is updated in place by each pass.  streams[0..2] = H2D,
 * compute, D2H (Fig. 5).  Creates CUDA events; allocates no device memory. */
ooc_status ooc_plan_bind(ooc_plan *plan, void *device_arena, size_t device_bytes, void *host_arena,
                         size_t host_bytes, void *const streams[3]);

/* Store / fetch a whole FP32 field (host pointers, nx*ny*nz floats) into /
 * out of the plan's host storage, encoding / decoding on the GPU.  Blocks
 * until done.  Must not overlap an ooc_step on the same plan.  FP32 plans
 * only (OOC_E_INVALID otherwise). */
ooc_status ooc_set_field(ooc_plan *plan, int field, const float *host_src);
ooc_status ooc_get_field(ooc_plan *plan, int field, float *host_dst);

/* The same for FP64 plans, with nx*ny*nz doubles. */
ooc_status ooc_set_field64(ooc_plan *plan, int field, const double *host_src);
ooc_status ooc_get_field64(ooc_plan *plan, int field, double *host_dst);

/* Point source of the wave stencil: p^{n+1}(sx,sy,sz) += w[n] for n < nw
 * (host array, copied).  nw = 0 removes it. */
ooc_status ooc_set_source(ooc_plan *plan, int64_t sx, int64_t sy, int64_t sz, const float *w, int64_t nw);

/* Advance nsteps time steps: ceil(nsteps/k) passes of the slab pipeline
 * (the last pass may be shorter).  Returns after the last D2H has landed,
 * or OOC_E_TIMEOUT if that takes longer than wait_timeout_ms.  After a
 * timeout the enqueued passes still run to completion on the plan's
 * streams.  The plan's later ooc_step, ooc_set_field and ooc_get_field
 * calls wait for them first (under the same deadline, OOC_E_TIMEOUT
 * again if they have not finished); a caller who touches the arenas
 * directly synchronises those streams first.  The call's steps are
 * enqueued before the wait, so a timed-out call still
 * advances the plan's time (host and device copies alike) and counts its
 * steps, passes and launches in the statistics. */
ooc_status ooc_step(ooc_plan *plan, int64_t nsteps);

/* Change the plan's host-wait deadline (ms; 0 = 600000).  The waits of
 * ooc_step, ooc_set_field and ooc_get_field use it. */
ooc_status ooc_plan_set_wait_timeout(ooc_plan *plan, int64_t wait_timeout_ms);

/* Switch per-launch CUDA-event timing (ooc_config.profile) on (1) or off
 * (0) for later ooc_step calls.  The events separate every launch and copy,
 * which keeps consecutive kernels from overlapping their ramp-down and
 * ramp-up: on the 1024^3 heat7 pipeline they cost about 10 % of the
 * throughput. */
ooc_status ooc_plan_set_profile(ooc_plan *plan, int profile);

ooc_status ooc_get_stats(const ooc_plan *plan, ooc_stats *stats);
ooc_status ooc_reset_stats(ooc_plan *plan);

/* One timed interval of a profiled ooc_step call (the per-operation
 * breakdown of Section VI-B, Fig. 7): a decode, a slab's group of stencil
 * launches, an encode, or a slab's host-to-device or device-to-host copies. */
#define OOC_TRACE_DECODE 0
#define OOC_TRACE_STENCIL 1
#define OOC_TRACE_ENCODE 2
#define OOC_TRACE_H2D 3
#define OOC_TRACE_D2H 4
typedef struct {
    int32_t kind;            /* OOC_TRACE_* */
    int32_t count;           /* launches or copies inside the interval */
    int64_t pass;            /* pass of the call, from 0 */
    int64_t slab;            /* slab of the pass, from 0 */
    double start_ms, end_ms; /* CUDA-event times from the start of the call's first interval */
} ooc_trace_rec;

/* Intervals of the last ooc_step call made with profile = 1, in the order
 * they were enqueued (stream by stream they are in time order).  Copies
 * min(*n, cap) records to out (out may be NULL when cap = 0) and sets *n to
 * the number recorded; 0 when the last call was not profiled.  The plan
 * owns the records until its next ooc_step. */
ooc_status ooc_plan_get_trace(const ooc_plan *plan, ooc_trace_rec *out, int64_t cap, int64_t *n);

/* Releases the plan's events and host bookkeeping (not the arenas). */
void ooc_plan_destroy(ooc_plan *plan);

#ifdef __cplusplus
}
#endif
#endif /* OOC_H */
