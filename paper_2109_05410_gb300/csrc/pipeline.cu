// pipeline.cu -- the out-of-core slab scheduler (host side) of the C ABI.
//
// The grid lives in the pinned host arena, one image per field in its
// storage format (FP32, BF16 or FR4 codec).  A pass advances the whole grid
// k time steps (temporal blocking, Section VI setup) by sweeping z-slabs of
// T planes in increasing z (Section III decomposition):
//
//   slab i owns planes [a_i, b_i), a_i = i T.  Its output is the two units
//   C_{i-1} = [a_i, a_i + W) and R_i = [a_i + W, b_i), compressed separately
//   (Section V-A, Fig. 4); its input is R_i and C_i = [a_i + W, b_i + W)
//   (slab 0 also C_{-1} = [0, W)), W = k h rounded up to 4 planes.
//
//   Step s = 1..k updates level s on [a_i + (k - s) h, b_i + (k - s) h)
//   (slab 0 from 0, the last slab to nz): a parallelogram in (z, t).  The
//   2h planes each level needs below its window were computed by slab i-1
//   and are still in the level's ring buffer, so nothing is recomputed and
//   the halo never crosses the host link (region sharing, Fig. 2).
//
// Each level parity has one ring of Z planes (plane z in slot
// (z + zbase) mod Z); p^{s} overwrites p^{s-2} in place.  Passes continue
// the ring addressing (zbase advances by nz per pass), so the pipeline never
// drains between passes.  Three streams overlap the copies with the kernels
// (Section V-B, Fig. 5): H2D(i+1) || decode, k steps, encode (i) || D2H(i-1),
// ordered by events.  FP32 slabs land directly in the ring (no staging);
// BF16/FR4 slabs go through double-buffered staging and a decode kernel.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace ooc;

namespace {

constexpr int kEv = 4;  // event ring depth (waits look back at most 2 slabs)
constexpr int64_t kSrcTable = 16384;  // source amplitudes kept on the device (graph replay)
constexpr size_t kGuard = 256;        // guard bytes after each arena region (debug_checks)
constexpr int kMaxGuards = 32;
constexpr unsigned char kGuardByte = 0xA5;

struct GuardList {
    uint64_t off[kMaxGuards];
    int n;
};

// Sets *flag when a guard region no longer holds kGuardByte in every byte
// (one CTA of 64 threads per region, one 32-bit word each).
__global__ void check_guards_kernel(const unsigned char *base, GuardList g, int *flag)
{
    for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
        const uint32_t w = reinterpret_cast<const uint32_t *>(base + g.off[i])[threadIdx.x];
        if (w != 0xA5A5A5A5u)
            atomicOr(flag, 1);
    }
}

// debug_checks: sets bit 2 of *flag when a value of the n 32-bit words at w
// is not finite (exponent bits all ones).  FP32 values are every word; FP64
// values have their exponent in the high word of each pair (stride 2).
__global__ void check_finite_kernel(const uint32_t *w, int64_t n, int stride, int *flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i * stride < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = w[i * stride + stride - 1];
        const uint32_t e = stride == 1 ? 0x7f800000u : 0x7ff00000u;
        if ((v & e) == e)
            atomicOr(flag, 2);
    }
}

int64_t round4(int64_t v) { return (v + 3) / 4 * 4; }
size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int fmt_bits(int fmt, int rate)
{
    if (fmt == OOC_FMT_FP32)
        return 32;
    if (fmt == OOC_FMT_FP64)
        return 64;
    if (fmt == OOC_FMT_BF16)
        return 16;
    return rate;
}

struct ProfPair {
    cudaEvent_t a, b;
    int kind;   // 0 decode, 1 stencil, 2 encode, 3 h2d, 4 d2h
    int count;  // launches or copies between a and b
    int64_t pass, slab;
};

}  // namespace

struct ooc_plan {
    ooc_config cfg{};
    int64_t T = 0, nslab = 0, W = 0, h = 0, Z = 0;
    int nrw = 0, nfield = 0, nring = 0;
    int spl = 1;  // heat7 steps per stencil launch (1 or 2)
    int esize = 4;  // bytes per value in the rings: 4 (FP32 plans) or 8 (FP64)
    size_t off_band = 0, band_bytes = 0;  // level-s bands of the fused launches
    size_t off_src = 0;                   // wave source table (kSrcTable floats) and the device time
    int fmt[3] = {0, 0, 0}, rate[3] = {0, 0, 0};
    int64_t fplane[3] = {0, 0, 0};  // storage bytes per plane, per field
    int64_t plane_elems = 0;
    size_t off_ring[3] = {0, 0, 0};
    size_t off_in[2][3] = {{0}}, off_out[2][3] = {{0}};
    size_t in_bytes_field[3] = {0, 0, 0}, out_bytes_field[3] = {0, 0, 0};
    size_t dev_bytes = 0;
    size_t off_host[3] = {0, 0, 0};
    size_t host_bytes = 0;
    // bound state
    bool bound = false;
    char *dev = nullptr;
    char *host = nullptr;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_h2d[kEv], ev_dec[kEv], ev_comp[kEv], ev_d2h[kEv];
    bool events_made = false;
    // CUDA graph of one ooc_step(graph_nsteps) call, replayed while the
    // call's launches stay the same (heat7 without per-launch profiling)
    cudaGraphExec_t graph = nullptr;
    int64_t graph_nsteps = 0;
    ooc_stats graph_delta{};  // counters one replay adds
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr}, ev_done = nullptr;
    cudaEvent_t ev_tail[3] = {nullptr, nullptr, nullptr};  // drain(): the streams' tails
    std::vector<ProfPair> prof;
    size_t prof_used = 0;
    int64_t prof_pass = 0, prof_slab = 0;  // pass and slab being enqueued
    std::vector<ooc_trace_rec> trace;      // intervals of the last profiled ooc_step
    // debug_checks: arena offsets of the guard regions, and of the device flag
    std::vector<size_t> guards;
    size_t off_flag = 0;
    // run state
    int64_t time = 0;
    int64_t sx = -1, sy = -1, sz = -1;
    std::vector<float> w;
    bool src_uploaded = false;  // w is in the device table
    ooc_stats stats{};
};

namespace {

bool staged(const ooc_plan *p, int f) { return p->fmt[f] != OOC_FMT_FP32 && p->fmt[f] != OOC_FMT_FP64; }

// Layout of the device arena for slab thickness T; returns total bytes.
size_t layout(ooc_plan *p, int64_t T)
{
    const int64_t W = p->W, h = p->h;
    // FP32 slabs land in the ring while the previous slab computes (2T);
    // staged slabs land in staging buffers and are decoded in stream order.
    bool direct = false;
    for (int f = 0; f < p->nfield; ++f)
        direct |= !staged(p, f);
    const int64_t Z = round4((direct ? 2 * T : T) + W + 2 * h);
    size_t off = 0;
    const bool dbg = p->cfg.debug_checks != 0;
    p->guards.clear();
    auto guard = [&]() {
        if (dbg) {
            p->guards.push_back(off);
            off += kGuard;
        }
    };
    const size_t ring_bytes = (size_t)Z * p->plane_elems * p->esize;
    for (int r = 0; r < p->nring; ++r) {
        p->off_ring[r] = off;
        off += align256(ring_bytes);
        guard();
    }
    for (int f = 0; f < p->nfield; ++f) {
        p->in_bytes_field[f] = staged(p, f) ? (size_t)(T + W) * p->fplane[f] : 0;
        p->out_bytes_field[f] = (staged(p, f) && f < p->nrw) ? (size_t)T * p->fplane[f] : 0;
    }
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < p->nfield; ++f) {
            p->off_in[b][f] = off;
            off += align256(p->in_bytes_field[f]);
            if (p->in_bytes_field[f] > 0)
                guard();
            p->off_out[b][f] = off;
            off += align256(p->out_bytes_field[f]);
            if (p->out_bytes_field[f] > 0)
                guard();
        }
    // Fused heat7 pairs: the intermediate level's top 2h planes of each slab,
    // for the next slab; one band per pair of the pass and slab parity.
    p->off_band = off;
    p->band_bytes = p->spl == 2 ? (size_t)(2 * h) * p->plane_elems * p->esize : 0;
    off += align256(p->band_bytes) * 2 * (size_t)(p->cfg.k / 2);
    if (p->band_bytes > 0)
        guard();
    // the plan's time on the device, then the wave's source amplitudes
    p->off_src = off;
    off += 256 + (p->cfg.stencil == OOC_WAVE25 ? align256(kSrcTable * sizeof(float)) : 0);
    guard();
    if (dbg) {
        p->off_flag = off;  // the guard checks' flag
        off += 256;
    }
    p->Z = Z;
    return off;
}

Ring ring_view(ooc_plan *p, int r, int64_t zbase)
{
    return Ring{(float *)(p->dev + p->off_ring[r]), p->Z, zbase};
}

ConstRing cring(const Ring &r) { return ConstRing{r.base, r.nslot, r.zbase}; }

// The same rings of an FP64 plan.
DRing dring_view(ooc_plan *p, int r, int64_t zbase)
{
    return DRing{(double *)(p->dev + p->off_ring[r]), p->Z, zbase};
}

DConstRing dcring(const DRing &r) { return DConstRing{r.base, r.nslot, r.zbase}; }

int64_t *dev_time(ooc_plan *p) { return (int64_t *)(p->dev + p->off_src); }
float *dev_src(ooc_plan *p) { return (float *)(p->dev + p->off_src + 256); }

// Band of pair j written by slabs of parity `parity`.
float *band(ooc_plan *p, int64_t j, int64_t parity)
{
    return (float *)(p->dev + p->off_band + align256(p->band_bytes) * (size_t)(2 * j + parity));
}

// Stencil launches of a pass of kp steps (heat7 pairs when fused).
int64_t stencil_launches(const ooc_plan *p, int64_t kp) { return p->spl == 2 ? kp / 2 + (kp & 1) : kp; }

// Copy planes [z0, z1) between a ring and contiguous memory (split at wrap).
cudaError_t copy_ring(ooc_plan *p, int r, int64_t zbase, int64_t z0, int64_t z1, char *hostp, bool to_device,
                      cudaStream_t st)
{
    const size_t pb = (size_t)p->plane_elems * p->esize;
    int64_t z = z0;
    while (z < z1) {
        const int64_t slot = ring_slot(z, zbase, p->Z);
        int64_t n = z1 - z;
        if (slot + n > p->Z)
            n = p->Z - slot;
        char *dptr = p->dev + p->off_ring[r] + (size_t)slot * pb;
        char *hptr = hostp + (size_t)(z - z0) * pb;
        cudaError_t e = to_device ? cudaMemcpyAsync(dptr, hptr, (size_t)n * pb, cudaMemcpyHostToDevice, st)
                                  : cudaMemcpyAsync(hptr, dptr, (size_t)n * pb, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess)
            return e;
        z += n;
    }
    return cudaSuccess;
}

ooc_status wait_event(ooc_plan *p, cudaEvent_t ev)
{
    const int64_t ms = p->cfg.wait_timeout_ms > 0 ? p->cfg.wait_timeout_ms : 600000;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(ms);
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess)
            return OOC_OK;
        if (e != cudaErrorNotReady)
            return OOC_E_CUDA;
        if (std::chrono::steady_clock::now() > deadline)
            return OOC_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// debug_checks: every guard region back to kGuardByte and the flag to 0.
ooc_status arm_guards(ooc_plan *p)
{
    if (!p->cfg.debug_checks)
        return OOC_OK;
    for (size_t off : p->guards)
        if (cudaMemset(p->dev + off, kGuardByte, kGuard) != cudaSuccess)
            return OOC_E_CUDA;
    return cudaMemset(p->dev + p->off_flag, 0, sizeof(int)) == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

ooc_status check_guards(ooc_plan *p);

// Host-side check of an internal invariant of the schedule (a window that
// leaves its ring, a unit outside the host image, a staging overflow): the
// call returns OOC_E_CORRUPT before anything reaches the GPU.
inline ooc_status expect(const ooc_plan *, bool ok) { return ok ? OOC_OK : OOC_E_CORRUPT; }

ooc_status prof_begin(ooc_plan *p, cudaStream_t st, int kind, size_t *idx)
{
    *idx = (size_t)-1;
    if (!p->cfg.profile)
        return OOC_OK;
    if (p->prof_used == p->prof.size()) {
        ProfPair pp{};
        pp.kind = kind;
        if (cudaEventCreate(&pp.a) != cudaSuccess || cudaEventCreate(&pp.b) != cudaSuccess)
            return OOC_E_CUDA;
        try {
            p->prof.push_back(pp);
        } catch (...) {
            return OOC_E_ALLOC;
        }
    }
    *idx = p->prof_used++;
    p->prof[*idx].kind = kind;
    p->prof[*idx].count = 1;
    p->prof[*idx].pass = p->prof_pass;
    p->prof[*idx].slab = p->prof_slab;
    return cudaEventRecord(p->prof[*idx].a, st) == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

ooc_status prof_end(ooc_plan *p, cudaStream_t st, size_t idx)
{
    if (idx == (size_t)-1)
        return OOC_OK;
    return cudaEventRecord(p->prof[idx].b, st) == cudaSuccess ? OOC_OK : OOC_E_CUDA;
}

#define OOC_TRY(x)                   \
    do {                             \
        ooc_status _s = (x);         \
        if (_s != OOC_OK)            \
            return _s;               \
    } while (0)
#define OOC_CUDA(x)                  \
    do {                             \
        if ((x) != cudaSuccess)      \
            return OOC_E_CUDA;       \
    } while (0)

// Decode planes [z0, z1) of field f from `src` (storage format) into ring r
// (FR4D on FP64 plans).
ooc_status decode_into(ooc_plan *p, int f, const char *src, int r, int64_t zb, int64_t z0, int64_t z1,
                       cudaStream_t st)
{
    const int64_t nx = p->cfg.nx, ny = p->cfg.ny;
    if (p->esize == 8)
        OOC_CUDA(launch_fr4d_decode((const uint32_t *)src, nx, ny, z0, z1, p->rate[f], dring_view(p, r, zb), st));
    else if (p->fmt[f] == OOC_FMT_FR4)
        OOC_CUDA(launch_fr4_decode((const uint32_t *)src, nx, ny, z0, z1, p->rate[f], ring_view(p, r, zb), st));
    else
        OOC_CUDA(launch_bf16_unpack_ring((const uint16_t *)src, nx, ny, z0, z1, ring_view(p, r, zb), st));
    return OOC_OK;
}

ooc_status encode_from(ooc_plan *p, int f, int r, int64_t zb, char *dst, int64_t z0, int64_t z1, cudaStream_t st)
{
    const int64_t nx = p->cfg.nx, ny = p->cfg.ny;
    if (p->esize == 8)
        OOC_CUDA(launch_fr4d_encode(dcring(dring_view(p, r, zb)), nx, ny, z0, z1, p->rate[f], (uint32_t *)dst, st));
    else if (p->fmt[f] == OOC_FMT_FR4)
        OOC_CUDA(launch_fr4_encode(cring(ring_view(p, r, zb)), nx, ny, z0, z1, p->rate[f], (uint32_t *)dst, st));
    else
        OOC_CUDA(launch_bf16_pack_ring(cring(ring_view(p, r, zb)), nx, ny, z0, z1, (uint16_t *)dst, st));
    return OOC_OK;
}

// Ring holding field f's input level (heat: u -> ring 0; wave: p^t -> 0,
// p^{t-1} -> 1, kappa -> 2) and its output after a pass of kp steps.
int input_ring(const ooc_plan *, int f) { return f; }
int output_ring(const ooc_plan *p, int f, int64_t kp)
{
    if (f == 0)
        return (int)(stencil_launches(p, kp) & 1);  // launch j reads ring j&1, writes the other
    return (int)((kp + 1) & 1);  // wave p^{t+kp-1}
}

struct SlabGeom {
    int64_t a, b, in_lo, in_hi;
};

SlabGeom slab_geom(const ooc_plan *p, int64_t i, int64_t Wp)
{
    const int64_t nz = p->cfg.nz;
    SlabGeom g;
    g.a = i * p->T;
    g.b = g.a + p->T < nz ? g.a + p->T : nz;
    g.in_lo = i == 0 ? 0 : (g.a + Wp < nz ? g.a + Wp : nz);
    g.in_hi = g.b + Wp < nz ? g.b + Wp : nz;
    if (g.in_hi < g.in_lo)
        g.in_hi = g.in_lo;
    return g;
}

void step_window(const ooc_plan *p, int64_t i, int64_t kp, int64_t s, int64_t *lo, int64_t *hi)
{
    const int64_t nz = p->cfg.nz;
    const SlabGeom g = slab_geom(p, i, 0);
    int64_t l = i == 0 ? 0 : g.a + (kp - s) * p->h;
    int64_t u = i == p->nslab - 1 ? nz : g.b + (kp - s) * p->h;
    if (l > nz)
        l = nz;
    if (u > nz)
        u = nz;
    *lo = l;
    *hi = u;
}

// Enqueue the passes of ooc_step(nsteps) on the plan's three streams; the
// last D2H records p->ev_d2h[(*slabs - 1) % kEv].  Counters go to `st`.
ooc_status enqueue_steps(ooc_plan *p, int64_t nsteps, ooc_stats *st, int64_t *slabs)
{
    const int64_t nx = p->cfg.nx, ny = p->cfg.ny, nz = p->cfg.nz, k = p->cfg.k;
    const bool wave = p->cfg.stencil == OOC_WAVE25;
    const float r = (float)p->cfg.r;
    cudaStream_t sH = p->st[0], sC = p->st[1], sD = p->st[2];
    p->prof_used = 0;
    const int64_t npass = (nsteps + k - 1) / k;
    bool direct = false;  // some field lands in its ring without staging
    for (int f = 0; f < p->nfield; ++f)
        direct |= !staged(p, f);
    int64_t g = 0;  // slab visits in this call
    for (int64_t pass = 0; pass < npass; ++pass) {
        const int64_t kp = (pass + 1) * k <= nsteps ? k : nsteps - pass * k;
        const int64_t Wp = round4(kp * p->h);
        const int64_t zb = (pass * nz) % p->Z;
        const int64_t t0 = p->time + pass * k;
        for (int64_t i = 0; i < p->nslab; ++i, ++g) {
            const SlabGeom sg = slab_geom(p, i, Wp);
            const int e = (int)(g % kEv);
            p->prof_pass = pass;
            p->prof_slab = i;
            // ---- H2D: input units R_i and C_i (slab 0 also C_{-1}) -------------
            // FP32 fields land in the rings, whose slots slab g-2's D2H may
            // still read; staged fields land in staging buffer g&1, free
            // once slab g-2's decode has run (ev_dec below).
            int64_t need = direct ? g - 2 : -1;
            if (pass > 0 && sg.in_hi > sg.in_lo) {
                // the host units read here, [in_lo, in_hi), were written by
                // the previous pass's slabs up to the one holding plane
                // in_hi - 1: slab i + 1 when W <= T, further when W > T.  The
                // event ring holds the last kEv slabs, so an older slab is
                // covered by waiting for slab g-3 (the D2H stream runs in
                // order).
                const int64_t last = (sg.in_hi - 1) / p->T;
                const int64_t jl = last < p->nslab - 1 ? last : p->nslab - 1;
                int64_t gp = g - p->nslab + (jl - i);
                if (gp < g - 3)
                    gp = g - 3;
                if (gp > need)
                    need = gp;
            }
            if (need >= 0)
                OOC_CUDA(cudaStreamWaitEvent(sH, p->ev_d2h[need % kEv], 0));
            if (g >= 2)
                OOC_CUDA(cudaStreamWaitEvent(sH, p->ev_dec[(g - 2) % kEv], 0));
            if (sg.in_hi > sg.in_lo) {
                size_t pi;
                OOC_TRY(prof_begin(p, sH, 3, &pi));
                for (int f = 0; f < p->nfield; ++f) {
                    char *src = p->host + p->off_host[f] + (size_t)sg.in_lo * p->fplane[f];
                    const size_t nb = (size_t)(sg.in_hi - sg.in_lo) * p->fplane[f];
                    // the units lie in the field's host image, 4-aligned, and
                    // fit the staging buffer (FP32: the ring)
                    OOC_TRY(expect(p, sg.in_lo >= 0 && sg.in_hi <= nz && sg.in_lo % 4 == 0 && sg.in_hi % 4 == 0 &&
                                          (staged(p, f) ? nb <= p->in_bytes_field[f]
                                                        : sg.in_hi - sg.in_lo <= p->Z)));
                    if (staged(p, f))
                        OOC_CUDA(cudaMemcpyAsync(p->dev + p->off_in[g & 1][f], src, nb, cudaMemcpyHostToDevice, sH));
                    else
                        OOC_CUDA(copy_ring(p, input_ring(p, f), zb, sg.in_lo, sg.in_hi, src, true, sH));
                    st->h2d_bytes += (int64_t)nb;
                }
                OOC_TRY(prof_end(p, sH, pi));
            }
            OOC_CUDA(cudaEventRecord(p->ev_h2d[e], sH));

            // ---- compute: decode, k stencil steps, encode ---------------------
            OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_h2d[e], 0));
            if (sg.in_hi > sg.in_lo) {
                for (int f = 0; f < p->nfield; ++f) {
                    if (!staged(p, f))
                        continue;
                    size_t pi;
                    OOC_TRY(prof_begin(p, sC, 0, &pi));
                    OOC_TRY(decode_into(p, f, p->dev + p->off_in[g & 1][f], input_ring(p, f), zb, sg.in_lo,
                                        sg.in_hi, sC));
                    OOC_TRY(prof_end(p, sC, pi));
                    st->kernel_launches++;
                }
            }
            OOC_CUDA(cudaEventRecord(p->ev_dec[e], sC));
            // one event pair around the slab's stencil launches (events
            // between consecutive kernels would keep them from overlapping)
            size_t pst = (size_t)-1;
            int nst = 0;
            for (int64_t s = 1, j = 0; s <= kp; ++j) {
                // launch j: steps s (and s+1 when paired), ring j&1 -> the other
                const int64_t len = p->spl == 2 && s + 1 <= kp ? 2 : 1;
                int64_t lo, hi;
                step_window(p, i, kp, s + len - 1, &lo, &hi);
                if (hi <= lo) {
                    s += len;
                    continue;
                }
                // the planes a launch reads (h beyond its window on each side)
                // and the 2h below it that the next level needs fit the ring
                OOC_TRY(expect(p, lo >= 0 && hi <= nz && (hi - lo) + 2 * p->h <= p->Z));
                if (nst++ == 0)
                    OOC_TRY(prof_begin(p, sC, 1, &pst));
                if (p->esize == 8 && !wave) {
                    OOC_CUDA(launch_heat7_f64_ring(dcring(dring_view(p, (int)(j & 1), zb)),
                                                   dring_view(p, (int)((j + 1) & 1), zb), nx, ny, nz, lo, hi, p->cfg.r,
                                                   sC));
                } else if (!wave && len == 2) {
                    // level s on [lo_s, hi_s) stays on chip; its 2h planes
                    // below lo_s come from slab i-1's band, its top 2h
                    // planes go to this slab's band
                    int64_t lo_s, hi_s;
                    step_window(p, i, kp, s, &lo_s, &hi_s);
                    const float *bin = i > 0 ? band(p, j, (i - 1) & 1) : nullptr;
                    float *bout = i + 1 < p->nslab ? band(p, j, i & 1) : nullptr;
                    OOC_CUDA(launch_heat7x2(cring(ring_view(p, (int)(j & 1), zb)), ring_view(p, (int)((j + 1) & 1), zb),
                                            nx, ny, nz, lo, hi, lo_s, hi_s, bin, lo_s - 2 * p->h, bout,
                                            hi_s - 2 * p->h, r, sC));
                } else if (!wave) {
                    OOC_CUDA(launch_heat7(cring(ring_view(p, (int)(j & 1), zb)), ring_view(p, (int)((j + 1) & 1), zb),
                                          nx, ny, nz, lo, hi, r, sC));
                } else {
                    const int64_t n = t0 + s - 1;  // computing p^{n+1}
                    WaveSrcTable tab{};
                    bool src;
                    if (p->src_uploaded) {  // amplitude read on the device: the launch is time-invariant
                        tab = WaveSrcTable{dev_src(p), dev_time(p), pass * k + s - 1, (int64_t)p->w.size()};
                        src = p->sx >= 0 && p->sz >= lo && p->sz < hi;
                    } else {
                        src = p->sx >= 0 && n < (int64_t)p->w.size() && p->sz >= lo && p->sz < hi;
                    }
                    if (p->esize == 8)
                        OOC_CUDA(launch_wave25_f64(dcring(dring_view(p, (int)((s - 1) & 1), zb)),
                                                   dring_view(p, (int)(s & 1), zb), dcring(dring_view(p, 2, zb)), nx,
                                                   ny, nz, lo, hi, src ? p->sx : -1, p->sy, p->sz,
                                                   src && !p->src_uploaded ? (double)p->w[n] : 0.0, sC, tab));
                    else
                        OOC_CUDA(launch_wave25(cring(ring_view(p, (int)((s - 1) & 1), zb)),
                                               ring_view(p, (int)(s & 1), zb), cring(ring_view(p, 2, zb)), nx, ny, nz,
                                               lo, hi, src ? p->sx : -1, p->sy, p->sz,
                                               src && !p->src_uploaded ? p->w[n] : 0.0f, sC, tab));
                }
                st->kernel_launches++;
                s += len;
            }
            if (nst > 0) {
                OOC_TRY(prof_end(p, sC, pst));
                if (pst != (size_t)-1)
                    p->prof[pst].count = nst;
            }
            bool any_enc = false;
            for (int f = 0; f < p->nrw; ++f)
                any_enc |= staged(p, f);
            if (any_enc && g >= 2)
                OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_d2h[(g - 2) % kEv], 0));
            for (int f = 0; f < p->nrw; ++f) {
                if (!staged(p, f))
                    continue;
                OOC_TRY(expect(p, sg.a % 4 == 0 && sg.b % 4 == 0 && sg.b <= nz &&
                                      (size_t)(sg.b - sg.a) * p->fplane[f] <= p->out_bytes_field[f]));
                size_t pi;
                OOC_TRY(prof_begin(p, sC, 2, &pi));
                OOC_TRY(encode_from(p, f, output_ring(p, f, kp), zb, p->dev + p->off_out[g & 1][f], sg.a, sg.b,
                                    sC));
                OOC_TRY(prof_end(p, sC, pi));
                st->kernel_launches++;
            }
            OOC_CUDA(cudaEventRecord(p->ev_comp[e], sC));

            // ---- D2H: units C_{i-1} and R_i ---------------------------------
            OOC_CUDA(cudaStreamWaitEvent(sD, p->ev_comp[e], 0));
            {
                size_t pi;
                OOC_TRY(prof_begin(p, sD, 4, &pi));
                for (int f = 0; f < p->nrw; ++f) {
                    char *dst = p->host + p->off_host[f] + (size_t)sg.a * p->fplane[f];
                    const size_t nb = (size_t)(sg.b - sg.a) * p->fplane[f];
                    if (staged(p, f))
                        OOC_CUDA(cudaMemcpyAsync(dst, p->dev + p->off_out[g & 1][f], nb, cudaMemcpyDeviceToHost, sD));
                    else
                        OOC_CUDA(copy_ring(p, output_ring(p, f, kp), zb, sg.a, sg.b, dst, false, sD));
                    st->d2h_bytes += (int64_t)nb;
                }
                OOC_TRY(prof_end(p, sD, pi));
            }
            OOC_CUDA(cudaEventRecord(p->ev_d2h[e], sD));
            st->slabs++;
        }
        st->passes++;
    }
    // the plan's time on the device advances with the call (read by the
    // table-driven source of the wave kernel)
    OOC_CUDA(launch_add_time(dev_time(p), nsteps, sC));
    *slabs = g;
    return OOC_OK;
}

ooc_status ensure_graph_events(ooc_plan *p)
{
    cudaEvent_t *evs[] = {&p->ev_fork,    &p->ev_join[0], &p->ev_join[1], &p->ev_done,
                          &p->ev_tail[0], &p->ev_tail[1], &p->ev_tail[2]};
    for (cudaEvent_t *e : evs)
        if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
            *e = nullptr;
            return OOC_E_CUDA;
        }
    return OOC_OK;
}

// A call that returned OOC_E_TIMEOUT left its copies and kernels queued.  A
// later call that reads or writes the host image or the rings starts only
// once the plan's three streams have drained, under the same deadline as
// every host wait (OOC_E_TIMEOUT again if they have not).  Streams that are
// idle, the normal case, cost three event records.
ooc_status drain(ooc_plan *p)
{
    OOC_TRY(ensure_graph_events(p));
    for (int i = 0; i < 3; ++i)
        OOC_CUDA(cudaEventRecord(p->ev_tail[i], p->st[i]));
    for (int i = 0; i < 3; ++i)
        OOC_TRY(wait_event(p, p->ev_tail[i]));
    return OOC_OK;
}

ooc_status check_guards(ooc_plan *p)
{
    if (!p->cfg.debug_checks)
        return OOC_OK;
    GuardList g{};
    if (p->guards.size() > (size_t)kMaxGuards)
        return OOC_E_INVALID;
    g.n = (int)p->guards.size();
    for (int i = 0; i < g.n; ++i)
        g.off[i] = p->guards[(size_t)i];
    OOC_TRY(ensure_graph_events(p));
    cudaStream_t sC = p->st[1];
    check_guards_kernel<<<g.n, (unsigned)(kGuard / 4), 0, sC>>>((const unsigned char *)p->dev, g,
                                                                 (int *)(p->dev + p->off_flag));
    OOC_CUDA(cudaGetLastError());
    OOC_CUDA(cudaEventRecord(p->ev_done, sC));
    OOC_TRY(wait_event(p, p->ev_done));
    int flag = 0;
    OOC_CUDA(cudaMemcpy(&flag, p->dev + p->off_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 1)
        return OOC_E_CORRUPT;
    if (flag & 2) {  // a non-finite input value (ooc_set_field): reported once
        OOC_CUDA(cudaMemset(p->dev + p->off_flag, 0, sizeof(int)));
        return OOC_E_INVALID;
    }
    return OOC_OK;
}

void drop_graph(ooc_plan *p)
{
    if (p->graph)
        cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
    p->graph_nsteps = 0;
}

// Capture ooc_step(nsteps) into p->graph: the compute stream forks to the
// copy streams and joins them back, so one launch on it replays the call.
ooc_status capture_graph(ooc_plan *p, int64_t nsteps)
{
    drop_graph(p);
    OOC_TRY(ensure_graph_events(p));
    cudaStream_t sH = p->st[0], sC = p->st[1], sD = p->st[2];
    OOC_CUDA(cudaStreamBeginCapture(sC, cudaStreamCaptureModeThreadLocal));
    ooc_stats delta{};
    int64_t slabs = 0;
    ooc_status s = OOC_OK;
    if (cudaEventRecord(p->ev_fork, sC) != cudaSuccess || cudaStreamWaitEvent(sH, p->ev_fork, 0) != cudaSuccess ||
        cudaStreamWaitEvent(sD, p->ev_fork, 0) != cudaSuccess)
        s = OOC_E_CUDA;
    if (s == OOC_OK)
        s = enqueue_steps(p, nsteps, &delta, &slabs);
    if (s == OOC_OK &&
        (cudaEventRecord(p->ev_join[0], sH) != cudaSuccess || cudaEventRecord(p->ev_join[1], sD) != cudaSuccess ||
         cudaStreamWaitEvent(sC, p->ev_join[0], 0) != cudaSuccess ||
         cudaStreamWaitEvent(sC, p->ev_join[1], 0) != cudaSuccess))
        s = OOC_E_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(sC, &graph);
    if (s == OOC_OK && e != cudaSuccess)
        s = OOC_E_CUDA;
    if (s == OOC_OK && cudaGraphInstantiate(&p->graph, graph, 0) != cudaSuccess) {
        p->graph = nullptr;
        s = OOC_E_CUDA;
    }
    if (graph)
        cudaGraphDestroy(graph);
    if (s != OOC_OK) {
        cudaGetLastError();
        drop_graph(p);
        return s;
    }
    p->graph_nsteps = nsteps;
    p->graph_delta = delta;
    return OOC_OK;
}

void add_counters(ooc_stats *to, const ooc_stats &d)
{
    to->passes += d.passes;
    to->slabs += d.slabs;
    to->h2d_bytes += d.h2d_bytes;
    to->d2h_bytes += d.d2h_bytes;
    to->kernel_launches += d.kernel_launches;
}

}  // namespace

extern "C" {

ooc_status ooc_plan_create(const ooc_config *cfg, ooc_plan **out, size_t *device_bytes, size_t *host_bytes)
{
    if (!cfg || !out)
        return OOC_E_INVALID;
    *out = nullptr;
    const ooc_config c = *cfg;
    if (c.nx <= 0 || c.ny <= 0 || c.nz <= 0 || c.nx % 4 || c.ny % 4 || c.nz % 4 || c.nx > (1 << 20) ||
        c.ny > (1 << 20) || c.nz > (1 << 20) || c.k < 1 || c.k > 4096)
        return OOC_E_INVALID;
    if (c.stencil != OOC_HEAT7 && c.stencil != OOC_WAVE25)
        return OOC_E_INVALID;
    if (c.precision != OOC_PREC_FP32 && c.precision != OOC_PREC_FP64)
        return OOC_E_INVALID;
    const bool f64 = c.precision == OOC_PREC_FP64;
    auto fmt_ok = [f64](int f, int r) {
        if (f == OOC_FMT_FR4)
            return r >= 1 && r <= 64;
        return f64 ? f == OOC_FMT_FP64 : (f == OOC_FMT_FP32 || f == OOC_FMT_BF16);
    };
    if (!fmt_ok(c.rw_format, c.rw_rate) || (c.stencil == OOC_WAVE25 && !fmt_ok(c.ro_format, c.ro_rate)))
        return OOC_E_INVALID;
    if (c.slab_planes < 0 || c.slab_planes % 4 || c.device_budget_bytes < 0)
        return OOC_E_INVALID;
    if (c.graph_mode < 0 || c.graph_mode > 1)
        return OOC_E_INVALID;
    if (c.heat_steps_per_launch < 0 || c.heat_steps_per_launch > 2 ||
        ((c.stencil == OOC_WAVE25 || f64) && c.heat_steps_per_launch > 1))
        return OOC_E_INVALID;
    ooc_plan *p = new (std::nothrow) ooc_plan();
    if (!p)
        return OOC_E_ALLOC;
    p->cfg = c;
    p->h = c.stencil == OOC_HEAT7 ? 1 : 4;
    // heat7 runs the k steps of a pass as fused pairs unless one step per
    // launch is asked for (heat_steps_per_launch = 1) or k = 1
    p->spl = !f64 && c.stencil == OOC_HEAT7 &&
                     (c.heat_steps_per_launch == 2 || (c.heat_steps_per_launch == 0 && c.k >= 2))
                 ? 2
                 : 1;
    p->esize = f64 ? 8 : 4;
    p->W = round4((int64_t)c.k * p->h);
    p->nrw = c.stencil == OOC_HEAT7 ? 1 : 2;
    p->nfield = c.stencil == OOC_HEAT7 ? 1 : 3;
    p->nring = c.stencil == OOC_HEAT7 ? 2 : 3;
    p->plane_elems = c.nx * c.ny;
    for (int f = 0; f < p->nfield; ++f) {
        const bool ro = f >= p->nrw;
        p->fmt[f] = ro ? c.ro_format : c.rw_format;
        p->rate[f] = ro ? c.ro_rate : c.rw_rate;
        p->fplane[f] = p->plane_elems * fmt_bits(p->fmt[f], p->rate[f]) / 8;
    }
    size_t off = 0;
    for (int f = 0; f < p->nfield; ++f) {
        p->off_host[f] = off;
        off += align256((size_t)p->fplane[f] * c.nz);
    }
    p->host_bytes = off;

    const int64_t nz = c.nz;
    int64_t T = 0;
    size_t bytes = 0;
    if (c.slab_planes > 0) {
        T = c.slab_planes < nz ? c.slab_planes : nz;
        bytes = layout(p, T);
        if (c.device_budget_bytes > 0 && bytes > (size_t)c.device_budget_bytes) {
            delete p;
            return OOC_E_BUDGET;
        }
    } else {
        if (c.device_budget_bytes <= 0) {
            delete p;
            return OOC_E_INVALID;
        }
        for (int64_t t = 4; t <= nz; t += 4) {
            const size_t b = layout(p, t);
            if (b > (size_t)c.device_budget_bytes)
                break;
            T = t;
        }
        if (T == 0) {
            delete p;
            return OOC_E_BUDGET;
        }
        bytes = layout(p, T);
    }
    p->T = T;
    p->nslab = (nz + T - 1) / T;
    p->dev_bytes = bytes;
    *out = p;
    if (device_bytes)
        *device_bytes = p->dev_bytes;
    if (host_bytes)
        *host_bytes = p->host_bytes;
    return OOC_OK;
}

ooc_status ooc_plan_get_info(const ooc_plan *p, ooc_plan_info *info)
{
    if (!p || !info)
        return OOC_E_INVALID;
    info->slab_planes = p->T;
    info->nslab = p->nslab;
    info->common_planes = p->W;
    info->halo = p->h;
    info->ring_planes = p->Z;
    info->nrings = p->nring;
    info->device_bytes = (int64_t)p->dev_bytes;
    info->host_bytes = (int64_t)p->host_bytes;
    info->staging_in_bytes = (int64_t)p->in_bytes_field[0];
    info->staging_out_bytes = (int64_t)p->out_bytes_field[0];
    return OOC_OK;
}

ooc_status ooc_plan_bind(ooc_plan *p, void *device_arena, size_t device_bytes, void *host_arena, size_t host_bytes,
                         void *const streams[3])
{
    if (!p || !device_arena || !host_arena || !streams || device_bytes < p->dev_bytes ||
        host_bytes < p->host_bytes || ((uintptr_t)device_arena % 256) || ((uintptr_t)host_arena % 16))
        return OOC_E_INVALID;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host_arena) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return OOC_E_INVALID;  // host arena must be pinned (page-locked) memory
    }
    if (cudaPointerGetAttributes(&at, device_arena) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return OOC_E_INVALID;
    }
    if (!p->events_made) {
        for (int i = 0; i < kEv; ++i) {
            if (cudaEventCreateWithFlags(&p->ev_h2d[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_dec[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_comp[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_d2h[i], cudaEventDisableTiming) != cudaSuccess)
                return OOC_E_CUDA;
        }
        p->events_made = true;
    }
    p->dev = (char *)device_arena;
    p->host = (char *)host_arena;
    for (int i = 0; i < 3; ++i)
        p->st[i] = (cudaStream_t)streams[i];
    drop_graph(p);
    p->src_uploaded = false;
    // stream-ordered on the compute stream: after the last kernel of any
    // earlier call on it (which may still advance the device time)
    if (cudaMemcpyAsync(dev_time(p), &p->time, sizeof(int64_t), cudaMemcpyHostToDevice, p->st[1]) != cudaSuccess)
        return OOC_E_CUDA;
    OOC_TRY(arm_guards(p));
    p->bound = true;
    return OOC_OK;
}

ooc_status ooc_set_source(ooc_plan *p, int64_t sx, int64_t sy, int64_t sz, const float *w, int64_t nw)
{
    if (!p || nw < 0 || (nw > 0 && !w))
        return OOC_E_INVALID;
    drop_graph(p);
    p->src_uploaded = false;
    if (nw == 0) {
        p->sx = p->sy = p->sz = -1;
        p->w.clear();
        return OOC_OK;
    }
    if (p->cfg.stencil != OOC_WAVE25 || sx < 0 || sy < 0 || sz < 0 || sx >= p->cfg.nx || sy >= p->cfg.ny ||
        sz >= p->cfg.nz)
        return OOC_E_INVALID;
    try {
        p->w.assign(w, w + nw);
    } catch (...) {
        return OOC_E_ALLOC;
    }
    p->sx = sx;
    p->sy = sy;
    p->sz = sz;
    return OOC_OK;
}

}  // extern "C"

namespace {

// ooc_set_field / ooc_set_field64: host_src holds nx*ny*nz values of the
// plan's precision.
// debug_checks on fields stored raw: every value finite (FP32 or FP64)
bool all_finite(const void *src, int64_t n, int esize)
{
    if (esize == 8) {
        const double *d = (const double *)src;
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(d[i]))
                return false;
        return true;
    }
    const float *f = (const float *)src;
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(f[i]))
            return false;
    return true;
}

ooc_status set_field_impl(ooc_plan *p, int field, const void *host_src)
{
    if (!p || !p->bound || !host_src || field < 0 || field >= p->nfield)
        return OOC_E_INVALID;
    OOC_TRY(drain(p));
    const int64_t nz = p->cfg.nz;
    const size_t pb = (size_t)p->plane_elems * p->esize;
    char *img = p->host + p->off_host[field];
    if (!staged(p, field)) {
        if (p->cfg.debug_checks && !all_finite(host_src, p->plane_elems * nz, p->esize))
            return OOC_E_INVALID;
        std::memcpy(img, host_src, pb * nz);
        return OOC_OK;
    }
    // Slab j lands in ring j&1 (H2D stream), is encoded into staging buffer
    // j&1 (compute stream) and copied to the host image (D2H stream), so
    // the three overlap across slabs; events guard the reuse of ring and
    // staging buffer j&1 by slab j+2.
    cudaStream_t sH = p->st[0], sC = p->st[1], sD = p->st[2];
    int64_t j = 0;
    for (int64_t z0 = 0; z0 < nz; z0 += p->T, ++j) {
        const int64_t z1 = z0 + p->T < nz ? z0 + p->T : nz;
        const int64_t zb = (p->Z - z0 % p->Z) % p->Z;  // plane z0 -> slot 0
        const int b = (int)(j & 1);
        const int e = (int)(j % kEv), e2 = (int)((j + kEv - 2) % kEv);
        if (j >= 2)
            OOC_CUDA(cudaStreamWaitEvent(sH, p->ev_comp[e2], 0));
        OOC_CUDA(copy_ring(p, b, zb, z0, z1, (char *)host_src + (size_t)z0 * pb, true, sH));
        OOC_CUDA(cudaEventRecord(p->ev_h2d[e], sH));
        OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_h2d[e], 0));
        if (j >= 2)
            OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_d2h[e2], 0));
        if (p->cfg.debug_checks) {  // the slab fills ring slots 0 .. z1 - z0 - 1
            check_finite_kernel<<<152 * 4, 256, 0, sC>>>((const uint32_t *)(p->dev + p->off_ring[b]),
                                                         (z1 - z0) * (int64_t)(pb / 4), p->esize / 4,
                                                         (int *)(p->dev + p->off_flag));
            OOC_CUDA(cudaGetLastError());
        }
        char *stage = p->dev + p->off_in[b][field];
        OOC_TRY(encode_from(p, field, b, zb, stage, z0, z1, sC));
        OOC_CUDA(cudaEventRecord(p->ev_comp[e], sC));
        OOC_CUDA(cudaStreamWaitEvent(sD, p->ev_comp[e], 0));
        OOC_CUDA(cudaMemcpyAsync(img + (size_t)z0 * p->fplane[field], stage, (size_t)(z1 - z0) * p->fplane[field],
                                 cudaMemcpyDeviceToHost, sD));
        OOC_CUDA(cudaEventRecord(p->ev_d2h[e], sD));
    }
    OOC_TRY(wait_event(p, p->ev_d2h[(j - 1) % kEv]));
    return check_guards(p);
}

ooc_status get_field_impl(ooc_plan *p, int field, void *host_dst)
{
    if (!p || !p->bound || !host_dst || field < 0 || field >= p->nfield)
        return OOC_E_INVALID;
    OOC_TRY(drain(p));
    const int64_t nz = p->cfg.nz;
    const size_t pb = (size_t)p->plane_elems * p->esize;
    char *img = p->host + p->off_host[field];
    if (!staged(p, field)) {
        std::memcpy(host_dst, img, pb * nz);
        return OOC_OK;
    }
    // Mirror of ooc_set_field: H2D of slab j's storage into staging buffer
    // j&1, decode into ring j&1, D2H of the FP32 planes, overlapped.
    cudaStream_t sH = p->st[0], sC = p->st[1], sD = p->st[2];
    int64_t j = 0;
    for (int64_t z0 = 0; z0 < nz; z0 += p->T, ++j) {
        const int64_t z1 = z0 + p->T < nz ? z0 + p->T : nz;
        const int64_t zb = (p->Z - z0 % p->Z) % p->Z;
        const int b = (int)(j & 1);
        const int e = (int)(j % kEv), e2 = (int)((j + kEv - 2) % kEv);
        char *stage = p->dev + p->off_in[b][field];
        if (j >= 2)
            OOC_CUDA(cudaStreamWaitEvent(sH, p->ev_dec[e2], 0));
        OOC_CUDA(cudaMemcpyAsync(stage, img + (size_t)z0 * p->fplane[field], (size_t)(z1 - z0) * p->fplane[field],
                                 cudaMemcpyHostToDevice, sH));
        OOC_CUDA(cudaEventRecord(p->ev_h2d[e], sH));
        OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_h2d[e], 0));
        if (j >= 2)
            OOC_CUDA(cudaStreamWaitEvent(sC, p->ev_d2h[e2], 0));
        OOC_TRY(decode_into(p, field, stage, b, zb, z0, z1, sC));
        OOC_CUDA(cudaEventRecord(p->ev_dec[e], sC));
        OOC_CUDA(cudaStreamWaitEvent(sD, p->ev_dec[e], 0));
        OOC_CUDA(copy_ring(p, b, zb, z0, z1, (char *)host_dst + (size_t)z0 * pb, false, sD));
        OOC_CUDA(cudaEventRecord(p->ev_d2h[e], sD));
    }
    OOC_TRY(wait_event(p, p->ev_d2h[(j - 1) % kEv]));
    return check_guards(p);
}

}  // namespace

extern "C" {

ooc_status ooc_set_field(ooc_plan *p, int field, const float *host_src)
{
    if (!p || p->esize != 4)
        return OOC_E_INVALID;
    return set_field_impl(p, field, host_src);
}

ooc_status ooc_get_field(ooc_plan *p, int field, float *host_dst)
{
    if (!p || p->esize != 4)
        return OOC_E_INVALID;
    return get_field_impl(p, field, host_dst);
}

ooc_status ooc_set_field64(ooc_plan *p, int field, const double *host_src)
{
    if (!p || p->esize != 8)
        return OOC_E_INVALID;
    return set_field_impl(p, field, host_src);
}

ooc_status ooc_get_field64(ooc_plan *p, int field, double *host_dst)
{
    if (!p || p->esize != 8)
        return OOC_E_INVALID;
    return get_field_impl(p, field, host_dst);
}

ooc_status ooc_step(ooc_plan *p, int64_t nsteps)
{
    if (!p || !p->bound || nsteps < 0)
        return OOC_E_INVALID;
    if (nsteps == 0)
        return OOC_OK;
    const auto t_start = std::chrono::steady_clock::now();
    OOC_TRY(drain(p));
    p->prof_used = 0;
    p->trace.clear();
    // A call's launches depend only on nsteps (the wave's source amplitudes
    // are read on the device from a table, at the device copy of the plan's
    // time), so calls without per-launch profiling replay a captured graph.
    const bool wave = p->cfg.stencil == OOC_WAVE25;
    if (wave && p->sx >= 0 && !p->src_uploaded && (int64_t)p->w.size() <= kSrcTable) {
        // Stream-ordered on the compute stream: it lands after every kernel
        // of earlier calls that reads the table (even of a call that timed
        // out) and before every kernel of this one.  A copy from pageable
        // memory has taken its source when it returns, so nothing waits.
        OOC_CUDA(cudaMemcpyAsync(dev_src(p), p->w.data(), p->w.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 p->st[1]));
        p->src_uploaded = true;
        drop_graph(p);
    }
    const bool graphed = !p->cfg.profile && p->cfg.graph_mode == 0 && (!wave || p->sx < 0 || p->src_uploaded);
    cudaEvent_t last = nullptr;
    if (graphed) {
        if (!p->graph || p->graph_nsteps != nsteps)
            OOC_TRY(capture_graph(p, nsteps));
        OOC_CUDA(cudaGraphLaunch(p->graph, p->st[1]));
        OOC_CUDA(cudaEventRecord(p->ev_done, p->st[1]));
        add_counters(&p->stats, p->graph_delta);
        last = p->ev_done;
    } else {
        ooc_stats delta{};
        int64_t g = 0;
        OOC_TRY(enqueue_steps(p, nsteps, &delta, &g));
        add_counters(&p->stats, delta);
        last = p->ev_d2h[(g - 1) % kEv];
    }
    // Every pass is enqueued, and the device copy of the time advances with
    // the call's last kernel, so the host time and the step count advance
    // now: a call whose wait below times out has still done its steps once
    // the streams drain, and the next call (or a rebind, which copies the
    // host time to the device) continues from the right time.
    p->time += nsteps;
    p->stats.steps_done += nsteps;
    OOC_TRY(wait_event(p, last));
    // a kernel whose bounded wait gave up left planes unwritten
    unsigned fault = 0u;
    OOC_CUDA(take_stencil_fault(&fault));
    if (fault)
        return OOC_E_TIMEOUT;
    if (p->cfg.profile) {
        try {
            p->trace.reserve(p->prof_used);
        } catch (...) {
            return OOC_E_ALLOC;
        }
        for (size_t j = 0; j < p->prof_used; ++j) {
            float ms = 0.0f, t0 = 0.0f, t1 = 0.0f;
            OOC_CUDA(cudaEventElapsedTime(&ms, p->prof[j].a, p->prof[j].b));
            OOC_CUDA(cudaEventElapsedTime(&t0, p->prof[0].a, p->prof[j].a));
            OOC_CUDA(cudaEventElapsedTime(&t1, p->prof[0].a, p->prof[j].b));
            p->trace.push_back(ooc_trace_rec{p->prof[j].kind, p->prof[j].count, p->prof[j].pass, p->prof[j].slab,
                                             (double)t0, (double)t1});
            switch (p->prof[j].kind) {
            case 0: p->stats.ms_decode += ms; p->stats.n_decode++; break;
            case 1: p->stats.ms_stencil += ms; p->stats.n_stencil += p->prof[j].count; break;
            case 2: p->stats.ms_encode += ms; p->stats.n_encode++; break;
            case 3: p->stats.ms_h2d += ms; p->stats.n_h2d++; break;
            default: p->stats.ms_d2h += ms; p->stats.n_d2h++; break;
            }
        }
    }
    p->stats.ms_last_step =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return check_guards(p);
}

ooc_status ooc_get_stats(const ooc_plan *p, ooc_stats *s)
{
    if (!p || !s)
        return OOC_E_INVALID;
    *s = p->stats;
    return OOC_OK;
}

ooc_status ooc_reset_stats(ooc_plan *p)
{
    if (!p)
        return OOC_E_INVALID;
    const int64_t steps = p->stats.steps_done;
    p->stats = ooc_stats{};
    p->stats.steps_done = steps;
    return OOC_OK;
}

ooc_status ooc_plan_set_wait_timeout(ooc_plan *p, int64_t wait_timeout_ms)
{
    if (!p || wait_timeout_ms < 0)
        return OOC_E_INVALID;
    p->cfg.wait_timeout_ms = wait_timeout_ms;
    return OOC_OK;
}

ooc_status ooc_plan_get_trace(const ooc_plan *p, ooc_trace_rec *out, int64_t cap, int64_t *n)
{
    if (!p || !n || cap < 0 || (cap > 0 && !out))
        return OOC_E_INVALID;
    const int64_t have = (int64_t)p->trace.size();
    for (int64_t j = 0; j < have && j < cap; ++j)
        out[j] = p->trace[(size_t)j];
    *n = have;
    return OOC_OK;
}

ooc_status ooc_plan_set_profile(ooc_plan *p, int profile)
{
    if (!p || (profile != 0 && profile != 1))
        return OOC_E_INVALID;
    p->cfg.profile = profile;
    return OOC_OK;
}

void ooc_plan_destroy(ooc_plan *p)
{
    if (!p)
        return;
    if (p->events_made) {
        for (int i = 0; i < kEv; ++i) {
            cudaEventDestroy(p->ev_h2d[i]);
            cudaEventDestroy(p->ev_dec[i]);
            cudaEventDestroy(p->ev_comp[i]);
            cudaEventDestroy(p->ev_d2h[i]);
        }
    }
    for (auto &pp : p->prof) {
        cudaEventDestroy(pp.a);
        cudaEventDestroy(pp.b);
    }
    drop_graph(p);
    for (cudaEvent_t e : {p->ev_fork, p->ev_join[0], p->ev_join[1], p->ev_done, p->ev_tail[0], p->ev_tail[1],
                          p->ev_tail[2]})
        if (e)
            cudaEventDestroy(e);
    delete p;
}

}  // extern "C"
