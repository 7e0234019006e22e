/*
 * oracle/codec.c -- TEST INFRASTRUCTURE ONLY.  Serial CPU reference of the
 * fixed-rate 4x4x4 block codec ("FR4") that stores FP32 slabs at R bits per
 * value.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg and reference arm may load it; the product path never does.
 *
 * The paper (Section IV) picks a fixed-rate lossy codec in the cuZFP family
 * because the user fixes the bits kept per value (so "32 bits per double"
 * gives 2:1) and the compressed size is therefore known in advance, letting
 * device buffers be preallocated.  The paper does not define the codec
 * itself.  FR4 is defined here, one step at a time, following the published
 * fixed-rate method of Lindstrom ("Fixed-Rate Compressed Floating-Point
 * Arrays", IEEE TVCG 2014): block floating point, a decorrelating integer
 * transform, sequency reordering, negabinary, and embedded bit-plane coding
 * with group tests.  The transform is this project's own reversible
 * lifting (S-transform pairs plus a linear-trend prediction, in the manner
 * of Said and Pearlman's S+P transform), not ZFP's.  This file is the
 * definition that the GPU codec must match bit for bit.
 *
 * Stream layout: a field of nx*ny*nz values (x fastest) is cut into 4^3
 * blocks ordered bx fastest, then by, then bz.  Each block
 * takes exactly B = 64*R bits = 2*R 32-bit little-endian words.  Bit j of a
 * block is bit (j mod 32) of its word j/32; multi-bit fields are written
 * least-significant bit first.
 *
 * Steps for one block x[64], index x + 4y + 16z:
 *  1. emax = max over nonzero values of the frexp exponent, clamped below
 *     at -126.  No nonzero value: write a single 0 bit, rest zero.
 *     Otherwise write a 1 bit and 8 bits of (emax + 127).
 *  2. q_i = trunc(x_i * 2^(26 - emax)), an exact int32 with |q_i| < 2^26.
 *  3. Forward lifting on every line of 4 along x, then y, then z:
 *        d0 = a0 - a1; s0 = a1 + floor(d0/2)
 *        d1 = a2 - a3; s1 = a3 + floor(d1/2)
 *        D  = s0 - s1; S  = s1 + floor(D/2)
 *        d0 -= floor(D/2); d1 -= floor(D/2)
 *        line := (S, D, d0, d1)
 *     Arithmetic is wrapping int32; floor(v/2) is the arithmetic shift.
 *     Every output satisfies |y| <= 2.5 M + 1.25 when |a| <= M, so three
 *     passes keep |coefficient| < 2^30 and nothing wraps on encode.
 *  4. Reorder coefficient (i,j,k) by key lev(i)+lev(j)+lev(k), ties by
 *     i + 4j + 16k, with lev = (0, 1, 2, 2).
 *  5. Negabinary: u = (q + 0xAAAAAAAA) ^ 0xAAAAAAAA in wrapping uint32.
 *  6. Bit planes p = 31 .. 0 within the B - 9 remaining bits; n counts
 *     coefficients already significant (a prefix of the order):
 *       - write bit p of u_0 .. u_{n-1};
 *       - while n < 64: write a group bit g = OR of bit p of u_n .. u_63;
 *         stop the plane if g == 0; else write bits p of u_n, u_{n+1}, ...
 *         advancing n after each, stopping after the first 1; when n
 *         reaches 63 in that scan, bit p of u_63 must be 1 and is not
 *         written (n becomes 64).
 *     Every write first checks the budget; coding stops the moment the
 *     budget is spent, possibly mid-plane.  Unwritten bits stay 0.
 * Decoding mirrors every step; bits never received read as 0.  The value
 * is rebuilt as RN_float( RN_float(q) * 2^(emax - 26) ).
 *
 * Partial blocks.  A field whose sides are not multiples of 4 is cut into
 * ceil(n/4) blocks per axis; a block reaching past the field takes, for
 * each missing point, the value of the nearest point inside the field
 * (each coordinate clamped to [0, n-1]).  Decoding writes only the points
 * inside the field.
 *
 * Variable-size modes (codec variants beyond the paper's fixed rate; the
 * paper names the comparison of other compressors as future work):
 *  - fixed precision P (1..32): planes 31 .. 32-P are coded, with no bit
 *    budget;
 *  - fixed accuracy tol > 0: planes 31 .. pmin are coded, with
 *    pmin = clamp(L - (emax - 26) - 4, 0, 32) and L = floor(log2 tol).  The
 *    dropped planes carry less than (2/3) 2^pmin in negabinary, and the
 *    inverse lifting amplifies a coefficient error by at most 2.25 per axis
 *    (its largest row sum), 11.4 in 3D; 2^(pmin + emax - 26) <= tol/16 keeps
 *    that part below tol/2.  Blocks whose pmin clamps to 0 are coded to
 *    full precision.
 * Each variable-size block starts on a 32-bit word and is padded with zero
 * bits to a whole word; block b occupies words [index[b], index[b+1]) of
 * the stream, index[0] = 0.  A block takes at most FR4_VAR_MAX_WORDS words:
 * 9 header bits and at most 129 bits per plane (n refinement bits, at most
 * 64 - n scan bits and 64 - n + 1 group bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FR4_PREC 26
#define FR4_PLANES 32
#define FR4_VAR_MAX_WORDS 130
#define FR4_MODE_RATE 0
#define FR4_MODE_PRECISION 1
#define FR4_MODE_ACCURACY 2

/* ---- bit stream with a hard budget ------------------------------------ */
typedef struct {
    uint32_t *w;   /* block words */
    int64_t pos;   /* next bit */
    int64_t end;   /* budget: bits [0, end) */
} bitstream;

/* Write one bit; returns 0 (and writes nothing) once the budget is spent. */
static int put_bit(bitstream *s, unsigned bit)
{
    if (s->pos >= s->end)
        return 0;
    if (bit & 1u)
        s->w[s->pos >> 5] |= 1u << (s->pos & 31);
    s->pos++;
    return 1;
}

/* Read one bit into *bit; returns 0 once the budget is spent. */
static int get_bit(bitstream *s, unsigned *bit)
{
    if (s->pos >= s->end)
        return 0;
    *bit = (s->w[s->pos >> 5] >> (s->pos & 31)) & 1u;
    s->pos++;
    return 1;
}

/* ---- step 1: exponent ---------------------------------------------------- */
static int value_exponent(float x)
{
    int e;
    frexpf(x, &e);
    return e < -126 ? -126 : e;
}

/* ---- step 3: lifting ----------------------------------------------------- */
/* All lifting arithmetic is two's-complement 32-bit: sums wrap modulo 2^32
 * and floor(v/2) is the arithmetic right shift.  For encoder input the range
 * bound guarantees that nothing wraps; `fr4_forward_wrapped` records any
 * wrap in the forward direction so that tests can check that claim.  The
 * inverse may wrap only on streams that no finite input produces. */
static _Thread_local int fr4_forward_wrapped;  /* per thread: the dense loops run blocks in parallel */
static _Thread_local int fr4_inverse_wrapped;

static int32_t wrap32(int64_t v, int *flag)
{
    if (v > INT32_MAX || v < INT32_MIN)
        *flag = 1;
    return (int32_t)(uint32_t)(uint64_t)v;
}

static int32_t floor_half(int32_t v) { return (int32_t)floor((double)v / 2.0); }

static void lift_forward(int32_t *a, int stride)
{
    int *w = &fr4_forward_wrapped;
    int32_t a0 = a[0], a1 = a[stride], a2 = a[2 * stride], a3 = a[3 * stride];
    int32_t d0 = wrap32((int64_t)a0 - a1, w);
    int32_t s0 = wrap32((int64_t)a1 + floor_half(d0), w);
    int32_t d1 = wrap32((int64_t)a2 - a3, w);
    int32_t s1 = wrap32((int64_t)a3 + floor_half(d1), w);
    int32_t D = wrap32((int64_t)s0 - s1, w);
    int32_t S = wrap32((int64_t)s1 + floor_half(D), w);
    d0 = wrap32((int64_t)d0 - floor_half(D), w);
    d1 = wrap32((int64_t)d1 - floor_half(D), w);
    a[0] = S;
    a[stride] = D;
    a[2 * stride] = d0;
    a[3 * stride] = d1;
}

static void lift_inverse(int32_t *a, int stride)
{
    int *w = &fr4_inverse_wrapped;
    int32_t S = a[0], D = a[stride], d0 = a[2 * stride], d1 = a[3 * stride];
    d0 = wrap32((int64_t)d0 + floor_half(D), w);
    d1 = wrap32((int64_t)d1 + floor_half(D), w);
    int32_t s1 = wrap32((int64_t)S - floor_half(D), w);
    int32_t s0 = wrap32((int64_t)s1 + D, w);
    int32_t a3 = wrap32((int64_t)s1 - floor_half(d1), w);
    int32_t a2 = wrap32((int64_t)a3 + d1, w);
    int32_t a1 = wrap32((int64_t)s0 - floor_half(d0), w);
    int32_t a0 = wrap32((int64_t)a1 + d0, w);
    a[0] = a0;
    a[stride] = a1;
    a[2 * stride] = a2;
    a[3 * stride] = a3;
}

static void transform_forward(int32_t *c)
{
    for (int z = 0; z < 4; z++)
        for (int y = 0; y < 4; y++)
            lift_forward(c + 4 * y + 16 * z, 1);
    for (int z = 0; z < 4; z++)
        for (int x = 0; x < 4; x++)
            lift_forward(c + x + 16 * z, 4);
    for (int y = 0; y < 4; y++)
        for (int x = 0; x < 4; x++)
            lift_forward(c + x + 4 * y, 16);
}

static void transform_inverse(int32_t *c)
{
    for (int y = 0; y < 4; y++)
        for (int x = 0; x < 4; x++)
            lift_inverse(c + x + 4 * y, 16);
    for (int z = 0; z < 4; z++)
        for (int x = 0; x < 4; x++)
            lift_inverse(c + x + 16 * z, 4);
    for (int z = 0; z < 4; z++)
        for (int y = 0; y < 4; y++)
            lift_inverse(c + 4 * y + 16 * z, 1);
}

/* ---- step 4: sequency order (plain selection by key) ---------------------- */
static int order_table[64];
static int order_ready;

static void build_order(void)
{
    static const int lev[4] = {0, 1, 2, 2};
    int used[64] = {0};
    for (int r = 0; r < 64; r++) {
        int best = -1, bestkey = 1 << 30;
        for (int l = 0; l < 64; l++) {
            if (used[l])
                continue;
            int key = (lev[l & 3] + lev[(l >> 2) & 3] + lev[l >> 4]) * 64 + l;
            if (key < bestkey) {
                bestkey = key;
                best = l;
            }
        }
        used[best] = 1;
        order_table[r] = best;
    }
    order_ready = 1;
}

/* ---- step 5: negabinary -------------------------------------------------- */
static uint32_t to_negabinary(int32_t q)
{
    return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}

static int32_t from_negabinary(uint32_t u)
{
    return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu);
}

/* ---- step 6: embedded bit-plane coding ----------------------------------- */
static void encode_planes(bitstream *s, const uint32_t *u, int pmin)
{
    int n = 0;
    for (int p = FR4_PLANES - 1; p >= pmin; p--) {
        for (int i = 0; i < n; i++)
            if (!put_bit(s, u[i] >> p))
                return;
        while (n < 64) {
            unsigned g = 0;
            for (int i = n; i < 64; i++)
                g |= (u[i] >> p) & 1u;
            if (!put_bit(s, g))
                return;
            if (!g)
                break;
            for (;;) {
                if (n == 63) { /* the last coefficient's one is implied */
                    n = 64;
                    break;
                }
                unsigned b = (u[n] >> p) & 1u;
                if (!put_bit(s, b))
                    return;
                n++;
                if (b)
                    break;
            }
        }
    }
}

static void decode_planes(bitstream *s, uint32_t *u, int pmin)
{
    int n = 0;
    unsigned b;
    for (int p = FR4_PLANES - 1; p >= pmin; p--) {
        for (int i = 0; i < n; i++) {
            if (!get_bit(s, &b))
                return;
            u[i] |= b << p;
        }
        while (n < 64) {
            if (!get_bit(s, &b))
                return;
            if (!b)
                break;
            for (;;) {
                if (n == 63) {
                    u[63] |= 1u << p;
                    n = 64;
                    break;
                }
                if (!get_bit(s, &b))
                    return;
                u[n] |= b << p;
                n++;
                if (b)
                    break;
            }
        }
    }
}

/* ---- one block ------------------------------------------------------------ */
/* Lowest coded plane of a block with exponent emax (step 6's range). */
static int plane_floor(int mode, double param, int emax)
{
    if (mode == FR4_MODE_PRECISION)
        return FR4_PLANES - (int)param;
    if (mode == FR4_MODE_ACCURACY) {
        int e;
        frexp(param, &e); /* param = m 2^e, m in [0.5, 1): floor(log2) = e - 1 */
        int pmin = (e - 1) - (emax - FR4_PREC) - 4;
        return pmin < 0 ? 0 : (pmin > FR4_PLANES ? FR4_PLANES : pmin);
    }
    return 0;
}

/* Encode block x[64] into s (words zeroed by the caller): steps 1-6 with
 * the plane range of `mode`.  Returns the bits written. */
static int64_t encode_block_mode(const float *x, bitstream *s, int mode, double param)
{
    int emax = INT32_MIN;
    for (int i = 0; i < 64; i++)
        if (x[i] != 0.0f) {
            int e = value_exponent(x[i]);
            if (e > emax)
                emax = e;
        }
    if (emax == INT32_MIN) {
        put_bit(s, 0);
        return s->pos;
    }
    put_bit(s, 1);
    for (int j = 0; j < 8; j++)
        put_bit(s, (unsigned)(emax + 127) >> j);
    int32_t q[64];
    for (int i = 0; i < 64; i++)
        q[i] = (int32_t)trunc(ldexp((double)x[i], FR4_PREC - emax));
    transform_forward(q);
    uint32_t u[64];
    for (int r = 0; r < 64; r++)
        u[r] = to_negabinary(q[order_table[r]]);
    encode_planes(s, u, plane_floor(mode, param, emax));
    return s->pos;
}

static void decode_block_mode(bitstream *s, float *x, int mode, double param)
{
    unsigned b = 0;
    get_bit(s, &b);
    if (!b) {
        for (int i = 0; i < 64; i++)
            x[i] = 0.0f;
        return;
    }
    int field = 0;
    for (int j = 0; j < 8; j++) {
        b = 0;
        get_bit(s, &b);
        field |= (int)b << j;
    }
    int emax = field - 127;
    uint32_t u[64] = {0};
    decode_planes(s, u, plane_floor(mode, param, emax));
    int32_t q[64];
    for (int r = 0; r < 64; r++)
        q[order_table[r]] = from_negabinary(u[r]);
    transform_inverse(q);
    for (int i = 0; i < 64; i++) {
        float f = (float)q[i];                            /* RN int -> float */
        x[i] = (float)((double)f * ldexp(1.0, emax - FR4_PREC)); /* one rounding */
    }
}

/* Fixed rate: block x[64] into words[0 .. 2R-1] (zeroed here). */
static void encode_block(const float *x, int rate, uint32_t *words)
{
    bitstream s = {words, 0, 64 * (int64_t)rate};
    memset(words, 0, sizeof(uint32_t) * 2 * (size_t)rate);
    encode_block_mode(x, &s, FR4_MODE_RATE, 0.0);
}

static void decode_block(const uint32_t *words, int rate, float *x)
{
    bitstream s = {(uint32_t *)words, 0, 64 * (int64_t)rate};
    decode_block_mode(&s, x, FR4_MODE_RATE, 0.0);
}

/* ---- exported API (ctypes) ----------------------------------------------- */
static int64_t nblocks(int64_t n) { return (n + 3) / 4; }

/* Returns the compressed byte count of an nx*ny*nz field at `rate`. */
int64_t fr4_compressed_bytes(int64_t nx, int64_t ny, int64_t nz, int rate)
{
    return nblocks(nx) * nblocks(ny) * nblocks(nz) * 8 * (int64_t)rate;
}

static int64_t clamp_index(int64_t i, int64_t n) { return i < n ? i : n - 1; }

/* Block (bx, by, bz) of the field, missing points taken from the nearest
 * point inside (partial blocks). */
static void gather_block(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t bx, int64_t by, int64_t bz,
                         float *x)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++) {
                int64_t z = clamp_index(4 * bz + k, nz), y = clamp_index(4 * by + j, ny);
                int64_t xx = clamp_index(4 * bx + i, nx);
                x[i + 4 * j + 16 * k] = f[(z * ny + y) * nx + xx];
            }
}

static void scatter_block(float *f, int64_t nx, int64_t ny, int64_t nz, int64_t bx, int64_t by, int64_t bz,
                          const float *x)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++) {
                int64_t z = 4 * bz + k, y = 4 * by + j, xx = 4 * bx + i;
                if (z < nz && y < ny && xx < nx)
                    f[(z * ny + y) * nx + xx] = x[i + 4 * j + 16 * k];
            }
}

/* Encode a dense field.  Returns 0, or -1 on bad arguments, or -2 if a
 * forward lifting value left int32 (which the range bound rules out). */
int fr4_encode(const float *field, int64_t nx, int64_t ny, int64_t nz, int rate, uint32_t *out)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || rate < 1 || rate > 64)
        return -1;
    if (!order_ready)
        build_order();
    int64_t nbx = nblocks(nx), nby = nblocks(ny), nbz = nblocks(nz);
    int wrapped = 0;
    /* blocks are independent: one block per iteration, any order */
#pragma omp parallel reduction(| : wrapped)
    {
        fr4_forward_wrapped = 0;
#pragma omp for collapse(3) schedule(static)
        for (int64_t bz = 0; bz < nbz; bz++)
            for (int64_t by = 0; by < nby; by++)
                for (int64_t bx = 0; bx < nbx; bx++) {
                    float x[64];
                    int64_t b = bx + nbx * (by + nby * bz);
                    gather_block(field, nx, ny, nz, bx, by, bz, x);
                    encode_block(x, rate, out + b * 2 * rate);
                }
        wrapped |= fr4_forward_wrapped;
    }
    fr4_forward_wrapped = wrapped;
    return wrapped ? -2 : 0;
}

/* Decode a dense field.  Returns 0, -1 on bad arguments, or 1 when the
 * inverse lifting wrapped (possible only for streams no input produces). */
int fr4_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t nz, int rate, float *field)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || rate < 1 || rate > 64)
        return -1;
    if (!order_ready)
        build_order();
    int64_t nbx = nblocks(nx), nby = nblocks(ny), nbz = nblocks(nz);
    int wrapped = 0;
    /* blocks are independent: one block per iteration, any order */
#pragma omp parallel reduction(| : wrapped)
    {
        fr4_inverse_wrapped = 0;
#pragma omp for collapse(3) schedule(static)
        for (int64_t bz = 0; bz < nbz; bz++)
            for (int64_t by = 0; by < nby; by++)
                for (int64_t bx = 0; bx < nbx; bx++) {
                    float x[64];
                    int64_t b = bx + nbx * (by + nby * bz);
                    decode_block(in + b * 2 * rate, rate, x);
                    scatter_block(field, nx, ny, nz, bx, by, bz, x);
                }
        wrapped |= fr4_inverse_wrapped;
    }
    fr4_inverse_wrapped = wrapped;
    return wrapped ? 1 : 0;
}

static int var_mode_ok(int mode, double param)
{
    if (mode == FR4_MODE_PRECISION)
        return param >= 1.0 && param <= 32.0 && param == floor(param);
    if (mode == FR4_MODE_ACCURACY)
        return param > 0.0 && isfinite(param);
    return 0;
}

/* Variable-size modes: encode into out (capacity cap_words >= blocks *
 * FR4_VAR_MAX_WORDS is always enough) and index[0 .. blocks].  Returns the
 * total words, or -1 on bad arguments / too small a capacity. */
int64_t fr4_encode_var(const float *field, int64_t nx, int64_t ny, int64_t nz, int mode, double param, uint32_t *out,
                       int64_t cap_words, uint64_t *index)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || !var_mode_ok(mode, param))
        return -1;
    if (!order_ready)
        build_order();
    int64_t nbx = nblocks(nx), nby = nblocks(ny), nbz = nblocks(nz);
    float x[64];
    uint32_t words[FR4_VAR_MAX_WORDS];
    int64_t at = 0;
    for (int64_t bz = 0; bz < nbz; bz++)
        for (int64_t by = 0; by < nby; by++)
            for (int64_t bx = 0; bx < nbx; bx++) {
                int64_t b = bx + nbx * (by + nby * bz);
                gather_block(field, nx, ny, nz, bx, by, bz, x);
                memset(words, 0, sizeof(words));
                bitstream s = {words, 0, 32 * FR4_VAR_MAX_WORDS};
                int64_t nw = (encode_block_mode(x, &s, mode, param) + 31) / 32;
                if (at + nw > cap_words)
                    return -1;
                index[b] = (uint64_t)at;
                memcpy(out + at, words, sizeof(uint32_t) * (size_t)nw);
                at += nw;
            }
    index[nbx * nby * nbz] = (uint64_t)at;
    return at;
}

/* Decode a variable-size stream with its index.  Returns 0 or -1. */
int fr4_decode_var(const uint32_t *in, const uint64_t *index, int64_t nx, int64_t ny, int64_t nz, int mode,
                   double param, float *field)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || !var_mode_ok(mode, param))
        return -1;
    if (!order_ready)
        build_order();
    int64_t nbx = nblocks(nx), nby = nblocks(ny), nbz = nblocks(nz);
    float x[64];
    for (int64_t bz = 0; bz < nbz; bz++)
        for (int64_t by = 0; by < nby; by++)
            for (int64_t bx = 0; bx < nbx; bx++) {
                int64_t b = bx + nbx * (by + nby * bz);
                int64_t nw = (int64_t)(index[b + 1] - index[b]);
                bitstream s = {(uint32_t *)(in + index[b]), 0, 32 * nw};
                decode_block_mode(&s, x, mode, param);
                scatter_block(field, nx, ny, nz, bx, by, bz, x);
            }
    return 0;
}

int64_t fr4_var_max_words_per_block(void) { return FR4_VAR_MAX_WORDS; }

/* Test hooks: the individual steps, exposed so that tests can pin each one. */
void fr4_lift_forward4(int32_t *a) { lift_forward(a, 1); }
void fr4_lift_inverse4(int32_t *a) { lift_inverse(a, 1); }
int fr4_transform_forward(int32_t *c) { fr4_forward_wrapped = 0; transform_forward(c); return fr4_forward_wrapped ? -2 : 0; }
int fr4_transform_inverse(int32_t *c) { fr4_inverse_wrapped = 0; transform_inverse(c); return fr4_inverse_wrapped ? 1 : 0; }
void fr4_order(int *out)
{
    if (!order_ready)
        build_order();
    memcpy(out, order_table, sizeof(order_table));
}
/* Plane coder on raw negabinary words u[64] with an explicit bit budget. */
int64_t fr4_encode_planes(const uint32_t *u, int64_t budget_bits, uint32_t *words)
{
    bitstream s = {words, 0, budget_bits};
    encode_planes(&s, u, 0);
    return s.pos;
}
int64_t fr4_decode_planes(const uint32_t *words, int64_t budget_bits, uint32_t *u)
{
    bitstream s = {(uint32_t *)words, 0, budget_bits};
    memset(u, 0, 64 * sizeof(uint32_t));
    decode_planes(&s, u, 0);
    return s.pos;
}
