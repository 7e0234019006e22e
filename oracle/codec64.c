/*
 * oracle/codec64.c -- TEST INFRASTRUCTURE ONLY.  Serial CPU reference of
 * FR4D, the fixed-rate 4x4x4 block codec for FP64 fields.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg and reference arm
 * may load it; the product path never does.
 *
 * The paper ran its wave fields in double precision and stored them at 32
 * and 24 of every 64 bits (Section VI, codes 2-4); Section IV asks for a
 * fixed-rate codec, so that the compressed size of every unit is known in
 * advance.  FR4D is FR4 (codec.c) carried over to 64-bit values, following
 * the same published fixed-rate method (Lindstrom, IEEE TVCG 2014): block
 * floating point, the same reversible integer lifting, the same sequency
 * order, negabinary, and the same group-test bit-plane coder over 64 planes.
 * This file is the definition that the GPU's FP64 codec must match bit for
 * bit.
 *
 * Stream layout as FR4: a field of nx*ny*nz values (x fastest) is cut into
 * 4^3 blocks ordered bx fastest, then by, then bz; each block takes exactly
 * B = 64*R bits = 2*R 32-bit little-endian words; bit j of a block is bit
 * (j mod 32) of word j/32, multi-bit fields least-significant bit first.
 *
 * Steps for one block x[64], index x + 4y + 16z:
 *  1. emax = max over nonzero values of the frexp exponent, clamped below at
 *     -1022.  No nonzero value: a single 0 bit, rest zero.  Otherwise a 1
 *     bit and 11 bits of (emax + 1023).
 *  2. q_i = trunc(x_i * 2^(58 - emax)), an exact int64 with |q_i| < 2^58
 *     (53-bit significands fit with 5 bits to spare).
 *  3. FR4's lifting on every line of 4 along x, then y, then z, in wrapping
 *     int64 with floor(v/2) for the halving: each pass keeps |y| <= 2.5 M +
 *     1.25 for |a| <= M, so three passes keep |coefficient| < 2^62.
 *  4. Sequency order: coefficient (i,j,k) by key lev(i)+lev(j)+lev(k), ties
 *     by i + 4j + 16k, lev = (0, 1, 2, 2).
 *  5. Negabinary: u = (q + 0xAAAAAAAAAAAAAAAA) ^ 0xAAAAAAAAAAAAAAAA in
 *     wrapping uint64.
 *  6. Bit planes p = 63 .. 0 within the B - 12 remaining bits, n counting
 *     coefficients already significant: write bit p of u_0 .. u_{n-1}; then,
 *     while n < 64, a group bit g = OR of bit p of u_n .. u_63; stop the
 *     plane if g == 0; else write bits p of u_n, u_{n+1}, ..., advancing n
 *     after each and stopping after the first 1; when the scan reaches
 *     u_63 its bit must be 1 and is not written (n becomes 64).  Every write
 *     first checks the budget; coding stops when it is spent.
 * Decoding mirrors every step; bits never received read as 0.  The value
 * is rebuilt as RN_double( RN_double(q) * 2^(emax - 58) ).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define FR4D_PREC 58
#define FR4D_PLANES 64
#define FR4D_HEADER 12
#define FR4D_MAX_RATE 128 /* above 64 only for the full-precision checks */

typedef struct {
    uint32_t *w;
    int64_t pos, end; /* next bit; the budget is bits [0, end) */
} bits64;

static int put1(bits64 *s, unsigned b)
{
    if (s->pos >= s->end)
        return 0;
    if (b & 1u)
        s->w[s->pos >> 5] |= 1u << (s->pos & 31);
    s->pos++;
    return 1;
}

static int get1(bits64 *s, unsigned *b)
{
    if (s->pos >= s->end)
        return 0;
    *b = (s->w[s->pos >> 5] >> (s->pos & 31)) & 1u;
    s->pos++;
    return 1;
}

/* ---- lifting in wrapping int64 ------------------------------------------ */
static _Thread_local int d_fwd_wrapped;
static _Thread_local int d_inv_wrapped;

static int64_t add_w(int64_t a, int64_t b, int *flag)
{
    int64_t r;
    if (__builtin_add_overflow(a, b, &r))
        *flag = 1;
    return (int64_t)((uint64_t)a + (uint64_t)b);
}

static int64_t sub_w(int64_t a, int64_t b, int *flag)
{
    int64_t r;
    if (__builtin_sub_overflow(a, b, &r))
        *flag = 1;
    return (int64_t)((uint64_t)a - (uint64_t)b);
}

/* floor(v / 2) for every int64 v */
static int64_t half_floor(int64_t v) { return (v - (v & 1)) / 2; }

static void lift4_forward(int64_t *a, int stride)
{
    int *w = &d_fwd_wrapped;
    int64_t d0 = sub_w(a[0], a[stride], w);
    int64_t s0 = add_w(a[stride], half_floor(d0), w);
    int64_t d1 = sub_w(a[2 * stride], a[3 * stride], w);
    int64_t s1 = add_w(a[3 * stride], half_floor(d1), w);
    int64_t D = sub_w(s0, s1, w);
    int64_t S = add_w(s1, half_floor(D), w);
    d0 = sub_w(d0, half_floor(D), w);
    d1 = sub_w(d1, half_floor(D), w);
    a[0] = S;
    a[stride] = D;
    a[2 * stride] = d0;
    a[3 * stride] = d1;
}

static void lift4_inverse(int64_t *a, int stride)
{
    int *w = &d_inv_wrapped;
    int64_t S = a[0], D = a[stride];
    int64_t d0 = add_w(a[2 * stride], half_floor(D), w);
    int64_t d1 = add_w(a[3 * stride], half_floor(D), w);
    int64_t s1 = sub_w(S, half_floor(D), w);
    int64_t s0 = add_w(s1, D, w);
    int64_t x3 = sub_w(s1, half_floor(d1), w);
    int64_t x2 = add_w(x3, d1, w);
    int64_t x1 = sub_w(s0, half_floor(d0), w);
    int64_t x0 = add_w(x1, d0, w);
    a[0] = x0;
    a[stride] = x1;
    a[2 * stride] = x2;
    a[3 * stride] = x3;
}

static void forward3(int64_t *c)
{
    for (int z = 0; z < 4; z++)
        for (int y = 0; y < 4; y++)
            lift4_forward(c + 4 * y + 16 * z, 1);
    for (int z = 0; z < 4; z++)
        for (int x = 0; x < 4; x++)
            lift4_forward(c + x + 16 * z, 4);
    for (int y = 0; y < 4; y++)
        for (int x = 0; x < 4; x++)
            lift4_forward(c + x + 4 * y, 16);
}

static void inverse3(int64_t *c)
{
    for (int y = 0; y < 4; y++)
        for (int x = 0; x < 4; x++)
            lift4_inverse(c + x + 4 * y, 16);
    for (int z = 0; z < 4; z++)
        for (int x = 0; x < 4; x++)
            lift4_inverse(c + x + 16 * z, 4);
    for (int z = 0; z < 4; z++)
        for (int y = 0; y < 4; y++)
            lift4_inverse(c + 4 * y + 16 * z, 1);
}

/* ---- sequency order ------------------------------------------------------ */
static int seq[64];
static int seq_ready;

static void make_seq(void)
{
    static const int lev[4] = {0, 1, 2, 2};
    int r = 0;
    for (int key = 0; key <= 6; key++) /* by level sum, ties by linear index */
        for (int l = 0; l < 64; l++)
            if (lev[l & 3] + lev[(l >> 2) & 3] + lev[l >> 4] == key)
                seq[r++] = l;
    seq_ready = 1;
}

/* ---- negabinary ---------------------------------------------------------- */
#define NB64 0xAAAAAAAAAAAAAAAAull

static uint64_t nb_from_int(int64_t q) { return ((uint64_t)q + NB64) ^ NB64; }
static int64_t nb_to_int(uint64_t u) { return (int64_t)((u ^ NB64) - NB64); }

/* ---- plane coder ---------------------------------------------------------- */
static void put_planes(bits64 *s, const uint64_t *u)
{
    int n = 0;
    for (int p = FR4D_PLANES - 1; p >= 0; p--) {
        for (int i = 0; i < n; i++)
            if (!put1(s, (unsigned)(u[i] >> p)))
                return;
        while (n < 64) {
            unsigned g = 0;
            for (int i = n; i < 64; i++)
                g |= (unsigned)(u[i] >> p) & 1u;
            if (!put1(s, g))
                return;
            if (!g)
                break;
            for (;;) {
                if (n == 63) { /* the last coefficient's one is not written */
                    n = 64;
                    break;
                }
                unsigned b = (unsigned)(u[n] >> p) & 1u;
                if (!put1(s, b))
                    return;
                n++;
                if (b)
                    break;
            }
        }
    }
}

static void get_planes(bits64 *s, uint64_t *u)
{
    int n = 0;
    unsigned b;
    for (int p = FR4D_PLANES - 1; p >= 0; p--) {
        for (int i = 0; i < n; i++) {
            if (!get1(s, &b))
                return;
            u[i] |= (uint64_t)b << p;
        }
        while (n < 64) {
            if (!get1(s, &b))
                return;
            if (!b)
                break;
            for (;;) {
                if (n == 63) {
                    u[63] |= 1ull << p;
                    n = 64;
                    break;
                }
                if (!get1(s, &b))
                    return;
                u[n] |= (uint64_t)b << p;
                n++;
                if (b)
                    break;
            }
        }
    }
}

/* ---- one block ------------------------------------------------------------ */
static void encode_block64(const double *x, int rate, uint32_t *words)
{
    bits64 s = {words, 0, 64 * (int64_t)rate};
    memset(words, 0, sizeof(uint32_t) * 2 * (size_t)rate);
    int emax = INT32_MIN;
    for (int i = 0; i < 64; i++)
        if (x[i] != 0.0) {
            int e;
            frexp(x[i], &e);
            if (e < -1022)
                e = -1022;
            if (e > emax)
                emax = e;
        }
    if (emax == INT32_MIN) {
        put1(&s, 0);
        return;
    }
    put1(&s, 1);
    for (int j = 0; j < 11; j++)
        put1(&s, (unsigned)(emax + 1023) >> j);
    int64_t q[64];
    for (int i = 0; i < 64; i++)
        q[i] = (int64_t)trunc(ldexp(x[i], FR4D_PREC - emax));
    forward3(q);
    uint64_t u[64];
    for (int r = 0; r < 64; r++)
        u[r] = nb_from_int(q[seq[r]]);
    put_planes(&s, u);
}

static void decode_block64(const uint32_t *words, int rate, double *x)
{
    bits64 s = {(uint32_t *)words, 0, 64 * (int64_t)rate};
    unsigned b = 0;
    get1(&s, &b);
    if (!b) {
        for (int i = 0; i < 64; i++)
            x[i] = 0.0;
        return;
    }
    int field = 0;
    for (int j = 0; j < 11; j++) {
        b = 0;
        get1(&s, &b);
        field |= (int)b << j;
    }
    int emax = field - 1023;
    uint64_t u[64] = {0};
    get_planes(&s, u);
    int64_t q[64];
    for (int r = 0; r < 64; r++)
        q[seq[r]] = nb_to_int(u[r]);
    inverse3(q);
    for (int i = 0; i < 64; i++)
        x[i] = ldexp((double)q[i], emax - FR4D_PREC); /* RN conversion, then one rounding at most */
}

/* ---- exported API (ctypes) ----------------------------------------------- */
static int64_t nblk(int64_t n) { return (n + 3) / 4; }
static int64_t clampi(int64_t i, int64_t n) { return i < n ? i : n - 1; }

int fr4d_encode(const double *field, int64_t nx, int64_t ny, int64_t nz, int rate, uint32_t *out)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || rate < 1 || rate > FR4D_MAX_RATE)
        return -1;
    if (!seq_ready)
        make_seq();
    const int64_t nbx = nblk(nx), nby = nblk(ny), nbz = nblk(nz);
    int wrapped = 0;
#pragma omp parallel reduction(| : wrapped)
    {
        d_fwd_wrapped = 0;
#pragma omp for collapse(3) schedule(static)
        for (int64_t bz = 0; bz < nbz; bz++)
            for (int64_t by = 0; by < nby; by++)
                for (int64_t bx = 0; bx < nbx; bx++) {
                    double x[64];
                    for (int k = 0; k < 4; k++)
                        for (int j = 0; j < 4; j++)
                            for (int i = 0; i < 4; i++)
                                x[i + 4 * j + 16 * k] = field[(clampi(4 * bz + k, nz) * ny + clampi(4 * by + j, ny)) *
                                                                  nx + clampi(4 * bx + i, nx)];
                    encode_block64(x, rate, out + (bx + nbx * (by + nby * bz)) * 2 * rate);
                }
        wrapped |= d_fwd_wrapped;
    }
    return wrapped ? -2 : 0;
}

int fr4d_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t nz, int rate, double *field)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || rate < 1 || rate > FR4D_MAX_RATE)
        return -1;
    if (!seq_ready)
        make_seq();
    const int64_t nbx = nblk(nx), nby = nblk(ny), nbz = nblk(nz);
    int wrapped = 0;
#pragma omp parallel reduction(| : wrapped)
    {
        d_inv_wrapped = 0;
#pragma omp for collapse(3) schedule(static)
        for (int64_t bz = 0; bz < nbz; bz++)
            for (int64_t by = 0; by < nby; by++)
                for (int64_t bx = 0; bx < nbx; bx++) {
                    double x[64];
                    decode_block64(in + (bx + nbx * (by + nby * bz)) * 2 * rate, rate, x);
                    for (int k = 0; k < 4; k++)
                        for (int j = 0; j < 4; j++)
                            for (int i = 0; i < 4; i++) {
                                const int64_t z = 4 * bz + k, y = 4 * by + j, xx = 4 * bx + i;
                                if (z < nz && y < ny && xx < nx)
                                    field[(z * ny + y) * nx + xx] = x[i + 4 * j + 16 * k];
                            }
                }
        wrapped |= d_inv_wrapped;
    }
    return wrapped ? 1 : 0;
}

/* Test hooks: the steps on their own. */
int fr4d_transform_forward(int64_t *c)
{
    d_fwd_wrapped = 0;
    forward3(c);
    return d_fwd_wrapped ? -2 : 0;
}

int fr4d_transform_inverse(int64_t *c)
{
    d_inv_wrapped = 0;
    inverse3(c);
    return d_inv_wrapped ? 1 : 0;
}

int64_t fr4d_encode_planes(const uint64_t *u, int64_t budget_bits, uint32_t *words)
{
    bits64 s = {words, 0, budget_bits};
    put_planes(&s, u);
    return s.pos;
}

int64_t fr4d_decode_planes(const uint32_t *words, int64_t budget_bits, uint64_t *u)
{
    bits64 s = {(uint32_t *)words, 0, budget_bits};
    memset(u, 0, 64 * sizeof(uint64_t));
    get_planes(&s, u);
    return s.pos;
}
