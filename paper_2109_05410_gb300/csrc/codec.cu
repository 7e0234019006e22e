// codec.cu -- FR4 fixed-rate 4x4x4 block codec on sm_103a.
//
// Section IV of the paper asks for a fixed-rate lossy codec: the user fixes
// the bits kept per value, so every compressed unit has a known size and the
// device buffers are preallocated.  FR4 follows the published fixed-rate
// method (Lindstrom, IEEE TVCG 2014): block floating point on 4^3 blocks,
// a reversible integer decorrelating transform, sequency ordering,
// negabinary, and embedded bit-plane coding with group tests.  Its exact
// definition (header, lifting steps, ordering, plane coder, dequantisation)
// is stated in the oracle's codec; this file is an independent GPU
// implementation that must match it bit for bit.
//
// GPU design: one thread per 4^3 block.  The 64 values stay in registers
// (16 coalesced 128-bit loads: neighbouring threads own neighbouring blocks
// along x).  The bit-plane stage turns the 64 negabinary words into 32
// 64-bit plane masks with two in-register 32x32 bit transposes; the encoder
// then writes each plane with at most three 64-bit ORs (its significance
// part from a 256-entry table of "doubled ones", whatever its number of new
// coefficients), and the decoder parses all group-test segments inside a
// 32-bit stream window from one register.  The encoder
// stages its CTA's compressed words in shared memory and writes them with
// coalesced 32-bit stores; the decoder reads each block's words straight
// from the stream through L1, one word ahead of their use.
//
// Also here: dense-field kernels for any shape (partial blocks padded with
// the nearest inside value) and the variable-size fixed-precision and
// fixed-accuracy modes, with a prefix sum that turns block sizes into
// offsets.
#include <utility>

#include "common.cuh"

namespace ooc {

// Set by a kernel whose bounded wait gave up (the variable-size encoder's
// look-back); read and cleared by take_codec_fault().
__device__ unsigned g_codec_fault = 0u;

namespace {

constexpr int kPrec = 26;  // block-floating-point precision (bits)
constexpr int kThreads = 128;
constexpr int kPlaneStride = 65;  // words per thread for its plane masks
constexpr int kSlack = 8;         // words past a block's 2R that a coder may touch

// ---- sequency order ---------------------------------------------------------
// r-th coefficient of the coding order: sort by level sum of (i, j, k) with
// level (0, 1, 2, 2) per axis, ties by linear index (counting order).
__host__ __device__ constexpr int order_at(int r)
{
    int c = 0;
    for (int s = 0; s <= 6; ++s)
        for (int l = 0; l < 64; ++l) {
            const int li = (l & 3) == 0 ? 0 : ((l & 3) == 1 ? 1 : 2);
            const int lj = ((l >> 2) & 3) == 0 ? 0 : (((l >> 2) & 3) == 1 ? 1 : 2);
            const int lk = (l >> 4) == 0 ? 0 : ((l >> 4) == 1 ? 1 : 2);
            if (li + lj + lk == s) {
                if (c == r)
                    return l;
                ++c;
            }
        }
    return -1;
}

constexpr uint32_t kNB = 0xAAAAAAAAu;

template <int... R>
__device__ __forceinline__ void to_coding_order(uint32_t (&u)[64], const int32_t (&q)[64],
                                                std::integer_sequence<int, R...>)
{
    ((u[R] = ((uint32_t)q[std::integral_constant<int, order_at(R)>::value] + kNB) ^ kNB), ...);
}

template <int... R>
__device__ __forceinline__ void from_coding_order(int32_t (&q)[64], const uint32_t (&u)[64],
                                                  std::integer_sequence<int, R...>)
{
    ((q[std::integral_constant<int, order_at(R)>::value] = (int32_t)((u[R] ^ kNB) - kNB)), ...);
}

// ---- wrapping int32 lifting ---------------------------------------------------
__device__ __forceinline__ int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
__device__ __forceinline__ int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }

__device__ __forceinline__ void lift_fwd(int32_t &a0, int32_t &a1, int32_t &a2, int32_t &a3)
{
    int32_t d0 = wsub(a0, a1);
    const int32_t s0 = wadd(a1, d0 >> 1);
    int32_t d1 = wsub(a2, a3);
    const int32_t s1 = wadd(a3, d1 >> 1);
    const int32_t D = wsub(s0, s1);
    const int32_t S = wadd(s1, D >> 1);
    d0 = wsub(d0, D >> 1);
    d1 = wsub(d1, D >> 1);
    a0 = S;
    a1 = D;
    a2 = d0;
    a3 = d1;
}

__device__ __forceinline__ void lift_inv(int32_t &a0, int32_t &a1, int32_t &a2, int32_t &a3)
{
    const int32_t S = a0, D = a1;
    const int32_t d0 = wadd(a2, D >> 1);
    const int32_t d1 = wadd(a3, D >> 1);
    const int32_t s1 = wsub(S, D >> 1);
    const int32_t s0 = wadd(s1, D);
    const int32_t x3 = wsub(s1, d1 >> 1);
    const int32_t x2 = wadd(x3, d1);
    const int32_t x1 = wsub(s0, d0 >> 1);
    const int32_t x0 = wadd(x1, d0);
    a0 = x0;
    a1 = x1;
    a2 = x2;
    a3 = x3;
}

__device__ __forceinline__ void transform_fwd(int32_t (&c)[64])
{
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = 4 * y + 16 * z;
            lift_fwd(c[b], c[b + 1], c[b + 2], c[b + 3]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 16 * z;
            lift_fwd(c[b], c[b + 4], c[b + 8], c[b + 12]);
        }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 4 * y;
            lift_fwd(c[b], c[b + 16], c[b + 32], c[b + 48]);
        }
}

__device__ __forceinline__ void transform_inv(int32_t (&c)[64])
{
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 4 * y;
            lift_inv(c[b], c[b + 16], c[b + 32], c[b + 48]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 16 * z;
            lift_inv(c[b], c[b + 4], c[b + 8], c[b + 12]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = 4 * y + 16 * z;
            lift_inv(c[b], c[b + 1], c[b + 2], c[b + 3]);
        }
}

// ---- 32x32 bit transpose of a[OFF .. OFF+31] in registers --------------------
// Afterwards bit i of a[OFF + p] is the former bit p of a[OFF + i].
template <int OFF, int J, uint32_t M>
__device__ __forceinline__ void transpose_stage(uint32_t (&a)[64])
{
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (!(k & J)) {
            const uint32_t t = ((a[OFF + k] >> J) ^ a[OFF + k + J]) & M;
            a[OFF + k + J] ^= t;
            a[OFF + k] ^= t << J;
        }
    }
}

// The 16- and 8-bit stages are pure byte moves: one byte permute per word.
template <int OFF>
__device__ __forceinline__ void transpose_stage16(uint32_t (&a)[64])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t lo = a[OFF + k], hi = a[OFF + k + 16];
        a[OFF + k] = __byte_perm(lo, hi, 0x5410);
        a[OFF + k + 16] = __byte_perm(lo, hi, 0x7632);
    }
}

template <int OFF>
__device__ __forceinline__ void transpose_stage8(uint32_t (&a)[64])
{
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (!(k & 8)) {
            const uint32_t lo = a[OFF + k], hi = a[OFF + k + 8];
            a[OFF + k] = __byte_perm(lo, hi, 0x6240);
            a[OFF + k + 8] = __byte_perm(lo, hi, 0x7351);
        }
    }
}

template <int OFF>
__device__ __forceinline__ void transpose32(uint32_t (&a)[64])
{
    transpose_stage16<OFF>(a);
    transpose_stage8<OFF>(a);
    transpose_stage<OFF, 4, 0x0F0F0F0Fu>(a);
    transpose_stage<OFF, 2, 0x33333333u>(a);
    transpose_stage<OFF, 1, 0x55555555u>(a);
}

// ---- bit writer / reader over a thread's shared-memory words ------------------
__device__ __forceinline__ uint32_t low_mask(int l)  // l in [0, 32]
{
    return (uint32_t)((1ull << l) - 1ull);
}

// Reads bit fields of a thread's words through a 64-bit buffer holding at
// least 32 unread bits; it loads one shared-memory word per 32 bits read.
// The words past the block's 2R are zero (slack), so bits past the budget
// read as 0, which is what a truncated stream means; only the implied-one
// rule needs the budget.
// Reads a block's words straight from the stream (through the L1 cache);
// words past the block's nwords read as 0, so bits past the budget are 0.
struct BitReader {
    const uint32_t *src;
    uint64_t buf;  // unread bits, least significant first
    int avail;     // valid bits in buf, >= 32
    int wnext;     // index of the word held in `pre`
    int pos;       // bits consumed
    int nwords;    // words of the block
    uint32_t pre;  // word wnext, loaded one refill ahead so its latency hides

    __device__ __forceinline__ uint32_t word(int i) const { return i < nwords ? __ldg(src + i) : 0u; }
    __device__ __forceinline__ void init(const uint32_t *s, int start, int n)
    {
        src = s;
        nwords = n;
        const int w = start >> 5, sh = start & 31;
        buf = ((uint64_t)word(w) | ((uint64_t)word(w + 1) << 32)) >> sh;
        avail = 64 - sh;
        wnext = w + 2;
        pos = start;
        pre = word(wnext);
    }
    __device__ __forceinline__ void skip(int len)  // len in [0, 32]
    {
        buf >>= len;
        avail -= len;
        pos += len;
        if (avail < 32) {
            buf |= (uint64_t)pre << avail;
            avail += 32;
            pre = word(++wnext);
        }
    }
    __device__ __forceinline__ uint32_t peek32() const { return (uint32_t)buf; }
    __device__ __forceinline__ uint32_t get(int len)  // len in [0, 32]
    {
        const uint32_t v = (uint32_t)buf & low_mask(len);
        skip(len);
        return v;
    }
};

// OR a 64-bit field into a thread's zeroed words at bit offset `off`
// (least significant bit first); touches words off/32 .. off/32 + 2.
__device__ __forceinline__ void or_bits(uint32_t *w, int off, uint64_t v)
{
    const int i = off >> 5, sh = off & 31;
    const uint32_t a = (uint32_t)v, b = (uint32_t)(v >> 32);
    w[i] |= a << sh;
    w[i + 1] |= __funnelshift_l(a, b, sh);
    w[i + 2] |= __funnelshift_l(b, 0u, sh);
}

// Significance parts are written with "doubled ones": the bits of x with
// every one followed by an extra one.  In a plane's significance part each
// new one is followed by the group bit 1 of the next segment, so the part
// after its first group bit is the doubled bits before the last new one,
// then that one.  dtab[b] holds the doubled bits of byte b (8 + popc(b) <= 16
// bits); a CTA fills it once.
__device__ __forceinline__ void init_dup_table(uint16_t *dtab)
{
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        uint32_t d = 0u;
        int k = 0;
        for (int i = 0; i < 8; ++i)
            if ((b >> i) & 1) {
                d |= 3u << (i + k);
                ++k;
            }
        dtab[b] = (uint16_t)d;
    }
}

// Doubled ones of a 32-bit word: 32 + popc(x) <= 64 bits.
__device__ __forceinline__ uint64_t dup_ones(uint32_t x, const uint16_t *dtab)
{
    const uint32_t b0 = x & 0xFFu, b2 = (x >> 16) & 0xFFu;
    const uint32_t lo = (uint32_t)dtab[b0] | ((uint32_t)dtab[(x >> 8) & 0xFFu] << (8 + __popc(b0)));
    const uint32_t hi = (uint32_t)dtab[b2] | ((uint32_t)dtab[x >> 24] << (8 + __popc(b2)));
    return (uint64_t)lo | ((uint64_t)hi << (16 + __popc(x & 0xFFFFu)));
}

// ---- one block ----------------------------------------------------------------
// Lowest coded bit plane: 0 at a fixed rate; 32 - P at fixed precision P;
// at fixed accuracy with L = floor(log2 tol), L - (emax - 26) - 4 clamped to
// [0, 32] (the dropped planes then cost at most tol/2 after the inverse
// transform's gain of 2.25 per axis).
__device__ __forceinline__ int plane_floor(int mode, int mparam, int emax)
{
    if (mode == OOC_FR4_PRECISION)
        return 32 - mparam;
    if (mode == OOC_FR4_ACCURACY) {
        const int p = mparam - (emax - kPrec) - 4;
        return p < 0 ? 0 : (p > 32 ? 32 : p);
    }
    return 0;
}

// The bit-plane coder shared by FR4 (NP = 32 planes) and FR4D (NP = 64):
// pm[p] and pm[NP + p] hold bit p of coefficients 0..31 and 32..63; the
// planes NP-1 .. pmin are written from bit `off` of the zeroed words dst
// until the budget is spent.  Returns the coded length in bits.
//
// Plane p (NP-1 .. 0) is written as: the refinement bits of the n
// significant coefficients; then, for each new one at offset t past n,
// a group bit 1, the zeros before it and the one itself; then a closing
// group bit 0 if coefficients remain.  When a new one is the last
// coefficient its one is implied and not written.
//
// With rest = the plane's bits past n and tl its highest one, the part
// after the refinement bits is the group bit 1, the doubled bits of rest
// below tl, and the one at tl: the one of segment j lands at t_j + j past
// the first group bit, and the next segment's group bit right after it.
// Each plane is written with at most three 64-bit ORs, whatever its
// number of new ones.
template <int NP>
__device__ __forceinline__ int code_planes(const uint32_t *pm, uint32_t *dst, int off, int budget, int pmin,
                                           const uint16_t *dtab)
{
    int n = 0;
#pragma unroll 1
    for (int p = NP - 1; p >= pmin && off < budget; --p) {
        const uint64_t X = ((uint64_t)pm[NP + p] << 32) | pm[p];
        if (n >= 64) {
            or_bits(dst, off, X);
            off += 64;
            continue;
        }
        const uint64_t refine = X & ((1ull << n) - 1ull);
        const uint64_t rest = X >> n;
        if (rest == 0ull) {
            if (n > 0)
                or_bits(dst, off, refine);
            off += n + 1;  // refinement bits and the closing group bit 0
            continue;
        }
        or_bits(dst, off, refine | (1ull << n));  // ... and the first group bit
        const int m = __popcll((long long)rest);
        const int tl = 63 - __clzll((long long)rest);  // offset of the last new one
        const int n_new = n + tl + 1;
        const int at = off + n + 1;  // first bit past the first group bit
        const uint64_t before = rest ^ (1ull << tl);
        const uint64_t last = n_new == 64 ? 0ull : 1ull;  // the last coefficient's one is implied
        const int rel = tl + m - 1;                        // the last one's position past `at`
        if (tl < 32) {
            or_bits(dst, at, dup_ones((uint32_t)before, dtab) | (last << rel));
        } else {
            const uint32_t lo = (uint32_t)before;
            const int hs = 32 + __popc(lo);
            or_bits(dst, at, dup_ones(lo, dtab));
            or_bits(dst, at + hs, dup_ones((uint32_t)(before >> 32), dtab) | (last << (rel - hs)));
        }
        // n refinement bits, m group bits 1, tl + 1 scanned bits (the last
        // one implied when it is coefficient 63), a closing 0 if n_new < 64
        off += n + m + tl + 1 - (n_new == 64 ? 1 : 0) + (n_new < 64 ? 1 : 0);
        n = n_new;
    }
    return off;
}

// Encode one block into dst[0 .. words) (a bit budget of 32 words; words =
// 2R at a fixed rate) with the plane range of `mode`.  Returns the coded
// length in bits (exact for the variable-size modes, whose budget never
// binds).
__device__ __forceinline__ int encode_block(uint32_t (&v)[64], int words, int mode, int mparam, uint32_t *dst,
                                            uint32_t *pm, const uint16_t *dtab)
{
    uint32_t mx = 0;
#pragma unroll
    for (int i = 0; i < 64; ++i)
        mx = max(mx, v[i] & 0x7FFFFFFFu);
    const int budget = 32 * words;
    // The coder ORs bit fields into a zeroed buffer of `words` words plus
    // slack; bits it writes past the budget land in the slack and are not
    // kept.
    for (int i = 0; i < words + kSlack; ++i)
        dst[i] = 0u;
    if (mx == 0u)
        return 1;
    const int emax = (int)(mx >> 23) - 126;  // largest frexp exponent, >= -126
    dst[0] = 1u | ((uint32_t)((emax + 127) & 0xFF) << 1);
    const int pmin = plane_floor(mode, mparam, emax);

    // q = trunc(x * 2^(26 - emax)), with the power of two split in two
    // normal factors; the first product is exact whenever the result can be
    // nonzero, the second is exact or already below 1.
    const int kk = kPrec - emax;
    const int k1 = kk >> 1, k2 = kk - k1;
    const float s1 = __int_as_float((k1 + 127) << 23);
    const float s2 = __int_as_float((k2 + 127) << 23);
    int32_t q[64];
#pragma unroll
    for (int i = 0; i < 64; ++i)
        q[i] = __float2int_rz(__fmul_rn(__fmul_rn(__uint_as_float(v[i]), s1), s2));

    transform_fwd(q);
    to_coding_order(v, q, std::make_integer_sequence<int, 64>{});
    transpose32<0>(v);   // v[p]      = bits p of coefficients 0..31
    transpose32<32>(v);  // v[32 + p] = bits p of coefficients 32..63
    // The plane coder stays a compact loop (no unrolling) and reads the
    // plane masks from this thread's shared-memory slot.
#pragma unroll
    for (int i = 0; i < 64; ++i)
        pm[i] = v[i];

    return code_planes<32>(pm, dst, 9, budget, pmin, dtab);
}

// The plane parser shared by FR4 (NP = 32 planes) and FR4D (NP = 64): reads
// planes NP-1 .. pmin from r (positioned past the header) within `budget`
// bits into pm[p] (bit p of coefficients 0..31) and pm[NP + p] (32..63);
// planes not received are zero.
template <int NP>
__device__ __forceinline__ void parse_planes(BitReader &r, int budget, int pmin, uint32_t *pm)
{
    int n = 0;
    int p = NP - 1;
#pragma unroll 1
    for (; p >= pmin && r.pos < budget; --p) {
        const int n1 = n < 32 ? n : 32;
        uint32_t xl = r.get(n1);
        uint32_t xh = n > 32 ? r.get(n - 32) : 0u;
        if (n < 64) {
            uint64_t X = 0ull;  // the plane's new ones
            for (;;) {
                // The segments (group bit, scan) that end inside the next 32
                // stream bits are parsed from one register, k bits in; the
                // reader then advances once.  A segment that reaches past
                // the window is parsed again from a fresh window, and from
                // the long-scan path below when even that is too short.
                const uint32_t wv = r.peek32();
                int k = 0;
                int state = 0;  // 0: window used up; 1: plane done; 2: segment reaches past the window
                while (k < 32) {
                    const uint32_t w = wv >> k;
                    if ((w & 1u) == 0u) {  // group test: nothing more in this plane
                        ++k;
                        state = 1;
                        break;
                    }
                    const int len = 63 - n;  // explicit scan bits at most (after the group bit)
                    const uint32_t sc = w >> 1;  // the 31 - k scan bits inside the window
                    const int t = __ffs((int)sc) - 1;
                    if (sc != 0u && t < len) {
                        X |= 1ull << (n + t);
                        n += t + 1;
                        k += t + 2;
                        continue;
                    }
                    if (len <= 31 - k) {  // the len scan bits are zero: the last coefficient's one is implied
                        if (r.pos + k + 1 + len <= budget) {
                            X |= 1ull << 63;
                            n = 64;
                        }
                        k += 1 + len;
                        state = 1;
                        break;
                    }
                    state = 2;
                    break;
                }
                r.skip(k);
                if (state == 1)
                    break;
                if (state == 0 || k > 0)
                    continue;
                // long scan: group bit 1, then 31 zero bits of a scan of len > 31
                const int len = 63 - n;
                r.skip(32);
                int done = 31;
                bool found = false;
                for (;;) {
                    const int rem = len - done;
                    const int mm = rem < 32 ? rem : 32;
                    const uint32_t s2 = r.peek32() & low_mask(mm);
                    if (s2 != 0u) {
                        const int f = __ffs((int)s2);
                        const int t = done + f - 1;
                        r.skip(f);
                        X |= 1ull << (n + t);
                        n += t + 1;
                        found = true;
                        break;
                    }
                    if (rem <= 32) {
                        if (r.pos + rem <= budget) {
                            X |= 1ull << 63;
                            n = 64;
                        }
                        r.skip(rem);
                        break;
                    }
                    r.skip(32);
                    done += 32;
                }
                if (!found)
                    break;
            }
            xl |= (uint32_t)X;
            xh |= (uint32_t)(X >> 32);
        }
        pm[p] = xl;
        pm[NP + p] = xh;
    }
    for (; p >= 0; --p) {  // planes past the budget or below the coded range
        pm[p] = 0u;
        pm[NP + p] = 0u;
    }
}

// Decode one block of `nwords` words (2R at a fixed rate) with the plane
// range of `mode`.
__device__ __forceinline__ void decode_block(const uint32_t *src, int nwords, int mode, int mparam,
                                             float (&out)[64], uint32_t *pm)
{
    const int budget = 32 * nwords;
    const uint32_t w0 = nwords > 0 ? __ldg(src) : 0u;
    if ((w0 & 1u) == 0u) {
#pragma unroll
        for (int i = 0; i < 64; ++i)
            out[i] = 0.0f;
        return;
    }
    const int emax = (int)((w0 >> 1) & 0xFFu) - 127;
    const int pmin = plane_floor(mode, mparam, emax);
    BitReader r;
    r.init(src, 9, nwords);
    parse_planes<32>(r, budget, pmin, pm);
    uint32_t u[64];
#pragma unroll
    for (int i = 0; i < 64; ++i)
        u[i] = pm[i];
    transpose32<0>(u);
    transpose32<32>(u);
    int32_t q[64];
    from_coding_order(q, u, std::make_integer_sequence<int, 64>{});
    transform_inv(q);
    // x = RN(RN(q) * 2^(emax - 26)): one exact or correctly rounded scaling.
    const int k = emax - kPrec;
    const bool split = k < -126;
    const float sa = __int_as_float(((split ? k + 64 : k) + 127) << 23);
    const float sb = __int_as_float((-64 + 127) << 23);
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        float f = __fmul_rn(__int2float_rn(q[i]), sa);
        if (split)
            f = __fmul_rn(f, sb);
        out[i] = f;
    }
}

// ---- kernels ------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) fr4_encode_kernel(ConstRing in, int64_t nx, int64_t ny, int64_t z0,
                                                             int64_t nblk, int rate, uint32_t *__restrict__ out)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint16_t dtab[256];
    init_dup_table(dtab);
    __syncthreads();
    const int words = 2 * rate, stride = words + kSlack + 1;
    const int64_t first = (int64_t)blockIdx.x * kThreads;
    const int64_t b = first + threadIdx.x;
    if (b < nblk) {
        const int64_t nbx = nx >> 2, nby = ny >> 2;
        const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
        const int64_t slot = ring_slot(z0 + 4 * bz, in.zbase, in.nslot);
        const float *p = in.base + (slot * ny + 4 * by) * nx + 4 * bx;
        uint32_t v[64];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(p + ((int64_t)k * ny + j) * nx));
                v[16 * k + 4 * j + 0] = __float_as_uint(f.x);
                v[16 * k + 4 * j + 1] = __float_as_uint(f.y);
                v[16 * k + 4 * j + 2] = __float_as_uint(f.z);
                v[16 * k + 4 * j + 3] = __float_as_uint(f.w);
            }
        encode_block(v, words, OOC_FR4_RATE, 0, smem + threadIdx.x * stride,
                     smem + kThreads * stride + threadIdx.x * kPlaneStride, dtab);
    }
    __syncthreads();
    const int64_t left = nblk - first;
    const int nvalid = left < kThreads ? (int)left : kThreads;
    uint32_t *dst = out + first * words;
    if ((words & 3) == 0 && ((uintptr_t)out & 15) == 0) {
        // 16-byte stores: chunk c of the CTA's output is words 4 (c mod q) ..
        // of block c / q, q = words / 4; c advances by kThreads
        const int q = words >> 2;
        int blk = threadIdx.x / q, ch = threadIdx.x - blk * q;
        const int step_blk = kThreads / q, step_ch = kThreads - step_blk * q;
        for (int c = threadIdx.x; c < nvalid * q; c += kThreads) {
            const uint32_t *w = smem + blk * stride + 4 * ch;
            reinterpret_cast<uint4 *>(dst)[c] = make_uint4(w[0], w[1], w[2], w[3]);
            blk += step_blk;
            ch += step_ch;
            if (ch >= q) {
                ch -= q;
                ++blk;
            }
        }
        return;
    }
    // word o of the CTA's output is word (o mod words) of block (o / words);
    // o advances by kThreads, so block and word advance incrementally
    int blk = threadIdx.x / words, wd = threadIdx.x - blk * words;
    const int step_blk = kThreads / words, step_wd = kThreads - step_blk * words;
    for (int o = threadIdx.x; o < nvalid * words; o += kThreads) {
        dst[o] = smem[blk * stride + wd];
        blk += step_blk;
        wd += step_wd;
        if (wd >= words) {
            wd -= words;
            ++blk;
        }
    }
}

// MINB CTAs per SM: 6 (80 registers) for rates up to 16, 5 (96 registers,
// more L1 beside the plane masks) above.  1024^3 decode, 6 against 5:
// R = 8 3.35 against 3.60 ms, R = 16 4.19 against 4.30, R = 24 4.90
// against 4.59.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) fr4_decode_kernel(const uint32_t *__restrict__ in, int64_t nx, int64_t ny,
                                                             int64_t z0, int64_t nblk, int rate, Ring out)
{
    extern __shared__ uint32_t smem[];  // each thread's plane masks
    const int64_t b = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (b >= nblk)
        return;
    float f[64];
    decode_block(in + b * (2 * rate), 2 * rate, OOC_FR4_RATE, 0, f, smem + threadIdx.x * kPlaneStride);
    const int64_t nbx = nx >> 2, nby = ny >> 2;
    const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
    const int64_t slot = ring_slot(z0 + 4 * bz, out.zbase, out.nslot);
    float *p = out.base + (slot * ny + 4 * by) * nx + 4 * bx;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4 *>(p + ((int64_t)k * ny + j) * nx) =
                make_float4(f[16 * k + 4 * j], f[16 * k + 4 * j + 1], f[16 * k + 4 * j + 2], f[16 * k + 4 * j + 3]);
}

// ---- FR4D: the same codec for FP64 fields -------------------------------------
// 58-bit block floating point (emax clamped at -1022, 11 header bits), the
// FR4 lifting in wrapping int64, the same coding order, 64-bit negabinary
// and 64 bit planes through the shared plane coder and parser.  One thread
// owns one block; a CTA of 64 threads keeps each thread's 128 plane words
// (and, encoding, its staged output) in shared memory.
constexpr int kPrec64 = 58;
constexpr int kThreads64 = 64;
constexpr int kPlaneStride64 = 129;  // 128 plane words, odd stride
constexpr uint64_t kNB64 = 0xAAAAAAAAAAAAAAAAull;

__device__ __forceinline__ int64_t wadd64(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
__device__ __forceinline__ int64_t wsub64(int64_t a, int64_t b) { return (int64_t)((uint64_t)a - (uint64_t)b); }

__device__ __forceinline__ void lift_fwd64(int64_t &a0, int64_t &a1, int64_t &a2, int64_t &a3)
{
    int64_t d0 = wsub64(a0, a1);
    const int64_t s0 = wadd64(a1, d0 >> 1);
    int64_t d1 = wsub64(a2, a3);
    const int64_t s1 = wadd64(a3, d1 >> 1);
    const int64_t D = wsub64(s0, s1);
    const int64_t S = wadd64(s1, D >> 1);
    d0 = wsub64(d0, D >> 1);
    d1 = wsub64(d1, D >> 1);
    a0 = S;
    a1 = D;
    a2 = d0;
    a3 = d1;
}

__device__ __forceinline__ void lift_inv64(int64_t &a0, int64_t &a1, int64_t &a2, int64_t &a3)
{
    const int64_t S = a0, D = a1;
    const int64_t d0 = wadd64(a2, D >> 1);
    const int64_t d1 = wadd64(a3, D >> 1);
    const int64_t s1 = wsub64(S, D >> 1);
    const int64_t s0 = wadd64(s1, D);
    const int64_t x3 = wsub64(s1, d1 >> 1);
    const int64_t x2 = wadd64(x3, d1);
    const int64_t x1 = wsub64(s0, d0 >> 1);
    const int64_t x0 = wadd64(x1, d0);
    a0 = x0;
    a1 = x1;
    a2 = x2;
    a3 = x3;
}

__device__ __forceinline__ void transform_fwd64(int64_t (&c)[64])
{
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = 4 * y + 16 * z;
            lift_fwd64(c[b], c[b + 1], c[b + 2], c[b + 3]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 16 * z;
            lift_fwd64(c[b], c[b + 4], c[b + 8], c[b + 12]);
        }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 4 * y;
            lift_fwd64(c[b], c[b + 16], c[b + 32], c[b + 48]);
        }
}

__device__ __forceinline__ void transform_inv64(int64_t (&c)[64])
{
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 4 * y;
            lift_inv64(c[b], c[b + 16], c[b + 32], c[b + 48]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = x + 16 * z;
            lift_inv64(c[b], c[b + 4], c[b + 8], c[b + 12]);
        }
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int b = 4 * y + 16 * z;
            lift_inv64(c[b], c[b + 1], c[b + 2], c[b + 3]);
        }
}

// coefficient order_at(r) as 64-bit negabinary, split into its low and high
// words
template <int... R>
__device__ __forceinline__ void to_coding_order64(uint32_t (&lo)[64], uint32_t (&hi)[64], const int64_t (&q)[64],
                                                  std::integer_sequence<int, R...>)
{
    ((lo[R] = (uint32_t)(((uint64_t)q[std::integral_constant<int, order_at(R)>::value] + kNB64) ^ kNB64),
      hi[R] = (uint32_t)((((uint64_t)q[std::integral_constant<int, order_at(R)>::value] + kNB64) ^ kNB64) >> 32)),
     ...);
}

template <int... R>
__device__ __forceinline__ void from_coding_order64(int64_t (&q)[64], const uint32_t (&lo)[64],
                                                    const uint32_t (&hi)[64], std::integer_sequence<int, R...>)
{
    ((q[std::integral_constant<int, order_at(R)>::value] =
          (int64_t)(((((uint64_t)hi[R] << 32) | lo[R]) ^ kNB64) - kNB64)),
     ...);
}

// 64 coefficients' low and high words -> pm[p] (bit p of coefficients
// 0..31) and pm[64 + p] (32..63) for p = 0..63, and back.
__device__ __forceinline__ void words_to_planes64(uint32_t (&lo)[64], uint32_t (&hi)[64], uint32_t *pm)
{
    transpose32<0>(lo);
    transpose32<32>(lo);
    transpose32<0>(hi);
    transpose32<32>(hi);
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        pm[p] = lo[p];
        pm[32 + p] = hi[p];
        pm[64 + p] = lo[32 + p];
        pm[96 + p] = hi[32 + p];
    }
}

__device__ __forceinline__ void planes_to_words64(const uint32_t *pm, uint32_t (&lo)[64], uint32_t (&hi)[64])
{
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        lo[p] = pm[p];
        hi[p] = pm[32 + p];
        lo[32 + p] = pm[64 + p];
        hi[32 + p] = pm[96 + p];
    }
    transpose32<0>(lo);
    transpose32<32>(lo);
    transpose32<0>(hi);
    transpose32<32>(hi);
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ double pow2d(int k)  // k in [-1022, 1023]
{
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// Encode one FP64 block (bit patterns v) into dst[0 .. words) at a fixed
// rate: words = 2R, a budget of 64R bits.
__device__ __forceinline__ void encode_block64(const uint64_t (&v)[64], int words, uint32_t *dst, uint32_t *pm,
                                               const uint16_t *dtab)
{
    uint64_t mx = 0;
#pragma unroll
    for (int i = 0; i < 64; ++i)
        mx = umax64(mx, v[i] & 0x7FFFFFFFFFFFFFFFull);
    for (int i = 0; i < words + kSlack; ++i)
        dst[i] = 0u;
    if (mx == 0ull)
        return;
    // largest frexp exponent (biased exponent - 1022; subnormals clamp to -1022)
    const int emax = (int)(mx >> 52) - 1022;
    dst[0] = 1u | ((uint32_t)(emax + 1023) << 1);
    // q = trunc(x * 2^(58 - emax)) in integer arithmetic on the bits (the
    // FP64 pipe is scarce on this GPU): x = m 2^e with the 53-bit significand
    // m, so |q| = m shifted by e + 58 - emax (left by at most 5, since |x| <
    // 2^emax; right past 63 is 0), then the sign
    const int kk = kPrec64 - emax;
    int64_t q[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        const uint64_t b = v[i];
        const int eb = (int)((b >> 52) & 0x7FFu);
        const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (eb != 0 ? (1ull << 52) : 0ull);
        const int sh = (eb != 0 ? eb - 1075 : -1074) + kk;
        const uint64_t a = sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ull);
        q[i] = (b >> 63) ? -(int64_t)a : (int64_t)a;
    }
    transform_fwd64(q);
    uint32_t lo[64], hi[64];
    to_coding_order64(lo, hi, q, std::make_integer_sequence<int, 64>{});
    words_to_planes64(lo, hi, pm);
    code_planes<64>(pm, dst, 12, 32 * words, 0, dtab);
}

__device__ __forceinline__ void decode_block64(const uint32_t *src, int nwords, double (&out)[64], uint32_t *pm)
{
    const uint32_t w0 = nwords > 0 ? __ldg(src) : 0u;
    if ((w0 & 1u) == 0u) {
#pragma unroll
        for (int i = 0; i < 64; ++i)
            out[i] = 0.0;
        return;
    }
    const int emax = (int)((w0 >> 1) & 0x7FFu) - 1023;
    BitReader r;
    r.init(src, 12, nwords);
    parse_planes<64>(r, 32 * nwords, 0, pm);
    uint32_t lo[64], hi[64];
    planes_to_words64(pm, lo, hi);
    int64_t q[64];
    from_coding_order64(q, lo, hi, std::make_integer_sequence<int, 64>{});
    transform_inv64(q);
    // x = RN(RN(q) * 2^(emax - 58)): one exact or correctly rounded scaling
    // (on the FP64 pipe: the same in integer arithmetic measured slower)
    const int k = emax - kPrec64;
    const bool split = k < -1022;
    const double sa = pow2d(split ? k + 64 : k), sb = pow2d(-64);
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        double f = __dmul_rn(__ll2double_rn((long long)q[i]), sa);
        if (split)
            f = __dmul_rn(f, sb);
        out[i] = f;
    }
}

__global__ void __launch_bounds__(kThreads64) fr4d_encode_kernel(DConstRing in, int64_t nx, int64_t ny, int64_t z0,
                                                                 int64_t nblk, int rate, uint32_t *__restrict__ out)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint16_t dtab[256];
    init_dup_table(dtab);
    __syncthreads();
    const int words = 2 * rate, stride = words + kSlack + 1;
    const int64_t first = (int64_t)blockIdx.x * kThreads64;
    const int64_t b = first + threadIdx.x;
    if (b < nblk) {
        const int64_t nbx = nx >> 2, nby = ny >> 2;
        const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
        const int64_t slot = ring_slot(z0 + 4 * bz, in.zbase, in.nslot);
        const double *p = in.base + (slot * ny + 4 * by) * nx + 4 * bx;
        uint64_t v[64];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double2 *row = reinterpret_cast<const double2 *>(p + ((int64_t)k * ny + j) * nx);
                const double2 a = __ldg(row), c = __ldg(row + 1);
                v[16 * k + 4 * j + 0] = (uint64_t)__double_as_longlong(a.x);
                v[16 * k + 4 * j + 1] = (uint64_t)__double_as_longlong(a.y);
                v[16 * k + 4 * j + 2] = (uint64_t)__double_as_longlong(c.x);
                v[16 * k + 4 * j + 3] = (uint64_t)__double_as_longlong(c.y);
            }
        encode_block64(v, words, smem + threadIdx.x * stride, smem + kThreads64 * stride + threadIdx.x * kPlaneStride64,
                       dtab);
    }
    __syncthreads();
    const int64_t left = nblk - first;
    const int nvalid = left < kThreads64 ? (int)left : kThreads64;
    uint32_t *dst = out + first * words;
    // word o of the CTA's output is word (o mod words) of block (o / words)
    for (int o = threadIdx.x; o < nvalid * words; o += kThreads64)
        dst[o] = smem[(o / words) * stride + (o % words)];
}

__global__ void __launch_bounds__(kThreads64) fr4d_decode_kernel(const uint32_t *__restrict__ in, int64_t nx,
                                                                 int64_t ny, int64_t z0, int64_t nblk, int rate,
                                                                 DRing out)
{
    extern __shared__ uint32_t smem[];  // each thread's plane words
    const int64_t b = (int64_t)blockIdx.x * kThreads64 + threadIdx.x;
    if (b >= nblk)
        return;
    double f[64];
    decode_block64(in + b * (2 * rate), 2 * rate, f, smem + threadIdx.x * kPlaneStride64);
    const int64_t nbx = nx >> 2, nby = ny >> 2;
    const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
    const int64_t slot = ring_slot(z0 + 4 * bz, out.zbase, out.nslot);
    double *p = out.base + (slot * ny + 4 * by) * nx + 4 * bx;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double2 *row = reinterpret_cast<double2 *>(p + ((int64_t)k * ny + j) * nx);
            row[0] = make_double2(f[16 * k + 4 * j], f[16 * k + 4 * j + 1]);
            row[1] = make_double2(f[16 * k + 4 * j + 2], f[16 * k + 4 * j + 3]);
        }
}

size_t smem_bytes64(int rate, bool encoder)
{
    if (!encoder)
        return (size_t)kThreads64 * kPlaneStride64 * sizeof(uint32_t);
    return ((size_t)kThreads64 * (2 * rate + kSlack + 1) + (size_t)kThreads64 * kPlaneStride64) * sizeof(uint32_t);
}

cudaError_t ensure_smem_attr64()
{
    // set once per process (thread-safe); the attribute is per function
    static const cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(fr4d_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes64(64, true));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fr4d_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes64(64, false));
        return e;
    }();
    return once;
}

// ---- dense fields of any shape, fixed rate and variable-size modes -------------
constexpr int kVarWords = 130;  // largest variable-size block (9 + 32 * 129 bits)

// Block (bx, by, bz) of a dense field; a block reaching past the field takes
// the value of the nearest point inside it (each coordinate clamped).
__device__ __forceinline__ void gather_clamped(const float *in, int64_t nx, int64_t ny, int64_t nz, int64_t bx,
                                               int64_t by, int64_t bz, uint32_t (&v)[64])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t z = min(4 * bz + k, nz - 1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float *row = in + (z * ny + min(4 * by + j, ny - 1)) * nx;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                v[16 * k + 4 * j + i] = __float_as_uint(__ldg(row + min(4 * bx + i, nx - 1)));
        }
    }
}

// Fixed rate for any shape: `words` words per block, the CTA's output
// staged and written with coalesced stores.
__global__ void __launch_bounds__(kThreads)
    fr4_encode_dense_kernel(const float *__restrict__ in, int64_t nx, int64_t ny, int64_t nz, int64_t nblk, int words,
                            uint32_t *__restrict__ out)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint16_t dtab[256];
    init_dup_table(dtab);
    __syncthreads();
    const int stride = words + kSlack + 1;
    const int64_t first = (int64_t)blockIdx.x * kThreads;
    const int64_t b = first + threadIdx.x;
    uint32_t *mine = smem + threadIdx.x * stride;
    if (b < nblk) {
        const int64_t nbx = (nx + 3) >> 2, nby = (ny + 3) >> 2;
        const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
        uint32_t v[64];
        gather_clamped(in, nx, ny, nz, bx, by, bz, v);
        encode_block(v, words, OOC_FR4_RATE, 0, mine, smem + kThreads * stride + threadIdx.x * kPlaneStride, dtab);
    }
    __syncthreads();
    const int64_t left = nblk - first;
    const int nvalid = left < kThreads ? (int)left : kThreads;
    uint32_t *dst = out + first * words;
    int blk = threadIdx.x / words, wd = threadIdx.x - blk * words;
    const int step_blk = kThreads / words, step_wd = kThreads - step_blk * words;
    for (int o = threadIdx.x; o < nvalid * words; o += kThreads) {
        dst[o] = smem[blk * stride + wd];
        blk += step_blk;
        wd += step_wd;
        if (wd >= words) {
            wd -= words;
            ++blk;
        }
    }
}

// Fixed rate: block b is words [b * words, (b + 1) * words).  Variable-size:
// words [index[b], index[b + 1]), clamped to the stream and to kVarWords.
// Only the points inside the field are written.
__global__ void __launch_bounds__(kThreads)
    fr4_decode_dense_kernel(const uint32_t *__restrict__ in, int64_t in_words, const uint64_t *__restrict__ index,
                            int64_t nx, int64_t ny, int64_t nz, int64_t nblk, int words, int mode, int mparam,
                            float *__restrict__ out)
{
    extern __shared__ uint32_t smem[];  // each thread's plane masks
    const int64_t b = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (b >= nblk)
        return;
    const uint32_t *src;
    int nw;
    if (mode == OOC_FR4_RATE) {
        src = in + b * words;
        nw = words;
    } else {
        uint64_t lo = __ldg(index + b), hi = __ldg(index + b + 1);
        lo = lo < (uint64_t)in_words ? lo : (uint64_t)in_words;
        hi = hi < (uint64_t)in_words ? hi : (uint64_t)in_words;
        const uint64_t n = hi > lo ? hi - lo : 0;
        nw = (int)(n < (uint64_t)kVarWords ? n : (uint64_t)kVarWords);
        src = in + lo;
    }
    float f[64];
    decode_block(src, nw, mode, mparam, f, smem + threadIdx.x * kPlaneStride);
    const int64_t nbx = (nx + 3) >> 2, nby = (ny + 3) >> 2;
    const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t z = 4 * bz + k, y = 4 * by + j, x = 4 * bx + i;
                if (z < nz && y < ny && x < nx)
                    out[(z * ny + y) * nx + x] = f[16 * k + 4 * j + i];
            }
}

// ---- variable-size modes: one pass with a decoupled look-back ---------------------
// Tile t is the kThreads blocks of the t-th CTA to start: an atomic counter
// numbers the CTAs as they begin, so every tile a CTA waits on is already
// running and never waits on a later one.  status[t] holds the tile's state
// in bits 62-63 and a word count in bits 0-61: kTileAgg its own words,
// kTilePrefix the words of tiles 0 .. t, kTileFailed a look-back that gave up.
// Each published value carries everything its reader needs, so relaxed
// 64-bit loads and stores suffice.
constexpr uint64_t kTileAgg = 1ull << 62, kTilePrefix = 2ull << 62, kTileFailed = 3ull << 62;
constexpr uint64_t kTileValue = (1ull << 62) - 1;
constexpr int kLookbackSpins = 1 << 24;  // about a second of 64 ns sleeps per tile waited on

__device__ __forceinline__ uint64_t ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Block b's words at out + index[b]; index[nblk] = total words.  A block is
// written only if it ends within out_words.  scratch: the tile counter, then
// one status word per tile, all zero at launch.
__global__ void __launch_bounds__(kThreads)
    fr4_encode_var_kernel(const float *__restrict__ in, int64_t nx, int64_t ny, int64_t nz, int64_t nblk, int mode,
                          int mparam, uint32_t *__restrict__ out, uint64_t out_words, uint64_t *__restrict__ index,
                          unsigned long long *scratch)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint16_t dtab[256];
    __shared__ uint64_t warp_tot[kThreads / 32];
    __shared__ int64_t s_tile;
    __shared__ uint64_t s_prefix;
    __shared__ int s_fail;
    unsigned long long *status = scratch + 1;
    if (threadIdx.x == 0) {
        s_tile = (int64_t)atomicAdd(scratch, 1ull);
        s_fail = 0;
    }
    init_dup_table(dtab);
    __syncthreads();
    const int64_t tile = s_tile;
    constexpr int stride = kVarWords + kSlack + 1;
    const int64_t b = tile * kThreads + threadIdx.x;
    uint32_t *mine = smem + threadIdx.x * stride;
    uint64_t nw = 0;
    if (b < nblk) {
        const int64_t nbx = (nx + 3) >> 2, nby = (ny + 3) >> 2;
        const int64_t bx = b % nbx, t2 = b / nbx, by = t2 % nby, bz = t2 / nby;
        uint32_t v[64];
        gather_clamped(in, nx, ny, nz, bx, by, bz, v);
        const int bits = encode_block(v, kVarWords, mode, mparam, mine,
                                      smem + kThreads * stride + threadIdx.x * kPlaneStride, dtab);
        nw = (uint64_t)((bits + 31) >> 5);
    }
    // exclusive scan of the word counts over the CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = nw;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d)
            incl += t;
    }
    if (lane == 31)
        warp_tot[warp] = incl;
    __syncthreads();
    uint64_t before = incl - nw, total = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp)
            before += warp_tot[w];
        total += warp_tot[w];
    }
    if (threadIdx.x == 0) {
        uint64_t prefix = 0;
        if (tile == 0) {
            st_relaxed_u64(&status[0], kTilePrefix | total);
        } else {
            st_relaxed_u64(&status[tile], kTileAgg | total);
            bool failed = false;
            for (int64_t j = tile - 1;; --j) {  // tile 0 publishes a prefix, so j stays >= 0
                uint64_t v = ld_relaxed_u64(&status[j]);
                for (int spins = 0; (v >> 62) == 0 && spins < kLookbackSpins; ++spins) {
                    __nanosleep(64);
                    v = ld_relaxed_u64(&status[j]);
                }
                const uint64_t state = v & ~kTileValue;
                if (state == 0 || state == kTileFailed) {
                    failed = true;
                    break;
                }
                prefix += v & kTileValue;
                if (state == kTilePrefix)
                    break;
            }
            if (failed) {
                st_relaxed_u64(&status[tile], kTileFailed);  // later tiles stop at once
                atomicOr(&g_codec_fault, 1u);
                s_fail = 1;
            } else {
                st_relaxed_u64(&status[tile], kTilePrefix | (prefix + total));
            }
        }
        s_prefix = prefix;
    }
    __syncthreads();
    if (s_fail || b >= nblk)
        return;
    const uint64_t off = s_prefix + before;
    index[b] = off;
    if (b == nblk - 1)
        index[nblk] = off + nw;
    if (off + nw <= out_words)
        for (uint64_t i = 0; i < nw; ++i)
            out[off + i] = mine[i];
}

size_t dense_smem_bytes(int words, bool encoder)
{
    if (!encoder)
        return (size_t)kThreads * kPlaneStride * sizeof(uint32_t);
    return (size_t)kThreads * (words + kSlack + 1 + kPlaneStride) * sizeof(uint32_t);
}

cudaError_t ensure_dense_smem_attr()
{
    // set once per process (thread-safe); the attribute is per function
    static const cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(fr4_encode_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dense_smem_bytes(kVarWords, true));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fr4_encode_var_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dense_smem_bytes(kVarWords, true));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fr4_decode_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dense_smem_bytes(kVarWords, false));
        return e;
    }();
    return once;
}

// Shared memory per CTA (encoder): each thread's compressed words plus
// kSlack words of slack (stride 2R + kSlack + 1, odd, so that the threads'
// slots start in different banks), then each thread's 64 plane masks
// (stride 65).  The decoder keeps only the plane masks.
size_t smem_bytes(int rate, bool encoder)
{
    if (!encoder)  // the decoder reads its words from the stream directly
        return (size_t)kThreads * kPlaneStride * sizeof(uint32_t);
    return ((size_t)kThreads * (2 * rate + kSlack + 1) + (size_t)kThreads * kPlaneStride) * sizeof(uint32_t);
}

cudaError_t ensure_smem_attr()
{
    // set once per process (thread-safe); the attribute is per function
    static const cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(fr4_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes(64, true));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fr4_decode_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes(64, false));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fr4_decode_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes(64, false));
        return e;
    }();
    return once;
}

}  // namespace

cudaError_t launch_fr4_encode(ConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                              uint32_t *out, cudaStream_t st)
{
    const int64_t nblk = (nx / 4) * (ny / 4) * ((z1 - z0) / 4);
    if (nblk <= 0)
        return cudaSuccess;
    cudaError_t e = ensure_smem_attr();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads - 1) / kThreads;
    fr4_encode_kernel<<<(unsigned)grid, kThreads, smem_bytes(rate, true), st>>>(in, nx, ny, z0, nblk, rate, out);
    return cudaGetLastError();
}

cudaError_t launch_fr4_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                              Ring out, cudaStream_t st)
{
    const int64_t nblk = (nx / 4) * (ny / 4) * ((z1 - z0) / 4);
    if (nblk <= 0)
        return cudaSuccess;
    cudaError_t e = ensure_smem_attr();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads - 1) / kThreads;
    if (rate > 16)
        fr4_decode_kernel<5><<<(unsigned)grid, kThreads, smem_bytes(rate, false), st>>>(in, nx, ny, z0, nblk, rate, out);
    else
        fr4_decode_kernel<6><<<(unsigned)grid, kThreads, smem_bytes(rate, false), st>>>(in, nx, ny, z0, nblk, rate, out);
    return cudaGetLastError();
}

cudaError_t launch_fr4d_encode(DConstRing in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                               uint32_t *out, cudaStream_t st)
{
    const int64_t nblk = (nx / 4) * (ny / 4) * ((z1 - z0) / 4);
    if (nblk <= 0)
        return cudaSuccess;
    if (rate < 1 || rate > 64)
        return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_attr64();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads64 - 1) / kThreads64;
    fr4d_encode_kernel<<<(unsigned)grid, kThreads64, smem_bytes64(rate, true), st>>>(in, nx, ny, z0, nblk, rate, out);
    return cudaGetLastError();
}

cudaError_t launch_fr4d_decode(const uint32_t *in, int64_t nx, int64_t ny, int64_t z0, int64_t z1, int rate,
                               DRing out, cudaStream_t st)
{
    const int64_t nblk = (nx / 4) * (ny / 4) * ((z1 - z0) / 4);
    if (nblk <= 0)
        return cudaSuccess;
    if (rate < 1 || rate > 64)
        return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_attr64();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads64 - 1) / kThreads64;
    fr4d_decode_kernel<<<(unsigned)grid, kThreads64, smem_bytes64(rate, false), st>>>(in, nx, ny, z0, nblk, rate, out);
    return cudaGetLastError();
}

int64_t fr4_blocks(int64_t nx, int64_t ny, int64_t nz) { return ((nx + 3) / 4) * ((ny + 3) / 4) * ((nz + 3) / 4); }

cudaError_t launch_fr4_encode_dense(const float *in, int64_t nx, int64_t ny, int64_t nz, int words, uint32_t *out,
                                    cudaStream_t st)
{
    const int64_t nblk = fr4_blocks(nx, ny, nz);
    if (nblk <= 0)
        return cudaSuccess;
    if (words < 1 || words > kVarWords)
        return cudaErrorInvalidValue;
    cudaError_t e = ensure_dense_smem_attr();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads - 1) / kThreads;
    fr4_encode_dense_kernel<<<(unsigned)grid, kThreads, dense_smem_bytes(words, true), st>>>(in, nx, ny, nz, nblk,
                                                                                             words, out);
    return cudaGetLastError();
}

cudaError_t launch_fr4_encode_var(const float *in, int64_t nx, int64_t ny, int64_t nz, int mode, int mparam,
                                  uint32_t *out, uint64_t out_words, uint64_t *index, void *scratch, cudaStream_t st)
{
    const int64_t nblk = fr4_blocks(nx, ny, nz);
    if (nblk <= 0)
        return cudaSuccess;
    cudaError_t e = ensure_dense_smem_attr();
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(scratch, 0, var_scratch_bytes(nblk), st);
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads - 1) / kThreads;
    fr4_encode_var_kernel<<<(unsigned)grid, kThreads, dense_smem_bytes(kVarWords, true), st>>>(
        in, nx, ny, nz, nblk, mode, mparam, out, out_words, index, (unsigned long long *)scratch);
    return cudaGetLastError();
}

cudaError_t take_codec_fault(unsigned *fault)
{
    unsigned v = 0u;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_codec_fault, sizeof(v));
    if (e == cudaSuccess && v != 0u) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_codec_fault, &zero, sizeof(zero));
    }
    *fault = v;
    return e;
}

cudaError_t launch_fr4_decode_dense(const uint32_t *in, int64_t in_words, const uint64_t *index, int64_t nx,
                                    int64_t ny, int64_t nz, int words, int mode, int mparam, float *out,
                                    cudaStream_t st)
{
    const int64_t nblk = fr4_blocks(nx, ny, nz);
    if (nblk <= 0)
        return cudaSuccess;
    cudaError_t e = ensure_dense_smem_attr();
    if (e != cudaSuccess)
        return e;
    const int64_t grid = (nblk + kThreads - 1) / kThreads;
    fr4_decode_dense_kernel<<<(unsigned)grid, kThreads, dense_smem_bytes(words, false), st>>>(
        in, in_words, index, nx, ny, nz, nblk, words, mode, mparam, out);
    return cudaGetLastError();
}

// the tile counter and one status word per tile of the variable-size encoder
size_t var_scratch_bytes(int64_t nblk) { return sizeof(uint64_t) * (size_t)((nblk + kThreads - 1) / kThreads + 1); }


}  // namespace ooc
