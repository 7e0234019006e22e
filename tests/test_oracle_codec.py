"""Pins for the oracle's FR4 codec (CPU only).

The paper fixes only the codec's contract (Section IV): a user-chosen number
of bits per value, hence a compressed size known in advance so that buffers
can be preallocated.  Each step of the codec is pinned here against
something other than the oracle itself: closed forms, exhaustive small
cases, the independent per-plane length formula, and the paper's fixed-size
contract.
"""
import itertools

import numpy as np
import pytest

import oracle
from synth import random_blocks

RATES = (8, 12, 16, 24)
KINDS = ("normal", "wide", "smooth", "constant", "zero", "denormal", "sparse", "bits")


def closed_form_quantised(x):
    """sign(x) * floor(|x| 2^(26-emax)) * 2^(emax-26) per 4^3 block, with emax
    the largest frexp exponent of the block's nonzero values clamped at -126,
    computed in float64 with numpy (independent of the C oracle)."""
    x = np.asarray(x, dtype=np.float32)
    nz, ny, nx = x.shape
    b = x.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64).astype(np.float64)
    _, e = np.frexp(b)
    e = np.where(b != 0, np.maximum(e, -126), -100000)
    emax = e.max(axis=1, keepdims=True)
    zero_block = emax < -1000
    emax = np.where(zero_block, 0, emax)
    q = np.trunc(np.ldexp(b, 26 - emax)) + 0.0  # integer q: a zero is +0
    y = np.ldexp(q, emax - 26)
    y = np.where(zero_block, 0.0, y)
    y = y.reshape(nz // 4, ny // 4, nx // 4, 4, 4, 4).transpose(0, 3, 1, 4, 2, 5).reshape(nz, ny, nx)
    return y.astype(np.float32)


@pytest.mark.parametrize("rate", [1, 2, 8, 12, 16, 24, 32, 40])
def test_compressed_size_is_fixed(rate):
    # Section IV: R bits per value -> exactly N*R/8 bytes, for any content.
    shape = (8, 12, 16)
    assert oracle.compressed_bytes(shape, rate) == 8 * 12 * 16 * rate // 8
    for kind in ("normal", "zero", "bits"):
        x = random_blocks(kind, 24, seed=rate)[: 8].reshape(8, 4, 4)
        x = np.resize(random_blocks(kind, 24, seed=rate).ravel(), shape).astype(np.float32)
        w = oracle.fr4_encode(x, rate)
        assert w.nbytes == 8 * 12 * 16 * rate // 8


def test_paper_ratio_example():
    # Section IV: 32 bits kept per 64-bit double is 2:1.  FR4 keeps R bits
    # per 32-bit float, so R = 16 is the same 2:1 and R = 8 is 4:1.
    shape = (4, 4, 4)
    assert 64 * 4 / oracle.compressed_bytes(shape, 16) == 2.0
    assert 64 * 4 / oracle.compressed_bytes(shape, 8) == 4.0


@pytest.mark.parametrize("rate", [2, 4, 8, 12, 16, 24])
def test_constant_blocks_exact(rate):
    vals = [0.0, -0.0, 1.0, -1.0, 3.0, 1e-30, -7.25e20, 2.0 ** -126, 2.0 ** -149 * 12345, 3.4e38, -1.17549435e-38]
    rng = np.random.default_rng(5)
    vals += list(rng.normal(size=20) * np.ldexp(1.0, rng.integers(-100, 100, size=20)))
    x = np.repeat(np.asarray(vals, dtype=np.float32), 64).reshape(-1, 4, 4)
    y = oracle.fr4_roundtrip(x, rate)
    assert np.array_equal(y, np.where(x == 0, np.float32(0), x))


@pytest.mark.parametrize("kind", KINDS)
def test_full_precision_equals_block_truncation(kind):
    # With enough bits (R = 40 > worst case 2153 bits / 64) every plane is
    # coded, so decode(encode(x)) must equal the closed-form block-floating-
    # point truncation: the transform and the plane coder are then lossless.
    x = random_blocks(kind, 256, seed=11)
    y = oracle.fr4_roundtrip(x, 40)
    ref = closed_form_quantised(x)
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))


def test_zero_block_stream_is_all_zero():
    x = random_blocks("zero", 16, seed=3)
    for rate in RATES:
        w = oracle.fr4_encode(x, rate)
        assert not w.any()
        y = oracle.fr4_decode(w, x.shape, rate)
        assert np.array_equal(y.view(np.uint32), np.zeros_like(y).view(np.uint32))


def test_header_holds_biased_exponent():
    x = np.zeros((4, 4, 4), dtype=np.float32)
    x[1, 2, 3] = 5.0  # frexp exponent 3
    x[0, 0, 0] = -0.25
    w = oracle.fr4_encode(x, 8)
    assert w[0] & 1 == 1
    assert (w[0] >> 1) & 0xFF == 3 + 127
    d = np.zeros((4, 4, 4), dtype=np.float32)
    d[0, 0, 1] = np.float32(2.0 ** -140)  # subnormal: exponent clamps to -126
    w = oracle.fr4_encode(d, 8)
    assert (w[0] >> 1) & 0xFF == -126 + 127


def test_lift_exact_inverse_and_range_bound_exhaustive():
    B = 9
    rng_vals = range(-B, B + 1)
    worst = 0
    for t in itertools.product(rng_vals, repeat=4):
        a = np.array(t, dtype=np.int32)
        y = oracle.lift_forward4(a)
        worst = max(worst, int(np.abs(y.astype(np.int64)).max()))
        assert np.array_equal(oracle.lift_inverse4(y), a)
    assert worst <= 2.5 * B + 1.25


def test_lift_range_bound_at_extremes():
    M = 2 ** 26 - 1
    for t in itertools.product((-M, -M + 1, -1, 0, 1, M - 1, M), repeat=4):
        a = np.array(t, dtype=np.int32)
        y = oracle.lift_forward4(a).astype(np.int64)
        assert np.abs(y).max() <= 2.5 * M + 1.25
        assert np.array_equal(oracle.lift_inverse4(y.astype(np.int32)), a)


def test_transform_headroom_on_extreme_blocks():
    # Three passes from |q| < 2^26 stay below 2^30: no int32 wrap on encode.
    M = 2 ** 26 - 1
    rng = np.random.default_rng(7)
    pats = [rng.choice([-M, M], size=64) for _ in range(3000)]
    pats += [rng.integers(-M, M + 1, size=64) for _ in range(1000)]
    pats += [np.full(64, M), np.full(64, -M), np.resize([M, -M], 64), np.resize([M, M, -M, -M], 64)]
    for p in pats:
        c, wrapped = oracle.transform_forward(p)
        assert not wrapped
        assert np.abs(c.astype(np.int64)).max() < 2 ** 30
        back, _ = oracle.transform_inverse(c)
        assert np.array_equal(back, np.asarray(p, dtype=np.int32))


def test_lift_properties_constant_and_linear():
    # A constant line maps to DC only; a linear ramp leaves only S and D
    # (the trend prediction removes it from the details).  This pins the
    # prediction's sign and the output positions.
    for c in (-1000, -1, 0, 7, 123456):
        assert np.array_equal(oracle.lift_forward4([c] * 4), [c, 0, 0, 0])
    for beta in (-40, -3, 1, 2, 5, 64, 1000):
        for off in (-17, 0, 9):
            a = np.array([off + beta * i for i in range(4)], dtype=np.int32)
            S, D, d0, d1 = oracle.lift_forward4(a)
            assert D == -2 * beta
            assert d0 == 0 and d1 == 0
            assert abs(S - (off + 1.5 * beta)) <= 1
    c, _ = oracle.transform_forward(np.full(64, 99))
    assert c[0] == 99 and not c[1:].any()


def test_sequency_order_is_a_sorted_permutation():
    order = oracle.sequency_order()
    assert sorted(order.tolist()) == list(range(64))
    lev = np.array([0, 1, 2, 2])
    key = [lev[l & 3] + lev[(l >> 2) & 3] + lev[l >> 4] for l in order]
    assert key == sorted(key)
    assert order[0] == 0 and set(order[1:4]) == {1, 4, 16}


def test_negabinary_digits_of_the_dc_coefficient():
    # For a constant block the only nonzero coefficient is the DC one, equal
    # to q = trunc(c 2^(26-emax)).  Strip the 9 header bits from the stream,
    # decode the planes, and read the DC word's bits as base -2 digits: they
    # must sum to q.  This pins the encoder's negabinary map itself.
    rng = np.random.default_rng(2)
    vals = np.concatenate([rng.normal(size=300) * np.ldexp(1.0, rng.integers(-60, 60, size=300)),
                           [1.0, -1.0, 0.75, -0.75, 3.0, -5.5]]).astype(np.float32)
    for c in vals:
        x = np.full((4, 4, 4), c, dtype=np.float32)
        w = oracle.fr4_encode(x, 40)
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")
        body = np.packbits(bits[9:], bitorder="little")
        body = np.concatenate([body, np.zeros((-body.size) % 4 + 8, np.uint8)]).view(np.uint32)
        u, _ = oracle.decode_planes(body, 64 * 40 - 9)
        assert not u[1:].any()
        _, e = np.frexp(np.float64(c))
        q = int(np.trunc(np.ldexp(np.float64(c), 26 - max(int(e), -126))))
        val = sum(((int(u[0]) >> j) & 1) * (-2) ** j for j in range(32))
        assert val == q


def plane_length_formula(u):
    """Independent count of the bits the plane coder writes at full budget,
    per plane from the plane masks: refinement n_p bits, then one group bit
    per newly significant coefficient plus the scanned bits (the last
    coefficient's one implied), plus a closing 0 group bit if any
    coefficient is left insignificant."""
    total = 0
    n = 0
    for p in range(31, -1, -1):
        X = 0
        for i in range(64):
            X |= ((int(u[i]) >> p) & 1) << i
        total += n
        rest = X >> n if n < 64 else 0
        if n == 64:
            continue
        if rest == 0:
            total += 1
            continue
        ones = bin(rest).count("1")
        t_last = rest.bit_length() - 1
        total += ones + (t_last + 1)
        if n + t_last == 63:
            total -= 1  # implied one of the last coefficient
        n_new = n + t_last + 1
        if n_new < 64:
            total += 1  # closing group bit 0
        n = n_new
    return total


def plane_test_vectors():
    rng = np.random.default_rng(9)
    vecs = [np.zeros(64, np.uint32), np.full(64, 0xFFFFFFFF, np.uint32)]
    one = np.zeros(64, np.uint32); one[63] = 1; vecs.append(one)
    top = np.zeros(64, np.uint32); top[63] = 1 << 31; vecs.append(top)
    mid = np.zeros(64, np.uint32); mid[62] = 5; mid[63] = 3; vecs.append(mid)
    for _ in range(150):
        v = rng.integers(0, 1 << 32, size=64, dtype=np.uint64).astype(np.uint32)
        shift = rng.integers(0, 32, size=64)
        vecs.append((v >> shift.astype(np.uint32)).astype(np.uint32))
    for _ in range(50):
        v = np.zeros(64, np.uint32)
        idx = rng.choice(64, size=rng.integers(1, 6), replace=False)
        v[idx] = rng.integers(1, 1 << 32, size=idx.size, dtype=np.uint64).astype(np.uint32)
        vecs.append(v)
    return vecs


def test_plane_coder_lossless_and_length_formula():
    for u in plane_test_vectors():
        words, nbits = oracle.encode_planes(u, 4096)
        assert nbits == plane_length_formula(u)
        back, nread = oracle.decode_planes(words, 4096)
        assert nread == nbits
        assert np.array_equal(back, u)


def test_plane_coder_embedded_prefix_and_truncation():
    # Embedded coding: the stream at a smaller budget is a prefix of the
    # stream at a larger one, and a truncated decode only drops bits.
    rng = np.random.default_rng(4)
    for u in plane_test_vectors()[::4]:
        full, nfull = oracle.encode_planes(u, 4096)
        for budget in sorted(set(rng.integers(0, nfull + 2, size=12).tolist() + [0, 1, nfull])):
            w, n = oracle.encode_planes(u, budget)
            assert n == min(budget, nfull)
            bits = np.unpackbits(w.view(np.uint8), bitorder="little")[:n]
            fbits = np.unpackbits(full.view(np.uint8), bitorder="little")[:n]
            assert np.array_equal(bits, fbits)
            assert not np.unpackbits(w.view(np.uint8), bitorder="little")[n:].any()
            back, _ = oracle.decode_planes(w, budget)
            assert not np.any(back & ~u)


@pytest.mark.parametrize("kind", ["smooth", "normal"])
def test_error_decreases_with_rate(kind):
    x = random_blocks(kind, 400, seed=21).astype(np.float64)
    errs = []
    for rate in (4, 8, 12, 16, 24, 32):
        y = oracle.fr4_roundtrip(x, rate).astype(np.float64)
        errs.append(np.linalg.norm(y - x) / np.linalg.norm(x))
    assert all(a >= b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6


def test_separate_compression_units_are_independent():
    # Section V-A: the remainder and the common region are compressed
    # separately.  With 4^3 blocks and 4-aligned z boundaries, the stream of
    # any plane range is exactly the matching byte range of the whole-field
    # stream, so either unit can be rewritten without touching the other.
    x, _ = __import__("synth").sine_modes_field((32, 16, 12), seed=0)
    for rate in RATES:
        whole = oracle.fr4_encode(x, rate)
        per_plane_words = 16 * 12 * rate // 8 // 4
        for z0, z1 in ((0, 4), (4, 12), (12, 32), (8, 28)):
            part = oracle.fr4_encode(x[z0:z1], rate)
            assert np.array_equal(part, whole[z0 * per_plane_words: z1 * per_plane_words])


def test_smooth_field_accuracy_by_rate():
    # Sanity on a smooth field: 16 bits/value keeps ~1e-4 relative L2 or better.
    from synth import smooth_random_field
    x = smooth_random_field((32, 32, 32), corr_len=8.0, seed=2)
    e = {}
    for rate in RATES:
        y = oracle.fr4_roundtrip(x, rate)
        e[rate] = np.linalg.norm(y - x) / np.linalg.norm(x)
    assert e[16] < 1e-4 and e[24] < 1e-6, e


def test_single_spike_block_error_bound():
    # One nonzero value in a block: the lifting spreads it over many
    # coefficients, so R = 24 (1527 bits after the header) does not hold all
    # 32 planes.  The block floating point holds a normal FP32 spike exactly
    # (24 significant bits in 26), so the error comes from the planes the
    # budget drops.  Here the coder delivers every plane from 31 down to 6;
    # the dropped negabinary planes 0..5 carry less than (2/3) 2^6 per
    # coefficient and the inverse lifting amplifies by at most 11.4 (its
    # largest row sum, 2.25 per axis), so the error stays below
    # 11.4 * (2/3) * 2^6 < 2^9 units of 2^(emax - 26) (the worst case
    # measured over these spikes is 142 units).  A higher rate never does
    # worse on the same spike.
    rng = np.random.default_rng(3)
    order = oracle.sequency_order()
    nb = np.uint32(0xAAAAAAAA)
    for i in range(64):
        for _ in range(4):
            b = np.zeros((4, 4, 4), np.float32)
            v = np.float32(rng.normal() * 10.0 ** rng.integers(-20, 20))
            b.flat[i] = v
            emax = np.frexp(np.float64(v))[1]
            unit = 2.0 ** (emax - 26)
            # the planes the R = 24 budget delivers: all of 31 .. 6
            q = np.zeros(64, np.int32)
            q[i] = int(np.trunc(np.float64(v) * 2.0 ** (26 - emax)))
            coef, wrapped = oracle.transform_forward(q)
            assert not wrapped
            u = ((coef.astype(np.int64)[order].astype(np.uint32) + nb) ^ nb).astype(np.uint32)
            words, _ = oracle.encode_planes(u, 24 * 64 - 9)
            back, _ = oracle.decode_planes(words, 24 * 64 - 9)
            top = np.uint32(0xFFFFFFFF << 6 & 0xFFFFFFFF)
            assert np.array_equal(np.asarray(back, np.uint32) & top, u & top)
            e24 = np.abs(oracle.fr4_roundtrip(b, 24).astype(np.float64) - b).max()
            e16 = np.abs(oracle.fr4_roundtrip(b, 16).astype(np.float64) - b).max()
            assert e24 <= 2.0 ** 9 * unit, (i, v, e24 / unit)
            assert e24 <= e16
