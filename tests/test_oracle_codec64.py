"""Pins for the oracle's FR4D codec, the FP64 form of FR4 (CPU only).

Section VI ran double-precision fields stored at 32 and 24 of every 64 bits;
Section IV fixes the codec's contract: a user-chosen number of bits per
value and a compressed size known in advance.  Each step is pinned against
something other than the oracle itself: closed forms computed with numpy,
exact inverses, the per-plane length formula and the fixed-size contract.
"""
import itertools

import numpy as np
import pytest

import oracle
from synth import random_blocks64

KINDS = ("normal", "wide", "smooth", "constant", "zero", "denormal", "sparse", "bits")
NB = 0xAAAAAAAAAAAAAAAA


def blocks_of(x):
    nz, ny, nx = x.shape
    return x.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)


def unblock(b, shape):
    nz, ny, nx = shape
    return b.reshape(nz // 4, ny // 4, nx // 4, 4, 4, 4).transpose(0, 3, 1, 4, 2, 5).reshape(nz, ny, nx)


def closed_form_quantised64(x):
    """sign(x) floor(|x| 2^(58-emax)) 2^(emax-58) per 4^3 block, emax the
    largest frexp exponent of the block's nonzero values clamped at -1022,
    computed with numpy (independent of the C oracle)."""
    x = np.asarray(x, dtype=np.float64)
    b = blocks_of(x)
    _, e = np.frexp(b)
    e = np.where(b != 0, np.maximum(e, -1022), -100000)
    emax = e.max(axis=1, keepdims=True)
    zero_block = emax < -10000
    emax = np.where(zero_block, 0, emax)
    q = np.trunc(np.ldexp(b, 58 - emax)) + 0.0
    y = np.ldexp(q, emax - 58)
    y = np.where(zero_block, 0.0, y)
    return unblock(y, x.shape)


@pytest.mark.parametrize("rate", [1, 8, 16, 24, 32, 64])
def test_compressed_size_is_fixed(rate):
    # Section IV: R bits per value -> exactly N*R/8 bytes, for any content.
    shape = (8, 12, 16)
    for kind in ("normal", "zero", "bits"):
        x = np.resize(random_blocks64(kind, 24, seed=rate).ravel(), shape)
        w = oracle.fr4d_encode(x, rate)
        assert w.nbytes == 8 * 12 * 16 * rate // 8


def test_paper_rates():
    # Section VI: 32 of 64 bits per double is 2:1, 24 of 64 is 8:3.
    x = random_blocks64("normal", 1, seed=0)
    assert 64 * 8 / oracle.fr4d_encode(x, 32).nbytes == 2.0
    assert 64 * 8 / oracle.fr4d_encode(x, 24).nbytes == 64 / 24


@pytest.mark.parametrize("rate", [2, 4, 8, 24, 32])
def test_constant_blocks_exact(rate):
    vals = [0.0, -0.0, 1.0, -1.0, 3.0, 1e-300, -7.25e280, 2.0 ** -1022, 2.0 ** -1074 * 12345, 1.7e308,
            -2.2250738585072014e-308, 1.0 + 2.0 ** -52, np.pi]
    rng = np.random.default_rng(5)
    vals += list(rng.normal(size=20) * np.ldexp(1.0, rng.integers(-900, 900, size=20)))
    x = np.repeat(np.asarray(vals, dtype=np.float64), 64).reshape(-1, 4, 4)
    y = oracle.fr4d_roundtrip(x, rate)
    assert np.array_equal(y, np.where(x == 0, 0.0, x))


@pytest.mark.parametrize("kind", KINDS)
def test_full_precision_equals_block_truncation(kind):
    # With 128 bits per value (8192 bits per block; the coder needs at most
    # 12 + 64 * 64 + 2 * 64 + 64) every plane is coded, so decode(encode(x))
    # must equal the closed-form block-floating-point truncation: the
    # transform and the plane coder are then lossless.
    x = random_blocks64(kind, 128, seed=11)
    y = oracle.fr4d_roundtrip(x, 128)
    ref = closed_form_quantised64(x)
    assert np.array_equal(y.view(np.uint64), ref.view(np.uint64))


def test_zero_block_stream_is_all_zero():
    x = random_blocks64("zero", 16, seed=3)
    for rate in (8, 24, 32):
        w = oracle.fr4d_encode(x, rate)
        assert not w.any()
        y = oracle.fr4d_decode(w, x.shape, rate)
        assert not y.view(np.uint64).any()


def test_header_holds_biased_exponent():
    x = np.zeros((4, 4, 4))
    x[1, 2, 3] = 5.0  # frexp exponent 3
    x[0, 0, 0] = -0.25
    w = oracle.fr4d_encode(x, 8)
    assert w[0] & 1 == 1
    assert (w[0] >> 1) & 0x7FF == 3 + 1023
    d = np.zeros((4, 4, 4))
    d[0, 0, 1] = 2.0 ** -1060  # subnormal: the exponent clamps to -1022
    w = oracle.fr4d_encode(d, 8)
    assert (w[0] >> 1) & 0x7FF == -1022 + 1023
    h = np.zeros((4, 4, 4))
    h[3, 3, 3] = -1.5e308  # frexp exponent 1024
    w = oracle.fr4d_encode(h, 8)
    assert (w[0] >> 1) & 0x7FF == 1024 + 1023


def lift_ref(a):
    """FR4's 4-point lift written out with Python integers (floor halving)."""
    a0, a1, a2, a3 = (int(v) for v in a)
    d0 = a0 - a1
    s0 = a1 + (d0 >> 1)
    d1 = a2 - a3
    s1 = a3 + (d1 >> 1)
    D = s0 - s1
    S = s1 + (D >> 1)
    return [S, D, d0 - (D >> 1), d1 - (D >> 1)]


def test_transform_is_three_passes_of_the_lift_and_inverts_exactly():
    rng = np.random.default_rng(7)
    for _ in range(200):
        q = rng.integers(-(1 << 58) + 1, 1 << 58, size=64, dtype=np.int64)
        c, wrapped = oracle.fr4d_transform_forward(q)
        assert not wrapped
        ref = [int(v) for v in q]
        for lines in ([[4 * y + 16 * z + i for i in range(4)] for z in range(4) for y in range(4)],
                      [[x + 16 * z + 4 * i for i in range(4)] for z in range(4) for x in range(4)],
                      [[x + 4 * y + 16 * i for i in range(4)] for y in range(4) for x in range(4)]):
            for idx in lines:
                out = lift_ref([ref[j] for j in idx])
                for j, v in zip(idx, out):
                    ref[j] = v
        assert [int(v) for v in c] == ref
        back, wrapped = oracle.fr4d_transform_inverse(c)
        assert not wrapped and np.array_equal(back, q)


def test_transform_headroom_on_extreme_blocks():
    # |q| < 2^58 on input: every extreme sign pattern along one line, with
    # the rest of the block at the extremes too, stays below 2^62.
    m = (1 << 58) - 1
    for signs in itertools.product((-1, 1), repeat=4):
        for rest in (-1, 1):
            q = np.full(64, rest * m, dtype=np.int64)
            q[:4] = np.asarray(signs, dtype=np.int64) * m
            c, wrapped = oracle.fr4d_transform_forward(q)
            assert not wrapped
            assert np.abs(c.astype(object)).max() < 2 ** 62


def test_negabinary_digits_of_the_dc_coefficient():
    # A constant block has only its DC coefficient, q = trunc(c 2^(58-emax));
    # its stream's planes, read as base -2 digits, must sum to q.
    rng = np.random.default_rng(2)
    vals = np.concatenate([rng.normal(size=200) * np.ldexp(1.0, rng.integers(-500, 500, size=200)),
                           [1.0, -1.0, 0.75, -0.75, 3.0, -5.5]])
    for c in vals:
        x = np.full((4, 4, 4), c)
        w = oracle.fr4d_encode(x, 128)
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")
        body = np.packbits(bits[12:], bitorder="little")
        body = np.concatenate([body, np.zeros((-body.size) % 4 + 8, np.uint8)]).view(np.uint32)
        u, _ = oracle.fr4d_decode_planes(body, 64 * 128 - 12)
        assert not u[1:].any()
        _, e = np.frexp(c)
        q = int(np.trunc(np.ldexp(c, 58 - max(int(e), -1022))))
        val = sum(((int(u[0]) >> j) & 1) * (-2) ** j for j in range(64))
        assert val == q
        assert int(u[0]) == ((q + NB) ^ NB) % (1 << 64)


def plane_length_formula64(u):
    """Bits the 64-plane coder writes at full budget, from the plane masks:
    per plane the n refinement bits; then one group bit per new coefficient
    and the scanned bits up to its one (the last coefficient's one implied);
    a closing group bit 0 while coefficients remain."""
    total, n = 0, 0
    for p in range(63, -1, -1):
        X = 0
        for i in range(64):
            X |= ((int(u[i]) >> p) & 1) << i
        total += n
        if n == 64:
            continue
        rest = X >> n
        if rest == 0:
            total += 1
            continue
        t_last = rest.bit_length() - 1
        total += bin(rest).count("1") + t_last + 1
        if n + t_last == 63:
            total -= 1
        n += t_last + 1
        if n < 64:
            total += 1
    return total


def plane_vectors64():
    rng = np.random.default_rng(9)
    vecs = [np.zeros(64, np.uint64), np.full(64, np.iinfo(np.uint64).max, np.uint64)]
    one = np.zeros(64, np.uint64); one[63] = 1; vecs.append(one)
    top = np.zeros(64, np.uint64); top[63] = np.uint64(1 << 63); vecs.append(top)
    for _ in range(100):
        v = rng.integers(0, np.iinfo(np.uint64).max, size=64, dtype=np.uint64, endpoint=True)
        vecs.append(v >> rng.integers(0, 64, size=64).astype(np.uint64))
    for _ in range(40):
        v = np.zeros(64, np.uint64)
        idx = rng.choice(64, size=rng.integers(1, 6), replace=False)
        v[idx] = rng.integers(1, np.iinfo(np.uint64).max, size=idx.size, dtype=np.uint64)
        vecs.append(v)
    return vecs


def test_plane_coder_lossless_and_length_formula():
    for u in plane_vectors64():
        words, nbits = oracle.fr4d_encode_planes(u, 16384)
        assert nbits == plane_length_formula64(u)
        back, nread = oracle.fr4d_decode_planes(words, 16384)
        assert nread == nbits
        assert np.array_equal(back, u)


def test_plane_coder_embedded_prefix_and_truncation():
    rng = np.random.default_rng(4)
    for u in plane_vectors64()[::5]:
        full, nfull = oracle.fr4d_encode_planes(u, 16384)
        for budget in sorted(set(rng.integers(0, nfull + 2, size=10).tolist() + [0, 1, nfull])):
            w, n = oracle.fr4d_encode_planes(u, budget)
            assert n == min(budget, nfull)
            bits = np.unpackbits(w.view(np.uint8), bitorder="little")
            fbits = np.unpackbits(full.view(np.uint8), bitorder="little")
            assert np.array_equal(bits[:n], fbits[:n]) and not bits[n:].any()
            back, _ = oracle.fr4d_decode_planes(w, budget)
            assert not np.any(back & ~u)


@pytest.mark.parametrize("kind", ["smooth", "normal"])
def test_error_decreases_with_rate(kind):
    x = random_blocks64(kind, 200, seed=21)
    errs = []
    for rate in (8, 16, 24, 32, 48, 64):
        y = oracle.fr4d_roundtrip(x, rate)
        errs.append(np.linalg.norm(y - x) / np.linalg.norm(x))
    assert all(a >= b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-15


def test_separate_compression_units_are_independent():
    # Section V-A: remainder and common region are compressed separately;
    # with 4-aligned z boundaries a plane range's stream is the matching
    # byte range of the whole field's stream.
    from synth import sine_modes_field
    x, _ = sine_modes_field((32, 16, 12), seed=0)
    x = np.asarray(x, dtype=np.float64)
    for rate in (24, 32):
        whole = oracle.fr4d_encode(x, rate)
        per_plane_words = 16 * 12 * rate // 8 // 4
        for z0, z1 in ((0, 4), (4, 12), (12, 32), (8, 28)):
            part = oracle.fr4d_encode(x[z0:z1], rate)
            assert np.array_equal(part, whole[z0 * per_plane_words: z1 * per_plane_words])


def test_paper_rates_accuracy_on_a_smooth_field():
    # Sanity for Section VI's rates on a smooth double field: 32/64 keeps
    # about 1e-9 relative L2, 24/64 about 1e-6 (FR4 at 16/32 keeps ~1e-5).
    from synth import smooth_random_field
    x = smooth_random_field((32, 32, 32), corr_len=8.0, seed=2, dtype=np.float64)
    e = {r: np.linalg.norm(oracle.fr4d_roundtrip(x, r) - x) / np.linalg.norm(x) for r in (24, 32)}
    assert e[32] < 1e-8 and e[24] < 1e-5 and e[32] < e[24] / 50, e


def test_fp64_storage_pipeline_reduces_to_plain_runs():
    # With FP64 storage the FP64 plan's oracle pipeline is the plain FP64
    # run, exactly: no rounding happens at the pass boundaries.
    from synth import sine_modes_field
    u0, _ = sine_modes_field((16, 12, 20), seed=1)
    u0 = np.asarray(u0, dtype=np.float64)
    a = oracle.heat7_storage_pipeline(u0, 9, 4, "fp64", precision="fp64")
    assert np.array_equal(a, oracle.heat7_run(u0, 9))
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=(16, 12, 20)) * 1e-3
    kap = 0.05 + 0.01 * rng.random((16, 12, 20))
    p, q = oracle.wave25_storage_pipeline(p0, 0.9 * p0, kap, 7, 3, "fp64", precision="fp64")
    pr, qr = oracle.wave25_run(p0, 0.9 * p0, kap, 7)
    assert np.array_equal(p, pr) and np.array_equal(q, qr)
    # and FR4D storage applies exactly the codec's round trip at each boundary
    b = oracle.heat7_storage_pipeline(u0, 4, 4, "fr4", rate=24, precision="fp64")
    ref = oracle.fr4d_roundtrip(oracle.heat7_run(oracle.fr4d_roundtrip(u0, 24), 4), 24)
    assert np.array_equal(b, ref)
