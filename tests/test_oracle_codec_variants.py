"""Pins of the oracle's codec variants (beyond the paper's fixed rate):
partial blocks for sides that are not multiples of 4, and the two
variable-size modes, fixed precision and fixed accuracy.

Partial blocks are pinned against the fixed-rate coder on an explicitly
edge-padded field (numpy's np.pad, not the oracle).  Fixed precision 32 is
pinned against block floating point computed here with numpy (the coder
then loses nothing beyond the quantisation).  Fixed accuracy is pinned by
its error guarantee and by its two limits (everything dropped, nothing
dropped)."""
import numpy as np
import pytest

import oracle
from synth import random_blocks, smooth_random_field

SHAPES = [(5, 6, 7), (1, 1, 1), (4, 9, 13), (3, 4, 8), (9, 2, 4)]


def padded(f):
    nz, ny, nx = f.shape
    return np.pad(f, ((0, -nz % 4), (0, -ny % 4), (0, -nx % 4)), mode="edge")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("rate", [4, 16])
def test_partial_blocks_equal_edge_padded_field(shape, rate):
    f = smooth_random_field(shape, 3.0, seed=1) * 7.0
    words = oracle.fr4_encode(f, rate)
    ref = oracle.fr4_encode(padded(f), rate)
    assert np.array_equal(words, ref)
    nz, ny, nx = shape
    assert words.nbytes == oracle.compressed_bytes(shape, rate)
    dec = oracle.fr4_decode(words, shape, rate)
    assert np.array_equal(dec, oracle.fr4_decode(ref, padded(f).shape, rate)[:nz, :ny, :nx])


def bfp_dequantised(block):
    """Block floating point of one 4^3 block written out with numpy:
    q = trunc(x 2^(26 - emax)), back as RN(RN(q) 2^(emax - 26))."""
    x = block.astype(np.float64)
    nz = x[x != 0]
    if nz.size == 0:
        return np.zeros_like(block)
    emax = max(max(int(np.frexp(v)[1]) for v in nz), -126)
    q = np.trunc(np.ldexp(x, 26 - emax)) + 0.0  # an integer zero is +0
    return (q.astype(np.float32).astype(np.float64) * 2.0 ** (emax - 26)).astype(np.float32)


@pytest.mark.parametrize("kind", ["normal", "wide", "smooth", "sparse"])
def test_precision_32_loses_nothing_beyond_quantisation(kind):
    f = random_blocks(kind, 200, seed=3)  # 4^3 blocks stacked in z
    words, index = oracle.fr4_encode_var(f, oracle.MODE_PRECISION, 32)
    dec = oracle.fr4_decode_var(words, index, f.shape, oracle.MODE_PRECISION, 32)
    for b in range(f.shape[0] // 4):
        got = dec[4 * b:4 * b + 4]
        assert np.array_equal(got.view(np.uint32), bfp_dequantised(f[4 * b:4 * b + 4]).view(np.uint32)), b


def test_precision_error_is_monotone_and_size_bounded():
    f = smooth_random_field((16, 20, 24), 4.0, seed=5) * 3.0
    errs, sizes = [], []
    for P in (4, 8, 12, 16, 20, 24, 28, 32):
        words, index = oracle.fr4_encode_var(f, oracle.MODE_PRECISION, P)
        dec = oracle.fr4_decode_var(words, index, f.shape, oracle.MODE_PRECISION, P)
        errs.append(float(np.abs(dec.astype(np.float64) - f).max()))
        sizes.append(words.size)
        per_block = np.diff(index.astype(np.int64))
        assert per_block.max() <= (9 + 129 * P + 31) // 32
        assert index[0] == 0 and int(index[-1]) == words.size
    assert all(a >= b for a, b in zip(errs, errs[1:])), errs
    assert all(a <= b for a, b in zip(sizes, sizes[1:])), sizes


def test_precision_stream_is_a_prefix_of_the_fixed_rate_stream():
    # Both modes run the same embedded coder; with a budget past the P-plane
    # length the fixed-rate block starts with the P-plane block's bits.
    f = smooth_random_field((4, 4, 8), 2.0, seed=6)
    fixed = oracle.fr4_encode(f, 64).reshape(2, 128)
    for P in (3, 9, 17):
        words, index = oracle.fr4_encode_var(f, oracle.MODE_PRECISION, P)
        for b in range(2):
            blk = words[int(index[b]):int(index[b + 1])]
            nbits = blk.size * 32
            assert nbits <= 64 * 64
            bits_var = np.unpackbits(blk.view(np.uint8), bitorder="little")
            bits_fix = np.unpackbits(fixed[b].view(np.uint8), bitorder="little")[:nbits]
            # the variable block is zero-padded to a word after its last plane
            last = np.nonzero(bits_var)[0].max() + 1 if bits_var.any() else 0
            assert np.array_equal(bits_var[:last], bits_fix[:last])


@pytest.mark.parametrize("kind", ["normal", "wide", "smooth"])
@pytest.mark.parametrize("rel_tol", [2.0 ** -4, 2.0 ** -9, 2.0 ** -15])
def test_accuracy_mode_meets_its_tolerance(kind, rel_tol):
    f = random_blocks(kind, 300, seed=7)
    scale = float(np.abs(f).max())
    tol = rel_tol * scale
    words, index = oracle.fr4_encode_var(f, oracle.MODE_ACCURACY, tol)
    dec = oracle.fr4_decode_var(words, index, f.shape, oracle.MODE_ACCURACY, tol)
    assert float(np.abs(dec.astype(np.float64) - f).max()) <= tol


def test_accuracy_mode_limits():
    f = smooth_random_field((8, 8, 12), 3.0, seed=9) * 5.0
    scale = float(np.abs(f).max())
    # a tolerance above every value drops every plane: header words only
    words, index = oracle.fr4_encode_var(f, oracle.MODE_ACCURACY, 2.0 ** 40 * scale)
    assert np.all(np.diff(index.astype(np.int64)) == 1)
    dec = oracle.fr4_decode_var(words, index, f.shape, oracle.MODE_ACCURACY, 2.0 ** 40 * scale)
    assert not dec.any()
    # a tolerance below the format's resolution keeps every plane: the
    # stream is the 32-plane fixed-precision stream
    wa, ia = oracle.fr4_encode_var(f, oracle.MODE_ACCURACY, 1e-30)
    wp, ip = oracle.fr4_encode_var(f, oracle.MODE_PRECISION, 32)
    assert np.array_equal(wa, wp) and np.array_equal(ia, ip)


def test_accuracy_size_shrinks_with_tolerance():
    f = smooth_random_field((16, 16, 16), 4.0, seed=10)
    sizes = [oracle.fr4_encode_var(f, oracle.MODE_ACCURACY, t)[0].size for t in (1e-7, 1e-5, 1e-3, 1e-1)]
    assert all(a > b for a, b in zip(sizes, sizes[1:])), sizes


def test_bad_arguments():
    f = np.zeros((4, 4, 4), np.float32)
    for mode, param in ((oracle.MODE_PRECISION, 0), (oracle.MODE_PRECISION, 33), (oracle.MODE_PRECISION, 2.5),
                        (oracle.MODE_ACCURACY, 0.0), (oracle.MODE_ACCURACY, -1.0), (7, 1.0)):
        with pytest.raises(RuntimeError):
            oracle.fr4_encode_var(f, mode, param)
