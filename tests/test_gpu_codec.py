"""GPU codec parity: the FR4 kernels behind ooc_compress / ooc_decompress
must reproduce the oracle's streams and values bit for bit (Section IV's
fixed-rate codec, defined in the oracle)."""
import numpy as np
import pytest

import oracle
from synth import random_blocks, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ("normal", "wide", "smooth", "constant", "zero", "denormal", "sparse", "bits")


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def gpu_encode(ooc, x, rate):
    d = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    w = ooc.ooc_compress(d, rate)
    torch.cuda.synchronize()
    return w.cpu().numpy().view(np.uint32)


def gpu_decode(ooc, words, shape, rate):
    d = torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.uint8)).cuda()
    out = ooc.ooc_decompress(d, shape, rate)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("rate", [1, 2, 3, 8, 12, 16, 24, 32, 40, 64])
@pytest.mark.parametrize("kind", KINDS)
def test_encode_decode_bit_exact(ooc, kind, rate):
    x = random_blocks(kind, 700, seed=rate * 31 + len(kind))  # 700 blocks: several CTAs and a ragged tail
    ref_w = oracle.fr4_encode(x, rate)
    got_w = gpu_encode(ooc, x, rate)
    assert np.array_equal(got_w, ref_w)
    ref_x = oracle.fr4_decode(ref_w, x.shape, rate)
    got_x = gpu_decode(ooc, ref_w, x.shape, rate)
    assert np.array_equal(got_x.view(np.uint32), ref_x.view(np.uint32))


@pytest.mark.parametrize("kind,rate", [(k, 16) for k in KINDS] + [("normal", 8), ("normal", 24), ("smooth", 8),
                                                                    ("smooth", 24)])
def test_million_blocks_bit_exact(ooc, kind, rate):
    # 10^6 blocks of each class, streams and decoded values word for word
    # against the oracle.  Smooth blocks are cut from a smooth field (the
    # same block order on both sides); the other classes come from the
    # block generator.
    n = 1_000_000
    if kind == "smooth":
        x = smooth_random_field((40, 1000, 1600), 3.0, seed=rate, nterms=64)
        assert x.size == 64 * n
    else:
        x = random_blocks(kind, n, seed=rate * 7 + len(kind))
    ref_w = oracle.fr4_encode(x, rate)
    got_w = gpu_encode(ooc, x, rate)
    assert got_w.size == n * 2 * rate
    mism = np.flatnonzero(got_w != ref_w)
    assert mism.size == 0, f"{mism.size} words differ, first at block {mism[0] // (2 * rate)}"
    ref_x = oracle.fr4_decode(ref_w, x.shape, rate)
    got_x = gpu_decode(ooc, ref_w, x.shape, rate)
    assert np.array_equal(got_x.view(np.uint32), ref_x.view(np.uint32))


@pytest.mark.parametrize("shape", [(4, 4, 4), (12, 20, 36), (8, 4, 132), (36, 28, 8)])
def test_non_cubic_shapes(ooc, shape):
    x = smooth_random_field(shape, 3.0, seed=sum(shape)).astype(np.float32)
    for rate in (8, 16):
        ref_w = oracle.fr4_encode(x, rate)
        assert np.array_equal(gpu_encode(ooc, x, rate), ref_w)
        assert np.array_equal(gpu_decode(ooc, ref_w, shape, rate).view(np.uint32),
                              oracle.fr4_decode(ref_w, shape, rate).view(np.uint32))


@pytest.mark.parametrize("rate", [4, 16, 24])
def test_decode_of_arbitrary_words(ooc, rate):
    # Any word content must decode without faulting and exactly as the oracle
    # decodes it (wrapping int32 inverse lifting included).
    rng = np.random.default_rng(rate)
    shape = (16, 16, 16)
    words = rng.integers(0, 1 << 32, size=16 * 16 * 16 * rate // 32, dtype=np.uint64).astype(np.uint32)
    got = gpu_decode(ooc, words, shape, rate)
    ref = oracle.fr4_decode(words, shape, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_bf16_pack_bit_exact(ooc):
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 1 << 32, size=1 << 18, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    d = torch.from_numpy(x.copy()).cuda()
    packed = ooc.ooc_bf16_pack(d)
    back = ooc.ooc_bf16_unpack(packed)
    torch.cuda.synchronize()
    assert np.array_equal(packed.cpu().numpy().view(np.uint16), oracle.bf16_bits(x))
    assert np.array_equal(back.cpu().numpy().view(np.uint32), oracle.bf16_to_f32(oracle.bf16_bits(x)).view(np.uint32))


@pytest.mark.parametrize("n", [1, 3, 4, 7, 1025, 4096 * 5 + 3, (1 << 22) + 2])
def test_bf16_ragged_lengths(ooc, n):
    # quads of 4 values per vector access, the n mod 4 tail separately, and
    # lengths spanning several rounds of the grid-stride loop
    rng = np.random.default_rng(n)
    x = rng.normal(size=n).astype(np.float32) * np.float32(3.0)
    packed = ooc.ooc_bf16_pack(torch.from_numpy(x).cuda())
    back = ooc.ooc_bf16_unpack(packed)
    torch.cuda.synchronize()
    assert np.array_equal(packed.cpu().numpy().view(np.uint16), oracle.bf16_bits(x))
    assert np.array_equal(back.cpu().numpy().view(np.uint32), oracle.bf16_to_f32(oracle.bf16_bits(x)).view(np.uint32))


def test_bf16_misaligned_pointers_refused(ooc):
    d = torch.zeros(65, device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_bf16_pack(d[1:])


def test_full_size_sampled_blocks(ooc):
    # The 1024^3 field of the heat benchmark, compressed on the GPU in one
    # launch; sampled 4^3 blocks are encoded by the oracle one by one and
    # must equal the matching words of the GPU stream (and decode equally).
    n = 1024
    x = smooth_random_field((n, n, n), 32.0, seed=2)
    rate = 16
    d = torch.from_numpy(x).cuda()
    w = ooc.ooc_compress(d, rate)
    back = ooc.ooc_decompress(w, (n, n, n), rate)
    torch.cuda.synchronize()
    wv = w.view(torch.int32)
    rng = np.random.default_rng(1)
    nb = n // 4
    for _ in range(64):
        bx, by, bz = (int(v) for v in rng.integers(0, nb, size=3))
        blk = x[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
        ref = oracle.fr4_encode(blk, rate)
        b = bx + nb * (by + nb * bz)
        got = wv[b * 2 * rate:(b + 1) * 2 * rate].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref)
        gb = back[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].cpu().numpy()
        assert np.array_equal(gb.view(np.uint32), oracle.fr4_decode(ref, (4, 4, 4), rate).view(np.uint32))
    # stated accuracy of the whole field at this rate
    err = (torch.linalg.vector_norm((back - d).double()) / torch.linalg.vector_norm(d.double())).item()
    assert err < 1e-4, err


def test_compress_argument_errors(ooc):
    d = torch.zeros((8, 8, 8), device="cuda")
    out = torch.empty(8 * 8 * 8 * 2 - 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress(d, 16, d_out=out)  # capacity one word short
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress(d, 0)
    # whole-block shapes take 128-bit loads: the input must be 16-byte aligned
    shifted = torch.zeros(8 * 8 * 8 + 1, device="cuda")[1:].view(8, 8, 8)
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress(shifted, 16)
