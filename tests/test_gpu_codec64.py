"""GPU parity of the FR4D codec (FP64 fields): ooc_compress64 /
ooc_decompress64 must reproduce the oracle's FR4D streams and values bit
for bit (Section VI's double fields at R of 64 bits per value, with the
fixed-rate contract of Section IV)."""
import numpy as np
import pytest

import oracle
from synth import random_blocks64, smooth_random_field

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
    d = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    w = ooc.ooc_compress64(d, rate)
    torch.cuda.synchronize()
    return w.cpu().numpy().view(np.uint32)


def gpu_decode(ooc, words, shape, rate):
    d = torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.uint8)).cuda()
    out = ooc.ooc_decompress64(d, shape, rate)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("rate", [1, 2, 8, 16, 24, 32, 48, 64])
@pytest.mark.parametrize("kind", KINDS)
def test_encode_decode_bit_exact(ooc, kind, rate):
    x = random_blocks64(kind, 300, seed=rate * 17 + len(kind))  # 300 blocks: several CTAs and a ragged tail
    ref_w = oracle.fr4d_encode(x, rate)
    got_w = gpu_encode(ooc, x, rate)
    assert np.array_equal(got_w, ref_w)
    ref_x = oracle.fr4d_decode(ref_w, x.shape, rate)
    got_x = gpu_decode(ooc, ref_w, x.shape, rate)
    assert np.array_equal(got_x.view(np.uint64), ref_x.view(np.uint64))


@pytest.mark.parametrize("kind,rate", [(k, 32) for k in KINDS] + [("normal", 24), ("smooth", 24)])
def test_million_blocks_bit_exact(ooc, kind, rate):
    # 10^6 blocks of each class at the paper's 32 (and 24) of 64 bits,
    # streams and values word for word against the oracle; smooth blocks are
    # cut from a smooth FP64 field
    n = 1_000_000
    if kind == "smooth":
        x = smooth_random_field((40, 1000, 1600), 3.0, seed=rate, nterms=64, dtype=np.float64)
    else:
        x = random_blocks64(kind, n, seed=rate * 5 + len(kind))
    ref_w = oracle.fr4d_encode(x, rate)
    got_w = gpu_encode(ooc, x, rate)
    assert got_w.size == n * 2 * rate
    mism = np.flatnonzero(got_w != ref_w)
    assert mism.size == 0, f"{mism.size} words differ, first at block {mism[0] // (2 * rate)}"
    ref_x = oracle.fr4d_decode(ref_w, x.shape, rate)
    got_x = gpu_decode(ooc, ref_w, x.shape, rate)
    assert np.array_equal(got_x.view(np.uint64), ref_x.view(np.uint64))


@pytest.mark.parametrize("shape", [(4, 4, 4), (12, 20, 36), (8, 4, 132), (36, 28, 8)])
def test_fields_of_several_shapes(ooc, shape):
    x = smooth_random_field(shape, 3.0, seed=sum(shape), dtype=np.float64)
    for rate in (24, 32):
        ref_w = oracle.fr4d_encode(x, rate)
        assert np.array_equal(gpu_encode(ooc, x, rate), ref_w)
        assert np.array_equal(gpu_decode(ooc, ref_w, shape, rate).view(np.uint64),
                              oracle.fr4d_decode(ref_w, shape, rate).view(np.uint64))


@pytest.mark.parametrize("rate", [4, 24, 32])
def test_decode_of_arbitrary_words(ooc, rate):
    # Any word content decodes without faulting and exactly as the oracle
    # decodes it (wrapping int64 inverse lifting included).
    rng = np.random.default_rng(rate)
    shape = (16, 16, 16)
    words = rng.integers(0, 1 << 32, size=16 * 16 * 16 * rate // 32, dtype=np.uint64).astype(np.uint32)
    got = gpu_decode(ooc, words, shape, rate)
    ref = oracle.fr4d_decode(words, shape, rate)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_invalid_arguments_are_refused(ooc):
    d = torch.zeros((4, 4, 6), dtype=torch.float64, device="cuda")  # nx not a multiple of 4
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress64(d, 32)
    d = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress64(d, 65)
