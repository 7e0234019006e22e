"""GPU codec variants against the oracle, bit for bit: fixed-rate streams of
fields whose sides are not multiples of 4 (edge-padded partial blocks), and
the variable-size fixed-precision and fixed-accuracy modes (stream words,
block index and decoded values)."""
import numpy as np
import pytest

import oracle
from synth import random_blocks, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


SHAPES = [(5, 6, 7), (1, 1, 1), (13, 9, 4), (4, 4, 130), (37, 45, 133), (8, 3, 8)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("rate", [1, 8, 16, 24, 64])
def test_partial_blocks_fixed_rate(ooc, shape, rate):
    f = smooth_random_field(shape, 3.0, seed=2) * 5.0
    d = torch.from_numpy(f).cuda()
    words = ooc.ooc_compress(d, rate).cpu().numpy().view(np.uint32)
    ref = oracle.fr4_encode(f, rate)
    assert np.array_equal(words, ref)
    got = ooc.ooc_decompress(torch.from_numpy(ref.view(np.uint8)).cuda(), shape, rate).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), oracle.fr4_decode(ref, shape, rate).view(np.uint32))


VAR_CASES = [(1, 1), (1, 8), (1, 16), (1, 32), (2, 1e-6), (2, 1e-3), (2, 0.25), (2, 1e-30), (2, 1e30)]


@pytest.mark.parametrize("mode,param", VAR_CASES)
@pytest.mark.parametrize("shape", [(8, 12, 16), (5, 6, 7), (37, 45, 133)])
def test_variable_modes_match_oracle(ooc, mode, param, shape):
    f = smooth_random_field(shape, 4.0, seed=3) * 3.0
    d = torch.from_numpy(f).cuda()
    stream, index = ooc.ooc_compress_var(d, mode, param)
    torch.cuda.synchronize()
    words_ref, index_ref = oracle.fr4_encode_var(f, mode, param)
    assert np.array_equal(index.cpu().numpy().astype(np.uint64), index_ref)
    assert np.array_equal(stream.cpu().numpy().view(np.uint32), words_ref)
    got = ooc.ooc_decompress_var(stream, index, shape, mode, param).cpu().numpy()
    ref = oracle.fr4_decode_var(words_ref, index_ref, shape, mode, param)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("kind", ["normal", "wide", "constant", "zero", "denormal", "sparse", "bits"])
def test_variable_modes_block_classes(ooc, kind):
    f = random_blocks(kind, 500, seed=11)
    d = torch.from_numpy(f).cuda()
    for mode, param in ((1, 12), (2, 1e-4 * float(np.abs(f).max() + 1e-30))):
        stream, index = ooc.ooc_compress_var(d, mode, param)
        words_ref, index_ref = oracle.fr4_encode_var(f, mode, param)
        assert np.array_equal(stream.cpu().numpy().view(np.uint32), words_ref)
        got = ooc.ooc_decompress_var(stream, index, f.shape, mode, param).cpu().numpy()
        ref = oracle.fr4_decode_var(words_ref, index_ref, f.shape, mode, param)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_accuracy_tolerance_on_gpu(ooc):
    f = smooth_random_field((64, 64, 64), 8.0, seed=4)
    d = torch.from_numpy(f).cuda()
    for tol in (1e-2, 1e-4, 1e-6):
        stream, index = ooc.ooc_compress_var(d, ooc.OOC_FR4_ACCURACY, tol)
        got = ooc.ooc_decompress_var(stream, index, f.shape, ooc.OOC_FR4_ACCURACY, tol).cpu().numpy()
        assert float(np.abs(got.astype(np.float64) - f).max()) <= tol


def test_small_capacity_and_bad_arguments(ooc):
    f = torch.from_numpy(smooth_random_field((16, 16, 16), 3.0, seed=5)).cuda()
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_compress_var(f, ooc.OOC_FR4_PRECISION, 20, d_out=small)
    for mode, param in ((1, 0), (1, 33), (1, 2.5), (2, 0.0), (2, float("inf")), (3, 1.0)):
        with pytest.raises(ooc.OocError):
            ooc.ooc_compress_var(f, mode, param)


def test_overflow_writes_whole_blocks_within_the_capacity_only(ooc):
    # A stream larger than the capacity: the call reports the size it needs,
    # every offset, and the leading blocks that fit; nothing lands past the
    # capacity (checked on a guard region behind it).
    f = torch.from_numpy(smooth_random_field((16, 24, 40), 3.0, seed=8)).cuda()
    full, index = ooc.ooc_compress_var(f, ooc.OOC_FR4_PRECISION, 20)
    need = full.numel()
    cap = (need // 2) // 4 * 4
    buf = torch.full((cap + 4096,), 0xA5, dtype=torch.uint8, device="cuda")
    idx2 = torch.empty_like(index)
    with pytest.raises(ooc.OocError) as err:
        ooc.ooc_compress_var(f, ooc.OOC_FR4_PRECISION, 20, d_out=buf[:cap], d_index=idx2)
    assert err.value.status == 1
    assert torch.equal(idx2, index)
    assert bool((buf[cap:] == 0xA5).all())
    words = full.view(torch.int32).cpu().numpy()
    got = buf[:cap].view(torch.int32).cpu().numpy()
    offs = index.cpu().numpy()
    fits = offs[1:] * 4 <= cap
    assert fits.any() and not fits.all()
    last = int(offs[1:][fits][-1])  # end of the last block that fits
    assert np.array_equal(got[:last], words[:last])


def test_corrupt_index_decodes_without_fault(ooc):
    # offsets are clamped to the stream and blocks to 130 words
    f = torch.from_numpy(smooth_random_field((12, 12, 12), 3.0, seed=6)).cuda()
    stream, index = ooc.ooc_compress_var(f, ooc.OOC_FR4_PRECISION, 16)
    rng = np.random.default_rng(0)
    bad = torch.from_numpy(rng.integers(0, 1 << 62, size=index.numel(), dtype=np.int64)).cuda()
    out = ooc.ooc_decompress_var(stream, bad, (12, 12, 12), ooc.OOC_FR4_PRECISION, 16)
    torch.cuda.synchronize()
    assert out.shape == (12, 12, 12)


@pytest.mark.parametrize("mode,param", [(1, 16), (2, 1e-4)])
def test_variable_modes_full_size(ooc, mode, param):
    # The 512^3 field the kernel workload times (2 M blocks, 16 K tiles of
    # the one-pass encoder's look-back): the whole stream and index word for
    # word against the oracle, and the decoded field.
    n = 512
    f = smooth_random_field((n, n, n), 32.0, seed=2)
    d = torch.from_numpy(f).cuda()
    stream, index = ooc.ooc_compress_var(d, mode, param)
    torch.cuda.synchronize()
    words_ref, index_ref = oracle.fr4_encode_var(f, mode, param)
    assert np.array_equal(index.cpu().numpy().astype(np.uint64), index_ref)
    assert np.array_equal(stream.cpu().numpy().view(np.uint32), words_ref)
    got = ooc.ooc_decompress_var(stream, index, f.shape, mode, param).cpu().numpy()
    ref = oracle.fr4_decode_var(words_ref, index_ref, f.shape, mode, param)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert ooc.ooc_take_device_fault() == 0
