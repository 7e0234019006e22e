"""The binding checks every tensor it hands to the library against what the
call reads or writes (the C ABI sees plain pointers and cannot): device,
dtype, contiguity and length.  Wrong tensors raise ValueError before any
kernel runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def test_wrong_dtype_is_refused(ooc):
    u = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ooc.ooc_heat7_steps(u, torch.empty_like(u), 1)
    with pytest.raises(ValueError):
        ooc.ooc_compress(u, 16)
    with pytest.raises(ValueError):
        ooc.ooc_bf16_unpack(torch.zeros(64, dtype=torch.float32, device="cuda"))
    f = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(ValueError):
        ooc.ooc_heat7_steps_f64(f, torch.empty_like(f), 1)
    with pytest.raises(ValueError):
        ooc.ooc_gather(f.flatten(), torch.zeros(4, dtype=torch.int32, device="cuda"))


def test_broadcast_and_strided_views_are_refused(ooc):
    # an expanded view holds one value for many elements: a kernel reading
    # the full extent would leave its allocation
    one = torch.zeros(1, device="cuda").expand(16, 16, 16)
    with pytest.raises(ValueError):
        ooc.ooc_compress(one, 16)
    big = torch.zeros((16, 16, 32), device="cuda")
    with pytest.raises(ValueError):
        ooc.ooc_heat7_steps(big[:, :, ::2], torch.empty((16, 16, 16), device="cuda"), 1)
    with pytest.raises(ValueError):
        ooc.ooc_wave25_steps(big, big, big.transpose(0, 2), 1)


def test_short_buffers_are_refused(ooc):
    u = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(ValueError):
        ooc.ooc_heat7_steps(u, torch.empty(8 * 8 * 7, device="cuda"), 1)
    with pytest.raises(ValueError):
        ooc.ooc_wave25_steps(u, torch.zeros_like(u), torch.zeros(100, device="cuda"), 1)
    with pytest.raises(ValueError):
        ooc.ooc_decompress(torch.zeros(1024, dtype=torch.uint8, device="cuda"), (8, 8, 8), 16,
                           d_out=torch.empty(8 * 8 * 8 - 4, device="cuda"))
    with pytest.raises(ValueError):
        ooc.ooc_bf16_pack(u, d_out=torch.empty(100, dtype=torch.int16, device="cuda"))
    # traces shorter than nsteps x receivers
    shape, N, every, rate = (8, 8, 8), 6, 3, 16
    h_ckpt = torch.empty(ooc.ooc_wave25_ckpt_bytes(shape, N, every, rate), dtype=torch.uint8, pin_memory=True)
    work = torch.empty(ooc.ooc_wave25_adjoint_work_bytes(shape, every, rate), dtype=torch.uint8, device="cuda")
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    rec = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        ooc.ooc_wave25_forward_ckpt(torch.full(shape, 0.05, device="cuda"), N, rec, torch.zeros((N - 1, 2), device="cuda"),
                                    every, rate, h_ckpt, work, streams)
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 0
    assert np.all(u.cpu().numpy() == 0)
