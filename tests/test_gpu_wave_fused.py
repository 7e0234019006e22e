"""Two wave25 steps per launch (temporal blocking inside the kernel, with
the intermediate level on chip): bit-identical to the single-step kernel
over ragged shapes, odd and even step counts, and a source on the tiles'
overlaps (Table I's HALO = 4: level n+1 is recomputed on a 4-wide halo)."""
import numpy as np
import pytest

from synth import smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


@pytest.mark.parametrize("shape,nsteps,src", [
    ((36, 44, 136), 6, (120, 8, 17)),     # source on the first column of x-tile 1 and row 0 of y-tile 1
    ((68, 36, 260), 5, (119, 7, 33)),     # source on the last output column / row of tile 0
    ((20, 132, 1000), 4, None),
    ((64, 64, 64), 7, (32, 32, 32)),
    ((8, 8, 8), 3, (4, 4, 4)),
    ((40, 12, 16), 10, (0, 0, 0)),        # source on the grid's corner
    ((24, 20, 248), 8, (124, 9, 11)),     # an even number of pairs: results land in place
    ((16, 16, 16), 1, (8, 8, 8)),         # one step: the single-step kernel alone
    ((16, 16, 16), 0, None),
])
def test_fused_pairs_bit_identical_to_single_steps(ooc, shape, nsteps, src):
    nz, ny, nx = shape
    g = np.random.default_rng(sum(shape))
    p0 = (1e-3 * smooth_random_field(shape, 3.0, seed=sum(shape))).astype(np.float32)
    pm1 = (0.9 * p0 + 1e-5 * g.normal(size=shape)).astype(np.float32)
    kap = (0.02 + 0.1 * g.random(shape)).astype(np.float32)
    w = np.linspace(0.5, -0.25, 64, dtype=np.float32)
    out = []
    for fused in (False, True):
        p, pp = torch.from_numpy(p0.copy()).cuda(), torch.from_numpy(pm1.copy()).cuda()
        k = torch.from_numpy(kap).cuda()
        if fused:
            ooc.ooc_wave25_steps_fused(p, pp, k, nsteps, src=src, w=w if src else None, t=3)
        else:
            ooc.ooc_wave25_steps(p, pp, k, nsteps, src=src, w=w if src else None, t=3)
        torch.cuda.synchronize()
        out.append((p.cpu().numpy(), pp.cpu().numpy()))
    assert np.abs(out[0][0]).max() > 0
    assert np.array_equal(out[1][0].view(np.uint32), out[0][0].view(np.uint32))
    assert np.array_equal(out[1][1].view(np.uint32), out[0][1].view(np.uint32))
    assert ooc.ooc_take_device_fault() == 0


def test_fused_pairs_refuse_aliased_buffers(ooc):
    d = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_wave25_steps_fused(d, d, torch.zeros_like(d), 2)
