"""Grids past 2^32 points.  The codec, the in-core stencils and the
out-of-core pipeline address fields with 64-bit offsets (element, stream
word and host-image byte offsets all pass 2^32 here): a 1024 x 1024 x 4104
field (4.30 G points, 17.2 GB in FP32, 8.6 GB at FR4-16) is checked at its
far end, where 32-bit offsets would wrap, against the oracle: sampled
codec blocks bit for bit, stencil sub-boxes on their exact dependency cones
against the FP64 runs, and the pipeline bit-identical to the in-core path
with the same storage round trips and within the storage error of the
oracle's pipeline."""
import numpy as np
import pytest

import oracle
from synth import smooth_random_field_torch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NZ, NY, NX = 4104, 1024, 1024


def _host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def big(ooc):
    assert NZ * NY * NX > 1 << 32
    free, _ = torch.cuda.mem_get_info()
    if free < 96e9:
        pytest.skip("needs about 90 GB of free device memory")
    f = smooth_random_field_torch((NZ, NY, NX), 24.0, seed=11)
    torch.cuda.synchronize()
    yield f
    del f
    torch.cuda.empty_cache()


def cone(lo, hi, n, m):
    return max(lo - m, 0), min(hi + m, n)


def oracle_box(fields, box, m, fn):
    """fn applied to the sub-boxes of `fields` (device tensors) that hold the
    output box `box` and every input within m cells of it, cropped to the
    box.  Sub-box faces on the grid's faces carry the grid's zero ghost, the
    others lie m cells out: exact for a dependency radius up to m."""
    (z0, z1), (y0, y1), (x0, x1) = box
    zs, ys, xs = cone(z0, z1, NZ, m), cone(y0, y1, NY, m), cone(x0, x1, NX, m)
    subs = [f[zs[0]:zs[1], ys[0]:ys[1], xs[0]:xs[1]].cpu().numpy().astype(np.float64) for f in fields]
    out = fn(*subs)
    return out[z0 - zs[0]:z1 - zs[0], y0 - ys[0]:y1 - ys[0], x0 - xs[0]:x1 - xs[0]]


# output boxes across the plane where the element offset reaches 2^32
# (z = 4096), on the grid's last planes, and on its x / y faces
BOXES = [((4092, 4100), (0, 8), (1016, 1024)), ((4096, 4104), (1016, 1024), (0, 8)),
         ((4100, 4104), (500, 508), (508, 516))]


def test_codec_blocks_past_2_32(ooc, big):
    rate = 16
    w = ooc.ooc_compress(big, rate)
    back = ooc.ooc_decompress(w, (NZ, NY, NX), rate)
    torch.cuda.synchronize()
    assert w.numel() == NZ * NY * NX * rate // 8
    wv = w.view(torch.int32)
    nbz, nby, nbx = NZ // 4, NY // 4, NX // 4
    rng = np.random.default_rng(4)
    picks = [(nbz - 1, nby - 1, nbx - 1), (1024, 0, 0), (1023, nby - 1, nbx - 1), (nbz // 2, 7, 9)]
    picks += [(int(rng.integers(1024, nbz)), int(rng.integers(0, nby)), int(rng.integers(0, nbx))) for _ in range(24)]
    for bz, by, bx in picks:
        blk = big[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].cpu().numpy()
        ref = oracle.fr4_encode(blk, rate)
        b = bx + nbx * (by + nby * bz)
        got = wv[b * 2 * rate:(b + 1) * 2 * rate].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref), (bz, by, bx)
        gb = back[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].cpu().numpy()
        assert np.array_equal(gb.view(np.uint32), oracle.fr4_decode(ref, (4, 4, 4), rate).view(np.uint32))
    err = (torch.linalg.vector_norm((back[4096:] - big[4096:]).double()) /
           torch.linalg.vector_norm(big[4096:].double())).item()
    assert err < 1e-4, err
    del w, back, wv
    torch.cuda.empty_cache()


def test_heat7_incore_past_2_32(ooc, big):
    nsteps = 2
    u = big.clone()
    tmp = torch.empty_like(u)
    ooc.ooc_heat7_steps(u, tmp, nsteps)
    torch.cuda.synchronize()
    for box in BOXES:
        ref = oracle_box([big], box, nsteps, lambda s: oracle.heat7_run(s, nsteps))
        (z0, z1), (y0, y1), (x0, x1) = box
        got = u[z0:z1, y0:y1, x0:x1].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max(), box
    del u, tmp
    torch.cuda.empty_cache()


def test_wave25_incore_past_2_32(ooc, big):
    nsteps = 2
    kap = 0.05 + 0.02 * torch.tanh(big)
    p, pp = big.clone(), 0.5 * big
    ooc.ooc_wave25_steps(p, pp, kap, nsteps)
    torch.cuda.synchronize()
    for box in BOXES:
        # p_prev = p / 2 exactly (a power-of-two scaling of normal floats)
        ref = oracle_box([big, kap], box, 4 * nsteps, lambda a, c: oracle.wave25_run(a, 0.5 * a, c, nsteps)[0])
        (z0, z1), (y0, y1), (x0, x1) = box
        got = p[z0:z1, y0:y1, x0:x1].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), box
    del p, pp, kap
    torch.cuda.empty_cache()


def test_heat7_pipeline_past_2_32(ooc, big):
    # 1 GiB device budget, k = 4, FR4 at 16 bits/value, 8 steps (two passes):
    # the host image is 8.6 GB, so slab units lie past byte offset 2^32
    if _host_available_bytes() < 64e9:
        pytest.skip("needs about 50 GB of free host memory")
    nsteps, k, rate = 8, 4, 16
    u0 = big.cpu().numpy()
    plan = ooc.Plan(nx=NX, ny=NY, nz=NZ, stencil="heat7", k=k, rw_format="fr4", rw_rate=rate,
                    device_budget_bytes=1 << 30)
    try:
        assert plan.info()["nslab"] > 1
        plan.set_field(0, u0)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    # the in-core path with the same round trips, compared on the device
    u = ooc.ooc_decompress(ooc.ooc_compress(big, rate), (NZ, NY, NX), rate)
    tmp = torch.empty_like(u)
    for _ in range(nsteps // k):
        ooc.ooc_heat7_steps(u, tmp, k)
        w = ooc.ooc_compress(u, rate)
        ooc.ooc_decompress(w, (NZ, NY, NX), rate, d_out=u)
        del w
    del tmp
    g = torch.from_numpy(got).cuda()
    assert torch.equal(g.view(torch.int32), u.view(torch.int32))
    del g, u
    torch.cuda.empty_cache()
    # against the oracle's pipeline on a 4-aligned sub-box at the far end:
    # 24 cells of margin cover the 8-cell dependency cone plus a block of
    # spreading per round trip
    m = 24
    (z0, z1), (y0, y1), (x0, x1) = (4080, 4104), (512, 528), (1000, 1024)
    zs, ys, xs = cone(z0, z1, NZ, m), cone(y0, y1, NY, m), cone(x0, x1, NX, m)
    sub = u0[zs[0]:zs[1], ys[0]:ys[1], xs[0]:xs[1]]
    crop = (slice(z0 - zs[0], z1 - zs[0]), slice(y0 - ys[0], y1 - ys[0]), slice(x0 - xs[0], x1 - xs[0]))
    pipe = oracle.heat7_storage_pipeline(sub, nsteps, k, "fr4", rate)[crop]
    exact = oracle.heat7_run(sub.astype(np.float64), nsteps)[crop]
    mine = got[z0:z1, y0:y1, x0:x1]
    assert oracle.error_metrics(mine, pipe)["rel_l2"] < 5e-5
    assert oracle.error_metrics(mine, exact)["rel_l2"] < 1e-4
    del u0, got
