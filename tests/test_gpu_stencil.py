"""GPU stencil parity: the heat7 and wave25 kernels (in-core entry points,
the same kernels the pipeline launches) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from synth import layered_velocity, ricker, sine_mode, sine_modes_field, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 compute against FP64: each heat step rounds a few ulps (u in [-3,3]).
HEAT_TOL = 1e-6
# The leapfrog accumulates rounding roughly linearly in time.
WAVE_TOL_PER_100 = 2e-5


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def run_heat_gpu(ooc, u0, nsteps):
    d = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    tmp = torch.empty_like(d)
    ooc.ooc_heat7_steps(d, tmp, nsteps)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("shape,nsteps", [((128, 128, 128), 8), ((36, 20, 44), 5), ((4, 4, 4), 3), ((68, 132, 8), 7)])
def test_heat7_matches_fp64(ooc, shape, nsteps):
    u0, _ = sine_modes_field(shape, seed=0)
    got = run_heat_gpu(ooc, u0, nsteps)
    ref = oracle.heat7_run(u0.astype(np.float64), nsteps)
    m = oracle.error_metrics(got, ref)
    assert m["rel_l2"] < HEAT_TOL, m
    assert m["max_abs"] < 2e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", [(36, 20, 44), (4, 4, 4), (8, 20, 244), (24, 36, 124), (40, 68, 256), (12, 8, 120),
                                   (24, 1024, 1024), (20, 1000, 1016)])
@pytest.mark.parametrize("nsteps", [1, 2, 3, 6])
def test_heat7_fused_pairs_bit_identical(ooc, shape, nsteps):
    # Two steps per launch (level s on chip) against one step per launch:
    # same arithmetic, so the bits agree.  The shapes span several 120-wide
    # x tiles and 14-row y tiles with ragged tails, and nz down to one block;
    # the 1024^2 and 1000 x 1016 planes have more tiles than one wave holds,
    # so the launch marches whole waves of whole tiles and z-chunks of the
    # remaining ones.
    if shape[1] * shape[2] < 100000:
        u0 = smooth_random_field(shape, 6.0, seed=11)
    else:  # large planes: any values do for bit identity
        u0 = np.random.default_rng(11).standard_normal(shape).astype(np.float32)
    a = torch.from_numpy(u0).cuda()
    b = a.clone()
    ooc.ooc_heat7_steps(a, torch.empty_like(a), nsteps)
    ooc.ooc_heat7_steps_fused(b, torch.empty_like(b), nsteps)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("scale", ["subnormal", "mixed", "large"])
def test_heat7_fused_pairs_bit_identical_on_special_values(ooc, scale):
    # The fused pairs compute their point updates in packed FP32 pairs, the
    # single steps in scalar FP32; neither flushes subnormals, and both round
    # each operation to nearest even.  Fields of subnormals (with +-0 and
    # signs mixed), of values spread over the whole exponent range, and of
    # values near the top of the range (sums of six stay finite) give the
    # same bits.
    g = np.random.default_rng({"subnormal": 1, "mixed": 2, "large": 3}[scale])
    shape = (20, 36, 260)
    if scale == "subnormal":
        u0 = (g.standard_normal(shape) * 1e-40).astype(np.float32)
        u0[g.random(shape) < 0.1] = 0.0
        u0[g.random(shape) < 0.05] = -0.0
    elif scale == "mixed":
        u0 = (g.standard_normal(shape) * 10.0 ** g.integers(-44, 38, size=shape)).astype(np.float32)
    else:
        u0 = (g.uniform(-1.0, 1.0, shape) * 5e37).astype(np.float32)
    assert np.all(np.isfinite(u0))
    a = torch.from_numpy(u0).cuda()
    b = a.clone()
    ooc.ooc_heat7_steps(a, torch.empty_like(a), 4)
    ooc.ooc_heat7_steps_fused(b, torch.empty_like(b), 4)
    torch.cuda.synchronize()
    got_a, got_b = a.cpu().numpy(), b.cpu().numpy()
    if scale == "subnormal":
        assert np.any((got_a != 0) & (np.abs(got_a) < np.finfo(np.float32).tiny))  # subnormals survive
    assert np.array_equal(got_a.view(np.uint32), got_b.view(np.uint32))


def test_heat7_fused_matches_fp64(ooc):
    u0, _ = sine_modes_field((64, 72, 136), seed=2)
    d = torch.from_numpy(u0).cuda()
    ooc.ooc_heat7_steps_fused(d, torch.empty_like(d), 8)
    torch.cuda.synchronize()
    m = oracle.error_metrics(d.cpu().numpy(), oracle.heat7_run(u0.astype(np.float64), 8))
    assert m["rel_l2"] < HEAT_TOL, m


@pytest.mark.parametrize("shape,nsteps", [((64, 48, 80), 6), ((36, 20, 132), 5), ((4, 4, 4), 3)])
def test_heat7_f64_matches_fp64_oracle(ooc, shape, nsteps):
    # the same step in double precision: agreement to FP64 rounding
    u0, _ = sine_modes_field(shape, seed=1)
    d = torch.from_numpy(u0.astype(np.float64)).cuda()
    ooc.ooc_heat7_steps_f64(d, torch.empty_like(d), nsteps)
    ref = oracle.heat7_run(u0.astype(np.float64), nsteps)
    got = d.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref) * nsteps
    assert np.abs(got - ref).max() <= 1e-14 * nsteps * max(1.0, np.abs(ref).max())


def test_heat7_f64_sine_mode_closed_form(ooc):
    shape, k = (64, 48, 80), (3, 2, 1)
    u0 = sine_mode(shape, k).astype(np.float64)
    lam = 1.0 - 2.0 / 6.0 * sum(1 - math.cos(math.pi * ka / (na + 1)) for ka, na in zip(k, (80, 48, 64)))
    d = torch.from_numpy(u0).cuda()
    ooc.ooc_heat7_steps_f64(d, torch.empty_like(d), 20)
    assert np.abs(d.cpu().numpy() - lam ** 20 * u0).max() < 1e-13


def test_heat7_sine_mode_closed_form(ooc):
    shape, k = (64, 48, 80), (3, 2, 1)
    u0 = sine_mode(shape, k)
    lam = 1.0 - 2.0 / 6.0 * sum(1 - math.cos(math.pi * ka / (na + 1)) for ka, na in zip(k, (80, 48, 64)))
    got = run_heat_gpu(ooc, u0, 20)
    assert np.abs(got - lam ** 20 * u0).max() < 5e-6


def wave_problem(n, nsteps, seed=3):
    shape = (n, n, n)
    v = layered_velocity(shape, seed=seed)
    dx = 10.0
    dt = 0.4 * dx / v.max()
    kappa = ((v * dt / dx) ** 2).astype(np.float32)
    src = (n // 2, n // 2, n // 2)
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    return kappa, src, w


@pytest.mark.parametrize("n,nsteps", [(64, 200), (44, 60)])
def test_wave25_matches_fp64(ooc, n, nsteps):
    kappa, (sx, sy, sz), w = wave_problem(n, nsteps)
    p = torch.zeros((n, n, n), device="cuda")
    pp = torch.zeros_like(p)
    k = torch.from_numpy(kappa).cuda()
    ooc.ooc_wave25_steps(p, pp, k, nsteps, src=(sx, sy, sz), w=w)
    torch.cuda.synchronize()
    src = (sz * n + sy) * n + sx
    rp, rpp = oracle.wave25_run(np.zeros((n, n, n)), np.zeros((n, n, n)), kappa.astype(np.float64), nsteps, src=src,
                                w=w.astype(np.float64))
    tol = WAVE_TOL_PER_100 * max(1.0, nsteps / 100)
    for got, ref in ((p, rp), (pp, rpp)):
        m = oracle.error_metrics(got.cpu().numpy(), ref)
        assert m["rel_l2"] < tol, m


def test_wave25_random_state_one_step(ooc):
    rng = np.random.default_rng(5)
    shape = (20, 28, 36)
    p0, p1 = rng.normal(size=(2,) + shape).astype(np.float32)
    kap = (rng.uniform(0.0, 0.16, size=shape)).astype(np.float32)
    a, b, k = (torch.from_numpy(v.copy()).cuda() for v in (p0, p1, kap))
    ooc.ooc_wave25_steps(a, b, k, 1)
    torch.cuda.synchronize()
    ref = oracle.wave25_step(p0.astype(np.float64), p1.astype(np.float64), kap.astype(np.float64))
    assert np.abs(a.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()
    assert np.array_equal(b.cpu().numpy(), p0)  # p^{t} moves to the previous level
