"""FP64 fields, as the paper ran them (Section VI: double-precision fields at
32 and 24 of every 64 bits): the FP64 kernels against the FP64 oracle, FP64
out-of-core plans against in-core runs of the same kernels (bit for bit),
and FR4D-compressed FP64 plans against the oracle's FP64 pipeline with the
same storage round trips."""
import numpy as np
import pytest

import oracle
from synth import layered_velocity, ricker, sine_modes_field, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def pass_lengths(calls, k):
    out = []
    for n in calls:
        full, rem = divmod(n, k)
        out += [k] * full + ([rem] if rem else [])
    return out


def roundtrip64(ooc, d, fmt, rate):
    if fmt == "fp64":
        return d.clone()
    return ooc.ooc_decompress64(ooc.ooc_compress64(d, rate), tuple(d.shape), rate)


def wave_case(shape, nsteps, seed=3):
    v = layered_velocity(shape, seed=seed)
    dt = 0.4 * 10.0 / v.max()
    kappa = (v * dt / 10.0) ** 2
    nz, ny, nx = shape
    src = (nx // 2 + 1, ny // 2, nz // 2)  # odd x: the second point of its thread's pair
    # FP32-exact amplitudes: the plans' source series is FP32 in both precisions
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32).astype(np.float64)
    return kappa.astype(np.float64), src, w


@pytest.mark.parametrize("shape,nsteps", [((48, 40, 136), 30), ((20, 16, 64), 12)])
def test_incore_wave25_f64_against_oracle(ooc, shape, nsteps):
    # FP64 on both sides: they differ only in rounding order (fused
    # multiply-adds on the GPU), about 1e-16 relative per step.
    kappa, src, w = wave_case(shape, nsteps)
    rng = np.random.default_rng(1)
    p0 = 1e-3 * smooth_random_field(shape, 4.0, seed=5, dtype=np.float64)
    pm1 = 0.97 * p0 + 1e-6 * rng.normal(size=shape)
    nz, ny, nx = shape
    p, pp = torch.from_numpy(p0.copy()).cuda(), torch.from_numpy(pm1.copy()).cuda()
    ooc.ooc_wave25_steps_f64(p, pp, torch.from_numpy(kappa).cuda(), nsteps, src=src, w=w)
    torch.cuda.synchronize()
    srcf = (src[2] * ny + src[1]) * nx + src[0]
    want_p, want_pp = oracle.wave25_run(p0, pm1, kappa, nsteps, src=srcf, w=w)
    for got, want in ((p.cpu().numpy(), want_p), (pp.cpu().numpy(), want_pp)):
        m = oracle.error_metrics(got, want)
        assert m["rel_l2"] < 1e-13, m


def test_incore_heat7_f64_against_oracle_on_a_ring_window(ooc):
    u0, _ = sine_modes_field((40, 24, 72), seed=2)
    u0 = np.asarray(u0, dtype=np.float64)
    d, tmp = torch.from_numpy(u0.copy()).cuda(), torch.empty((40, 24, 72), dtype=torch.float64, device="cuda")
    ooc.ooc_heat7_steps_f64(d, tmp, 7)
    torch.cuda.synchronize()
    assert oracle.error_metrics(d.cpu().numpy(), oracle.heat7_run(u0, 7))["rel_l2"] < 1e-14


@pytest.mark.parametrize("fmt,rate", [("fp64", 64), ("fr4", 32), ("fr4", 24)])
@pytest.mark.parametrize("T,k,calls", [(8, 1, [5]), (12, 3, [10]), (28, 2, [3, 4]), (64, 4, [9])])
def test_heat7_f64_ooc_bit_identical_to_incore(ooc, fmt, rate, T, k, calls):
    shape = (64, 24, 72)  # thin last slabs for T = 12, 28; 72-wide rows: a ragged 64-point x tile
    u0, _ = sine_modes_field(shape, seed=4)
    u0 = np.asarray(u0, dtype=np.float64)
    plan = ooc.Plan(nx=72, ny=24, nz=64, stencil="heat7", k=k, rw_format=fmt, rw_rate=rate, slab_planes=T,
                    precision="fp64")
    try:
        plan.set_field(0, u0)
        for n in calls:
            plan.step(n)
        got = plan.get_field(0)
    finally:
        plan.close()
    u = roundtrip64(ooc, torch.from_numpy(u0).cuda(), fmt, rate)
    tmp = torch.empty_like(u)
    for kp in pass_lengths(calls, k):
        ooc.ooc_heat7_steps_f64(u, tmp, kp)
        u = roundtrip64(ooc, u, fmt, rate)
    torch.cuda.synchronize()
    assert got.dtype == np.float64
    assert np.array_equal(got.view(np.uint64), u.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("rw,rw_rate,ro,ro_rate", [("fp64", 64, "fp64", 64), ("fr4", 32, "fr4", 32),
                                                   ("fr4", 24, "fp64", 64)])
def test_wave25_f64_ooc_bit_identical_to_incore(ooc, rw, rw_rate, ro, ro_rate):
    shape = (96, 24, 72)
    kappa, src, w = wave_case(shape, 40)
    p0 = 1e-3 * smooth_random_field(shape, 4.0, seed=7, dtype=np.float64)
    pm1 = 0.95 * p0
    calls, k = [10, 11], 10
    plan = ooc.Plan(nx=72, ny=24, nz=96, stencil="wave25", k=k, rw_format=rw, rw_rate=rw_rate, ro_format=ro,
                    ro_rate=ro_rate, slab_planes=24, precision="fp64")
    try:
        assert plan.info()["nslab"] == 4
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w.astype(np.float32))
        for n in calls:
            plan.step(n)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
    finally:
        plan.close()
    kap = roundtrip64(ooc, torch.from_numpy(kappa).cuda(), ro, ro_rate)
    p = roundtrip64(ooc, torch.from_numpy(p0).cuda(), rw, rw_rate)
    pp = roundtrip64(ooc, torch.from_numpy(pm1).cuda(), rw, rw_rate)
    t = 0
    for kp in pass_lengths(calls, k):
        ooc.ooc_wave25_steps_f64(p, pp, kap, kp, src=src, w=w, t=t)
        t += kp
        p = roundtrip64(ooc, p, rw, rw_rate)
        pp = roundtrip64(ooc, pp, rw, rw_rate)
    torch.cuda.synchronize()
    assert np.array_equal(got_p.view(np.uint64), p.cpu().numpy().view(np.uint64))
    assert np.array_equal(got_pp.view(np.uint64), pp.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("rate,tol_pipe,tol_exact", [(32, 1e-10, 1e-7), (24, 1e-8, 1e-4)])
def test_fr4d_heat_plan_against_oracle_pipeline(ooc, rate, tol_pipe, tol_exact):
    # Both sides round-trip identical FR4D streams at identical points, so
    # they differ by FP64 rounding order (~1e-16 relative) carried through
    # the round trips; a value on the other side of the last kept bit plane
    # moves by one unit of it (about 1e-9 relative at 32 bits per value,
    # 1e-6 at 24), which at these odds touches a few values at most.
    # Against the FP64 run without storage, the storage error itself adds.
    shape = (64, 32, 64)
    u0 = smooth_random_field(shape, 6.0, seed=9, dtype=np.float64)
    plan = ooc.Plan(nx=64, ny=32, nz=64, stencil="heat7", k=4, rw_format="fr4", rw_rate=rate, slab_planes=16,
                    precision="fp64")
    try:
        plan.set_field(0, u0)
        plan.step(12)
        got = plan.get_field(0)
    finally:
        plan.close()
    want = oracle.heat7_storage_pipeline(u0, 12, 4, "fr4", rate=rate, precision="fp64")
    exact = oracle.heat7_run(u0, 12)
    mp, me = oracle.error_metrics(got, want), oracle.error_metrics(got, exact)
    print(f"FR4D-{rate} heat plan: vs oracle pipeline {mp}, vs FP64 run {me}")
    assert mp["rel_l2"] < tol_pipe, mp
    assert me["rel_l2"] < tol_exact, me


def test_fr4d_wave_code4_against_oracle_pipeline(ooc):
    # Section VI's code 4 in double precision at 32 of 64 bits: both levels
    # and kappa FR4D-32, 3 slabs, k = 10, the source on, two calls.
    #
    # Tolerance: FP64 rounding order flips a coded bit only rarely, but a
    # flipped value moves by one unit of the last kept plane (about the
    # storage error), the wave carries that change to its neighbours within
    # the pass, and at the next round trip it flips some of theirs: unlike
    # the diffusive heat plans, the two wave pipelines drift apart by up to
    # the storage error itself (measured 2.7e-10 against the oracle
    # pipeline, 2.5e-10 against the FP64 run without storage).
    shape = (96, 32, 64)
    kappa, src, w = wave_case(shape, 25)
    p0 = 1e-3 * smooth_random_field(shape, 5.0, seed=11, dtype=np.float64)
    pm1 = 0.96 * p0
    nz, ny, nx = shape
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="wave25", k=10, rw_format="fr4", rw_rate=32, ro_format="fr4",
                    ro_rate=32, slab_planes=32, precision="fp64")
    try:
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w.astype(np.float32))
        plan.step(12)
        plan.step(13)
        got = plan.get_field(0)
    finally:
        plan.close()
    srcf = (src[2] * ny + src[1]) * nx + src[0]
    want, _ = oracle.wave25_storage_pipeline(p0, pm1, kappa, 25, 10, "fr4", 32, ro_fmt="fr4", ro_rate=32, src=srcf,
                                             w=w, precision="fp64")
    exact, _ = oracle.wave25_run(p0, pm1, kappa, 25, src=srcf, w=w)
    mp, me = oracle.error_metrics(got, want), oracle.error_metrics(got, exact)
    print(f"FR4D-32 wave code 4: vs oracle pipeline {mp}, vs FP64 run {me}")
    assert mp["rel_l2"] < 2e-9, mp
    assert me["rel_l2"] < 1e-7, me


def test_precision_and_format_combinations_are_checked(ooc):
    for kw in (dict(precision="fp64", rw_format="bf16"), dict(precision="fp64", rw_format="fp32"),
               dict(precision="fp32", rw_format="fp64"),
               dict(precision="fp64", rw_format="fp64", heat_steps_per_launch=2),
               dict(precision=2)):
        with pytest.raises(ooc.OocError):
            ooc.Plan(nx=16, ny=16, nz=16, stencil="heat7", k=2, slab_planes=8, **kw)
    plan = ooc.Plan(nx=16, ny=16, nz=16, stencil="heat7", k=2, slab_planes=8, precision="fp64", rw_format="fp64")
    try:
        # the FP32 entry points refuse an FP64 plan
        buf = np.zeros((16, 16, 16), dtype=np.float32)
        assert ooc.lib().ooc_set_field(plan._h, 0, buf.ctypes.data) != 0
        assert ooc.lib().ooc_get_field(plan._h, 0, buf.ctypes.data) != 0
    finally:
        plan.close()


@pytest.mark.parametrize("fmt,rate", [("fp64", 64), ("fr4", 32)])
def test_fp64_plans_with_debug_checks_budget_and_graph_replay(ooc, fmt, rate):
    # The FP64 plans go through the same scheduler machinery as the FP32
    # ones: with debug checks (guard bytes and window/copy checks) on, with
    # the slab thickness derived from a budget that forces streaming, and
    # with calls replayed as CUDA graphs or launched directly, the bits stay
    # those of a single-slab plan launched directly.
    shape = (96, 32, 36)
    u0 = smooth_random_field(shape, 5.0, seed=41, dtype=np.float64)
    outs = {}
    for name, kw in (("ref", dict(slab_planes=96, graph_mode=1)),
                     ("debug", dict(slab_planes=12, debug_checks=1)),
                     ("budget", dict(device_budget_bytes=1_200_000)),
                     ("graph", dict(slab_planes=24, graph_mode=0))):
        plan = ooc.Plan(nx=36, ny=32, nz=96, stencil="heat7", k=3, rw_format=fmt, rw_rate=rate, precision="fp64",
                        **kw)
        try:
            plan.set_field(0, u0)
            for n in (6, 6, 4, 6):
                plan.step(n)
            outs[name] = (plan.info()["nslab"], plan.get_field(0))
            assert plan.stats()["steps_done"] == 22
        finally:
            plan.close()
    assert outs["ref"][0] == 1 and outs["budget"][0] > 3
    for name in ("debug", "budget", "graph"):
        assert np.array_equal(outs[name][1].view(np.uint64), outs["ref"][1].view(np.uint64)), name


def test_fp64_wave_graph_replay_with_the_source_table(ooc):
    # graph replay reads the source amplitude from the device table at the
    # plan's device time: replayed calls give the bits of direct launches
    shape = (64, 24, 72)
    kappa, src, w = wave_case(shape, 40)
    p0 = 1e-3 * smooth_random_field(shape, 4.0, seed=13, dtype=np.float64)
    outs = {}
    for mode in (0, 1):
        plan = ooc.Plan(nx=72, ny=24, nz=64, stencil="wave25", k=5, rw_format="fr4", rw_rate=32, ro_format="fp64",
                        ro_rate=64, slab_planes=16, graph_mode=mode, precision="fp64")
        try:
            plan.set_field(0, p0)
            plan.set_field(1, 0.9 * p0)
            plan.set_field(2, kappa)
            plan.set_source(*src, w.astype(np.float32))
            for n in (10, 10, 10, 7):
                plan.step(n)
            outs[mode] = plan.get_field(0)
        finally:
            plan.close()
    assert np.abs(outs[1]).max() > 0
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))


def test_fp64_reference_of_the_precision_configuration(ooc):
    # The precision and wave1024_error workloads take their errors against an
    # FP64 run by this kernel: here it runs the 384^3 configuration's inputs
    # (layered velocity, FP32 kappa, the Ricker source at the centre, from
    # rest) for 40 steps and meets the FP64 oracle over the whole field.
    import bench
    n, nsteps = 384, 40
    kappa, src, dt = bench.wave_inputs(n)
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32).astype(np.float64)
    k64 = kappa.astype(np.float64)
    p = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp = torch.zeros_like(p)
    ooc.ooc_wave25_steps_f64(p, pp, torch.from_numpy(k64).cuda(), nsteps, src=src, w=w)
    torch.cuda.synchronize()
    srcf = (src[2] * n + src[1]) * n + src[0]
    want, _ = oracle.wave25_run(np.zeros((n, n, n)), np.zeros((n, n, n)), k64, nsteps, src=srcf, w=w)
    m = oracle.error_metrics(p.cpu().numpy(), want)
    assert m["rel_l2"] < 1e-13, m


def test_fp64_reference_of_the_1024_wave_configuration(ooc):
    # The same at 1024^3 (the wave1024_error workload): after 20 steps from
    # rest the field is nonzero only within 4 x 20 = 80 cells of the source,
    # so the oracle on the 208^3 box around it (104 cells out, zero ghosts
    # beyond) gives every nonzero value exactly; outside the box the GPU
    # field must be exactly zero.
    import bench
    n, nsteps, m = 1024, 20, 104
    kappa, src, dt = bench.wave_inputs(n)
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32).astype(np.float64)
    p = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp = torch.zeros_like(p)
    ooc.ooc_wave25_steps_f64(p, pp, torch.from_numpy(kappa.astype(np.float64)).cuda(), nsteps, src=src, w=w)
    torch.cuda.synchronize()
    lo = [c - m for c in src]
    box = (slice(lo[2], lo[2] + 2 * m), slice(lo[1], lo[1] + 2 * m), slice(lo[0], lo[0] + 2 * m))
    sub_k = kappa[box].astype(np.float64)
    srcf = (m * 2 * m + m) * 2 * m + m
    want, _ = oracle.wave25_run(np.zeros(sub_k.shape), np.zeros(sub_k.shape), sub_k, nsteps, src=srcf, w=w)
    got = p[box].cpu().numpy()
    assert np.abs(want).max() > 0
    e = oracle.error_metrics(got, want)
    assert e["rel_l2"] < 1e-13, e
    p[box] = 0.0
    assert int(torch.count_nonzero(p)) == 0


@pytest.mark.parametrize("fmt,rate", [("fp64", 64), ("fr4", 32)])
@pytest.mark.parametrize("shape,T,k,calls", [((4, 4, 4), 4, 8, [0, 3, 9]), ((16, 4, 4), 4, 9, [20]),
                                             ((12, 8, 4), 4, 2, [5, 0, 3])])
def test_fp64_heat_degenerate_plans(ooc, fmt, rate, shape, T, k, calls):
    # FP64 plans on one-block grids, k h beyond the grid and common regions
    # up to 3 slabs wide (inputs from several slabs of the previous pass):
    # bit-identical to the in-core FP64 path with the same round trips
    nz, ny, nx = shape
    u0 = np.random.default_rng(sum(shape) + k).normal(size=shape)
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="heat7", k=k, rw_format=fmt, rw_rate=rate, slab_planes=T,
                    precision="fp64")
    try:
        assert plan.info()["nslab"] == nz // T
        plan.set_field(0, u0)
        for n in calls:
            plan.step(n)
        got = plan.get_field(0)
    finally:
        plan.close()
    u = roundtrip64(ooc, torch.from_numpy(u0).cuda(), fmt, rate)
    tmp = torch.empty_like(u)
    for kp in pass_lengths(calls, k):
        ooc.ooc_heat7_steps_f64(u, tmp, kp)
        u = roundtrip64(ooc, u, fmt, rate)
    torch.cuda.synchronize()
    assert np.array_equal(got.view(np.uint64), u.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("shape,T,k,calls", [((24, 8, 4), 4, 3, [7]), ((8, 4, 4), 4, 10, [13])])
def test_fp64_wave_degenerate_plans(ooc, shape, T, k, calls):
    nz, ny, nx = shape
    kappa, src, w = wave_case(shape, sum(calls))
    rng = np.random.default_rng(nz)
    p0 = 1e-3 * rng.normal(size=shape)
    pm1 = 0.9 * p0
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="wave25", k=k, rw_format="fr4", rw_rate=32, ro_format="fp64",
                    ro_rate=64, slab_planes=T, precision="fp64")
    try:
        assert plan.info()["nslab"] == nz // T
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w.astype(np.float32))
        for n in calls:
            plan.step(n)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
    finally:
        plan.close()
    kap = torch.from_numpy(kappa).cuda()
    p = roundtrip64(ooc, torch.from_numpy(p0).cuda(), "fr4", 32)
    pp = roundtrip64(ooc, torch.from_numpy(pm1).cuda(), "fr4", 32)
    t = 0
    for kp in pass_lengths(calls, k):
        ooc.ooc_wave25_steps_f64(p, pp, kap, kp, src=src, w=w, t=t)
        t += kp
        p = roundtrip64(ooc, p, "fr4", 32)
        pp = roundtrip64(ooc, pp, "fr4", 32)
    torch.cuda.synchronize()
    assert np.abs(got_p).max() > 0
    assert np.array_equal(got_p.view(np.uint64), p.cpu().numpy().view(np.uint64))
    assert np.array_equal(got_pp.view(np.uint64), pp.cpu().numpy().view(np.uint64))


def test_full_size_fp64_heat_configuration(ooc):
    # The fp64 workload's heat configuration at its size: 1024^3 FP64, 2 GiB
    # device budget, k = 4, FR4D at 32 of 64 bits, one call of 32 steps.
    # Bit-identical over the whole field to the in-core FP64 kernel with the
    # same round trips (compared on the device), and on the central 128^3
    # sub-box (exact dependency cone) within FR4D-32's storage error of the
    # FP64 oracle run without storage.
    n, k, nsteps, rate = 1024, 4, 32, 32
    u0 = smooth_random_field((n, n, n), 32.0, seed=2, dtype=np.float64)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=k, rw_format="fr4", rw_rate=rate,
                    device_budget_bytes=2 << 30, precision="fp64")
    try:
        assert plan.device_bytes <= 2 << 30 and plan.info()["nslab"] > 1
        plan.set_field(0, u0)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    u = roundtrip64(ooc, torch.from_numpy(u0).cuda(), "fr4", rate)
    tmp = torch.empty_like(u)
    for kp in pass_lengths([nsteps], k):
        ooc.ooc_heat7_steps_f64(u, tmp, kp)
        u = roundtrip64(ooc, u, "fr4", rate)
    del tmp
    g = torch.from_numpy(got).cuda()
    assert torch.equal(g.view(torch.int64), u.view(torch.int64))
    del g, u
    torch.cuda.empty_cache()
    c0, c1 = n // 2 - 64, n // 2 + 64
    sub = u0[c0 - nsteps:c1 + nsteps, c0 - nsteps:c1 + nsteps, c0 - nsteps:c1 + nsteps]
    exact = oracle.heat7_run(sub, nsteps)[nsteps:-nsteps, nsteps:-nsteps, nsteps:-nsteps]
    m = oracle.error_metrics(got[c0:c1, c0:c1, c0:c1], exact)
    assert m["rel_l2"] < 1e-7, m


def test_full_size_fp64_wave_configuration(ooc):
    # The fp64 workload's wave configuration at its size: 1024^3 FP64, 8 GiB
    # budget, k = 10, code 4 (both levels and kappa FR4D-32), from rest with
    # the source, 20 steps.  Bit-identical over the whole field to the
    # in-core FP64 kernel with the same round trips; and the central 32^3
    # box against the FP64 oracle run without storage on a 208^3 sub-box
    # (20 steps move information 80 cells, the field is zero beyond that
    # from the source, so the sub-box's zero ghosts are exact).
    from synth import layered_velocity
    n, k, nsteps, rate, m = 1024, 10, 20, 32, 104
    v = layered_velocity((n, n, n), seed=3)
    dt = 0.4 * 10.0 / float(v.max())
    kappa = (np.asarray(v, dtype=np.float64) * (dt / 10.0)) ** 2
    del v
    src = (n // 2, n // 2, n // 2)
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float64)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format="fr4", rw_rate=rate, ro_format="fr4",
                    ro_rate=rate, device_budget_bytes=8 << 30, precision="fp64")
    try:
        assert plan.device_bytes <= 8 << 30 and plan.info()["nslab"] > 1
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    del zero
    kap = roundtrip64(ooc, torch.from_numpy(kappa).cuda(), "fr4", rate)
    p = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp = torch.zeros_like(p)
    w64 = w.astype(np.float64)
    t = 0
    for kp in pass_lengths([nsteps], k):
        ooc.ooc_wave25_steps_f64(p, pp, kap, kp, src=src, w=w64, t=t)
        t += kp
        p = roundtrip64(ooc, p, "fr4", rate)
        pp = roundtrip64(ooc, pp, "fr4", rate)
    del kap, pp
    g = torch.from_numpy(got).cuda()
    assert torch.equal(g.view(torch.int64), p.view(torch.int64))
    del g, p
    torch.cuda.empty_cache()
    lo = [c - m for c in src]
    box = (slice(lo[2], lo[2] + 2 * m), slice(lo[1], lo[1] + 2 * m), slice(lo[0], lo[0] + 2 * m))
    srcf = (m * 2 * m + m) * 2 * m + m
    exact, _ = oracle.wave25_run(np.zeros((2 * m,) * 3), np.zeros((2 * m,) * 3), kappa[box], nsteps, src=srcf,
                                 w=w64)
    cen = (slice(m - 16, m + 16),) * 3
    e = oracle.error_metrics(got[box][cen], exact[cen])
    assert np.abs(exact[cen]).max() > 0
    assert e["rel_l2"] < 1e-6, e
