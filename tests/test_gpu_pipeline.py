"""Out-of-core pipeline parity (ooc_plan / ooc_step through the C ABI).

The scheduler must not change arithmetic: a run streamed slab by slab with
region sharing and temporal blocking is bit-identical to an in-core GPU run
of the same kernels that applies the same storage round trip (FP32 identity,
BF16 rounding, FR4 encode+decode) to every stored field at load and after
every pass.  The in-core kernels and the codec are checked against the
oracle elsewhere; here the oracle bounds the end-to-end error."""
import numpy as np
import pytest

import oracle
from synth import layered_velocity, ricker, sine_mode, sine_modes_field, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def roundtrip(ooc, d, fmt, rate):
    if fmt == "fp32":
        return d.clone()
    if fmt == "bf16":
        return ooc.ooc_bf16_unpack(ooc.ooc_bf16_pack(d)).reshape(d.shape)
    return ooc.ooc_decompress(ooc.ooc_compress(d, rate), tuple(d.shape), rate)


def pass_lengths(calls, k):
    out = []
    for n in calls:
        full, rem = divmod(n, k)
        out += [k] * full + ([rem] if rem else [])
    return out


def incore_heat(ooc, u0, calls, k, fmt, rate):
    u = roundtrip(ooc, torch.from_numpy(u0).cuda(), fmt, rate)
    tmp = torch.empty_like(u)
    for kp in pass_lengths(calls, k):
        ooc.ooc_heat7_steps(u, tmp, kp)
        u = roundtrip(ooc, u, fmt, rate)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def incore_wave(ooc, p0, pm1, kappa, calls, k, fmt, rate, ro_fmt, ro_rate, src, w):
    kap = roundtrip(ooc, torch.from_numpy(kappa).cuda(), ro_fmt, ro_rate)
    p = roundtrip(ooc, torch.from_numpy(p0).cuda(), fmt, rate)
    pp = roundtrip(ooc, torch.from_numpy(pm1).cuda(), fmt, rate)
    t = 0
    for kp in pass_lengths(calls, k):
        ooc.ooc_wave25_steps(p, pp, kap, kp, src=src, w=w, t=t)
        t += kp
        p = roundtrip(ooc, p, fmt, rate)
        pp = roundtrip(ooc, pp, fmt, rate)
    torch.cuda.synchronize()
    return p.cpu().numpy(), pp.cpu().numpy()


FMTS = [("fp32", 16), ("bf16", 16), ("fr4", 8), ("fr4", 16), ("fr4", 24)]


@pytest.mark.parametrize("spl", [1, 2])
@pytest.mark.parametrize("fmt,rate", FMTS)
@pytest.mark.parametrize("T,k,calls", [(4, 1, [5]), (8, 2, [7]), (12, 3, [10]), (28, 2, [3, 4]), (64, 4, [9]),
                                       (32, 5, [11]), (8, 6, [13])])
def test_heat7_ooc_bit_identical_to_incore(ooc, fmt, rate, T, k, calls, spl):
    # spl = heat7 steps per launch (2: pairs fused, level s on chip); the
    # in-core reference always runs one step per launch
    shape = (64, 24, 32)  # nz = 64: thin last slabs for T = 12, 28
    u0, _ = sine_modes_field(shape, seed=4)
    plan = ooc.Plan(nx=32, ny=24, nz=64, stencil="heat7", k=k, rw_format=fmt, rw_rate=rate, slab_planes=T,
                    heat_steps_per_launch=spl)
    try:
        plan.set_field(0, u0)
        for n in calls:
            plan.step(n)
        got = plan.get_field(0)
        st = plan.stats()
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, calls, k, fmt, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert st["steps_done"] == sum(calls)
    assert st["passes"] == len(pass_lengths(calls, k))


@pytest.mark.parametrize("fmt,rate", [("fp32", 16), ("fr4", 16)])
@pytest.mark.parametrize("T,k,calls", [(8, 2, [6]), (12, 4, [8, 3]), (16, 5, [10]), (4, 4, [4])])
def test_heat7_fused_ooc_several_tiles(ooc, fmt, rate, T, k, calls):
    # several 120-wide x tiles and 8-row y tiles with ragged tails, so the
    # bands of the fused pairs cross tile edges
    nz, ny, nx = 48, 36, 248
    u0 = smooth_random_field((nz, ny, nx), 5.0, seed=8)
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="heat7", k=k, rw_format=fmt, rw_rate=rate, slab_planes=T,
                    heat_steps_per_launch=2)
    try:
        plan.set_field(0, u0)
        for n in calls:
            plan.step(n)
        got = plan.get_field(0)
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, calls, k, fmt, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def wave_inputs(shape, nsteps, seed=3):
    v = layered_velocity(shape, seed=seed)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    nz, ny, nx = shape
    src = (nx // 2, ny // 2, nz // 2)
    w = (ricker(nsteps + 8, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    rng = np.random.default_rng(seed)
    p0 = (1e-3 * rng.normal(size=shape)).astype(np.float32)
    pm1 = (0.9 * p0).astype(np.float32)
    return kappa, p0, pm1, src, w


@pytest.mark.parametrize("fmt,rate,ro_fmt,ro_rate", [("fp32", 16, "fp32", 16), ("fr4", 16, "fr4", 16),
                                                     ("fr4", 12, "fp32", 16), ("bf16", 16, "bf16", 16),
                                                     ("fp32", 16, "fr4", 8)])
@pytest.mark.parametrize("T,k,calls", [(8, 1, [5]), (16, 2, [7]), (8, 3, [9]), (64, 2, [4]), (24, 3, [2, 5]),
                                       (40, 10, [12])])
def test_wave25_ooc_bit_identical_to_incore(ooc, fmt, rate, ro_fmt, ro_rate, T, k, calls):
    shape = (64, 20, 24)
    kappa, p0, pm1, src, w = wave_inputs(shape, sum(calls))
    plan = ooc.Plan(nx=24, ny=20, nz=64, stencil="wave25", k=k, rw_format=fmt, rw_rate=rate, ro_format=ro_fmt,
                    ro_rate=ro_rate, slab_planes=T)
    try:
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        for n in calls:
            plan.step(n)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
    finally:
        plan.close()
    ref_p, ref_pp = incore_wave(ooc, p0, pm1, kappa, calls, k, fmt, rate, ro_fmt, ro_rate, src, w)
    assert np.array_equal(got_p.view(np.uint32), ref_p.view(np.uint32))
    assert np.array_equal(got_pp.view(np.uint32), ref_pp.view(np.uint32))


@pytest.mark.parametrize("fmt,rate", FMTS)
def test_set_get_field_roundtrip(ooc, fmt, rate):
    x = smooth_random_field((32, 16, 20), 4.0, seed=8)
    plan = ooc.Plan(nx=20, ny=16, nz=32, stencil="heat7", k=2, rw_format=fmt, rw_rate=rate, slab_planes=8)
    try:
        plan.set_field(0, x)
        got = plan.get_field(0)
    finally:
        plan.close()
    ref = oracle.storage_roundtrip(x, fmt, rate).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("fmt,rate", [("bf16", 16), ("fr4", 12)])
def test_set_get_many_slabs_pinned_wave_fields(ooc, fmt, rate):
    # 8 slabs with a ragged last one, so the overlapped set/get reuse each
    # ring and staging buffer several times; pinned host buffers (fully
    # asynchronous copies); the three wave fields must not disturb each other.
    nz, ny, nx = 92, 12, 16
    xs = [smooth_random_field((nz, ny, nx), 3.0 + f, seed=20 + f) for f in range(3)]
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="wave25", k=1, rw_format=fmt, rw_rate=rate, ro_format=fmt,
                    ro_rate=rate, slab_planes=12)
    try:
        for f in range(3):
            src = torch.from_numpy(xs[f]).pin_memory()
            plan.set_field(f, src.numpy())
        for f in range(3):
            dst = torch.empty((nz, ny, nx), dtype=torch.float32, pin_memory=True)
            plan.get_field(f, out=dst.numpy())
            ref = oracle.storage_roundtrip(xs[f], fmt, rate).astype(np.float32)
            assert np.array_equal(dst.numpy().view(np.uint32), ref.view(np.uint32)), f
    finally:
        plan.close()


def test_heat7_ooc_against_oracle_pipeline(ooc):
    # The configuration of the 128^3 heat case: 4 slabs of 32 planes, k = 2,
    # 8 steps, FR4 at 16 bits/value.
    shape = (128, 128, 128)
    u0, _ = sine_modes_field(shape, seed=0)
    plan = ooc.Plan(nx=128, ny=128, nz=128, stencil="heat7", k=2, rw_format="fr4", rw_rate=16, slab_planes=32)
    try:
        plan.set_field(0, u0)
        plan.step(8)
        got = plan.get_field(0)
        info = plan.info()
    finally:
        plan.close()
    assert info["nslab"] == 4
    pipe = oracle.heat7_storage_pipeline(u0, 8, 2, "fr4", 16)
    exact = oracle.heat7_run(u0.astype(np.float64), 8)
    assert oracle.error_metrics(got, pipe)["rel_l2"] < 5e-5
    assert oracle.error_metrics(got, exact)["rel_l2"] < 1e-4


def test_budget_forces_streaming_and_matches_single_slab(ooc):
    shape = (96, 32, 32)
    u0, _ = sine_modes_field(shape, seed=2)
    outs = []
    for budget in (1 << 28, 300_000):
        plan = ooc.Plan(nx=32, ny=32, nz=96, stencil="heat7", k=3, rw_format="fr4", rw_rate=12,
                        device_budget_bytes=budget)
        try:
            plan.set_field(0, u0)
            plan.step(9)
            outs.append((plan.info()["nslab"], plan.get_field(0)))
        finally:
            plan.close()
    assert outs[0][0] == 1 and outs[1][0] > 3
    assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))


def test_full_size_heat_benchmark_configuration(ooc):
    # The 1024^3 heat workload exactly as bench.py runs it (1 GiB device
    # budget, k = 4, 64 steps, FR4 at 16 bits/value): bit-identical to the
    # in-core GPU reference, and within the stated error of the FP64 oracle
    # on a sampled sub-box (central 128^3, exact dependency cone).
    n, nsteps, k = 1024, 64, 4
    u0 = smooth_random_field((n, n, n), 32.0, seed=2)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=k, rw_format="fr4", rw_rate=16,
                    device_budget_bytes=1 << 30)
    try:
        assert plan.device_bytes <= 1 << 30
        plan.set_field(0, u0)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, [nsteps], k, "fr4", 16)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    c0, c1 = n // 2 - 64, n // 2 + 64
    sub = u0[c0 - nsteps:c1 + nsteps, c0 - nsteps:c1 + nsteps, c0 - nsteps:c1 + nsteps].astype(np.float64)
    exact = oracle.heat7_run(sub, nsteps)[nsteps:-nsteps, nsteps:-nsteps, nsteps:-nsteps]
    m = oracle.error_metrics(got[c0:c1, c0:c1, c0:c1], exact)
    assert m["rel_l2"] < 1e-4, m


def test_full_size_wave_benchmark_configuration(ooc):
    # The 1024^3 wave workload's code 4 (read-write levels and kappa at FR4-16,
    # 4 GiB device budget, k = 10) over two passes with the source on:
    # bit-identical to the in-core GPU reference with the same storage round
    # trips, at the size the bench runs.
    n, k, nsteps = 1024, 10, 20
    kappa, p0, pm1, src, w = wave_inputs((n, n, n), nsteps)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format="fr4", rw_rate=16, ro_format="fr4",
                    ro_rate=16, device_budget_bytes=4 << 30)
    try:
        assert plan.device_bytes <= 4 << 30 and plan.info()["nslab"] > 1
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plan.step(nsteps)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
    finally:
        plan.close()
    ref_p, ref_pp = incore_wave(ooc, p0, pm1, kappa, [nsteps], k, "fr4", 16, "fr4", 16, src, w)
    assert np.array_equal(got_p.view(np.uint32), ref_p.view(np.uint32))
    assert np.array_equal(got_pp.view(np.uint32), ref_pp.view(np.uint32))
    del ref_p, ref_pp
    # Against the FP64 oracle on sampled outputs: the central 32^3 box after
    # 20 steps depends only on inputs within 4 x 20 = 80 planes of it, so the
    # oracle runs on a 208^3 sub-box (88 planes of margin, 4-aligned so that
    # its codec blocks are the full grid's blocks) with the same storage
    # round trips.  Errors entering from the sub-box's edges travel 4 planes
    # per step and cross at most one block per round trip: 80 + 6 < 88.
    c0, c1, m = n // 2 - 16, n // 2 + 16, 88
    lo, hi = c0 - m, c1 + m
    sub = (slice(lo, hi),) * 3
    srcf = ((src[2] - lo) * (hi - lo) + (src[1] - lo)) * (hi - lo) + (src[0] - lo)
    want_p, _ = oracle.wave25_storage_pipeline(p0[sub], pm1[sub], kappa[sub], nsteps, k, "fr4", 16, ro_fmt="fr4",
                                               ro_rate=16, src=srcf, w=w.astype(np.float64))
    exact_p, _ = oracle.wave25_run(p0[sub].astype(np.float64), pm1[sub].astype(np.float64),
                                   kappa[sub].astype(np.float64), nsteps, src=srcf, w=w.astype(np.float64))
    cen = (slice(m, m + 32),) * 3
    mp = oracle.error_metrics(got_p[c0:c1, c0:c1, c0:c1], want_p[cen])
    me = oracle.error_metrics(got_p[c0:c1, c0:c1, c0:c1], exact_p[cen])
    print(f"1024^3 wave code 4, central 32^3 after {nsteps} steps: vs oracle pipeline {mp}, vs FP64 run {me}")
    # measured 7.6e-5 and 1.5e-3: the codec flips of the other wave tests at
    # white-noise data, and FR4-16's storage error on white noise
    assert mp["rel_l2"] < 3e-4, mp
    assert me["rel_l2"] < 5e-3, me


@pytest.mark.parametrize("rw,rw_rate,ro,ro_rate", [("fr4", 16, "fr4", 16), ("fr4", 16, "fp32", 16),
                                                   ("bf16", 16, "bf16", 16)])
def test_wave25_compressed_pipeline_against_oracle(ooc, rw, rw_rate, ro, ro_rate):
    # Section VI's codes 4 (read-write levels and kappa at 16 bits/value) and
    # 2 (read-write levels only), and BF16 storage, against the oracle's FP64
    # leapfrog with the same storage round trips (at load, kappa once, both
    # levels after every pass).  4 slabs of 32 planes with k = 10 (the common
    # region, 40 planes, is wider than a slab), the source on, two calls of
    # 10 and 11 steps (passes of 10, 10 and 1 steps), planes spanning two
    # 128-wide x tiles and six 8-row y tiles of the wave kernel.
    #
    # Tolerance: both sides round-trip identical formats at identical points,
    # so they differ by the GPU's FP32 arithmetic (about 10 steps x 2^-24
    # relative between round trips) carried through each round trip, where a
    # value next to a rounding or truncation boundary lands on the other side
    # and moves by one unit of what the format keeps: one BF16 ulp (2^-8
    # relative), or one unit of the last FR4 bit plane kept (about the codec's
    # own error, 1e-5 relative here at 16 bits/value).  Such flips hit a
    # fraction of the points (the FP32 error over the quantum, ~1e-4 for BF16)
    # and spread with the wave: rel-L2 below 2e-3 (BF16) and 5e-5 (FR4-16),
    # max-abs below two units (2^-7 of the largest value for BF16).  Against
    # the FP64 run without storage, the storage error itself (Section VI-C)
    # adds on top.
    nz, ny, nx = 128, 48, 136
    shape = (nz, ny, nx)
    v = layered_velocity(shape, seed=3)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    p0 = (1e-3 * smooth_random_field(shape, 6.0, seed=41)).astype(np.float32)
    pm1 = (0.95 * p0).astype(np.float32)
    src = (nx // 2, ny // 2, nz // 2)
    srcf = (src[2] * ny + src[1]) * nx + src[0]
    w = (ricker(40, dt) * float(kappa[src[2], src[1], src[0]]) * 1e-2).astype(np.float32)
    calls = [10, 11]
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="wave25", k=10, rw_format=rw, rw_rate=rw_rate, ro_format=ro,
                    ro_rate=ro_rate, slab_planes=32)
    try:
        assert plan.info()["nslab"] == 4 and plan.info()["common_planes"] == 40
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        for n in calls:
            plan.step(n)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
        assert plan.stats()["passes"] == 3
    finally:
        plan.close()
    want_p, want_pp = oracle.wave25_storage_pipeline(p0, pm1, kappa, sum(calls), 10, rw, rw_rate, ro_fmt=ro,
                                                     ro_rate=ro_rate, src=srcf, w=w.astype(np.float64))
    exact_p, _ = oracle.wave25_run(p0.astype(np.float64), pm1.astype(np.float64), kappa.astype(np.float64),
                                   sum(calls), src=srcf, w=w.astype(np.float64))
    bf16 = rw == "bf16"
    for got, want in ((got_p, want_p), (got_pp, want_pp)):
        m = oracle.error_metrics(got, want)
        print(f"{rw}-{rw_rate}/{ro}-{ro_rate} vs oracle pipeline: {m}")
        assert m["rel_l2"] < (2e-3 if bf16 else 5e-5), m
        assert m["max_abs"] < (2.0 ** -7 if bf16 else 1e-3) * np.abs(want).max(), m
    m = oracle.error_metrics(got_p, exact_p)
    print(f"{rw}-{rw_rate}/{ro}-{ro_rate} vs FP64 run without storage: {m}")
    assert m["rel_l2"] < (2e-2 if bf16 else 1e-4), m


@pytest.mark.parametrize("table", [True, False])
def test_wave_step_deadline_keeps_the_source_in_step(ooc, table):
    # A wave plan with a source whose call times out: the call still advances
    # the plan's time, so a rebind (which copies the host time to the device
    # time that the table-driven source reads) and the next call inject the
    # right amplitudes; with a series longer than the device table the
    # amplitudes come from the host at the host time.  The bits equal a plan
    # that waited normally.
    n, k = 256, 10
    shape = (n, n, n)
    v = layered_velocity(shape, seed=3)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    zero = np.zeros(shape, dtype=np.float32)
    src = (n // 2, n // 2, n // 2)
    nw = 100 if table else 20000  # the device table holds 16384 amplitudes
    w = np.zeros(nw, dtype=np.float32)
    w[:80] = ricker(80, dt) * float(kappa[src[2], src[1], src[0]])
    out = []
    for hurried in (True, False):
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format="fr4", rw_rate=16, ro_format="fr4",
                        ro_rate=16, slab_planes=64)
        try:
            plan.set_field(0, zero)
            plan.set_field(1, zero)
            plan.set_field(2, kappa)
            plan.set_source(*src, w)
            if hurried:
                plan.set_wait_timeout(1)
                with pytest.raises(ooc.OocError) as err:
                    plan.step(40)
                assert err.value.status == 5
                torch.cuda.synchronize()
                plan.set_wait_timeout(0)
                plan.rebind()
            else:
                plan.step(40)
            assert plan.stats()["steps_done"] == 40
            plan.step(30)
            out.append((plan.get_field(0), plan.get_field(1)))
        finally:
            plan.close()
    assert np.abs(out[1][0]).max() > 0
    assert np.array_equal(out[0][0].view(np.uint32), out[1][0].view(np.uint32))
    assert np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))


def test_precision_configuration_against_oracle(ooc):
    # The long-horizon precision configuration at its stated size: wave25 at
    # 384^3, 6 slabs of 64 planes, k = 10, both levels and kappa at FR4-16,
    # the source at the centre, from rest; after 100 steps (10 passes) the
    # whole field against the FP64 oracle with the same storage round trips,
    # and against the FP64 run without them.
    #
    # Tolerance: as in the other compressed wave tests, the two pipelines
    # differ where FP32 arithmetic puts a value on the other side of the last
    # FR4 bit plane kept, which moves it by one unit of that plane: about the
    # storage error itself.  Here there are 10 round trips instead of 3, and
    # the field is nonzero only within some 40 cells of the source, so such
    # flips weigh more in the norm; the bound is a few times the storage
    # error against the FP64 run (measured 5.8e-5 against the oracle pipeline
    # and 5.3e-5 against the FP64 run).
    n, k, nsteps = 384, 10, 100
    v = layered_velocity((n, n, n), seed=3)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    src = (n // 2, n // 2, n // 2)
    srcf = (src[2] * n + src[1]) * n + src[0]
    w = (ricker(nsteps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float32)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format="fr4", rw_rate=16, ro_format="fr4",
                    ro_rate=16, slab_planes=64)
    try:
        assert plan.info()["nslab"] == 6
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    want, _ = oracle.wave25_storage_pipeline(zero, zero, kappa, nsteps, k, "fr4", 16, ro_fmt="fr4", ro_rate=16,
                                             src=srcf, w=w.astype(np.float64))
    exact, _ = oracle.wave25_run(np.zeros((n, n, n)), np.zeros((n, n, n)), kappa.astype(np.float64), nsteps,
                                 src=srcf, w=w.astype(np.float64))
    mp = oracle.error_metrics(got, want)
    me = oracle.error_metrics(got, exact)
    print(f"384^3 wave FR4-16 after {nsteps} steps: vs oracle pipeline {mp}, vs FP64 run {me}")
    assert mp["rel_l2"] < 2e-4, mp
    assert me["rel_l2"] < 5e-4, me


def test_step_deadline_reports_timeout_and_work_completes(ooc):
    # A host wait that runs past the plan's deadline returns OOC_E_TIMEOUT
    # (status 5) without faulting anything: the enqueued passes still run,
    # and after synchronising the plan gives the same field as a plan that
    # waited normally.  64 steps of a 256^3 FR4-16 field take several
    # milliseconds, far past a 1 ms deadline.
    n = 256
    u0 = smooth_random_field((n, n, n), 8.0, seed=12)
    plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format="fr4", rw_rate=16, slab_planes=32)
    ref = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format="fr4", rw_rate=16, slab_planes=32)
    try:
        plan.set_field(0, u0)
        plan.set_wait_timeout(1)
        with pytest.raises(ooc.OocError) as err:
            plan.step(64)
        assert err.value.status == 5
        torch.cuda.synchronize()
        plan.set_wait_timeout(0)
        assert plan.stats()["steps_done"] == 64  # enqueued before the wait, so counted
        got = plan.get_field(0)
        ref.set_field(0, u0)
        ref.step(64)
        want = ref.get_field(0)
    finally:
        plan.close()
        ref.close()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("fmt,rate,graph_mode", [("fp32", 16, 0), ("fp32", 16, 1), ("fr4", 16, 1)])
def test_calls_after_a_timeout_wait_for_its_queued_work(ooc, fmt, rate, graph_mode):
    # A call that returns OOC_E_TIMEOUT leaves its copies and kernels queued.
    # The plan's next calls wait for them (under the deadline) before they
    # touch the host image or the rings, so the caller need not synchronise:
    # a get_field straight after the timed-out call (a plain host copy of the
    # image with FP32 storage), then more steps, give the bits of a plan that
    # waited normally.
    n = 256
    u0 = smooth_random_field((n, n, n), 8.0, seed=13)
    out = []
    for hurried in (True, False):
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate, slab_planes=32,
                        graph_mode=graph_mode)
        try:
            plan.set_field(0, u0)
            if hurried:
                plan.set_wait_timeout(1)
                with pytest.raises(ooc.OocError) as err:
                    plan.step(64)
                assert err.value.status == 5
                plan.set_wait_timeout(0)
            else:
                plan.step(64)
            mid = plan.get_field(0)
            plan.step(8)
            out.append((mid, plan.get_field(0)))
        finally:
            plan.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("k", [1, 2])
def test_heat7_8cube_two_slabs_against_brute_force(ooc, k):
    # The smallest pipeline: 8^3, two slabs of 4 planes, h = 1.  FP32 storage
    # is bit-identical to the in-core kernel, and both agree with a per-point
    # FP64 evaluation (each step written out with an explicit neighbour
    # lookup, as in the oracle's brute-force pin) to FP32 rounding.
    rng = np.random.default_rng(21)
    u0 = rng.normal(size=(8, 8, 8)).astype(np.float32)
    nsteps = 4
    plan = ooc.Plan(nx=8, ny=8, nz=8, stencil="heat7", k=k, rw_format="fp32", slab_planes=4)
    try:
        assert plan.info()["nslab"] == 2
        plan.set_field(0, u0)
        plan.step(nsteps)
        got = plan.get_field(0)
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, [nsteps], k, "fp32", 16)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    u = u0.astype(np.float64)
    for _ in range(nsteps):
        v = np.empty_like(u)
        for z in range(8):
            for y in range(8):
                for x in range(8):
                    def at(dz, dy, dx):
                        zz, yy, xx = z + dz, y + dy, x + dx
                        return u[zz, yy, xx] if 0 <= zz < 8 and 0 <= yy < 8 and 0 <= xx < 8 else 0.0
                    nb = at(0, 0, -1) + at(0, 0, 1) + at(0, -1, 0) + at(0, 1, 0) + at(-1, 0, 0) + at(1, 0, 0)
                    v[z, y, x] = u[z, y, x] + (nb - 6.0 * u[z, y, x]) / 6.0
        u = v
    assert np.abs(got.astype(np.float64) - u).max() < 1e-6 * max(1.0, np.abs(u).max())


# Degenerate plans: grids of one or two 4-plane slabs, k h far beyond the
# grid (the common region is wider than the grid itself), common regions
# wider than a slab (a slab's input units then come from several slabs of
# the previous pass, whose write-backs it must wait for), the smallest grid
# (one codec block), and calls of zero steps between others.
@pytest.mark.parametrize("fmt,rate", [("fp32", 16), ("fr4", 16), ("bf16", 16), ("fr4", 8)])
@pytest.mark.parametrize("shape,T,k,calls", [((4, 4, 4), 4, 8, [0, 3, 9]), ((8, 4, 4), 4, 5, [7, 0]),
                                             ((4, 8, 12), None, 1, [2, 0, 1]), ((12, 4, 8), 4, 3, [4, 4]),
                                             ((16, 4, 4), 4, 9, [20])])
def test_heat7_degenerate_plans(ooc, fmt, rate, shape, T, k, calls):
    nz, ny, nx = shape
    u0 = np.random.default_rng(sum(shape) + k).normal(size=shape).astype(np.float32)
    kw = {"slab_planes": T} if T else {"device_budget_bytes": 1 << 24}
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="heat7", k=k, rw_format=fmt, rw_rate=rate, **kw)
    try:
        if T:
            assert plan.info()["nslab"] == nz // T
        plan.set_field(0, u0)
        for n in calls:
            plan.step(n)
        got = plan.get_field(0)
        st = plan.stats()
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, calls, k, fmt, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert st["steps_done"] == sum(calls)
    assert st["passes"] == len(pass_lengths(calls, k))


@pytest.mark.parametrize("fmt,rate,ro_fmt,ro_rate", [("fp32", 16, "fp32", 16), ("fr4", 16, "fr4", 16),
                                                     ("bf16", 16, "fr4", 12)])
@pytest.mark.parametrize("shape,T,k,calls", [((8, 4, 4), 4, 10, [13]), ((4, 4, 4), 4, 3, [0, 4, 1]),
                                             ((12, 8, 4), 4, 2, [5]), ((24, 8, 4), 4, 3, [7]),
                                             ((32, 4, 8), 8, 5, [11, 4])])
def test_wave25_degenerate_plans(ooc, fmt, rate, ro_fmt, ro_rate, shape, T, k, calls):
    nz, ny, nx = shape
    kappa, p0, pm1, src, w = wave_inputs(shape, sum(calls))
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="wave25", k=k, rw_format=fmt, rw_rate=rate, ro_format=ro_fmt,
                    ro_rate=ro_rate, slab_planes=T)
    try:
        assert plan.info()["nslab"] == nz // T
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        for n in calls:
            plan.step(n)
        got_p, got_pp = plan.get_field(0), plan.get_field(1)
    finally:
        plan.close()
    ref_p, ref_pp = incore_wave(ooc, p0, pm1, kappa, calls, k, fmt, rate, ro_fmt, ro_rate, src, w)
    assert np.abs(ref_p).max() > 0
    assert np.array_equal(got_p.view(np.uint32), ref_p.view(np.uint32))
    assert np.array_equal(got_pp.view(np.uint32), ref_pp.view(np.uint32))


@pytest.mark.parametrize("fmt,rate", [("fp32", 16), ("fr4", 16), ("bf16", 16)])
def test_graph_replay_matches_direct_launches(ooc, fmt, rate):
    # heat7 calls without profiling are captured as a CUDA graph per
    # distinct nsteps and replayed; calls of 8, 8, 5, 8 steps (replay,
    # recapture, recapture) give the bits of direct launches
    shape = (48, 40, 36)
    u0 = smooth_random_field(shape, 5.0, seed=31)
    out = {}
    for mode in (0, 1):
        plan = ooc.Plan(nx=36, ny=40, nz=48, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate, slab_planes=12,
                        graph_mode=mode)
        try:
            plan.set_field(0, u0)
            for n in (8, 8, 5, 8):
                plan.step(n)
            out[mode] = plan.get_field(0)
            st = plan.stats()
        finally:
            plan.close()
        assert st["steps_done"] == 29 and st["passes"] == 2 + 2 + 2 + 2
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
    ref = incore_heat(ooc, u0, [8, 8, 5, 8], 4, fmt, rate)
    assert np.array_equal(out[0].view(np.uint32), ref.view(np.uint32))


def test_wave_graph_replay_with_source_matches_direct(ooc):
    # wave plans replay graphs too: the source amplitude of each step is read
    # on the device from a table at the device copy of the plan's time, so
    # calls of 6, 6, 6, 4 steps (replays, then a recapture) inject the same
    # amplitudes as direct launches and as the in-core reference
    shape = (64, 20, 24)
    kappa, p0, pm1, src, w = wave_inputs(shape, 22)
    calls = [6, 6, 6, 4]
    out = {}
    for mode in (0, 1):
        plan = ooc.Plan(nx=24, ny=20, nz=64, stencil="wave25", k=3, rw_format="fr4", rw_rate=16, ro_format="fp32",
                        ro_rate=16, slab_planes=16, graph_mode=mode)
        try:
            plan.set_field(0, p0)
            plan.set_field(1, pm1)
            plan.set_field(2, kappa)
            plan.set_source(*src, w)
            for n in calls:
                plan.step(n)
            out[mode] = (plan.get_field(0), plan.get_field(1))
        finally:
            plan.close()
    ref_p, ref_pp = incore_wave(ooc, p0, pm1, kappa, calls, 3, "fr4", 16, "fp32", 16, src, w)
    for mode in (0, 1):
        assert np.array_equal(out[mode][0].view(np.uint32), ref_p.view(np.uint32)), mode
        assert np.array_equal(out[mode][1].view(np.uint32), ref_pp.view(np.uint32)), mode


@pytest.mark.parametrize("fmt,rate,spl", [("fr4", 16, 2), ("fr4", 16, 1), ("fp32", 16, 2), ("bf16", 16, 1)])
def test_profiled_trace_follows_each_slab_stages(ooc, fmt, rate, spl):
    # With profiling on, ooc_plan_get_trace returns the intervals of the last
    # call: every slab's stages run in dependency order (H2D -> decode ->
    # stencil launches -> encode -> D2H), each stream's intervals are in time
    # order, the counts match ooc_get_stats, and the bits match direct runs.
    shape = (48, 40, 36)
    u0 = smooth_random_field(shape, 5.0, seed=33)
    plan = ooc.Plan(nx=36, ny=40, nz=48, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate, slab_planes=12,
                    profile=1, heat_steps_per_launch=spl)
    try:
        plan.set_field(0, u0)
        plan.step(8)
        plan.reset_stats()
        plan.step(6)
        tr = plan.trace()
        st = plan.stats()
        got = plan.get_field(0)
        plan.set_profile(False)
        plan.step(4)
        assert plan.trace() == []
    finally:
        plan.close()
    assert tr and {r["pass"] for r in tr} == {0, 1} and {r["slab"] for r in tr} == {0, 1, 2, 3}
    by = {}
    for r in tr:
        assert r["end_ms"] >= r["start_ms"] >= -1e-3
        by.setdefault(r["kind"], []).append(r)
    assert len(by.get("decode", [])) == st["n_decode"] and len(by.get("encode", [])) == st["n_encode"]
    assert len(by["h2d"]) == st["n_h2d"] and len(by["d2h"]) == st["n_d2h"]
    # launches: 4 slabs x (4 steps, then 2), one step or a fused pair each
    assert sum(r["count"] for r in by["stencil"]) == st["n_stencil"] == (4 * 4 + 4 * 2) // spl
    staged = fmt != "fp32"
    assert ("decode" in by) == staged and ("encode" in by) == staged
    eps = 2e-3  # event timestamps are good to about a microsecond
    for stream in (("h2d",), ("decode", "stencil", "encode"), ("d2h",)):
        seq = [r for r in tr if r["kind"] in stream]
        for a, b in zip(seq, seq[1:]):
            assert b["start_ms"] >= a["end_ms"] - eps, (a, b)
    order = ("h2d", "decode", "stencil", "encode", "d2h")
    for ps in {(r["pass"], r["slab"]) for r in tr}:
        stages = {r["kind"]: r for r in tr if (r["pass"], r["slab"]) == ps}
        present = [k for k in order if k in stages]
        for a, b in zip(present, present[1:]):
            assert stages[b]["start_ms"] >= stages[a]["end_ms"] - eps, (ps, a, b)
    ref = incore_heat(ooc, u0, [8, 6], 4, fmt, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("fmt,rate", [("fr4", 16), ("fp32", 16)])
def test_debug_checks_pass_and_keep_the_bits(ooc, fmt, rate):
    # debug_checks = 1: guard bytes after every arena region stay intact and
    # every launch window and copy range passes its host check over ragged
    # slabs, a short last pass and set/get; the bits are those of the in-core
    # reference.
    shape = (48, 40, 36)
    u0 = smooth_random_field(shape, 5.0, seed=35)
    plan = ooc.Plan(nx=36, ny=40, nz=48, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate, slab_planes=12,
                    debug_checks=1)
    try:
        plan.set_field(0, u0)
        plan.step(8)
        plan.step(6)
        got = plan.get_field(0)
    finally:
        plan.close()
    ref = incore_heat(ooc, u0, [8, 6], 4, fmt, rate)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_debug_checks_wave_fields(ooc):
    shape = (64, 20, 24)
    kappa, p0, pm1, src, w = wave_inputs(shape, 12)
    plan = ooc.Plan(nx=24, ny=20, nz=64, stencil="wave25", k=3, rw_format="fr4", rw_rate=16, ro_format="fr4",
                    ro_rate=16, slab_planes=16, debug_checks=1)
    try:
        plan.set_field(0, p0)
        plan.set_field(1, pm1)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plan.step(6)
        plan.step(4)
        got = (plan.get_field(0), plan.get_field(1))
    finally:
        plan.close()
    ref_p, ref_pp = incore_wave(ooc, p0, pm1, kappa, [6, 4], 3, "fr4", 16, "fr4", 16, src, w)
    assert np.array_equal(got[0].view(np.uint32), ref_p.view(np.uint32))
    assert np.array_equal(got[1].view(np.uint32), ref_pp.view(np.uint32))


def test_debug_guard_overwrite_is_reported(ooc):
    # A byte of the guard that follows ring 0, overwritten here on purpose
    # from the host side (an in-bounds write to the caller's arena), makes
    # the next call return OOC_E_CORRUPT.
    nx, ny, nz = 36, 40, 48
    u0 = smooth_random_field((nz, ny, nx), 5.0, seed=36)
    plan = ooc.Plan(nx=nx, ny=ny, nz=nz, stencil="heat7", k=4, rw_format="fr4", rw_rate=16, slab_planes=12,
                    debug_checks=1)
    try:
        plan.set_field(0, u0)
        plan.step(4)
        ring_bytes = plan.info()["ring_planes"] * nx * ny * 4
        guard0 = (ring_bytes + 255) // 256 * 256
        assert guard0 + 256 <= plan.dev_arena.numel()
        with torch.cuda.stream(plan.streams[1]):
            plan.dev_arena[guard0 + 17] = 0
        torch.cuda.synchronize()
        with pytest.raises(ooc.OocError) as e:
            plan.step(4)
        assert e.value.status == 6
    finally:
        torch.cuda.synchronize()
        plan.close()


@pytest.mark.parametrize("fmt,rate", [("fr4", 16), ("fp32", 16), ("bf16", 16)])
def test_debug_checks_refuse_non_finite_input(ooc, fmt, rate):
    # With debug_checks, a NaN or infinity in ooc_set_field's input returns
    # OOC_E_INVALID (checked on the device for staged formats, on the host
    # for FP32 storage); the next finite field is accepted.  Without debug
    # checks the call does not look.
    u = np.random.default_rng(5).normal(size=(16, 12, 20)).astype(np.float32)
    for bad in (np.nan, np.inf):
        v = u.copy()
        v[9, 3, 17] = bad
        plan = ooc.Plan(nx=20, ny=12, nz=16, stencil="heat7", k=2, rw_format=fmt, rw_rate=rate, slab_planes=8,
                        debug_checks=1)
        try:
            with pytest.raises(ooc.OocError) as err:
                plan.set_field(0, v)
            assert err.value.status == 1
            plan.set_field(0, u)
            plan.step(2)
        finally:
            plan.close()
        quiet = ooc.Plan(nx=20, ny=12, nz=16, stencil="heat7", k=2, rw_format=fmt, rw_rate=rate, slab_planes=8)
        try:
            quiet.set_field(0, v)
        finally:
            quiet.close()
    assert ooc.ooc_take_device_fault() == 0


def test_fp64_debug_checks_refuse_non_finite_input(ooc):
    u = np.random.default_rng(6).normal(size=(8, 8, 12))
    u[2, 5, 7] = -np.inf
    plan = ooc.Plan(nx=12, ny=8, nz=8, stencil="heat7", k=2, rw_format="fp64", rw_rate=64, slab_planes=4,
                    precision="fp64", debug_checks=1)
    try:
        with pytest.raises(ooc.OocError) as err:
            plan.set_field(0, u)
        assert err.value.status == 1
    finally:
        plan.close()


def test_plans_run_concurrently_from_two_host_threads(ooc):
    # Two plans (a heat7 FR4-16 plan and a wave code-4 plan) stepped at the
    # same time from two host threads, each on its own streams: each gives
    # the bits of the same plan run alone.  The library's process-wide state
    # (launch constants, the tensor-map cache, fault words) is initialised
    # once, thread-safely.
    import threading
    n = 96
    u0 = smooth_random_field((n, n, n), 8.0, seed=31)
    kappa, p0, pm1, src, w = wave_inputs((n, n, n), 40)

    def heat():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format="fr4", rw_rate=16, slab_planes=24)
        try:
            plan.set_field(0, u0)
            for _ in range(4):
                plan.step(8)
            return plan.get_field(0)
        finally:
            plan.close()

    def wave():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=5, rw_format="fr4", rw_rate=16, ro_format="fr4",
                        ro_rate=16, slab_planes=24)
        try:
            plan.set_field(0, p0)
            plan.set_field(1, pm1)
            plan.set_field(2, kappa)
            plan.set_source(*src, w)
            for _ in range(4):
                plan.step(10)
            return plan.get_field(0)
        finally:
            plan.close()

    alone = [heat(), wave()]
    results, errors = [None, None], []

    def run(i, fn):
        try:
            results[i] = fn()
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(0, heat)), threading.Thread(target=run, args=(1, wave))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    for got, want in zip(results, alone):
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert ooc.ooc_take_device_fault() == 0
