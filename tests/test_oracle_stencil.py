"""Pins for the oracle's FP64 stencils (CPU only): closed forms, brute
force on 8^3, polynomial exactness, the stability limit and symmetry."""
import itertools
import math

import numpy as np
import pytest

import oracle
from synth import sine_mode, ricker

C8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


@pytest.mark.parametrize("shape,k", [((12, 10, 8), (1, 2, 3)), ((16, 16, 16), (4, 1, 2)), ((9, 13, 11), (2, 5, 1))])
def test_heat7_sine_mode_decays_by_discrete_eigenvalue(shape, k):
    # Section III's neighbour average in 3D: with zero ghosts a product of
    # sines is an eigenvector; one step multiplies it by
    # lambda = 1 - 2 r sum_a (1 - cos(pi k_a/(n_a+1))).
    r = 1.0 / 6.0
    nz, ny, nx = shape
    u0 = sine_mode(shape, k)
    lam = 1.0 - 2.0 * r * sum(1.0 - math.cos(math.pi * ka / (na + 1)) for ka, na in zip(k, (nx, ny, nz)))
    t = 7
    u = oracle.heat7_run(u0, t, r)
    assert np.allclose(u, lam ** t * u0, rtol=0, atol=1e-13 * np.abs(u0).max())


def test_heat7_constant_interior_stays_constant():
    c = 1.5
    u = np.full((20, 20, 20), c)
    t = 3
    v = oracle.heat7_run(u, t)
    inner = v[t:-t, t:-t, t:-t]
    assert np.all(inner == c)
    assert v[0, 0, 0] < c  # zero ghosts pull the boundary down


def brute_neighbours(f, z, y, x, dz, dy, dx):
    nz, ny, nx = f.shape
    zz, yy, xx = z + dz, y + dy, x + dx
    if 0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx:
        return f[zz, yy, xx]
    return 0.0


def test_brute_force_8cube_heat7_and_wave25():
    rng = np.random.default_rng(0)
    u = rng.normal(size=(8, 8, 8))
    r = 0.13
    ref = np.zeros_like(u)
    for z, y, x in itertools.product(range(8), repeat=3):
        nb = {d: brute_neighbours(u, z, y, x, *d) for d in
              [(0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]}
        ref[z, y, x] = u[z, y, x] + r * (sum(nb.values()) - 6 * u[z, y, x])
    assert np.allclose(oracle.heat7_step(u, r), ref, rtol=0, atol=1e-14)

    p, pp, kap = rng.normal(size=(3, 8, 8, 8))
    kap = np.abs(kap) * 0.1
    ref = np.zeros_like(p)
    for z, y, x in itertools.product(range(8), repeat=3):
        lap = 3 * C8[0] * p[z, y, x]
        for m in range(1, 5):
            for d in [(0, 0, m), (0, 0, -m), (0, m, 0), (0, -m, 0), (m, 0, 0), (-m, 0, 0)]:
                lap += C8[m] * brute_neighbours(p, z, y, x, *d)
        ref[z, y, x] = 2 * p[z, y, x] - pp[z, y, x] + kap[z, y, x] * lap
    src = 3 * 64 + 5 * 8 + 2
    ref.ravel()[src] += 0.7
    assert np.allclose(oracle.wave25_step(p, pp, kap, src=src, w=0.7), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 6, 8, 9])
def test_laplacian8_exact_on_polynomials(deg):
    # The 8th-order central second difference is exact for polynomials of
    # degree <= 9 (its truncation error starts with the 10th derivative).
    n = 24
    c = np.arange(n, dtype=np.float64) - (n - 1) / 2.0
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    s = 0.25
    f = (s * x) ** deg + 0.5 * (s * y) ** deg - 0.25 * (s * z) ** deg
    d2 = 0.0 if deg < 2 else deg * (deg - 1)
    exact = d2 * s * s * ((s * x) ** (deg - 2) + 0.5 * (s * y) ** (deg - 2) - 0.25 * (s * z) ** (deg - 2)) if deg >= 2 else np.zeros_like(f)
    got = oracle.laplacian8(f)
    i = slice(4, n - 4)
    scale = max(1.0, np.abs(f[i, i, i]).max())
    assert np.allclose(got[i, i, i], exact[i, i, i], rtol=0, atol=1e-10 * scale)


def test_wave25_plane_wave_follows_discrete_dispersion():
    # Away from the boundary (farther than 4 cells per step) a cosine mode of
    # a homogeneous medium obeys the leapfrog recurrence exactly:
    # p^n = cos(n theta) p^0 with cos theta = 1 + kappa mu / 2 and mu the
    # stencil's symbol sum_a [c0 + 2 sum_m c_m cos(m k_a)].
    n = 48
    kvec = (0.3, 0.55, 0.9)
    c = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mode = np.cos(kvec[0] * x + 0.1) * np.cos(kvec[1] * y) * np.cos(kvec[2] * z + 0.2)
    kappa = 0.15
    mu = sum(C8[0] + 2 * sum(C8[m] * math.cos(m * ka) for m in range(1, 5)) for ka in kvec)
    cos_t = 1.0 + kappa * mu / 2.0
    theta = math.acos(cos_t)
    steps = 4
    p, pp = oracle.wave25_run(mode, math.cos(theta) * mode, np.full(mode.shape, kappa), steps)
    i = slice(4 * steps, n - 4 * steps)
    assert np.allclose(p[i, i, i], math.cos(steps * theta) * mode[i, i, i], rtol=0, atol=1e-12)
    assert np.allclose(pp[i, i, i], math.cos((steps - 1) * theta) * mode[i, i, i], rtol=0, atol=1e-12)


def test_wave25_stability_limit():
    # For these coefficients the 3D leapfrog limit is C <= 2/sqrt(3*6.5016)
    # ~ 0.4529 (kappa = C^2).  CFL 0.4 stays bounded for 600 steps; 0.47
    # blows up from noise.
    sym = -(C8[0] + 2 * sum(C8[m] * (-1) ** m for m in range(1, 5)))  # |symbol| at k = pi
    cmax = 2.0 / math.sqrt(3 * sym)
    assert abs(cmax - 0.4529) < 1e-3
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=(20, 20, 20)) * 1e-3
    for C, bounded in ((0.40, True), (0.47, False)):
        p, _ = oracle.wave25_run(p0, p0, np.full(p0.shape, C * C), 600)
        amp = np.abs(p).max()
        assert (amp < 1.0) == bounded, (C, amp)


def test_wave25_source_symmetry():
    # Homogeneous medium, source at the centre of an odd cube: the field is
    # invariant under the 48 symmetries of the cube, to round-off.
    n = 17
    kap = np.full((n, n, n), 0.12)
    src = (n // 2) * n * n + (n // 2) * n + n // 2
    w = ricker(60, 1e-3 * 5, freq=15.0) * 0.12
    p, _ = oracle.wave25_run(np.zeros_like(kap), np.zeros_like(kap), kap, 60, src=src, w=w)
    assert np.abs(p).max() > 0
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            q = np.transpose(p, perm)
            for ax, f in enumerate(flips):
                if f:
                    q = np.flip(q, axis=ax)
            assert np.allclose(q, p, rtol=0, atol=1e-12 * np.abs(p).max())


def test_error_metrics_basic():
    ref = np.ones((4, 5, 6))
    a = ref * (1 + 1e-6)
    m = oracle.error_metrics(a, ref, nsample_per_plane=10)
    assert abs(m["rel_l2"] - 1e-6) < 1e-12
    assert abs(m["mean_rel_sampled"] - 1e-6) < 1e-12
    assert m["samples"] == 40 and m["excluded"] == 0


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000).astype(np.float32),
                        rng.integers(0, 1 << 32, size=20000, dtype=np.uint64).astype(np.uint32).view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8], np.float32)])
    x = x[~np.isnan(x)]
    ours = oracle.bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    nan = np.array([np.nan], np.float32)
    assert np.isnan(oracle.bf16_roundtrip(nan)).all()


def test_storage_pipeline_error_ordering():
    # Section VI-C's qualitative finding: fewer bits, more error; FP32
    # storage is far below any compressed format.
    from synth import smooth_random_field
    u0 = smooth_random_field((32, 32, 32), 8.0, seed=2).astype(np.float64)
    exact = oracle.heat7_run(u0.astype(np.float32).astype(np.float64), 8)
    errs = {}
    for fmt, rate in (("fp32", 0), ("fr4", 24), ("fr4", 16), ("bf16", 0), ("fr4", 8)):
        u = oracle.heat7_storage_pipeline(u0, 8, 2, fmt, rate or 16)
        errs[(fmt, rate)] = oracle.error_metrics(u, exact)["rel_l2"]
    assert errs[("fp32", 0)] < 1e-6
    assert errs[("fp32", 0)] < errs[("fr4", 24)] < errs[("fr4", 16)] < errs[("fr4", 8)]


def _paper():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_setup.json")
    return {k: v["value"] for k, v in json.load(open(path))["items"].items()}


def test_wave25_footprint_is_table_I_stencil():
    # Table I and Section VI: a 25-point stencil with HALO = 4.  One oracle
    # step from a unit impulse (p^{n-1} = 0, kappa = 1) changes exactly the
    # 1 + 6 HALO points on the three axes through it, none farther than HALO.
    P = _paper()
    h = P["table1_halo"]
    n = 2 * h + 5
    p = np.zeros((n, n, n))
    c = n // 2
    p[c, c, c] = 1.0
    q, _ = oracle.wave25_run(p, np.zeros_like(p), np.ones_like(p), 1)
    nzp = np.argwhere(q != 0.0) - c
    assert len(nzp) == P["stencil_points"] == 1 + 6 * h
    assert np.abs(nzp).max() == h
    assert all(np.count_nonzero(o) <= 1 for o in nzp)  # on an axis through the impulse


def test_table_I_sizes_and_schedule():
    # Table I's 46 GB lies between 4 double datasets of the 1152^3 interior
    # (45.6 GiB) and of the (1152 + 2 HALO)^3 padded grid (46.5 GiB); the
    # steps 480..4320 are whole multiples of the temporal block 12, and the
    # padded side splits into the 8 divisions.
    P = _paper()
    side = P["table1_interior_side"] + 2 * P["table1_halo"]
    per_point = P["table1_datasets"] * P["table1_data_type_bytes"]
    inner = per_point * P["table1_interior_side"] ** 3 / 2 ** 30
    padded = per_point * side ** 3 / 2 ** 30
    assert inner <= P["table1_entire_size_gb"] <= padded < P["table1_entire_size_gb"] + 1
    steps = range(P["total_steps_first"], P["total_steps_last"] + 1, P["total_steps_increment"])
    assert len(steps) == 9 and all(s % P["temporal_block_steps"] == 0 for s in steps)
    assert side % P["divisions"] == 0  # 8 slabs of 145 planes


def test_paper_rates_are_fr4_rates_for_float():
    # The codes keep 32 or 24 of 64 bits per double (ratios 2 and 8/3); on
    # 32-bit floats the same ratios are FR4 at R = 16 and R = 12, and the
    # oracle's stream has exactly that size.
    P = _paper()
    shape = (8, 8, 8)
    fp32 = 8 * 8 * 8 * 4
    for bits in (P["code2_rw_bits_per_double"], P["code4_bits_per_double"]):
        ratio = 64 / bits
        rate = int(round(32 / ratio))
        x = np.random.default_rng(bits).normal(size=shape).astype(np.float32)
        assert oracle.fr4_encode(x, rate).nbytes * ratio == fp32


def test_heat7_fp32_variant_is_the_fp32_update():
    # The FP32 CPU variant (timed beside the FP64 oracle) computes the same
    # update in float arithmetic: bit for bit the numpy float32 evaluation
    # with the same association (the oracle is compiled without contraction),
    # and within FP32 rounding of the FP64 definition.
    rng = np.random.default_rng(17)
    u0 = rng.normal(size=(10, 12, 14)).astype(np.float32)
    r = np.float32(1.0 / 6.0)
    u = u0.copy()
    for _ in range(3):
        p = np.pad(u, 1)  # zero ghosts
        s = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:]) + p[1:-1, :-2, 1:-1]
        s = ((s + p[1:-1, 2:, 1:-1]) + p[:-2, 1:-1, 1:-1]) + p[2:, 1:-1, 1:-1]
        u = (u + r * (s - np.float32(6.0) * u)).astype(np.float32)
    got = oracle.heat7_run_f32(u0, 3)
    assert got.dtype == np.float32
    assert np.array_equal(got.view(np.uint32), u.view(np.uint32))
    ref = oracle.heat7_run(u0.astype(np.float64), 5)
    got5 = oracle.heat7_run_f32(u0, 5)
    assert np.abs(got5 - ref).max() <= 1e-6 * np.abs(ref).max()
