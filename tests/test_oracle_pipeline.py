"""Pins for the oracle's storage pipelines (CPU only).

``oracle.wave25_storage_pipeline`` is the FP64 leapfrog of Section VI with
the storage round trip that the out-of-core pipeline applies (Section V-A:
each slab is compressed once per pass of k steps, so every stored value goes
through exactly one round trip per pass; kappa, read only, once at load).
It is pinned here by things other than itself:

- with kappa = 0 every point obeys p^{n+1} - 2 p^n + p^{n-1} = w[n] at the
  source and 0 elsewhere, whose sum has a closed form; on integer-valued
  states every storage format that holds those integers exactly (FP32, BF16
  below 256, FR4 with every bit plane coded) must reproduce it exactly,
  whatever the pass length, which fixes the level bookkeeping across passes
  and the source time index;
- with every bit plane coded, the FR4 round trip is the block-floating-point
  truncation, computed here with numpy alone; the pipeline must equal the
  oracle's pinned stencil run with that truncation at load and at each pass
  boundary (and kappa truncated once);
- Section VI-C's qualitative result: fewer bits per value, more error.
"""
import numpy as np
import pytest

import oracle
from synth import layered_velocity, ricker, smooth_random_field

from test_oracle_codec import closed_form_quantised


def closed_form_leapfrog(p0, pm1, src, w, nsteps):
    """p^N and p^{N-1} of p^{n+1} = 2 p^n - p^{n-1} + w[n] delta_src from
    (p^0, p^{-1}): with v^n = p^n - p^{n-1}, v^{n+1} = v^n + w[n] delta_src,
    so p^N = p^0 + N v^0 + sum_{m<N} (N - m) w[m] delta_src."""
    def at(n):
        if n == -1:
            return pm1.astype(np.float64).copy()
        out = p0.astype(np.float64) + n * (p0.astype(np.float64) - pm1.astype(np.float64))
        if src >= 0:
            flat = out.reshape(-1)
            flat[src] += sum((n - m) * float(w[m]) for m in range(n))
        return out
    return at(nsteps), at(nsteps - 1)


@pytest.mark.parametrize("fmt,rate,amp,wamp", [("fp32", 16, 50, 3), ("fr4", 40, 50, 3), ("bf16", 16, 2, 0)])
@pytest.mark.parametrize("k", [1, 4, 7, 23, 30])
def test_wave_storage_pipeline_zero_kappa_closed_form(fmt, rate, amp, wamp, k):
    rng = np.random.default_rng(k)
    shape = (12, 8, 8)
    nsteps = 23
    p0 = rng.integers(-amp, amp + 1, size=shape).astype(np.float32)
    v0 = rng.integers(-1, 2, size=shape).astype(np.float32)
    pm1 = (p0 - v0).astype(np.float32)
    kappa = np.zeros(shape, dtype=np.float32)
    src = (6 * 8 + 3) * 8 + 5
    w = rng.integers(-wamp, wamp + 1, size=nsteps + 5).astype(np.float64) if wamp else None
    p, q = oracle.wave25_storage_pipeline(p0, pm1, kappa, nsteps, k, fmt, rate, ro_fmt=fmt, ro_rate=rate,
                                          src=src if wamp else -1, w=w)
    want_p, want_q = closed_form_leapfrog(p0, pm1, src if wamp else -1, w, nsteps)
    assert np.abs(want_p).max() < (256 if fmt == "bf16" else 1 << 24)  # exactly representable
    assert np.array_equal(p, want_p)
    assert np.array_equal(q, want_q)


def test_wave_storage_pipeline_zero_kappa_catches_a_restarted_source():
    # The source series continues across passes (w[done + j] in step j of a
    # pass): a pipeline that restarted it at w[0] in every pass equals the
    # closed form of the series w' with w'[5 i + j] = w[j], not of w.
    shape = (8, 8, 8)
    z = np.zeros(shape, dtype=np.float32)
    src = 100
    w = np.arange(1.0, 31.0)
    p, _ = oracle.wave25_storage_pipeline(z, z, z, 20, 5, "fp32", src=src, w=w)
    want, _ = closed_form_leapfrog(z, z, src, w, 20)
    restarted, _ = closed_form_leapfrog(z, z, src, np.tile(w[:5], 4), 20)
    assert np.array_equal(p, want)
    assert not np.array_equal(p, restarted)


@pytest.mark.parametrize("k,nsteps", [(3, 8), (10, 21), (5, 5)])
def test_wave_storage_pipeline_full_precision_fr4_is_block_truncation(k, nsteps):
    shape = (16, 12, 20)
    v = layered_velocity(shape, seed=3)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    rng = np.random.default_rng(7)
    p0 = (1e-3 * rng.normal(size=shape)).astype(np.float32)
    pm1 = (0.9 * p0).astype(np.float32)
    src = (8 * 12 + 6) * 20 + 10
    w = ricker(nsteps + 4, dt) * float(kappa.reshape(-1)[src])
    got_p, got_q = oracle.wave25_storage_pipeline(p0, pm1, kappa, nsteps, k, "fr4", 40, ro_fmt="fr4", ro_rate=40,
                                                  src=src, w=w)
    Q = closed_form_quantised
    kap = Q(kappa).astype(np.float64)
    p, q = Q(p0).astype(np.float64), Q(pm1).astype(np.float64)
    done = 0
    while done < nsteps:
        s = min(k, nsteps - done)
        p, q = oracle.wave25_run(p, q, kap, s, src=src, w=w, t0=done)
        p, q = Q(p).astype(np.float64), Q(q).astype(np.float64)
        done += s
    assert np.array_equal(got_p, p) and np.array_equal(got_q, q)
    # the round trips change the state: an oracle that skipped them would fail
    raw_p, _ = oracle.wave25_run(p0.astype(np.float64), pm1.astype(np.float64), kappa.astype(np.float64), nsteps,
                                 src=src, w=w)
    assert not np.array_equal(raw_p, got_p)


def test_wave_storage_pipeline_error_ordering():
    # Section VI-C: fewer bits per value, more error against the uncompressed
    # run; FP32 storage far below every compressed format.
    shape = (24, 24, 24)
    v = layered_velocity(shape, seed=3)
    dt = 0.4 * 10.0 / v.max()
    kappa = ((v * dt / 10.0) ** 2).astype(np.float32)
    p0 = smooth_random_field(shape, 4.0, seed=9)
    pm1 = (0.95 * p0).astype(np.float32)
    exact, _ = oracle.wave25_run(p0.astype(np.float64), pm1.astype(np.float64), kappa.astype(np.float64), 30)
    errs = {}
    for fmt, rate in (("fp32", 16), ("fr4", 24), ("fr4", 16), ("bf16", 16), ("fr4", 8)):
        p, _ = oracle.wave25_storage_pipeline(p0, pm1, kappa, 30, 10, fmt, rate)
        errs[(fmt, rate)] = oracle.error_metrics(p, exact)["rel_l2"]
    assert errs[("fp32", 16)] < 1e-6
    assert errs[("fp32", 16)] < errs[("fr4", 24)] < errs[("fr4", 16)] < errs[("fr4", 8)]
    assert errs[("fr4", 16)] < errs[("bf16", 16)]
