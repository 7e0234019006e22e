"""GPU adjoint parity: the adjoint-step and gradient kernels against FP64
formulas, the checkpointed forward/backward entry points against the FP64
oracle adjoint, FP64 finite differences in 16 seeded directions, and the
torch.autograd.Function end to end."""
import numpy as np
import pytest

import oracle
from synth import layered_velocity, ricker, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_adjoint_step_and_grad_kernels(ooc):
    rng = np.random.default_rng(0)
    shape = (20, 28, 36)
    mu, mup = rng.normal(size=(2,) + shape).astype(np.float32)
    kap = rng.uniform(0.02, 0.16, size=shape).astype(np.float32)
    out = ooc.ooc_wave25_adjoint_step(cuda(mu), cuda(mup), cuda(kap), d_out=torch.empty(shape, device="cuda"))
    ref = 2.0 * mu - mup + oracle.laplacian8(kap.astype(np.float64) * mu.astype(np.float64))
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()
    # in place on mu_prev
    d_mup = cuda(mup)
    ooc.ooc_wave25_adjoint_step(cuda(mu), d_mup, cuda(kap))
    torch.cuda.synchronize()
    assert np.array_equal(d_mup.cpu().numpy(), out.cpu().numpy())
    p = rng.normal(size=shape).astype(np.float32)
    g0 = rng.normal(size=shape)
    g = cuda(g0, torch.float64)
    ooc.ooc_wave25_grad_accum(g, cuda(mu), cuda(p))
    ref = g0 + mu.astype(np.float64) * oracle.laplacian8(p.astype(np.float64))
    torch.cuda.synchronize()
    assert np.abs(g.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()


def test_gather_scatter(ooc):
    f = torch.arange(1000, dtype=torch.float32, device="cuda")
    idx = torch.tensor([5, 17, 999, 0], dtype=torch.int64, device="cuda")
    assert ooc.ooc_gather(f, idx).cpu().tolist() == [5.0, 17.0, 999.0, 0.0]
    ooc.ooc_scatter_add(f, idx, torch.ones(4, device="cuda"))
    assert f[17].item() == 18.0 and f[1].item() == 1.0
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 0


def test_gather_scatter_skip_indices_outside_the_field(ooc):
    # Indices outside [0, field size) never reach memory: the gather gives 0
    # there, the scatter skips them, and the device fault word reports it.
    # The field is a slice of a larger buffer whose other values must stay.
    buf = torch.arange(1200, dtype=torch.float32, device="cuda")
    f = buf[100:1100]
    idx = torch.tensor([5, -1, 1000, 999, 1 << 40], dtype=torch.int64, device="cuda")
    assert ooc.ooc_take_device_fault() == 0
    assert ooc.ooc_gather(f, idx).cpu().tolist() == [105.0, 0.0, 0.0, 1099.0, 0.0]
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 2
    ooc.ooc_scatter_add(f, idx, torch.full((5,), 0.5, device="cuda"))
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 2
    assert ooc.ooc_take_device_fault() == 0  # read and cleared
    want = np.arange(1200, dtype=np.float32)
    want[105] += 0.5
    want[1099] += 0.5
    assert np.array_equal(buf.cpu().numpy(), want)


def test_checkpointed_calls_refuse_receivers_outside_the_field(ooc):
    n, N, every, rate = 16, 12, 4, 16
    shape = (n, n, n)
    d_kap = torch.full(shape, 0.05, device="cuda")
    traces = torch.zeros((N, 3), device="cuda")
    h_ckpt = torch.empty(ooc.ooc_wave25_ckpt_bytes(shape, N, every, rate), dtype=torch.uint8, pin_memory=True)
    work = torch.empty(ooc.ooc_wave25_adjoint_work_bytes(shape, every, rate), dtype=torch.uint8, device="cuda")
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    w = np.ones(N, dtype=np.float32)
    for bad in (n ** 3, -3):
        d_rec = torch.tensor([0, bad, 7], dtype=torch.int64, device="cuda")
        with pytest.raises(ooc.OocError) as err:
            ooc.ooc_wave25_forward_ckpt(d_kap, N, d_rec, traces, every, rate, h_ckpt, work, streams, src=(8, 8, 8),
                                        w=w)
        assert err.value.status == 1
        g = torch.zeros(shape, dtype=torch.float64, device="cuda")
        with pytest.raises(ooc.OocError) as err:
            ooc.ooc_wave25_backward_ckpt(d_kap, N, d_rec, traces, every, rate, h_ckpt, g, work, streams,
                                         src=(8, 8, 8), w=w)
        assert err.value.status == 1
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 0
    assert not traces.any()
    # the same call with the receivers in the field runs
    d_rec = torch.tensor([0, n ** 3 - 1, 7], dtype=torch.int64, device="cuda")
    ooc.ooc_wave25_forward_ckpt(d_kap, N, d_rec, traces, every, rate, h_ckpt, work, streams, src=(8, 8, 8), w=w)
    torch.cuda.synchronize()
    assert ooc.ooc_take_device_fault() == 0


def problem(n, nsteps, seed=3, rec_stride=2):
    shape = (n, n, n)
    v_true = layered_velocity(shape, seed=seed)
    dx = 10.0
    dt = 0.4 * dx / (v_true.max() * 1.05)
    c = dt / dx
    pert = np.clip(smooth_random_field(shape, 6.0, seed=seed + 10, dtype=np.float64), -1, 1)
    v = (v_true * (1.0 + 0.02 * pert)).astype(np.float32)
    src = (n // 2, n // 2, n // 2)
    src_flat = (src[2] * n + src[1]) * n + src[0]
    kap_src = float((v_true[src[2], src[1], src[0]] * c) ** 2)
    w = (ricker(nsteps, dt) * kap_src * 1e3).astype(np.float32)
    zr = 8
    rec = np.array([(zr * n + y) * n + x for y in range(0, n, rec_stride) for x in range(0, n, rec_stride)],
                   dtype=np.int64)
    kap_true = (v_true.astype(np.float32).astype(np.float64) * c) ** 2
    d = oracle.wave25_traces(kap_true, src_flat, w.astype(np.float64), nsteps, rec)
    return dict(v=v, c=c, dt=dt, dx=dx, src=src, src_flat=src_flat, w=w, rec=rec, d=d, shape=shape)


def kappa_of(v, c):
    # same float32 arithmetic as the kappa kernel: (v*c)^2 in FP32
    s = (v.astype(np.float32) * np.float32(c)).astype(np.float32)
    return (s * s).astype(np.float32)


@pytest.mark.parametrize("rate,n,N,stride", [(0, 48, 120, 2), (16, 48, 120, 2), (16, 64, 150, 1)])
def test_checkpointed_gradient_matches_oracle(ooc, rate, n, N, stride):
    # (16, 64, 150, 1) is the adjoint configuration's oracle check: 64^3, a
    # 64 x 64 receiver plane at z = 8 (every cell), checkpoints every 10
    # steps at 16 bits/value
    every = 10
    P = problem(n, N, rec_stride=stride)
    assert P["rec"].size == (n // stride) ** 2
    kap = kappa_of(P["v"], P["c"])
    kap64 = kap.astype(np.float64)
    tr_ref = oracle.wave25_traces(kap64, P["src_flat"], P["w"].astype(np.float64), N, P["rec"])
    res = tr_ref - P["d"]
    g_ref = oracle.wave25_adjoint_grad(kap64, P["src_flat"], P["w"].astype(np.float64), N, P["rec"], res)

    shape = P["shape"]
    d_kap = cuda(kap)
    d_rec = torch.from_numpy(P["rec"]).cuda()
    traces = torch.empty((N, P["rec"].size), device="cuda")
    h_ckpt = torch.empty(ooc.ooc_wave25_ckpt_bytes(shape, N, every, rate), dtype=torch.uint8, pin_memory=True)
    work = torch.empty(ooc.ooc_wave25_adjoint_work_bytes(shape, every, rate), dtype=torch.uint8, device="cuda")
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    ooc.ooc_wave25_forward_ckpt(d_kap, N, d_rec, traces, every, rate, h_ckpt, work, streams, src=P["src"], w=P["w"])
    tr = traces.cpu().numpy()
    assert np.linalg.norm(tr - tr_ref) <= 1e-4 * np.linalg.norm(tr_ref)
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    ooc.ooc_wave25_backward_ckpt(d_kap, N, d_rec, cuda(res), every, rate, h_ckpt, g, work, streams, src=P["src"],
                                 w=P["w"])
    gg = g.cpu().numpy()
    err = np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref)
    assert err < (1e-3 if rate == 0 else 2e-2), err


def test_gradient_finite_differences_16_directions(ooc):
    # FP64 central differences of the misfit (oracle forward) along 16 seeded
    # random directions against <dJ/dkappa, delta> from the GPU adjoint with
    # 16-bit compressed checkpoints, at 64^3.
    n, N, every, rate = 64, 150, 10, 16
    P = problem(n, N, seed=5)
    kap = kappa_of(P["v"], P["c"]).astype(np.float64)
    tr_ref = oracle.wave25_traces(kap, P["src_flat"], P["w"].astype(np.float64), N, P["rec"])
    res = tr_ref - P["d"]
    shape = P["shape"]
    d_kap = cuda(kap.astype(np.float32))
    d_rec = torch.from_numpy(P["rec"]).cuda()
    traces = torch.empty((N, P["rec"].size), device="cuda")
    h_ckpt = torch.empty(ooc.ooc_wave25_ckpt_bytes(shape, N, every, rate), dtype=torch.uint8, pin_memory=True)
    work = torch.empty(ooc.ooc_wave25_adjoint_work_bytes(shape, every, rate), dtype=torch.uint8, device="cuda")
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    ooc.ooc_wave25_forward_ckpt(d_kap, N, d_rec, traces, every, rate, h_ckpt, work, streams, src=P["src"], w=P["w"])
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    ooc.ooc_wave25_backward_ckpt(d_kap, N, d_rec, cuda(res), every, rate, h_ckpt, g, work, streams, src=P["src"],
                                 w=P["w"])
    gg = g.cpu().numpy()
    errs = []
    for seed in range(100, 116):
        rng = np.random.default_rng(seed)
        delta = rng.normal(size=shape)
        delta *= np.abs(kap) / np.linalg.norm(delta) * np.sqrt(kap.size)  # relative-size perturbation pattern
        eps = 1e-6
        jp = oracle.misfit(oracle.wave25_traces(kap + eps * delta, P["src_flat"], P["w"].astype(np.float64), N,
                                                P["rec"]), P["d"])
        jm = oracle.misfit(oracle.wave25_traces(kap - eps * delta, P["src_flat"], P["w"].astype(np.float64), N,
                                                P["rec"]), P["d"])
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(gg * delta))
        errs.append(abs(fd - an) / max(abs(fd), 1e-300))
    assert max(errs) < 2e-2, errs


def test_wavefn_autograd_velocity_gradient(ooc):
    from paper_2109_05410_gb300.autograd import WaveConfig
    n, N = 32, 80
    P = problem(n, N, seed=7)
    rec = torch.from_numpy(P["rec"]).cuda()
    cfg = WaveConfig(dt=P["dt"], dx=P["dx"], nsteps=N, rec=rec, src=P["src"], w=P["w"], every=10, rate=16)
    v = cuda(P["v"]).requires_grad_(True)
    d = cuda(P["d"])
    tr = ooc.wave_forward(v, cfg)
    loss = 0.5 * ((tr - d) ** 2).sum()
    loss.backward()
    gv = v.grad.cpu().numpy().astype(np.float64)
    kap = kappa_of(P["v"], P["c"]).astype(np.float64)
    tr_ref = oracle.wave25_traces(kap, P["src_flat"], P["w"].astype(np.float64), N, P["rec"])
    g_ref = oracle.wave25_adjoint_grad(kap, P["src_flat"], P["w"].astype(np.float64), N, P["rec"], tr_ref - P["d"])
    gv_ref = g_ref * 2.0 * P["v"].astype(np.float64) * P["c"] ** 2
    assert np.linalg.norm(gv - gv_ref) / np.linalg.norm(gv_ref) < 1e-2
    assert abs(loss.item() - oracle.misfit(tr_ref, P["d"])) < 1e-3 * oracle.misfit(tr_ref, P["d"])
