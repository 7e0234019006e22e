"""Pins for the oracle's FP64 discrete adjoint of wave25: the dot-product
(transpose) identity against the Born linearisation, central finite
differences of the misfit in random directions, and a per-entry brute force
gradient on 8^3."""
import numpy as np

import oracle
from synth import ricker


def problem(n, nsteps, seed=0):
    rng = np.random.default_rng(seed)
    kappa = 0.08 + 0.06 * rng.random((n, n, n))
    src = (n // 2) * n * n + (n // 3) * n + n // 2
    w = ricker(nsteps, 0.004, freq=15.0)
    zr = n // 4
    rec = np.array([(zr * n + y) * n + x for y in range(1, n - 1, 2) for x in range(0, n, 2)], dtype=np.int64)
    return kappa, src, w, rec


def test_dot_product_adjoint_identity():
    kappa, src, w, rec = problem(12, 30)
    rng = np.random.default_rng(1)
    dk = rng.normal(size=kappa.shape) * 0.01
    dr = rng.normal(size=(30, rec.size))
    lhs = float(np.sum(oracle.wave25_born(kappa, dk, src, w, 30, rec) * dr))
    rhs = float(np.sum(dk * oracle.wave25_adjoint_grad(kappa, src, w, 30, rec, dr)))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_gradient_matches_central_differences():
    n, N = 16, 40
    kappa, src, w, rec = problem(n, N, seed=2)
    d = oracle.wave25_traces(kappa * 1.02, src, w, N, rec)  # data from a perturbed model
    tr = oracle.wave25_traces(kappa, src, w, N, rec)
    g = oracle.wave25_adjoint_grad(kappa, src, w, N, rec, tr - d)
    rng = np.random.default_rng(3)
    for _ in range(3):
        dk = rng.normal(size=kappa.shape)
        dk /= np.linalg.norm(dk)
        eps = 1e-4
        jp = oracle.misfit(oracle.wave25_traces(kappa + eps * dk, src, w, N, rec), d)
        jm = oracle.misfit(oracle.wave25_traces(kappa - eps * dk, src, w, N, rec), d)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * dk))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_brute_force_gradient_8cube():
    n, N = 8, 6
    kappa, src, w, rec = problem(n, N, seed=4)
    d = oracle.wave25_traces(kappa * 0.97, src, w, N, rec)
    tr = oracle.wave25_traces(kappa, src, w, N, rec)
    g = oracle.wave25_adjoint_grad(kappa, src, w, N, rec, tr - d)
    eps = 1e-5
    fd = np.zeros_like(kappa)
    flat = kappa.ravel()
    for i in range(flat.size):
        kp = flat.copy(); kp[i] += eps
        km = flat.copy(); km[i] -= eps
        fd.ravel()[i] = (oracle.misfit(oracle.wave25_traces(kp.reshape(kappa.shape), src, w, N, rec), d)
                         - oracle.misfit(oracle.wave25_traces(km.reshape(kappa.shape), src, w, N, rec), d)) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())


def test_zero_residual_zero_gradient():
    kappa, src, w, rec = problem(10, 12, seed=5)
    tr = oracle.wave25_traces(kappa, src, w, 12, rec)
    g = oracle.wave25_adjoint_grad(kappa, src, w, 12, rec, np.zeros_like(tr))
    assert not g.any()
    # traces agree with the plain stencil oracle
    p, _ = oracle.wave25_run(np.zeros_like(kappa), np.zeros_like(kappa), kappa, 12, src=src, w=w)
    assert np.allclose(tr[-1], p.ravel()[rec], rtol=0, atol=1e-15)
