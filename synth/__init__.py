"""Seeded synthetic inputs shared by the oracle checks and the GPU path.

This module holds input recipes only (initial fields, velocity models,
source wavelets).  It contains none of the stencil or codec arithmetic, so
both the CPU oracle and the CUDA path can consume the same arrays without
sharing any method code.

All generators evaluate in float64 and return C-contiguous arrays indexed
[z, y, x] (x fastest), cast to float32 where the field is an FP32 input.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "sine_mode",
    "sine_modes_field",
    "smooth_random_field",
    "smooth_random_field_torch",
    "layered_velocity",
    "ricker",
    "random_blocks",
]


def sine_mode(shape, k, amplitude=1.0, dtype=np.float64):
    """Product of sines sin(pi*k_a*(i_a+1)/(n_a+1)) over the three axes.

    This is an eigenvector of the 7-point Laplacian with zero Dirichlet
    ghosts, which gives the heat-equation tests a closed-form decay.
    ``shape`` is (nz, ny, nx) and ``k`` is (kx, ky, kz).
    """
    nz, ny, nx = shape
    kx, ky, kz = k
    sx = np.sin(math.pi * kx * (np.arange(nx) + 1) / (nx + 1))
    sy = np.sin(math.pi * ky * (np.arange(ny) + 1) / (ny + 1))
    sz = np.sin(math.pi * kz * (np.arange(nz) + 1) / (nz + 1))
    f = amplitude * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return np.ascontiguousarray(f, dtype=dtype)


def sine_modes_field(shape, seed=0, nmodes=3, kmax=4, noise_sigma=1e-3, noise_seed=1):
    """Sum of ``nmodes`` sine modes with wavenumbers drawn from U{1..kmax}^3
    (seed ``seed``), plus N(0, noise_sigma^2) noise (seed ``noise_seed``).

    Returns (field_float32, wavenumbers).  With noise_sigma=0 the field is an
    exact combination of Laplacian eigenvectors (before the FP32 cast).
    """
    rng = np.random.default_rng(seed)
    ks = [tuple(int(v) for v in rng.integers(1, kmax + 1, size=3)) for _ in range(nmodes)]
    f = np.zeros(shape, dtype=np.float64)
    for k in ks:
        f += sine_mode(shape, k)
    if noise_sigma > 0:
        f += np.random.default_rng(noise_seed).normal(0.0, noise_sigma, size=shape)
    return np.ascontiguousarray(f, dtype=np.float32), ks


def smooth_random_field(shape, corr_len, seed, nterms=256, dtype=np.float32, ychunk=32):
    """Smooth random field with correlation length ``corr_len`` cells.

    f(x,y,z) = sqrt(8/J) * sum_j cos(kx_j x + ax_j) cos(ky_j y + ay_j) cos(kz_j z + az_j)
    with k*_j ~ N(0, 1/corr_len^2) and phases ~ U[0, 2 pi).  Each term is a
    separable product, so the whole field is one dense product of an
    (nz x J) matrix and a (J x ny*nx) matrix, evaluated in float64 in chunks
    of ``ychunk`` rows.  The normalisation gives unit variance on average.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    J = nterms
    k = rng.normal(0.0, 1.0 / corr_len, size=(3, J))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(3, J))
    X = np.cos(np.outer(np.arange(nx), k[0]) + ph[0])  # (nx, J)
    Y = np.cos(np.outer(np.arange(ny), k[1]) + ph[1])  # (ny, J)
    Z = np.cos(np.outer(np.arange(nz), k[2]) + ph[2]) * math.sqrt(8.0 / J)  # (nz, J)
    out = np.empty(shape, dtype=dtype)
    for y0 in range(0, ny, ychunk):
        y1 = min(ny, y0 + ychunk)
        B = (Y[y0:y1, None, :] * X[None, :, :]).reshape(-1, J)  # ((y1-y0)*nx, J)
        out[:, y0:y1, :] = (Z @ B.T).reshape(nz, y1 - y0, nx)
    return out


def smooth_random_field_torch(shape, corr_len, seed, nterms=16, device="cuda", zchunk=64):
    """The recipe of ``smooth_random_field`` evaluated with torch on
    ``device`` (float64 terms, float32 result), for fields too large for the
    host-side product (billions of points).  The wavenumbers and phases are
    the same draws as ``smooth_random_field`` with the same seed and
    ``nterms``; values agree with it to float64 rounding of the cosines."""
    import torch

    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    J = nterms
    k = rng.normal(0.0, 1.0 / corr_len, size=(3, J))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(3, J))

    def axis(n, a):
        i = torch.arange(n, dtype=torch.float64, device=device)
        return torch.cos(torch.outer(i, torch.from_numpy(k[a]).to(device)) + torch.from_numpy(ph[a]).to(device))

    X, Y = axis(nx, 0), axis(ny, 1)
    Z = axis(nz, 2) * math.sqrt(8.0 / J)
    B = (Y[:, None, :] * X[None, :, :]).reshape(-1, J)  # (ny*nx, J)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    for z0 in range(0, nz, zchunk):
        z1 = min(nz, z0 + zchunk)
        out[z0:z1] = (Z[z0:z1] @ B.T).reshape(z1 - z0, ny, nx).to(torch.float32)
    return out


def layered_velocity(shape, vmin=1500.0, vmax=4500.0, nlayers=8, perturb=0.05,
                     corr_len=8.0, seed=3, white=False):
    """Layered velocity model (m/s): ``nlayers`` equal z-layers whose speed
    rises linearly from vmin to vmax, times (1 + perturb*g) with g a smooth
    random field (correlation ``corr_len`` cells, seed ``seed``) clipped to
    [-1, 1].  ``white=True`` uses uniform white noise in [-1, 1] instead.
    Returned in float64.
    """
    nz, ny, nx = shape
    layer = np.minimum((np.arange(nz) * nlayers) // nz, nlayers - 1)
    v_layer = vmin + (vmax - vmin) * layer / max(nlayers - 1, 1)
    if white:
        g = np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)
    else:
        g = np.clip(smooth_random_field(shape, corr_len, seed, dtype=np.float64), -1.0, 1.0)
    return v_layer[:, None, None] * (1.0 + perturb * g)


def ricker(nsteps, dt, freq=15.0, t0=None):
    """Ricker wavelet samples s(n*dt), n = 0..nsteps-1, in float64:
    s(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0,
    with t0 = 1/f by default."""
    if t0 is None:
        t0 = 1.0 / freq
    tau = np.arange(nsteps) * dt - t0
    a = (math.pi * freq * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def random_blocks(kind, nblocks, seed):
    """float32 arrays of shape (nblocks*4, 4, 4) (``nblocks`` 4^3 blocks
    stacked along z) for codec tests.

    kinds: 'normal' (N(0,1)), 'wide' (random sign, exponents spread over
    the full finite float range), 'smooth' (low-order polynomial plus small
    noise), 'constant', 'zero' (mixed +0/-0), 'denormal' (subnormal values
    and zeros), 'sparse' (mostly zeros with a few spikes), 'bits' (random
    finite bit patterns).
    """
    rng = np.random.default_rng(seed)
    n = nblocks * 64
    if kind == "normal":
        v = rng.normal(size=n)
    elif kind == "wide":
        v = rng.choice([-1.0, 1.0], size=n) * np.ldexp(rng.uniform(1.0, 2.0, size=n), rng.integers(-126, 127, size=n))
        return v.astype(np.float32).reshape(nblocks * 4, 4, 4)
    elif kind == "smooth":
        z, y, x = np.meshgrid(np.arange(4.0), np.arange(4.0), np.arange(4.0), indexing="ij")
        blocks = []
        c = rng.normal(size=(nblocks, 10))
        scale = np.ldexp(1.0, rng.integers(-20, 20, size=nblocks))
        for b in range(nblocks):
            a = c[b]
            f = (a[0] + a[1] * x + a[2] * y + a[3] * z + 0.1 * (a[4] * x * x + a[5] * y * y + a[6] * z * z)
                 + 0.05 * (a[7] * x * y + a[8] * y * z + a[9] * x * z))
            blocks.append(scale[b] * (f + 1e-4 * rng.normal(size=f.shape)))
        v = np.concatenate([bb.ravel() for bb in blocks])
    elif kind == "constant":
        vals = rng.normal(size=nblocks) * np.ldexp(1.0, rng.integers(-30, 30, size=nblocks))
        vals[: max(1, nblocks // 8)] = 0.0
        v = np.repeat(vals, 64)
    elif kind == "zero":
        v = np.where(rng.random(n) < 0.5, 0.0, -0.0)
    elif kind == "denormal":
        m = rng.integers(0, 1 << 23, size=n)
        v = np.ldexp(m.astype(np.float64), -149) * rng.choice([-1.0, 1.0], size=n)
        v[rng.random(n) < 0.2] = 0.0
    elif kind == "sparse":
        v = np.zeros(n)
        idx = rng.choice(n, size=max(1, n // 40), replace=False)
        v[idx] = rng.normal(size=idx.size) * 1e3
    elif kind == "bits":
        bits = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        expo = (bits >> 23) & 0xFF
        bits = np.where(expo == 0xFF, bits & ~np.uint32(0x40000000), bits)  # keep finite
        return bits.view(np.float32).reshape(nblocks * 4, 4, 4)
    else:
        raise ValueError(kind)
    return np.asarray(v, dtype=np.float32).reshape(nblocks * 4, 4, 4)


def random_blocks64(kind, nblocks, seed):
    """float64 arrays of shape (nblocks*4, 4, 4) for the FP64 codec's tests;
    the kinds of ``random_blocks`` over the double range ('wide': exponents
    over the full finite double range; 'denormal': double subnormals; 'bits':
    random finite 64-bit patterns).  'normal', 'smooth', 'constant' and
    'sparse' take ``random_blocks``' values and give them full double
    significands (one factor per block for 'constant'); 'zero' keeps its
    signed zeros."""
    rng = np.random.default_rng(seed)
    n = nblocks * 64
    if kind == "wide":
        v = rng.choice([-1.0, 1.0], size=n) * np.ldexp(rng.uniform(1.0, 2.0, size=n), rng.integers(-1022, 1023, size=n))
    elif kind == "denormal":
        m = rng.integers(0, 1 << 52, size=n, dtype=np.int64)
        v = np.ldexp(m.astype(np.float64), -1074) * rng.choice([-1.0, 1.0], size=n)
        v[rng.random(n) < 0.2] = 0.0
    elif kind == "bits":
        bits = rng.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)
        expo = (bits >> np.uint64(52)) & np.uint64(0x7FF)
        bits = np.where(expo == 0x7FF, bits & ~np.uint64(1 << 62), bits)  # keep finite
        v = bits.view(np.float64)
    elif kind == "zero":
        v = random_blocks(kind, nblocks, seed).astype(np.float64).ravel()
    elif kind in ("normal", "smooth", "constant", "sparse"):
        v = random_blocks(kind, nblocks, seed).astype(np.float64).ravel()
        if kind == "constant":
            f = np.repeat(1.0 + rng.uniform(-1e-9, 1e-9, size=nblocks), 64)
        else:
            f = 1.0 + rng.uniform(-1e-9, 1e-9, size=n)
        v = v * f
    else:
        raise ValueError(kind)
    return np.asarray(v, dtype=np.float64).reshape(nblocks * 4, 4, 4)
