"""torch.autograd.Function over the wave25 forward/adjoint entry points.

``WaveFn.apply(v, cfg)`` maps a velocity model v [nz, ny, nx] (float32, CUDA,
m/s) to the receiver traces [nsteps, nrec] of a wave25 run from rest; its
backward returns dJ/dv for any loss J of the traces.  The forward stores
(p^{kK}, p^{kK-1}) every K steps in pinned host memory, FR4-compressed at
``rate`` bits/value (0 = FP32); the backward replays each K-step segment
from its checkpoint and runs the discrete adjoint (all in libooc kernels).
With kappa = (v dt/dx)^2 and dt, dx fixed, dJ/dv = dJ/dkappa * 2 v (dt/dx)^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class WaveConfig:
    dt: float
    dx: float
    nsteps: int
    rec: "object"                 # int64 CUDA tensor of flat receiver indices (distinct)
    src: tuple | None = None      # (sx, sy, sz)
    w: np.ndarray | None = None   # source amplitude per step (float32, >= nsteps)
    every: int = 10               # checkpoint interval K
    rate: int = 16                # checkpoint bits/value (0 = FP32)
    extra: dict = field(default_factory=dict)


def _make_fn():
    import torch
    from . import (ooc_kappa_from_velocity, ooc_velocity_grad, ooc_wave25_adjoint_work_bytes,
                   ooc_wave25_backward_ckpt, ooc_wave25_ckpt_bytes, ooc_wave25_forward_ckpt)

    class _WaveFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, cfg):
            shape = tuple(v.shape)
            c = cfg.dt / cfg.dx
            kappa = ooc_kappa_from_velocity(v.contiguous(), c)
            nrec = cfg.rec.numel()
            traces = torch.empty((cfg.nsteps, nrec), dtype=torch.float32, device=v.device)
            h_ckpt = torch.empty(ooc_wave25_ckpt_bytes(shape, cfg.nsteps, cfg.every, cfg.rate), dtype=torch.uint8,
                                 pin_memory=True)
            work = torch.empty(ooc_wave25_adjoint_work_bytes(shape, cfg.every, cfg.rate), dtype=torch.uint8,
                               device=v.device)
            streams = [torch.cuda.current_stream(v.device), torch.cuda.Stream(device=v.device)]
            ooc_wave25_forward_ckpt(kappa, cfg.nsteps, cfg.rec, traces, cfg.every, cfg.rate, h_ckpt, work, streams,
                                    src=cfg.src, w=cfg.w)
            ctx.save_for_backward(v, kappa)
            ctx.cfg, ctx.h_ckpt, ctx.work = cfg, h_ckpt, work
            return traces

        @staticmethod
        def backward(ctx, grad_traces):
            v, kappa = ctx.saved_tensors
            cfg = ctx.cfg
            g = torch.empty(tuple(v.shape), dtype=torch.float64, device=v.device)
            streams = [torch.cuda.current_stream(v.device), torch.cuda.Stream(device=v.device)]
            ooc_wave25_backward_ckpt(kappa, cfg.nsteps, cfg.rec, grad_traces.contiguous().float(), cfg.every,
                                     cfg.rate, ctx.h_ckpt, g, ctx.work, streams, src=cfg.src, w=cfg.w)
            ctx.grad_kappa = g
            gv = ooc_velocity_grad(g, v.contiguous(), cfg.dt / cfg.dx)
            return gv, None

    return _WaveFn


try:
    WaveFn = _make_fn()
except Exception:  # torch missing: the binding still loads for host-side use
    WaveFn = None


def wave_forward(v, cfg):
    """Traces of a wave25 run for velocity v (differentiable w.r.t. v)."""
    if WaveFn is None:
        raise RuntimeError("torch is required for WaveFn")
    return WaveFn.apply(v, cfg)
