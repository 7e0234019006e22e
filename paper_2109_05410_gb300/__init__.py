"""Out-of-core stencil computation with on-the-fly fixed-rate compression
for one GB300 (sm_103a).

This package is a thin ctypes binding over the C ABI of ``libooc.so``
(declared in ``include/ooc.h``).  Every step of the computation runs in the
library's CUDA kernels; Python only marshals arguments and uses PyTorch for
device memory, pinned host memory and streams.  If the library is missing
the functions raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

__all__ = [
    "OOC_HEAT7", "OOC_WAVE25", "OOC_FMT_FP32", "OOC_FMT_BF16", "OOC_FMT_FR4",
    "OocConfig", "OocStats", "OocPlanInfo", "OocError", "lib", "build",
    "ooc_status_string", "ooc_take_device_fault", "ooc_compressed_bytes", "ooc_compress", "ooc_decompress", "ooc_compress64", "ooc_decompress64", "ooc_compress_var",
    "ooc_decompress_var", "ooc_compress_var_bound", "ooc_var_scratch_bytes", "OOC_FR4_PRECISION", "OOC_FR4_ACCURACY",
    "ooc_bf16_pack", "ooc_bf16_unpack", "ooc_heat7_steps", "ooc_heat7_steps_f64", "ooc_heat7_steps_fused", "ooc_heat7_steps_noalloc", "ooc_wave25_steps", "ooc_wave25_steps_f64", "ooc_wave25_steps_fused", "Plan",
    "ooc_gather", "ooc_scatter_add", "ooc_wave25_adjoint_step", "ooc_wave25_grad_accum", "ooc_kappa_from_velocity",
    "ooc_velocity_grad", "ooc_wave25_ckpt_bytes", "ooc_wave25_adjoint_work_bytes", "ooc_wave25_forward_ckpt",
    "ooc_wave25_backward_ckpt", "WaveFn", "wave_forward",
]

OOC_HEAT7, OOC_WAVE25 = 1, 2
OOC_FMT_FP32, OOC_FMT_BF16, OOC_FMT_FR4, OOC_FMT_FP64 = 0, 1, 2, 3
FORMATS = {"fp32": OOC_FMT_FP32, "bf16": OOC_FMT_BF16, "fr4": OOC_FMT_FR4, "fp64": OOC_FMT_FP64}
OOC_PREC_FP32, OOC_PREC_FP64 = 0, 1
PRECISIONS = {"fp32": OOC_PREC_FP32, "fp64": OOC_PREC_FP64}
STENCILS = {"heat7": OOC_HEAT7, "wave25": OOC_WAVE25}


class OocConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("stencil", ctypes.c_int32), ("k", ctypes.c_int32), ("r", ctypes.c_double),
        ("rw_format", ctypes.c_int32), ("rw_rate", ctypes.c_int32),
        ("ro_format", ctypes.c_int32), ("ro_rate", ctypes.c_int32),
        ("device_budget_bytes", ctypes.c_int64), ("slab_planes", ctypes.c_int32),
        ("profile", ctypes.c_int32), ("wait_timeout_ms", ctypes.c_int64),
        ("heat_steps_per_launch", ctypes.c_int32), ("graph_mode", ctypes.c_int32),
        ("debug_checks", ctypes.c_int32), ("precision", ctypes.c_int32),
    ]


class OocStats(ctypes.Structure):
    _fields_ = [
        ("steps_done", ctypes.c_int64), ("passes", ctypes.c_int64), ("slabs", ctypes.c_int64),
        ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("ms_decode", ctypes.c_double), ("ms_stencil", ctypes.c_double), ("ms_encode", ctypes.c_double),
        ("ms_h2d", ctypes.c_double), ("ms_d2h", ctypes.c_double),
        ("n_decode", ctypes.c_int64), ("n_stencil", ctypes.c_int64), ("n_encode", ctypes.c_int64),
        ("n_h2d", ctypes.c_int64), ("n_d2h", ctypes.c_int64),
        ("ms_last_step", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class OocPlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "slab_planes", "nslab", "common_planes", "halo", "ring_planes", "nrings",
        "device_bytes", "host_bytes", "staging_in_bytes", "staging_out_bytes")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class OocTraceRec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("count", ctypes.c_int32), ("pass_", ctypes.c_int64),
                ("slab", ctypes.c_int64), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


TRACE_KINDS = ("decode", "stencil", "encode", "h2d", "d2h")


class OocError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {ooc_status_string(status)} ({status})")
        self.status = status


_lib = None
_SIGS = {
    "ooc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ooc_compressed_bytes": (ctypes.c_size_t, [ctypes.c_int64] * 3 + [ctypes.c_int]),
    "ooc_compress": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 3 + [ctypes.c_int, ctypes.c_void_p,
                                                                              ctypes.c_size_t, ctypes.c_void_p]),
    "ooc_decompress": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_int64] * 3
                       + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ooc_compress64": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 3 + [ctypes.c_int, ctypes.c_void_p,
                                                                                ctypes.c_size_t, ctypes.c_void_p]),
    "ooc_decompress64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_int64] * 3
                         + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ooc_compress_var_bound": (ctypes.c_size_t, [ctypes.c_int64] * 3),
    "ooc_var_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64] * 3),
    "ooc_compress_var": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 3
                         + [ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p]),
    "ooc_decompress_var": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p] + [ctypes.c_int64] * 3
                           + [ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "ooc_bf16_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_bf16_unpack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_heat7_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int64] * 3
                        + [ctypes.c_double, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_heat7_steps_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int64] * 3
                            + [ctypes.c_double, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_heat7_steps_fused": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int64] * 3
                              + [ctypes.c_double, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_wave25_steps": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 6
                         + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_wave25_steps_fused": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int64] * 6
                               + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_wave25_steps_f64": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 6
                             + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_plan_create": (ctypes.c_int, [ctypes.POINTER(OocConfig), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "ooc_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(OocPlanInfo)]),
    "ooc_plan_bind": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p * 3]),
    "ooc_set_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ooc_get_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ooc_set_field64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ooc_get_field64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ooc_set_source": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 3 + [ctypes.c_void_p, ctypes.c_int64]),
    "ooc_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "ooc_take_device_fault": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "ooc_plan_set_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "ooc_plan_set_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ooc_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(OocStats)]),
    "ooc_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "ooc_plan_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(OocTraceRec), ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "ooc_plan_destroy": (None, [ctypes.c_void_p]),
    "ooc_heat7_steps_noalloc": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 3
                                + [ctypes.c_double, ctypes.c_int64, ctypes.c_void_p]),
    "ooc_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "ooc_scatter_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "ooc_wave25_adjoint_step": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64] * 3 + [ctypes.c_void_p]),
    "ooc_wave25_grad_accum": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 3 + [ctypes.c_void_p]),
    "ooc_kappa_from_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                               ctypes.c_void_p]),
    "ooc_velocity_grad": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]),
    "ooc_wave25_ckpt_bytes": (ctypes.c_size_t, [ctypes.c_int64] * 5 + [ctypes.c_int]),
    "ooc_wave25_adjoint_work_bytes": (ctypes.c_size_t, [ctypes.c_int64] * 4 + [ctypes.c_int]),
    "ooc_wave25_forward_ckpt": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 6
                                + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_void_p * 2]),
    "ooc_wave25_backward_ckpt": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int64] * 6
                                 + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p * 2]),
}


def build(force=False):
    """Compile libooc.so in-tree (nvcc, sm_103a)."""
    return _build_mod.build(force=force)


def lib():
    """The loaded libooc.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build_mod.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libooc.so is not built ({path}); call paper_2109_05410_gb300.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, what):
    if status != 0:
        raise OocError(status, what)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, name, numel=None, ndim=None):
    """Device pointer of a tensor checked against what the C call reads or
    writes through it: a CUDA tensor of ``dtype``, contiguous (no strides or
    broadcast views), with ``ndim`` dimensions and at least ``numel``
    elements when given.  The library cannot see a buffer's size, so a wrong
    tensor fails here instead of reaching memory it does not own."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name}: expected {ndim} dimensions, got {t.dim()}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: holds {t.numel()} elements, the call needs {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _host(t, name):
    """Pointer of a contiguous uint8 CPU tensor (the library checks its size
    and that it is pinned where it must be)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous uint8 CPU tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f32():
    import torch
    return torch.float32


def _dt(name):
    import torch
    return getattr(torch, name)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ooc_status_string(s):
    return lib().ooc_status_string(int(s)).decode()


def ooc_take_device_fault():
    """Bit set of the library's device fault words (read and cleared): 1 if
    a kernel gave up a bounded wait since the last call, 2 if a gather or
    scatter skipped an index outside its field; 0 when nothing went wrong."""
    f = ctypes.c_int()
    _check(lib().ooc_take_device_fault(ctypes.byref(f)), "ooc_take_device_fault")
    return f.value


def ooc_compressed_bytes(nx, ny, nz, rate):
    return int(lib().ooc_compressed_bytes(nx, ny, nz, rate))


def ooc_compress(d_in, rate, d_out=None, stream=None):
    """Encode a float32 CUDA tensor [nz, ny, nx] at ``rate`` bits/value into
    ``d_out`` (uint8 CUDA tensor, allocated if None); returns d_out."""
    import torch
    nz, ny, nx = d_in.shape
    nbytes = ooc_compressed_bytes(nx, ny, nz, rate)
    if d_out is None:
        d_out = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=d_in.device)
    _check(lib().ooc_compress(_dev(d_in, _f32(), "d_in", ndim=3), nx, ny, nz, rate, _dev(d_out, _dt("uint8"), "d_out"),
                              d_out.numel(), _stream(stream)), "ooc_compress")
    return d_out


def ooc_decompress(d_in, shape, rate, d_out=None, stream=None):
    import torch
    nz, ny, nx = shape
    if d_out is None:
        d_out = torch.empty(shape, dtype=torch.float32, device=d_in.device)
    _check(lib().ooc_decompress(_dev(d_in, _dt("uint8"), "d_in"), d_in.numel(), nx, ny, nz, rate,
                                _dev(d_out, _f32(), "d_out", numel=nx * ny * nz), _stream(stream)), "ooc_decompress")
    return d_out


def ooc_compress64(d_in, rate, d_out=None, stream=None):
    """FR4D: encode a float64 CUDA tensor [nz, ny, nx] (sides multiples of 4)
    at ``rate`` bits/value into ``d_out`` (uint8 CUDA tensor, allocated if
    None); returns d_out."""
    import torch
    nz, ny, nx = d_in.shape
    nbytes = ooc_compressed_bytes(nx, ny, nz, rate)
    if d_out is None:
        d_out = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=d_in.device)
    _check(lib().ooc_compress64(_dev(d_in, _dt("float64"), "d_in", ndim=3), nx, ny, nz, rate,
                                _dev(d_out, _dt("uint8"), "d_out"), d_out.numel(), _stream(stream)), "ooc_compress64")
    return d_out


def ooc_decompress64(d_in, shape, rate, d_out=None, stream=None):
    import torch
    nz, ny, nx = shape
    if d_out is None:
        d_out = torch.empty(shape, dtype=torch.float64, device=d_in.device)
    _check(lib().ooc_decompress64(_dev(d_in, _dt("uint8"), "d_in"), d_in.numel(), nx, ny, nz, rate,
                                  _dev(d_out, _dt("float64"), "d_out", numel=nx * ny * nz), _stream(stream)),
           "ooc_decompress64")
    return d_out


OOC_FR4_PRECISION = 1
OOC_FR4_ACCURACY = 2


def ooc_compress_var_bound(nx, ny, nz):
    return int(lib().ooc_compress_var_bound(nx, ny, nz))


def ooc_var_scratch_bytes(nx, ny, nz):
    return int(lib().ooc_var_scratch_bytes(nx, ny, nz))


def ooc_compress_var(d_in, mode, param, d_out=None, d_index=None, stream=None):
    """Variable-size modes (OOC_FR4_PRECISION: param = planes P;
    OOC_FR4_ACCURACY: param = tolerance).  Returns (stream bytes as a uint8
    CUDA tensor view of d_out, index as an int64 CUDA tensor of nblocks + 1
    word offsets).  Synchronises ``stream`` to learn the size."""
    import torch
    nz, ny, nx = d_in.shape
    nblk = ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 3) // 4)
    if d_out is None:
        d_out = torch.empty(max(ooc_compress_var_bound(nx, ny, nz), 4), dtype=torch.uint8, device=d_in.device)
    if d_index is None:
        d_index = torch.empty(nblk + 1, dtype=torch.int64, device=d_in.device)
    scratch = torch.empty(max(ooc_var_scratch_bytes(nx, ny, nz), 8), dtype=torch.uint8, device=d_in.device)
    used = ctypes.c_size_t(0)
    _check(lib().ooc_compress_var(_dev(d_in, _f32(), "d_in", ndim=3), nx, ny, nz, int(mode), float(param),
                                  _dev(d_out, _dt("uint8"), "d_out"), d_out.numel(),
                                  _dev(d_index, _dt("int64"), "d_index", numel=nblk + 1), _ptr(scratch),
                                  scratch.numel(), ctypes.byref(used), _stream(stream)), "ooc_compress_var")
    return d_out[:used.value], d_index


def ooc_decompress_var(d_in, d_index, shape, mode, param, d_out=None, stream=None):
    import torch
    nz, ny, nx = shape
    if d_out is None:
        d_out = torch.empty(shape, dtype=torch.float32, device=d_in.device)
    nblk = ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 3) // 4)
    _check(lib().ooc_decompress_var(_dev(d_in, _dt("uint8"), "d_in"), d_in.numel(),
                                    _dev(d_index, _dt("int64"), "d_index", numel=nblk + 1), nx, ny, nz, int(mode),
                                    float(param), _dev(d_out, _f32(), "d_out", numel=nx * ny * nz), _stream(stream)),
           "ooc_decompress_var")
    return d_out


def ooc_bf16_pack(d_in, d_out=None, stream=None):
    import torch
    if d_out is None:
        d_out = torch.empty(d_in.shape, dtype=torch.int16, device=d_in.device)
    _check(lib().ooc_bf16_pack(_dev(d_in, _f32(), "d_in"), _dev(d_out, _dt("int16"), "d_out", numel=d_in.numel()),
                               d_in.numel(), _stream(stream)), "ooc_bf16_pack")
    return d_out


def ooc_bf16_unpack(d_in, d_out=None, stream=None):
    import torch
    if d_out is None:
        d_out = torch.empty(d_in.shape, dtype=torch.float32, device=d_in.device)
    _check(lib().ooc_bf16_unpack(_dev(d_in, _dt("int16"), "d_in"), _dev(d_out, _f32(), "d_out", numel=d_in.numel()),
                                 d_in.numel(), _stream(stream)), "ooc_bf16_unpack")
    return d_out


def ooc_heat7_steps(d_u, d_tmp, nsteps, r=1.0 / 6.0, stream=None):
    nz, ny, nx = d_u.shape
    _check(lib().ooc_heat7_steps(_dev(d_u, _f32(), "d_u", ndim=3), _dev(d_tmp, _f32(), "d_tmp", numel=d_u.numel()),
                                 nx, ny, nz, float(r), int(nsteps), _stream(stream)), "ooc_heat7_steps")
    return d_u


def ooc_heat7_steps_f64(d_u, d_tmp, nsteps, r=1.0 / 6.0, stream=None):
    """heat7 in FP64 (float64 CUDA tensors [nz, ny, nx])."""
    nz, ny, nx = d_u.shape
    f64 = _dt("float64")
    _check(lib().ooc_heat7_steps_f64(_dev(d_u, f64, "d_u", ndim=3), _dev(d_tmp, f64, "d_tmp", numel=d_u.numel()), nx,
                                     ny, nz, float(r), int(nsteps), _stream(stream)), "ooc_heat7_steps_f64")
    return d_u


def ooc_heat7_steps_fused(d_u, d_tmp, nsteps, r=1.0 / 6.0, stream=None):
    """ooc_heat7_steps with each pair of steps in one launch (bit-identical)."""
    nz, ny, nx = d_u.shape
    _check(lib().ooc_heat7_steps_fused(_dev(d_u, _f32(), "d_u", ndim=3),
                                       _dev(d_tmp, _f32(), "d_tmp", numel=d_u.numel()), nx, ny, nz, float(r),
                                       int(nsteps), _stream(stream)), "ooc_heat7_steps_fused")
    return d_u


def ooc_heat7_steps_noalloc(d_u, nsteps, r=1.0 / 6.0, stream=None):
    """ooc_heat7_steps without a scratch field: the library's fixed scratch
    array (OOC_NOALLOC_MAX_POINTS points) holds the second field."""
    nz, ny, nx = d_u.shape
    _check(lib().ooc_heat7_steps_noalloc(_dev(d_u, _f32(), "d_u", ndim=3), nx, ny, nz, float(r), int(nsteps),
                                         _stream(stream)), "ooc_heat7_steps_noalloc")
    return d_u


OOC_NOALLOC_MAX_POINTS = 4 * 1024 * 1024


def ooc_wave25_steps(d_p, d_pprev, d_kappa, nsteps, src=None, w=None, t=0, stream=None):
    """Leapfrog in place on (d_p, d_pprev); ``src`` = (sx, sy, sz) and ``w`` a
    float32 numpy series indexed by absolute step."""
    nz, ny, nx = d_p.shape
    if src is None or w is None:
        sx, sy, sz, wp = -1, -1, -1, None
    else:
        sx, sy, sz = src
        w = np.ascontiguousarray(w, dtype=np.float32)
        if len(w) < t + nsteps:
            raise ValueError("source series shorter than t + nsteps")
        wp = w.ctypes.data_as(ctypes.c_void_p)
    n = d_p.numel()
    _check(lib().ooc_wave25_steps(_dev(d_p, _f32(), "d_p", ndim=3), _dev(d_pprev, _f32(), "d_pprev", numel=n),
                                  _dev(d_kappa, _f32(), "d_kappa", numel=n), nx, ny, nz, sx, sy, sz, wp, int(t),
                                  int(nsteps), _stream(stream)), "ooc_wave25_steps")
    return d_p, d_pprev


def ooc_wave25_steps_fused(d_p, d_pprev, d_kappa, nsteps, src=None, w=None, t=0, d_t1=None, d_t2=None,
                           stream=None):
    """ooc_wave25_steps with each pair of steps in one launch; d_t1, d_t2 are
    scratch fields (allocated if None)."""
    import torch
    nz, ny, nx = d_p.shape
    t1 = torch.empty_like(d_p) if d_t1 is None else d_t1
    t2 = torch.empty_like(d_p) if d_t2 is None else d_t2
    if src is None or w is None:
        sx, sy, sz, wp = -1, -1, -1, None
    else:
        sx, sy, sz = src
        w = np.ascontiguousarray(w, dtype=np.float32)
        if len(w) < t + nsteps:
            raise ValueError("source series shorter than t + nsteps")
        wp = w.ctypes.data_as(ctypes.c_void_p)
    n = d_p.numel()
    _check(lib().ooc_wave25_steps_fused(_dev(d_p, _f32(), "d_p", ndim=3), _dev(d_pprev, _f32(), "d_pprev", numel=n),
                                        _dev(d_kappa, _f32(), "d_kappa", numel=n), _dev(t1, _f32(), "d_t1", numel=n),
                                        _dev(t2, _f32(), "d_t2", numel=n), nx, ny, nz, sx, sy, sz, wp, int(t),
                                        int(nsteps), _stream(stream)), "ooc_wave25_steps_fused")
    return d_p, d_pprev


def ooc_wave25_steps_f64(d_p, d_pprev, d_kappa, nsteps, src=None, w=None, t=0, stream=None):
    """FP64 leapfrog in place on float64 CUDA tensors; ``w`` a float64 numpy
    series indexed by absolute step."""
    nz, ny, nx = d_p.shape
    if src is None or w is None:
        sx, sy, sz, wp = -1, -1, -1, None
    else:
        sx, sy, sz = src
        w = np.ascontiguousarray(w, dtype=np.float64)
        if len(w) < t + nsteps:
            raise ValueError("source series shorter than t + nsteps")
        wp = w.ctypes.data_as(ctypes.c_void_p)
    n, f64 = d_p.numel(), _dt("float64")
    _check(lib().ooc_wave25_steps_f64(_dev(d_p, f64, "d_p", ndim=3), _dev(d_pprev, f64, "d_pprev", numel=n),
                                      _dev(d_kappa, f64, "d_kappa", numel=n), nx, ny, nz, sx, sy, sz, wp, int(t),
                                      int(nsteps), _stream(stream)), "ooc_wave25_steps_f64")
    return d_p, d_pprev


def ooc_gather(d_field, d_idx, d_out=None, stream=None):
    import torch
    if d_out is None:
        d_out = torch.empty(d_idx.numel(), dtype=torch.float32, device=d_field.device)
    _check(lib().ooc_gather(_dev(d_field, _f32(), "d_field"), d_field.numel(), _dev(d_idx, _dt("int64"), "d_idx"),
                            d_idx.numel(), _dev(d_out, _f32(), "d_out", numel=d_idx.numel()), _stream(stream)),
           "ooc_gather")
    return d_out


def ooc_scatter_add(d_field, d_idx, d_val, stream=None):
    _check(lib().ooc_scatter_add(_dev(d_field, _f32(), "d_field"), d_field.numel(),
                                 _dev(d_idx, _dt("int64"), "d_idx"), d_idx.numel(),
                                 _dev(d_val, _f32(), "d_val", numel=d_idx.numel()), _stream(stream)),
           "ooc_scatter_add")
    return d_field


def ooc_wave25_adjoint_step(d_mu, d_mu_prev, d_kappa, d_out=None, stream=None):
    """d_out = 2 mu - mu_prev + L(kappa mu) (in place on d_mu_prev if d_out is None)."""
    nz, ny, nx = d_mu.shape
    if d_out is None:
        d_out = d_mu_prev
    n = d_mu.numel()
    _check(lib().ooc_wave25_adjoint_step(_dev(d_mu, _f32(), "d_mu", ndim=3), _dev(d_mu_prev, _f32(), "d_mu_prev", numel=n),
                                         _dev(d_out, _f32(), "d_out", numel=n), _dev(d_kappa, _f32(), "d_kappa", numel=n),
                                         nx, ny, nz, _stream(stream)), "ooc_wave25_adjoint_step")
    return d_out


def ooc_wave25_grad_accum(d_grad, d_mu, d_p, stream=None):
    nz, ny, nx = d_mu.shape
    n = d_mu.numel()
    _check(lib().ooc_wave25_grad_accum(_dev(d_grad, _dt("float64"), "d_grad", numel=n), _dev(d_mu, _f32(), "d_mu", ndim=3),
                                       _dev(d_p, _f32(), "d_p", numel=n), nx, ny, nz, _stream(stream)),
           "ooc_wave25_grad_accum")
    return d_grad


def ooc_kappa_from_velocity(d_v, dt_over_dx, d_kappa=None, stream=None):
    import torch
    if d_kappa is None:
        d_kappa = torch.empty_like(d_v)
    _check(lib().ooc_kappa_from_velocity(_dev(d_v, _f32(), "d_v"), _dev(d_kappa, _f32(), "d_kappa", numel=d_v.numel()),
                                         d_v.numel(), float(dt_over_dx), _stream(stream)), "ooc_kappa_from_velocity")
    return d_kappa


def ooc_velocity_grad(d_grad_kappa, d_v, dt_over_dx, d_grad_v=None, stream=None):
    import torch
    if d_grad_v is None:
        d_grad_v = torch.empty_like(d_v)
    n = d_v.numel()
    _check(lib().ooc_velocity_grad(_dev(d_grad_kappa, _dt("float64"), "d_grad_kappa", numel=n), _dev(d_v, _f32(), "d_v"),
                                   _dev(d_grad_v, _f32(), "d_grad_v", numel=n), n, float(dt_over_dx), _stream(stream)),
           "ooc_velocity_grad")
    return d_grad_v


def ooc_wave25_ckpt_bytes(shape, nsteps, every, rate):
    nz, ny, nx = shape
    return int(lib().ooc_wave25_ckpt_bytes(nx, ny, nz, nsteps, every, rate))


def ooc_wave25_adjoint_work_bytes(shape, every, rate):
    nz, ny, nx = shape
    return int(lib().ooc_wave25_adjoint_work_bytes(nx, ny, nz, every, rate))


def _src_args(src, w, nsteps):
    if src is None or w is None:
        return -1, -1, -1, None, None
    w = np.ascontiguousarray(w, dtype=np.float32)
    if w.size < nsteps:
        raise ValueError("source series shorter than nsteps")
    return src[0], src[1], src[2], w, w.ctypes.data_as(ctypes.c_void_p)


def ooc_wave25_forward_ckpt(d_kappa, nsteps, d_rec, d_traces, every, rate, h_ckpt, d_work, streams, src=None, w=None):
    nz, ny, nx = d_kappa.shape
    sx, sy, sz, w_keep, wp = _src_args(src, w, nsteps)
    arr = (ctypes.c_void_p * 2)(*[s.cuda_stream for s in streams])
    nrec = d_rec.numel()
    _check(lib().ooc_wave25_forward_ckpt(_dev(d_kappa, _f32(), "d_kappa", ndim=3), nx, ny, nz, sx, sy, sz, wp,
                                         int(nsteps), _dev(d_rec, _dt("int64"), "d_rec"), nrec,
                                         _dev(d_traces, _f32(), "d_traces", numel=int(nsteps) * nrec), int(every),
                                         int(rate), _host(h_ckpt, "h_ckpt"), h_ckpt.numel(),
                                         _dev(d_work, _dt("uint8"), "d_work"), d_work.numel(), arr),
           "ooc_wave25_forward_ckpt")
    return d_traces


def ooc_wave25_backward_ckpt(d_kappa, nsteps, d_rec, d_res, every, rate, h_ckpt, d_grad, d_work, streams, src=None,
                             w=None):
    nz, ny, nx = d_kappa.shape
    sx, sy, sz, w_keep, wp = _src_args(src, w, nsteps)
    arr = (ctypes.c_void_p * 2)(*[s.cuda_stream for s in streams])
    nrec = d_rec.numel()
    _check(lib().ooc_wave25_backward_ckpt(_dev(d_kappa, _f32(), "d_kappa", ndim=3), nx, ny, nz, sx, sy, sz, wp,
                                          int(nsteps), _dev(d_rec, _dt("int64"), "d_rec"), nrec,
                                          _dev(d_res, _f32(), "d_res", numel=int(nsteps) * nrec), int(every), int(rate),
                                          _host(h_ckpt, "h_ckpt"), h_ckpt.numel(),
                                          _dev(d_grad, _dt("float64"), "d_grad", numel=d_kappa.numel()),
                                          _dev(d_work, _dt("uint8"), "d_work"), d_work.numel(), arr),
           "ooc_wave25_backward_ckpt")
    return d_grad


def _fmt(v):
    return FORMATS[v] if isinstance(v, str) else int(v)


class Plan:
    """An out-of-core run bound to torch-allocated arenas and three torch
    streams (H2D, compute, D2H).  Configuration keys mirror ``ooc_config``:
    nx, ny, nz, stencil ('heat7'|'wave25'), k, r, rw_format, rw_rate,
    ro_format, ro_rate, device_budget_bytes, slab_planes, profile,
    wait_timeout_ms, heat_steps_per_launch, graph_mode, debug_checks,
    precision ('fp32'|'fp64'; FP64 plans store 'fp64' or 'fr4' fields and
    exchange float64 arrays)."""

    def __init__(self, device=0, **kw):
        import torch
        c = OocConfig()
        c.nx, c.ny, c.nz = kw["nx"], kw["ny"], kw["nz"]
        st = kw.get("stencil", "heat7")
        c.stencil = STENCILS[st] if isinstance(st, str) else int(st)
        c.k = kw.get("k", 1)
        c.r = kw.get("r", 1.0 / 6.0)
        c.rw_format = _fmt(kw.get("rw_format", "fp32"))
        c.rw_rate = kw.get("rw_rate", 16)
        c.ro_format = _fmt(kw.get("ro_format", "fp32"))
        c.ro_rate = kw.get("ro_rate", 16)
        c.device_budget_bytes = kw.get("device_budget_bytes", 0)
        c.slab_planes = kw.get("slab_planes", 0)
        c.profile = int(kw.get("profile", 0))
        c.wait_timeout_ms = kw.get("wait_timeout_ms", 0)
        c.heat_steps_per_launch = int(kw.get("heat_steps_per_launch", 0))
        c.graph_mode = int(kw.get("graph_mode", 0))
        c.debug_checks = int(kw.get("debug_checks", 0))
        prec = kw.get("precision", "fp32")
        c.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.dtype = np.float64 if c.precision == OOC_PREC_FP64 else np.float32
        self.config = c
        self.shape = (c.nz, c.ny, c.nx)
        self._h = ctypes.c_void_p()
        dev_b, host_b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().ooc_plan_create(ctypes.byref(c), ctypes.byref(self._h), ctypes.byref(dev_b),
                                     ctypes.byref(host_b)), "ooc_plan_create")
        self.device_bytes, self.host_bytes = dev_b.value, host_b.value
        self.device = torch.device("cuda", device)
        self.dev_arena = torch.empty(max(self.device_bytes, 256), dtype=torch.uint8, device=self.device)
        self.host_arena = torch.empty(max(self.host_bytes, 256), dtype=torch.uint8, pin_memory=True)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(3)]
        arr = (ctypes.c_void_p * 3)(*[s.cuda_stream for s in self.streams])
        _check(lib().ooc_plan_bind(self._h, _ptr(self.dev_arena), self.dev_arena.numel(), _ptr(self.host_arena),
                                   self.host_arena.numel(), arr), "ooc_plan_bind")

    def rebind(self):
        """Bind the plan again to its own arenas and streams (ooc_plan_bind):
        copies the plan's time to the device and drops any captured graph."""
        arr = (ctypes.c_void_p * 3)(*[s.cuda_stream for s in self.streams])
        _check(lib().ooc_plan_bind(self._h, _ptr(self.dev_arena), self.dev_arena.numel(), _ptr(self.host_arena),
                                   self.host_arena.numel(), arr), "ooc_plan_bind")

    def info(self):
        i = OocPlanInfo()
        _check(lib().ooc_plan_get_info(self._h, ctypes.byref(i)), "ooc_plan_get_info")
        return i.as_dict()

    def set_field(self, field, host_src):
        a = np.ascontiguousarray(host_src, dtype=self.dtype)
        if a.shape != self.shape:
            raise ValueError(f"field shape {a.shape} != {self.shape}")
        fn = "ooc_set_field64" if self.dtype == np.float64 else "ooc_set_field"
        _check(getattr(lib(), fn)(self._h, int(field), a.ctypes.data_as(ctypes.c_void_p)), fn)

    def get_field(self, field, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        if out.dtype != self.dtype or out.shape != self.shape or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous array of the plan's shape and precision")
        fn = "ooc_get_field64" if self.dtype == np.float64 else "ooc_get_field"
        _check(getattr(lib(), fn)(self._h, int(field), out.ctypes.data_as(ctypes.c_void_p)), fn)
        return out

    def set_source(self, sx, sy, sz, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib().ooc_set_source(self._h, sx, sy, sz, w.ctypes.data_as(ctypes.c_void_p), w.size),
               "ooc_set_source")

    def step(self, nsteps):
        _check(lib().ooc_step(self._h, int(nsteps)), "ooc_step")

    def set_wait_timeout(self, ms):
        _check(lib().ooc_plan_set_wait_timeout(self._h, int(ms)), "ooc_plan_set_wait_timeout")

    def set_profile(self, on):
        _check(lib().ooc_plan_set_profile(self._h, 1 if on else 0), "ooc_plan_set_profile")

    def stats(self):
        s = OocStats()
        _check(lib().ooc_get_stats(self._h, ctypes.byref(s)), "ooc_get_stats")
        return s.as_dict()

    def trace(self):
        """Intervals of the last ooc_step made with profiling on: a list of
        dicts (kind, count, pass, slab, start_ms, end_ms)."""
        n = ctypes.c_int64()
        _check(lib().ooc_plan_get_trace(self._h, None, 0, ctypes.byref(n)), "ooc_plan_get_trace")
        recs = (OocTraceRec * max(n.value, 1))()
        _check(lib().ooc_plan_get_trace(self._h, recs, n.value, ctypes.byref(n)), "ooc_plan_get_trace")
        return [{"kind": TRACE_KINDS[r.kind], "count": r.count, "pass": r.pass_, "slab": r.slab,
                 "start_ms": r.start_ms, "end_ms": r.end_ms} for r in recs[:n.value]]

    def reset_stats(self):
        _check(lib().ooc_reset_stats(self._h), "ooc_reset_stats")

    def close(self):
        if self._h:
            lib().ooc_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from .autograd import WaveFn, wave_forward  # noqa: E402
