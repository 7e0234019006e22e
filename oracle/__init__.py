"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations of everything the GPU
path computes: the FR4 fixed-rate block codec and its FP64 form FR4D
(serial definitions, C), the
FP64 heat7 and wave25 stencils (C, OpenMP over z), BF16 storage rounding
(numpy bit manipulation) and the storage round trips that the out-of-core
pipeline applies at pass boundaries.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg and reference arm (``--impl reference``) may import this package.  It
shares no code with the CUDA library in ``paper_2109_05410_gb300/csrc`` and
never imports the product package.

The C sources are compiled with gcc into ``oracle/_build/liboracle.so`` on
first use (or by :func:`build`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["codec.c", "codec64.c", "stencil.c", "adjoint.c", "util.c"]
_lock = threading.Lock()
_lib = None

FORMATS = ("fp32", "bf16", "fr4")


def build(force=False):
    """Compile the oracle's C sources into a shared library (gcc, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            i64, i32, vp, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
            sigs = {
                "fr4_compressed_bytes": (i64, [i64, i64, i64, i32]),
                "fr4_encode": (i32, [vp, i64, i64, i64, i32, vp]),
                "fr4_decode": (i32, [vp, i64, i64, i64, i32, vp]),
                "fr4_lift_forward4": (None, [vp]),
                "fr4_lift_inverse4": (None, [vp]),
                "fr4_transform_forward": (i32, [vp]),
                "fr4_transform_inverse": (i32, [vp]),
                "fr4_order": (None, [vp]),
                "fr4_encode_planes": (i64, [vp, i64, vp]),
                "fr4_encode_var": (i64, [vp, i64, i64, i64, i32, dbl, vp, i64, vp]),
                "fr4_decode_var": (i32, [vp, vp, i64, i64, i64, i32, dbl, vp]),
                "fr4_var_max_words_per_block": (i64, []),
                "fr4_decode_planes": (i64, [vp, i64, vp]),
                "fr4d_encode": (i32, [vp, i64, i64, i64, i32, vp]),
                "fr4d_decode": (i32, [vp, i64, i64, i64, i32, vp]),
                "fr4d_transform_forward": (i32, [vp]),
                "fr4d_transform_inverse": (i32, [vp]),
                "fr4d_encode_planes": (i64, [vp, i64, vp]),
                "fr4d_decode_planes": (i64, [vp, i64, vp]),
                "oracle_heat7_step": (None, [vp, vp, i64, i64, i64, dbl]),
                "oracle_heat7_run": (None, [vp, vp, i64, i64, i64, dbl, i64]),
                "oracle_heat7_run_f32": (None, [vp, vp, i64, i64, i64, ctypes.c_float, i64]),
                "oracle_laplacian8": (None, [vp, vp, i64, i64, i64]),
                "oracle_wave25_step": (None, [vp, vp, vp, vp, i64, i64, i64, i64, dbl]),
                "oracle_wave25_run": (None, [vp, vp, vp, vp, i64, i64, i64, i64, vp, i64, i64]),
                "oracle_threads": (i32, []),
                "oracle_wave25_traces": (i32, [vp, i64, i64, i64, i64, vp, i64, vp, i64, vp]),
                "oracle_wave25_adjoint_grad": (i32, [vp, i64, i64, i64, i64, vp, i64, vp, i64, vp, vp]),
                "oracle_wave25_born": (i32, [vp, vp, i64, i64, i64, i64, vp, i64, vp, i64, vp]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads():
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().oracle_threads())


# --------------------------------------------------------------------------- codec
def compressed_bytes(shape, rate):
    nz, ny, nx = shape
    return int(lib().fr4_compressed_bytes(nx, ny, nz, rate))


def _nblocks(shape):
    nz, ny, nx = shape
    return ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 3) // 4)


def fr4_encode(field, rate):
    """Encode a float32 [nz, ny, nx] field at ``rate`` bits per value;
    returns uint32 words (2*rate per 4^3 block; partial blocks at the far
    faces are padded with the nearest value inside the field)."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    out = np.zeros(_nblocks(f.shape) * 2 * rate, dtype=np.uint32)
    rc = lib().fr4_encode(_p(f), nx, ny, nz, rate, _p(out))
    if rc != 0:
        raise RuntimeError(f"fr4_encode failed ({rc})")
    return out


def fr4_decode(words, shape, rate):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    nz, ny, nx = shape
    if w.size != _nblocks(shape) * 2 * rate:
        raise ValueError("stream size does not match shape and rate")
    out = np.empty(shape, dtype=np.float32)
    rc = lib().fr4_decode(_p(w), nx, ny, nz, rate, _p(out))
    if rc < 0:
        raise RuntimeError(f"fr4_decode failed ({rc})")
    return out


MODE_PRECISION = 1
MODE_ACCURACY = 2


def fr4_encode_var(field, mode, param):
    """Variable-size modes (fixed precision: ``param`` planes; fixed
    accuracy: ``param`` = tolerance).  Returns (words, index) with block b in
    words[index[b]:index[b+1]]."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    nb = _nblocks(f.shape)
    cap = nb * int(lib().fr4_var_max_words_per_block())
    out = np.zeros(cap, dtype=np.uint32)
    index = np.zeros(nb + 1, dtype=np.uint64)
    n = lib().fr4_encode_var(_p(f), nx, ny, nz, mode, float(param), _p(out), cap, _p(index))
    if n < 0:
        raise RuntimeError("fr4_encode_var failed")
    return out[:n].copy(), index


def fr4_decode_var(words, index, shape, mode, param):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    idx = np.ascontiguousarray(index, dtype=np.uint64)
    nz, ny, nx = shape
    if idx.size != _nblocks(shape) + 1 or int(idx[-1]) > w.size:
        raise ValueError("index does not match shape or stream")
    out = np.empty(shape, dtype=np.float32)
    if lib().fr4_decode_var(_p(w), _p(idx), nx, ny, nz, mode, float(param), _p(out)) != 0:
        raise RuntimeError("fr4_decode_var failed")
    return out


def fr4_roundtrip(field, rate):
    f = np.ascontiguousarray(field, dtype=np.float32)
    return fr4_decode(fr4_encode(f, rate), f.shape, rate)


def lift_forward4(a):
    v = np.ascontiguousarray(a, dtype=np.int32).copy()
    lib().fr4_lift_forward4(_p(v))
    return v


def lift_inverse4(a):
    v = np.ascontiguousarray(a, dtype=np.int32).copy()
    lib().fr4_lift_inverse4(_p(v))
    return v


def transform_forward(block):
    """3D forward lifting of one block (64 int32, index x + 4y + 16z).
    Returns (coefficients, wrapped)."""
    v = np.ascontiguousarray(block, dtype=np.int32).reshape(64).copy()
    rc = lib().fr4_transform_forward(_p(v))
    return v, rc != 0


def transform_inverse(coef):
    v = np.ascontiguousarray(coef, dtype=np.int32).reshape(64).copy()
    rc = lib().fr4_transform_inverse(_p(v))
    return v, rc != 0


def sequency_order():
    v = np.zeros(64, dtype=np.int32)
    lib().fr4_order(_p(v))
    return v


def encode_planes(u, budget_bits):
    """Run only the bit-plane coder on 64 negabinary words; returns
    (words, bits_written)."""
    uu = np.ascontiguousarray(u, dtype=np.uint32)
    words = np.zeros((budget_bits + 31) // 32 + 1, dtype=np.uint32)
    n = lib().fr4_encode_planes(_p(uu), budget_bits, _p(words))
    return words, int(n)


def decode_planes(words, budget_bits):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    u = np.zeros(64, dtype=np.uint32)
    n = lib().fr4_decode_planes(_p(w), budget_bits, _p(u))
    return u, int(n)


# --------------------------------------------------------------------------- FP64 codec
def fr4d_encode(field, rate):
    """Encode a float64 [nz, ny, nx] field with FR4D at ``rate`` bits per
    value (2*rate uint32 words per 4^3 block).  Rates above 64 are for the
    full-precision checks only."""
    f = np.ascontiguousarray(field, dtype=np.float64)
    nz, ny, nx = f.shape
    out = np.zeros(_nblocks(f.shape) * 2 * rate, dtype=np.uint32)
    rc = lib().fr4d_encode(_p(f), nx, ny, nz, rate, _p(out))
    if rc != 0:
        raise RuntimeError(f"fr4d_encode failed ({rc})")
    return out


def fr4d_decode(words, shape, rate):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    nz, ny, nx = shape
    if w.size != _nblocks(shape) * 2 * rate:
        raise ValueError("stream size does not match shape and rate")
    out = np.empty(shape, dtype=np.float64)
    rc = lib().fr4d_decode(_p(w), nx, ny, nz, rate, _p(out))
    if rc < 0:
        raise RuntimeError(f"fr4d_decode failed ({rc})")
    return out


def fr4d_roundtrip(field, rate):
    f = np.ascontiguousarray(field, dtype=np.float64)
    return fr4d_decode(fr4d_encode(f, rate), f.shape, rate)


def fr4d_transform_forward(block):
    """FR4D's 3D forward lifting of one block (64 int64); returns
    (coefficients, wrapped)."""
    v = np.ascontiguousarray(block, dtype=np.int64).reshape(64).copy()
    rc = lib().fr4d_transform_forward(_p(v))
    return v, rc != 0


def fr4d_transform_inverse(coef):
    v = np.ascontiguousarray(coef, dtype=np.int64).reshape(64).copy()
    rc = lib().fr4d_transform_inverse(_p(v))
    return v, rc != 0


def fr4d_encode_planes(u, budget_bits):
    """Only FR4D's 64-plane coder on 64 negabinary uint64 words; returns
    (words, bits_written)."""
    uu = np.ascontiguousarray(u, dtype=np.uint64)
    words = np.zeros((budget_bits + 31) // 32 + 1, dtype=np.uint32)
    n = lib().fr4d_encode_planes(_p(uu), budget_bits, _p(words))
    return words, int(n)


def fr4d_decode_planes(words, budget_bits):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    u = np.zeros(64, dtype=np.uint64)
    n = lib().fr4d_decode_planes(_p(w), budget_bits, _p(u))
    return u, int(n)


# --------------------------------------------------------------------------- bf16
def bf16_bits(x):
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even,
    NaN kept quiet."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = (u & 0x7FFFFFFF) > 0x7F800000
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    quiet = (u >> 16) | 0x40
    return np.where(nan, quiet, rounded).astype(np.uint16)


def bf16_to_f32(b):
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def bf16_roundtrip(x):
    return bf16_to_f32(bf16_bits(x)).reshape(np.shape(x))


def storage_roundtrip(field, fmt, rate=16, precision="fp32"):
    """What a field looks like after being stored in ``fmt``.  FP32 plans:
    cast to float32 and, for bf16/fr4, rounded/encoded and decoded.  FP64
    plans (precision='fp64'): 'fp64' keeps the value, 'fr4' is the FR4D
    round trip.  Returns float64."""
    if precision == "fp64":
        d = np.array(field, dtype=np.float64)
        if fmt == "fp64":
            return d
        if fmt == "fr4":
            return fr4d_roundtrip(d, rate)
        raise ValueError(fmt)
    f = np.ascontiguousarray(field, dtype=np.float32)
    if fmt == "fp32":
        g = f
    elif fmt == "bf16":
        g = bf16_roundtrip(f)
    elif fmt == "fr4":
        g = fr4_roundtrip(f, rate)
    else:
        raise ValueError(fmt)
    return g.astype(np.float64)


# --------------------------------------------------------------------------- stencils
def heat7_step(u, r=1.0 / 6.0):
    a = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(a)
    nz, ny, nx = a.shape
    lib().oracle_heat7_step(_p(a), _p(out), nx, ny, nz, r)
    return out


def heat7_run(u, nsteps, r=1.0 / 6.0):
    a = np.array(u, dtype=np.float64, order="C", copy=True)
    tmp = np.empty_like(a)
    nz, ny, nx = a.shape
    lib().oracle_heat7_run(_p(a), _p(tmp), nx, ny, nz, r, nsteps)
    return a


def heat7_run_f32(u, nsteps, r=1.0 / 6.0):
    """The heat steps in FP32 arithmetic (not a reference: the CPU doing the
    GPU's FP32 work, timed beside the FP64 oracle)."""
    a = np.array(u, dtype=np.float32, order="C", copy=True)
    tmp = np.empty_like(a)
    nz, ny, nx = a.shape
    lib().oracle_heat7_run_f32(_p(a), _p(tmp), nx, ny, nz, r, nsteps)
    return a


def laplacian8(p):
    a = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(a)
    nz, ny, nx = a.shape
    lib().oracle_laplacian8(_p(a), _p(out), nx, ny, nz)
    return out


def wave25_step(p, p_prev, kappa, src=-1, w=0.0):
    a = np.ascontiguousarray(p, dtype=np.float64)
    b = np.ascontiguousarray(p_prev, dtype=np.float64)
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    out = np.empty_like(a)
    nz, ny, nx = a.shape
    lib().oracle_wave25_step(_p(a), _p(b), _p(k), _p(out), nx, ny, nz, int(src), float(w))
    return out


def wave25_run(p, p_prev, kappa, nsteps, src=-1, w=None, t0=0):
    """Leapfrog ``nsteps`` steps from (p^t, p^{t-1}); returns
    (p^{t+nsteps}, p^{t+nsteps-1}).  Step j adds w[t0 + j] at flat index src."""
    a = np.array(p, dtype=np.float64, order="C", copy=True)
    b = np.array(p_prev, dtype=np.float64, order="C", copy=True)
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    tmp = np.empty_like(a)
    nz, ny, nx = a.shape
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    lib().oracle_wave25_run(_p(a), _p(b), _p(k), _p(tmp), nx, ny, nz, int(src),
                            None if ww is None else _p(ww), int(t0), int(nsteps))
    return a, b


# --------------------------------------------------------------------------- adjoint
def _rec(rec):
    return np.ascontiguousarray(rec, dtype=np.int64)


def wave25_traces(kappa, src, w, nsteps, rec):
    """FP64 forward from rest; returns traces [nsteps, nrec] (p^1..p^N at
    the flat receiver indices ``rec``)."""
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    nz, ny, nx = k.shape
    r = _rec(rec)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((nsteps, r.size), dtype=np.float64)
    if lib().oracle_wave25_traces(_p(k), nx, ny, nz, int(src), _p(ww), int(nsteps), _p(r), r.size, _p(out)) != 0:
        raise MemoryError("oracle_wave25_traces")
    return out


def wave25_adjoint_grad(kappa, src, w, nsteps, rec, res):
    """dJ/dkappa for dJ/dtraces = ``res`` [nsteps, nrec] (FP64 discrete
    adjoint)."""
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    nz, ny, nx = k.shape
    r = _rec(rec)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    rr = np.ascontiguousarray(res, dtype=np.float64)
    g = np.zeros_like(k)
    if lib().oracle_wave25_adjoint_grad(_p(k), nx, ny, nz, int(src), _p(ww), int(nsteps), _p(r), r.size, _p(rr),
                                        _p(g)) != 0:
        raise MemoryError("oracle_wave25_adjoint_grad")
    return g


def wave25_born(kappa, dkappa, src, w, nsteps, rec):
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    dk = np.ascontiguousarray(dkappa, dtype=np.float64)
    nz, ny, nx = k.shape
    r = _rec(rec)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((nsteps, r.size), dtype=np.float64)
    if lib().oracle_wave25_born(_p(k), _p(dk), nx, ny, nz, int(src), _p(ww), int(nsteps), _p(r), r.size,
                                _p(out)) != 0:
        raise MemoryError("oracle_wave25_born")
    return out


def misfit(traces, d):
    r = np.asarray(traces, dtype=np.float64) - np.asarray(d, dtype=np.float64)
    return 0.5 * float(np.sum(r * r))


# --------------------------------------------------------------------------- pipelines
def heat7_storage_pipeline(u0, nsteps, k, fmt, rate=16, r=1.0 / 6.0, precision="fp32"):
    """FP64 heat7 with the storage round trip the out-of-core pipeline
    applies: once at load, then after every pass of ``k`` steps (the last
    pass may be shorter).  With fmt='fp32' this is FP64 compute on the
    FP32-rounded state at pass boundaries; precision='fp64' stores in the
    FP64 plan's formats ('fp64', or 'fr4' = FR4D)."""
    u = storage_roundtrip(u0, fmt, rate, precision)
    done = 0
    while done < nsteps:
        s = min(k, nsteps - done)
        u = heat7_run(u, s, r)
        u = storage_roundtrip(u, fmt, rate, precision)
        done += s
    return u


def wave25_storage_pipeline(p0, pm1, kappa, nsteps, k, fmt, rate=16, ro_fmt=None, ro_rate=None,
                            src=-1, w=None, precision="fp32"):
    """FP64 leapfrog with storage round trips of both time levels at load
    and after every pass of ``k`` steps; kappa (read-only) is stored once in
    ``ro_fmt`` (default: the plan's uncompressed format)."""
    raw = "fp64" if precision == "fp64" else "fp32"
    kap = storage_roundtrip(kappa, ro_fmt or raw, ro_rate or rate, precision)
    p = storage_roundtrip(p0, fmt, rate, precision)
    q = storage_roundtrip(pm1, fmt, rate, precision)
    done = 0
    while done < nsteps:
        s = min(k, nsteps - done)
        p, q = wave25_run(p, q, kap, s, src=src, w=w, t0=done)
        p = storage_roundtrip(p, fmt, rate, precision)
        q = storage_roundtrip(q, fmt, rate, precision)
        done += s
    return p, q


# --------------------------------------------------------------------------- metrics
def error_metrics(a, ref, nsample_per_plane=100, seed=0, floor_frac=1e-3):
    """rel-L2, max-abs and the paper-style mean pointwise relative error
    (Section VI-C: 100 sampled points per plane).  Samples with
    |ref| < floor_frac * max|ref| are excluded from the relative mean and
    counted."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    diff = a - ref
    nref = np.linalg.norm(ref.ravel())
    rel_l2 = float(np.linalg.norm(diff.ravel()) / nref) if nref > 0 else float(np.linalg.norm(diff.ravel()))
    max_abs = float(np.max(np.abs(diff))) if diff.size else 0.0
    nz, ny, nx = ref.shape
    rng = np.random.default_rng(seed)
    ys = rng.integers(0, ny, size=(nz, nsample_per_plane))
    xs = rng.integers(0, nx, size=(nz, nsample_per_plane))
    zs = np.repeat(np.arange(nz)[:, None], nsample_per_plane, axis=1)
    r = ref[zs, ys, xs].ravel()
    v = a[zs, ys, xs].ravel()
    floor = floor_frac * float(np.max(np.abs(ref))) if ref.size else 0.0
    keep = np.abs(r) >= floor
    mean_rel = float(np.mean(np.abs(v[keep] - r[keep]) / np.abs(r[keep]))) if keep.any() else 0.0
    return {"rel_l2": rel_l2, "max_abs": max_abs, "mean_rel_sampled": mean_rel,
            "samples": int(r.size), "excluded": int((~keep).sum())}
