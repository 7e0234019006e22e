"""Throughput of the out-of-core stencil pipeline with on-the-fly compression.

Workload (default): 3D 7-point heat equation, FP32 compute, 1024^3 grid held
in pinned host memory, device budget 1 GiB (the plan streams z-slabs),
temporal blocking k = 4, 64 time steps per bench step, slabs stored and
transferred as FR4 at 16 bits/value; the same run with uncompressed FP32
slabs (and BF16, FR4 at 8/12/24) is measured on the same GPU for the
compressed-vs-uncompressed comparison.  Error is stated against the FP64
oracle on a sampled central 128^3 sub-box (exact dependency cone).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload heat1024|kernels512|window56|wave1024|wave1024_error|precision|precision192|
                   adjoint512|fp64|window56_fp64]

Prints one JSON line (rank 0).  The default workload is the headline; the
others measure the remaining configurations: one launch of each kernel on a
512^3 field (kernels512), the headline's kernels on one 56-plane 1024^2
window (window56, the ncu capture case of the headline), the 1024^3 wave with
the paper's four storage codes (wave1024) and its accuracy over 2000 steps
against an FP64 run (wave1024_error), the long-horizon precision study over
4320 steps against an FP64 run (precision at 384^3, precision192), the
checkpointed adjoint at 512^3 (adjoint512) and FP64 fields (fp64,
window56_fp64).  The FP64 runs these errors are taken against use the
library's FP64 wave kernel, which the GPU tests hold to the FP64 oracle; the
CPU oracle itself runs only in the reference arm and the cpu_baseline leg.
N > 1 runs N independent replicas (the method works on one GPU; there is no
data-path collective).
"""
from __future__ import annotations

import argparse
import bisect
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1024
NSTEPS = 64
K = 4
BUDGET = 1 << 30
# heat7 steps per stencil launch: 2 = the k steps run as fused pairs with the
# intermediate level on chip (the library's default for k >= 2), 1 = one step
# per launch
SPL = int(os.environ.get("OOC_BENCH_HEAT_STEPS_PER_LAUNCH", "2"))
MAIN = ("fr4", 16)
COMPARE = [("fp32", 0), ("bf16", 0), ("fr4", 8), ("fr4", 12), ("fr4", 24)]
# ncu counters of the headline's three kernels, per launch, on one 56-plane
# window of 1024^2 planes (58,720,256 points or values; FR4 at 16 bits per
# value): `python bench.py --workload window56 --steps 1 --warmup 0` under
# `ncu --set full --clock-control none -k regex:"heat7x2t|fr4_encode_kernel|
# fr4_decode_kernel" -c 4`.  DRAM bytes (read + write) and executed warp
# instructions scale with the points a launch processes, so the bench scales
# them to its own launches.  They hold only for the kernel source they were
# taken on: `sha` is the hash of that .cu file without comments and blank
# lines, and a changed file gives null.
NCU_UNITS = 56 * 1024 * 1024
NCU_COUNTERS = {
    "heat7_stencil": {"src": ["heat_tma.cu", "tma.cuh", "stencil_common.cuh", "f32x2.cuh"], "sha": "0d363f8834289584",
                      "dram_bytes": 428.6e6, "warp_inst": 83.74e6},
    "fr4_encode": {"src": "codec.cu", "sha": "3d031d5fc8adc782", "dram_bytes": 320.7e6, "warp_inst": 180.37e6},
    "fr4_decode": {"src": "codec.cu", "sha": "3d031d5fc8adc782", "dram_bytes": 296.2e6, "warp_inst": 180.98e6},
}
# issue peak: 152 SMs x 4 schedulers x one warp instruction per clock at the
# maximum SM clock of 2070 MHz
ISSUE_PEAK_WARP_INST = 152 * 4 * 2070e6
METRIC = "Gpts/s out-of-core (compressed vs uncompressed, same GB300) at stated L2 error; % roofline"
WORKLOAD = "heat7 1024^3 FP32, device budget 1 GiB, k=4, 64 steps/bench step"


def fmt_name(fmt, rate):
    return f"fr4-{rate}" if fmt == "fr4" else fmt


def source_sha(names):
    """sha256 prefix of the csrc/ files `names` (one name or a list), with
    comments and blank lines removed."""
    import hashlib
    import re
    text = ""
    for name in [names] if isinstance(names, str) else names:
        with open(os.path.join(ROOT, "paper_2109_05410_gb300", "csrc", name)) as f:
            text += f.read() + "\n"
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    code = [" ".join(re.sub(r"//.*$", "", line).split()) for line in text.split("\n")]
    return hashlib.sha256("\n".join(l for l in code if l).encode()).hexdigest()[:16]


def ncu_counters(kernel):
    """The window56 ncu counters of `kernel`, or None when its source has
    changed since they were taken."""
    c = NCU_COUNTERS.get(kernel)
    if c is None or source_sha(c["src"]) != c["sha"]:
        return None
    return c


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle legs
def oracle_sample(nsample=128, steps=8):
    """The oracle's version of one bench step on a bounded sample: FP64 heat7
    with the FR4-16 storage round trip after every pass of k = 4 steps."""
    import oracle
    from synth import smooth_random_field
    u0 = smooth_random_field((nsample,) * 3, 32.0, seed=2)
    t = time.perf_counter()
    oracle.heat7_storage_pipeline(u0, steps, K, "fr4", 16)
    dt = time.perf_counter() - t
    return nsample ** 3 * steps / dt / 1e9, dt, oracle.threads()


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    ns, steps = 128, 8
    for _ in range(args.warmup):
        oracle_sample(ns, steps)
    vals, total = [], 0.0
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(ns, steps)
        vals.append(v)
        total += dt
    value = ns ** 3 * steps * args.steps / total / 1e9
    sample = f"{ns}^3 smooth field, {steps} steps (2 passes of k=4), FP64 heat7 + FR4-16 round trips, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "oracle_sample": sample},
            "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def make_plan(ooc, fmt, rate, profile=0):
    return ooc.Plan(nx=N, ny=N, nz=N, stencil="heat7", k=K, rw_format=fmt, rw_rate=rate or 16,
                    device_budget_bytes=BUDGET, profile=profile, heat_steps_per_launch=SPL)


def timed_steps(torch, plan, nsteps, reps):
    """reps calls of ooc_step(nsteps), each bracketed by CUDA events on the
    plan's H2D (first work) and D2H (last work) streams; returns ms list."""
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(plan.streams[0])
        plan.step(nsteps)
        e1.record(plan.streams[2])
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


SUB = slice(N // 2 - 64, N // 2 + 64)  # central 128^3 sub-box for the stated error


def overlap_summary(tr):
    """Per-operation breakdown of one profiled ooc_step call (Section VI-B,
    Fig. 7) from its trace: the busy time of each stream, the overlap
    efficiency (busiest stream / wall time of the call), and the compute
    stream's idle time split by what it waited for: the H2D of the slab it
    decodes next, or the D2H that frees the staging buffer it encodes into."""
    if not tr:
        return None
    t0 = min(r["start_ms"] for r in tr)
    wall = max(r["end_ms"] for r in tr) - t0
    busy = {"h2d": 0.0, "d2h": 0.0, "compute": 0.0}
    for r in tr:
        busy["compute" if r["kind"] in ("decode", "stencil", "encode") else r["kind"]] += r["end_ms"] - r["start_ms"]
    h2d_ends = sorted(r["end_ms"] for r in tr if r["kind"] == "h2d")
    d2h_ends = sorted(r["end_ms"] for r in tr if r["kind"] == "d2h")

    def near(ends, t, tol=0.02):
        i = bisect.bisect_left(ends, t - tol)
        return i < len(ends) and ends[i] <= t + tol

    idle = {"waiting_h2d": 0.0, "waiting_d2h": 0.0, "other": 0.0}
    prev = t0
    for r in (r for r in tr if r["kind"] in ("decode", "stencil", "encode")):
        gap = r["start_ms"] - prev
        if gap > 0:
            if r["kind"] == "decode" and near(h2d_ends, r["start_ms"]):
                idle["waiting_h2d"] += gap
            elif r["kind"] == "encode" and near(d2h_ends, r["start_ms"]):
                idle["waiting_d2h"] += gap
            else:
                idle["other"] += gap
        prev = r["end_ms"]
    return {"call_ms": wall, "busy_ms": busy, "efficiency": max(busy.values()) / wall if wall > 0 else None,
            "compute_idle_ms": idle,
            "source": "ooc_plan_get_trace of the last profiled ooc_step call (one bench step, with CUDA events)"}


def sub_box(field):
    return np.array(field[SUB, SUB, SUB], dtype=np.float64)


def cpu_oracle_leg(u0):
    """The only part of the bench that runs the CPU oracle (rank 0, N = 1):
    the FP64 reference of the central sub-box after 64 steps (its dependency
    cone fits in a 256^3 window) and the timed oracle sample."""
    import oracle
    oracle.build()
    s = NSTEPS
    lo, hi = N // 2 - 64 - s, N // 2 + 64 + s
    exact = oracle.heat7_run(u0[lo:hi, lo:hi, lo:hi].astype(np.float64), s)[s:-s, s:-s, s:-s]
    v, dt, cores = oracle_sample(384, 8)
    cpu = {"value": v, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
           "sample": f"384^3 smooth field, 8 steps (2 passes of k=4), FP64 heat7 + FR4-16 round trips, {dt:.1f} s"}
    # the same steps in FP32 on the host cores (the GPU's arithmetic, no
    # storage round trips): a CPU throughput for the FP32 work itself
    from synth import smooth_random_field
    u32 = smooth_random_field((384,) * 3, 32.0, seed=2)
    t = time.perf_counter()
    oracle.heat7_run_f32(u32, 8)
    dt32 = time.perf_counter() - t
    cpu["fp32_variant"] = {"value": 384 ** 3 * 8 / dt32 / 1e9, "unit": "Gpts/s", "cores": cores,
                           "sample": f"384^3 smooth field, 8 FP32 heat7 steps in place, {dt32:.2f} s"}
    return exact, cpu


def wave1024_summary(torch, ooc, nsteps=100, reps=2):
    """The paper's workload in brief, for the default line: the 1024^3 wave
    (4 GiB budget, k = 10, source at the centre, from rest) with FP32 storage
    (code 1) and with the read-write levels and kappa at FR4-16 (code 4),
    one untimed call and `reps` timed calls of `nsteps` steps each."""
    n, k = 1024, 10
    kappa, src, dt = wave_inputs(n)
    from synth import ricker
    w = (ricker(nsteps * (reps + 1), dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float32)
    out = {}
    fields = {}
    for name, (rw, ro) in (("code1_fp32", ("fp32", "fp32")), ("code4_rw_ro_fr4-16", ("fr4", "fr4"))):
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format=rw, rw_rate=16, ro_format=ro, ro_rate=16,
                        device_budget_bytes=4 << 30)
        try:
            plan.set_field(0, zero)
            plan.set_field(1, zero)
            plan.set_field(2, kappa)
            plan.set_source(*src, w)
            plan.step(nsteps)
            ms = timed_steps(torch, plan, nsteps, reps)
            out[name] = n ** 3 * nsteps / (statistics.mean(ms) / 1e3) / 1e9
            fields[name] = plan.get_field(0)
        finally:
            plan.close()
        del plan
        torch.cuda.empty_cache()
    out["speedup_code4_vs_code1"] = out["code4_rw_ro_fr4-16"] / out["code1_fp32"]
    # both codes' p after the same steps against an FP64 run of them (the
    # library's FP64 wave kernel, held to the FP64 oracle by the GPU tests)
    total = nsteps * (reps + 1)
    p64 = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp64 = torch.zeros_like(p64)
    ooc.ooc_wave25_steps_f64(p64, pp64, torch.from_numpy(kappa.astype(np.float64)).cuda(), total, src=src,
                             w=w.astype(np.float64))
    torch.cuda.synchronize()
    del pp64
    for name, f in fields.items():
        out[f"{name}_rel_l2_vs_fp64"] = field_errors(torch.from_numpy(f).cuda(), p64)["rel_l2"]
    del fields, p64
    torch.cuda.empty_cache()
    out["what"] = (f"wave25 1024^3, 4 GiB budget, k = {k}, {reps} timed calls of {nsteps} steps after one untimed; "
                   f"errors of p after all {total} steps against an FP64 run; "
                   "bench.py --workload wave1024 and wave1024_error have the full study")
    return out


def fp64_summary(torch, ooc, n=512, nsteps=16, reps=2):
    """FP64 fields in brief, for the default line: heat7 at n^3 in FP64 with
    a 256 MiB budget (streaming), k = 4, raw FP64 storage against FR4D at 32
    bits per value (the paper's 2:1 for doubles), one untimed call and
    `reps` timed calls of `nsteps` steps each, with the FR4D result's rel-L2
    against the raw-FP64 run."""
    from synth import smooth_random_field
    u0 = smooth_random_field((n, n, n), 16.0, seed=5, dtype=np.float64)
    out, ref = {}, None
    for name, (fmt, rate) in (("fp64", ("fp64", 64)), ("fr4d-32", ("fr4", 32))):
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate,
                        device_budget_bytes=256 << 20, precision="fp64")
        try:
            plan.set_field(0, u0)
            plan.step(nsteps)
            ms = timed_steps(torch, plan, nsteps, reps)
            out[name] = n ** 3 * nsteps / (statistics.mean(ms) / 1e3) / 1e9
            got = plan.get_field(0)
        finally:
            plan.close()
        del plan
        torch.cuda.empty_cache()
        if ref is None:
            ref = got
        else:
            out["fr4d-32_rel_l2_vs_fp64_storage"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    out["speedup_fr4d32_vs_fp64"] = out["fr4d-32"] / out["fp64"]
    out["what"] = (f"heat7 {n}^3 in FP64, 256 MiB budget, k = 4, {reps} timed calls of {nsteps} steps after one "
                   "untimed; bench.py --workload fp64 has the 1024^3 heat7 and wave25 study")
    return out


def run_gpu(args, world, rank, local):
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import smooth_random_field

    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    dev = torch.device("cuda", local)
    hbm_peak, peak_src = load_peaks()
    u0 = smooth_random_field((N, N, N), 32.0, seed=2)
    pts = N ** 3
    subs = {}

    # ---- headline: FR4-16 slabs --------------------------------------------------
    plan = make_plan(ooc, *MAIN)
    info = plan.info()
    plan.set_field(0, u0)
    plan.step(NSTEPS)  # first warm-up step: 64 steps from u0, checked for the stated error
    subs[fmt_name(*MAIN)] = sub_box(plan.get_field(0))
    for _ in range(max(args.warmup - 1, 0)):
        plan.step(NSTEPS)
    plan.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed_steps(torch, plan, NSTEPS, args.steps)
        torch.cuda.synchronize()
        barrier(world)
        # Second timed region, same steps, with a CUDA event pair around every
        # launch for the per-kernel rooflines.  The events keep consecutive
        # kernels from overlapping and cost about 10 % of the throughput, so
        # the headline value above is timed without them.
        plan.set_profile(True)
        plan.reset_stats()
        ms_prof = timed_steps(torch, plan, NSTEPS, args.steps)
        overlap = overlap_summary(plan.trace())
        plan.set_profile(False)
    torch.cuda.synchronize()
    barrier(world)
    st = plan.stats()
    total_ms = max_over_ranks(world, sum(ms), dev)
    ms_per_step = total_ms / args.steps
    value = world * pts * NSTEPS * args.steps / (total_ms / 1e3) / 1e9
    value_profiled = world * pts * NSTEPS * args.steps / (max_over_ranks(world, sum(ms_prof), dev) / 1e3) / 1e9

    # per-kernel rooflines from the live per-launch events of the second timed region
    nsten = pts * NSTEPS * args.steps
    rate = MAIN[1]
    kernels = {
        # 8 B per point per launch: one step per launch reads and writes each
        # point once per step; a fused pair once per two steps (the band of
        # the intermediate level, about 3 % more, is not counted)
        "heat7_stencil": {"ms": st["ms_stencil"], "launches": st["n_stencil"], "bytes": 8 * nsten / SPL,
                          "steps_per_launch": SPL},
        "fr4_decode": {"ms": st["ms_decode"], "launches": st["n_decode"], "bytes": (4 + rate / 8) * pts * st["passes"]},
        "fr4_encode": {"ms": st["ms_encode"], "launches": st["n_encode"], "bytes": (4 + rate / 8) * pts * st["passes"]},
    }
    # units (points or values) of each kernel class over the timed region
    units = {"heat7_stencil": nsten / SPL, "fr4_decode": pts * st["passes"], "fr4_encode": pts * st["passes"]}
    for name, kv in kernels.items():
        kv["GBs"] = kv["bytes"] / (kv["ms"] / 1e3) / 1e9 if kv["ms"] > 0 else None
        kv["frac_hbm"] = kv["GBs"] / hbm_peak if kv["GBs"] else None
        c = ncu_counters(name) if SPL == 2 or name != "heat7_stencil" else None
        per_launch = units[name] / max(kv["launches"], 1)
        kv["dram_bytes_per_launch_ncu"] = c["dram_bytes"] / NCU_UNITS * per_launch if c else None
        kv["issue_frac"] = (c["warp_inst"] / NCU_UNITS * units[name] / (kv["ms"] / 1e3) / ISSUE_PEAK_WARP_INST
                            if c and kv["ms"] > 0 else None)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    launches = max(dk["launches"], 1)
    timing = ("CUDA events on the compute stream around each slab's stencil launches and each codec launch, "
              "over a second timed region of the same steps; mean launch = bracketed time / launches (whole-job "
              "rate with the events: %.1f Gpts/s)" % value_profiled)
    if dom == "heat7_stencil":
        roofline = {"bound": "hbm", "kernel": "heat7x2t (two heat7 steps per launch)" if SPL == 2 else "heat7",
                    "achieved": dk["GBs"], "peak": hbm_peak, "unit": "GB/s", "frac": dk["frac_hbm"],
                    "traffic": dk["dram_bytes_per_launch_ncu"], "bytes_per_launch": dk["bytes"] / launches,
                    "ms_per_launch": dk["ms"] / launches, "peak_source": peak_src, "timing": timing}
    else:
        # the codec is bound by instruction issue (integer and shared-memory
        # work per block), not by HBM: its roofline is the issue rate, with
        # its HBM fraction beside it
        c = ncu_counters(dom)
        ach = c["warp_inst"] / NCU_UNITS * units[dom] / (dk["ms"] / 1e3) / 1e9 if c and dk["ms"] > 0 else None
        roofline = {"bound": "alu", "kernel": dom + "_kernel", "achieved": ach, "peak": ISSUE_PEAK_WARP_INST / 1e9,
                    "unit": "G warp-instructions/s", "frac": ach * 1e9 / ISSUE_PEAK_WARP_INST if ach else None,
                    "traffic": dk["dram_bytes_per_launch_ncu"], "bytes_per_launch": dk["bytes"] / launches,
                    "ms_per_launch": dk["ms"] / launches, "hbm_achieved_GBs": dk["GBs"], "hbm_frac": dk["frac_hbm"],
                    "peak_source": "152 SMs x 4 schedulers x 1 warp instruction per clock x 2070 MHz",
                    "achieved_source": "executed warp instructions per value from ncu on the window56 case "
                                       "(same kernel source), scaled to the values of the timed launches",
                    "timing": timing}
    h2d_GBs = st["h2d_bytes"] / (st["ms_h2d"] / 1e3) / 1e9 if st["ms_h2d"] > 0 else None
    d2h_GBs = st["d2h_bytes"] / (st["ms_d2h"] / 1e3) / 1e9 if st["ms_d2h"] > 0 else None
    plan.close()
    del plan
    torch.cuda.empty_cache()

    # ---- end to end through the public API with host FP32 buffers ---------------
    plan = make_plan(ooc, *MAIN, profile=0)
    e2e_ms = []
    # the user's FP32 input and output live in pinned host memory
    pinned_in = torch.from_numpy(u0).pin_memory()
    pinned_out = torch.empty((N, N, N), dtype=torch.float32, pin_memory=True)
    host_in, host_out = pinned_in.numpy(), pinned_out.numpy()
    for rep in range(1 + min(args.steps, 2)):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(plan.streams[0])
        plan.set_field(0, host_in)
        plan.step(NSTEPS)
        plan.get_field(0, out=host_out)
        e1.record(plan.streams[2])
        e1.synchronize()
        if rep > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    st_e2e = plan.stats()
    plan.close()
    del plan, pinned_in, pinned_out
    torch.cuda.empty_cache()
    e2e_ms_max = max_over_ranks(world, statistics.mean(e2e_ms), dev)
    e2e_value = world * pts * NSTEPS / (e2e_ms_max / 1e3) / 1e9
    field_bytes = pts * 4
    nrep = len(e2e_ms) + 1
    h2d_step = field_bytes + st_e2e["h2d_bytes"] // nrep
    d2h_step = field_bytes + st_e2e["d2h_bytes"] // nrep

    # ---- compressed vs uncompressed on the same GPU ----------------------------
    formats = {}
    for fmt, r in COMPARE:
        p = make_plan(ooc, fmt, r, profile=0)
        p.set_field(0, u0)
        p.step(NSTEPS)  # warm-up, and the state checked for the stated error
        subs[fmt_name(fmt, r)] = sub_box(p.get_field(0))
        # same warm-up and timed steps as the headline
        for _ in range(max(args.warmup - 1, 0)):
            p.step(NSTEPS)
        m = timed_steps(torch, p, NSTEPS, args.steps)
        formats[fmt_name(fmt, r)] = {"Gpts": pts * NSTEPS / (statistics.mean(m) / 1e3) / 1e9,
                                     "slab_planes": p.info()["slab_planes"], "nslab": p.info()["nslab"],
                                     "warmup": args.warmup, "steps": args.steps}
        p.close()
        del p
        torch.cuda.empty_cache()
    formats[fmt_name(*MAIN)] = {"Gpts": value / world, "slab_planes": info["slab_planes"], "nslab": info["nslab"]}

    # ---- the paper's own workload (25-point wave, Section VI) in brief ---------
    try:
        wave = wave1024_summary(torch, ooc)
    except Exception as exc:  # reported, never fatal to the headline
        wave = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
    # ---- FP64 fields, as the paper ran them, in brief ---------------------------
    try:
        f64 = fp64_summary(torch, ooc)
    except Exception as exc:  # reported, never fatal to the headline
        f64 = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()

    if rank != 0:
        return 0

    # ---- stated accuracy and the CPU oracle baseline (rank 0, N = 1 only) --------
    err = None
    cpu = None
    if world == 1:
        exact, cpu = cpu_oracle_leg(u0)
        for name, sb in subs.items():
            m = field_errors(torch.from_numpy(sb), torch.from_numpy(exact))
            formats[name]["rel_l2"] = m["rel_l2"]
            formats[name]["max_abs"] = m["max_abs"]
            formats[name]["mean_rel_sampled"] = m["mean_rel_sampled"]
        mm = formats[fmt_name(*MAIN)]
        err = {"rel_l2": mm["rel_l2"], "max_abs": mm["max_abs"], "mean_rel_sampled": mm["mean_rel_sampled"],
               "vs": "FP64 oracle, central 128^3 sub-box after 64 steps from the initial field"}

    fp32 = formats["fp32"]["Gpts"]
    link_dir = 170.0  # GB/s each way with both directions busy (measured H2D/D2H probe)
    link_roof = {f: link_dir * 1e9 * K / (bits / 8) / 1e9 for f, bits in
                 (("fp32", 32), ("bf16", 16), ("fr4-8", 8), ("fr4-12", 12), ("fr4-16", 16), ("fr4-24", 24))}
    # stencil bytes per point-step: 8 with one step per launch, 4 with fused pairs
    sten_b = 8.0 / SPL
    hbm_roof = hbm_peak / sten_b
    # HBM bound including the codec and DMA bytes of the storage format: per
    # point-step the stencil bytes, plus per pass (/k) decode R/8 + 4, encode
    # 4 + R/8 and the landing / sending of R/8 each way.
    fmt_bits = {"fp32": 32, "bf16": 16, "fr4-8": 8, "fr4-12": 12, "fr4-16": 16, "fr4-24": 24}
    hbm_refined = {f: hbm_peak / (sten_b + ((8 + b / 4 if f != "fp32" else 0) + b / 4) / K)
                   for f, b in fmt_bits.items()}
    line = {
        "metric": METRIC, "value": value, "unit": "Gpts/s",
        # the comparison the metric names, first so that it survives a cut tail
        "speedup_vs_fp32": value / world / fp32 if fp32 else None, "fp32_Gpts": fp32,
        "rel_l2_vs_fp64": err["rel_l2"] if err else None,
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "storage": fmt_name(*MAIN), "grid": [N, N, N], "k": K,
                   "heat_steps_per_launch": SPL, "time_steps_per_bench_step": NSTEPS, "device_budget_bytes": BUDGET,
                   "slab_planes": info["slab_planes"], "nslab": info["nslab"], "ring_planes": info["ring_planes"],
                   "device_bytes": info["device_bytes"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (4 GiB field streamed from pinned host memory each pass)"},
        "error": err,
        "compressed_vs_uncompressed": {"speedup": value / world / fp32 if fp32 else None, "formats": formats},
        "pipeline_roofline": {"hbm_Gpts": hbm_roof, "link_Gpts": link_roof,
                              "hbm_with_codec_and_dma_Gpts": hbm_refined,
                              "frac_of_min": (value / world) / min(hbm_roof, link_roof[fmt_name(*MAIN)]),
                              "frac_of_min_refined": (value / world) / min(hbm_refined[fmt_name(*MAIN)],
                                                                           link_roof[fmt_name(*MAIN)]),
                              "link_GBs_each_way_assumed": link_dir,
                              "h2d_GBs_per_copy": h2d_GBs, "d2h_GBs_per_copy": d2h_GBs},
        "roofline": roofline,
        "paper_workload_wave1024": wave,
        "fp64_fields_heat512": f64,
        "kernels": kernels,
        "overlap": overlap,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "Gpts/s", "h2d_bytes_per_step": int(h2d_step),
                "d2h_bytes_per_step": int(d2h_step),
                "what": "ooc_set_field(pinned host FP32) + ooc_step(64) + ooc_get_field(pinned host FP32)"},
        "gpu_launches": int(st["kernel_launches"]),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- other workloads
def _cuda_events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_kernels512(args, world, rank, local):
    """Each kernel once per step on a 512^3 smooth field (the ncu capture case):
    FR4 encode and decode at R = 16, two in-core heat7 steps, two fused heat7
    pairs (two steps per launch), two in-core wave25 steps, two fused wave25
    pairs, two FP64 heat7 steps, BF16 pack and unpack, one adjoint step and
    one gradient update; CUDA-event times per kernel class."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import smooth_random_field
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    n = 512
    pts = n ** 3
    d = torch.from_numpy(smooth_random_field((n, n, n), 32.0, seed=2)).cuda()
    d_codec = d.clone()  # the stencil ops below advance d in place; the codec variants get the field itself
    w = torch.empty(ooc.ooc_compressed_bytes(n, n, n, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(d)
    tmp = torch.empty_like(d)
    kap = torch.full_like(d, 0.1)
    pp = torch.zeros_like(d)
    d64 = d.double()
    t64 = torch.empty_like(d64)
    b16 = torch.empty(d.shape, dtype=torch.int16, device="cuda")
    w1, w2 = torch.empty_like(d), torch.empty_like(d)  # scratch of the fused wave pairs
    ops = {
        "fr4_encode": (lambda: ooc.ooc_compress(d, 16, d_out=w), 1, (4 + 2) * pts, 0),
        "fr4_decode": (lambda: ooc.ooc_decompress(w, (n, n, n), 16, d_out=out), 1, (4 + 2) * pts, 0),
        "heat7": (lambda: ooc.ooc_heat7_steps(d, tmp, 2), 2, 8 * pts, 1),
        "heat7_fused_pair": (lambda: ooc.ooc_heat7_steps_fused(d, tmp, 4), 2, 8 * pts, 2),
        "wave25": (lambda: ooc.ooc_wave25_steps(d, pp, kap, 2), 2, 16 * pts, 1),
        # two pairs land in place (no copy); p^n, p^{n-1}, kappa in and
        # p^{n+1}, p^{n+2} out: 20 B per point per launch
        "wave25_fused_pair": (lambda: ooc.ooc_wave25_steps_fused(d, pp, kap, 4, d_t1=w1, d_t2=w2), 2, 20 * pts, 2),
        "heat7_f64": (lambda: ooc.ooc_heat7_steps_f64(d64, t64, 2), 2, 16 * pts, 1),
        "bf16_pack": (lambda: ooc.ooc_bf16_pack(d, d_out=b16), 1, 6 * pts, 0),
        "bf16_unpack": (lambda: ooc.ooc_bf16_unpack(b16, d_out=out), 1, 6 * pts, 0),
        # adjoint kernels: mu_prev <- 2 mu - mu_prev + L(kappa mu) (reads mu,
        # kappa, mu_prev, writes 16 B per point); g += mu L(p) in FP64 (reads
        # mu, p, g, writes g: 24 B per point)
        "wave25_adjoint_step": (lambda: ooc.ooc_wave25_adjoint_step(d, pp, kap, d_out=out), 1, 16 * pts, 0),
        "wave25_grad_accum": (lambda: ooc.ooc_wave25_grad_accum(t64, d, out), 1, 24 * pts, 0),
    }
    res = {}
    for name, (fn, nl, by, spl) in ops.items():
        for _ in range(args.warmup):
            fn()
        e0, e1 = _cuda_events(torch)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(max(args.steps, 1)):
            fn()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1) / nl
        res[name] = {"ms_per_launch": ms, "GBs": by / (ms / 1e3) / 1e9}
        if spl:
            res[name]["steps_per_launch"] = spl
            res[name]["Gpts_steps_per_s"] = pts * spl / (ms / 1e3) / 1e9
    # codec variants: variable-size blocks (two encode passes with a prefix
    # sum and a host read of the size in between; one decode pass)
    var = {}
    d = d_codec
    for name, mode, param in (("precision16", ooc.OOC_FR4_PRECISION, 16), ("accuracy1e-4", ooc.OOC_FR4_ACCURACY, 1e-4)):
        stream, index = ooc.ooc_compress_var(d, mode, param)
        times = {}
        for what, fn in (("encode", lambda: ooc.ooc_compress_var(d, mode, param, d_out=stream_buf, d_index=index)),
                         ("decode", lambda: ooc.ooc_decompress_var(stream, index, (n, n, n), mode, param, d_out=out))):
            if what == "encode":
                stream_buf = torch.empty(ooc.ooc_compress_var_bound(n, n, n), dtype=torch.uint8, device="cuda")
            for _ in range(max(args.warmup, 1)):
                fn()
            e0, e1 = _cuda_events(torch)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(max(args.steps, 1)):
                fn()
            e1.record()
            e1.synchronize()
            times[what] = e0.elapsed_time(e1) / max(args.steps, 1)
        bits = stream.numel() * 8 / pts
        err = float((ooc.ooc_decompress_var(stream, index, (n, n, n), mode, param) - d).abs().max())
        var[name] = {"bits_per_value": bits, "max_abs_err": err, "encode_ms": times["encode"],
                     "decode_ms": times["decode"],
                     "encode_GBs": (4 + bits / 8) * pts / (times["encode"] / 1e3) / 1e9,
                     "decode_GBs": (4 + bits / 8) * pts / (times["decode"] / 1e3) / 1e9}
        del stream, index, stream_buf
    if rank == 0:
        print(json.dumps({"workload": "kernels512", "kernels": res, "codec_variants": var, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup}), flush=True)
    return 0


def run_window56(args, world, rank, local):
    """The headline pipeline's kernels on one of its windows, in-core: a
    56-plane window of 1024^2 planes (the slab thickness the 1 GiB budget
    gives at k = 4), a smooth field; per step one fused heat7 pair launch
    (two launches per call: levels 0 -> 2 -> 4, no copy back), one FR4-16
    encode and one decode of the window.  CUDA-event times per launch.  This
    is the small ncu capture case of the 1024^3 workload's kernels."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import smooth_random_field
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    shape = (56, 1024, 1024)
    pts = 56 * 1024 * 1024
    d = torch.from_numpy(smooth_random_field(shape, 32.0, seed=2)).cuda()
    tmp = torch.empty_like(d)
    out = torch.empty_like(d)
    w = torch.empty(ooc.ooc_compressed_bytes(1024, 1024, 56, 16), dtype=torch.uint8, device="cuda")
    ops = {
        # name: (call, launches per call, algorithmic bytes per launch)
        "heat7x2_pair": (lambda: ooc.ooc_heat7_steps_fused(d, tmp, 4), 2, 8 * pts),
        "fr4_encode": (lambda: ooc.ooc_compress(d, 16, d_out=w), 1, (4 + 2) * pts),
        "fr4_decode": (lambda: ooc.ooc_decompress(w, shape, 16, d_out=out), 1, (4 + 2) * pts),
    }
    res = {}
    for name, (fn, nl, by) in ops.items():
        for _ in range(args.warmup):
            fn()
        e0, e1 = _cuda_events(torch)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(max(args.steps, 1)):
            fn()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1) / nl
        res[name] = {"us_per_launch": 1e3 * ms, "GBs": by / (ms / 1e3) / 1e9, "bytes_per_launch": by}
    if rank == 0:
        print(json.dumps({"workload": "window56", "window": list(shape), "kernels": res,
                          "device_fault": ooc.ooc_take_device_fault(), "steps": args.steps,
                          "warmup": args.warmup}), flush=True)
    return 0


def wave_inputs(n, seed=3):
    from synth import layered_velocity, ricker
    shape = (n, n, n)
    v = layered_velocity(shape, seed=seed)
    dx = 10.0
    dt = 0.4 * dx / v.max()
    kappa = ((v * dt / dx) ** 2).astype(np.float32)
    src = (n // 2, n // 2, n // 2)
    return kappa, src, dt


def incore_wave_fusion(torch, ooc, kappa, src, w, nsteps=20, reps=2):
    """In-core 1024^3 wave25 from rest with the source on: nsteps single
    steps (16 B per point-step from HBM) against nsteps/2 fused pairs (two
    steps per launch, level n+1 on chip: 10 B per point-step), CUDA-event
    time per step, and whether the two give the same bits."""
    d_k = torch.from_numpy(kappa).cuda()
    res, fields = {}, {}
    for name in ("single", "fused_pair"):
        p, pp = torch.zeros_like(d_k), torch.zeros_like(d_k)
        t1, t2 = (torch.empty_like(d_k), torch.empty_like(d_k)) if name == "fused_pair" else (None, None)

        def run(t0):
            if name == "fused_pair":
                ooc.ooc_wave25_steps_fused(p, pp, d_k, nsteps, src=src, w=w, t=t0, d_t1=t1, d_t2=t2)
            else:
                ooc.ooc_wave25_steps(p, pp, d_k, nsteps, src=src, w=w, t=t0)
        run(0)  # warm-up; its steps are part of the compared history
        times = []
        for r in range(reps):
            e0, e1 = _cuda_events(torch)
            torch.cuda.synchronize()
            e0.record()
            run(nsteps * (r + 1))
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / nsteps)
        ms = min(times)
        res[name] = {"ms_per_step": ms, "Gpts_steps_per_s": kappa.size / (ms / 1e3) / 1e9,
                     "algorithmic_bytes_per_point_step": 16 if name == "single" else 10}
        fields[name] = (p, pp)
        del t1, t2
    a, b = fields["single"], fields["fused_pair"]
    res["bit_identical"] = bool(torch.equal(a[0].view(torch.int32), b[0].view(torch.int32)) and
                                torch.equal(a[1].view(torch.int32), b[1].view(torch.int32)))
    res["fused_over_single_time"] = res["fused_pair"]["ms_per_step"] / res["single"]["ms_per_step"]
    del fields, a, b, d_k
    torch.cuda.empty_cache()
    return res


def run_wave1024(args, world, rank, local):
    """3D acoustic wave, 25-point, 1024^3, device budget 4 GiB, k = 10: the
    paper's four codes (FP32; read-write fields at 16 bits/value; read-only
    kappa at 16 bits/value; both), 200 time steps per bench step."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import ricker
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    n, k, nsteps = 1024, 10, 200
    kappa, src, dt = wave_inputs(n)
    total_steps = nsteps * (args.warmup + args.steps + 1)
    w = (ricker(total_steps, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float32)
    codes = {"code1_fp32": ("fp32", "fp32"), "code2_rw_fr4-16": ("fr4", "fp32"),
             "code3_ro_fr4-16": ("fp32", "fr4"), "code4_rw_ro_fr4-16": ("fr4", "fr4")}
    out = {}
    finals = {}
    # untimed warm-up in calls of 100 steps, with the central 128 planes kept
    # every 100 steps for the self-consistency series (against code 1)
    series_ref, series = [], {}
    c0, c1 = n // 2 - 64, n // 2 + 64
    for name, (rw, ro) in codes.items():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format=rw, rw_rate=16, ro_format=ro,
                        ro_rate=16, device_budget_bytes=4 << 30, profile=0)
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        series[name] = []
        for j in range(args.warmup * nsteps // 100):
            plan.step(100)
            mid = plan.get_field(0)[c0:c1].astype(np.float64)
            if name == "code1_fp32":
                series_ref.append(mid)
            else:
                ref_mid = series_ref[j]
                series[name].append([100 * (j + 1), float(np.linalg.norm(mid - ref_mid) / np.linalg.norm(ref_mid))])
            del mid
        plan.step(nsteps)  # captures the graph of a bench step outside the timed region
        ms = timed_steps(torch, plan, nsteps, args.steps)
        t = sum(ms) / args.steps
        out[name] = {"Gpts": n ** 3 * nsteps / (t / 1e3) / 1e9, "ms_per_step": t,
                     "slab_planes": plan.info()["slab_planes"], "nslab": plan.info()["nslab"],
                     "device_bytes": plan.info()["device_bytes"]}
        finals[name] = plan.get_field(0)[n // 2 - 64:n // 2 + 64].astype(np.float64)
        plan.close()
        del plan
        torch.cuda.empty_cache()
    ref = finals["code1_fp32"]
    for name in codes:
        dd = finals[name] - ref
        out[name]["rel_l2_vs_fp32_storage"] = float(np.linalg.norm(dd) / np.linalg.norm(ref))
        if name != "code1_fp32":
            out[name]["rel_l2_vs_fp32_storage_every_100"] = series[name]
    del series_ref
    # the two-steps-per-launch kernel in-core at the same size (the pipeline
    # keeps single steps: the pair is slower per step on GB300)
    fusion = incore_wave_fusion(torch, ooc, kappa, src, w)
    if rank == 0:
        steps_done = nsteps * (args.warmup + args.steps + 1)
        print(json.dumps({"workload": "wave1024", "metric": "Gpts/s", "value": out["code4_rw_ro_fr4-16"]["Gpts"],
                          "unit": "Gpts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "time_steps_per_bench_step": nsteps, "k": k, "device_budget_bytes": 4 << 30,
                          "speedup_code4_vs_code1": out["code4_rw_ro_fr4-16"]["Gpts"] / out["code1_fp32"]["Gpts"],
                          "codes": out, "incore_fusion_1024": fusion,
                          "error_note": f"self-consistency, not oracle error: rel-L2 of the central "
                          f"128 planes against the same pipeline with FP32 storage, every 100 steps of the warm-up "
                          f"and after {steps_done} steps (an FP64 oracle at 1024^3 x 2000 steps is out of reach of "
                          "the host cores; the precision workload measures storage error against the FP64 oracle)"}),
              flush=True)
    return 0


def field_errors(got, ref, nsample_per_plane=100, seed=0, floor_frac=1e-3, zchunk=64):
    """Errors of a field against a reference, both CUDA tensors [nz, ny, nx]:
    rel-L2, max-abs and the paper-style mean pointwise relative error on 100
    sampled points per plane (Section VI-C), leaving out samples with |ref|
    below floor_frac * max|ref|.  The sample points are drawn from
    numpy.random.default_rng(seed): for each plane nsample_per_plane rows,
    then as many columns.  Sums run in FP64 over z-chunks."""
    import torch
    nz, ny, nx = ref.shape
    sq_d = sq_r = 0.0
    max_abs = max_ref = 0.0
    for z0 in range(0, nz, zchunk):
        r = ref[z0:z0 + zchunk].double()
        d = got[z0:z0 + zchunk].double() - r
        sq_d += float((d * d).sum())
        sq_r += float((r * r).sum())
        max_abs = max(max_abs, float(d.abs().max()))
        max_ref = max(max_ref, float(r.abs().max()))
        del r, d
    rng = np.random.default_rng(seed)
    ys = rng.integers(0, ny, size=(nz, nsample_per_plane))
    xs = rng.integers(0, nx, size=(nz, nsample_per_plane))
    flat = torch.from_numpy(((np.arange(nz)[:, None] * ny + ys) * nx + xs).ravel()).to(ref.device)
    rs = ref.reshape(-1)[flat].double()
    vs = got.reshape(-1)[flat].double()
    keep = rs.abs() >= floor_frac * max_ref
    mean_rel = float(((vs - rs).abs()[keep] / rs.abs()[keep]).mean()) if bool(keep.any()) else 0.0
    return {"rel_l2": (sq_d / sq_r) ** 0.5 if sq_r > 0 else sq_d ** 0.5, "max_abs": max_abs,
            "mean_rel_sampled": mean_rel, "samples": int(rs.numel()), "excluded": int((~keep).sum())}


FP64_REFERENCE_NOTE = ("FP64 reference: the same wave run in FP64 arithmetic by the library's FP64 wave25 kernel "
                       "(ooc_wave25_steps_f64, in-core, FP32 kappa values and source amplitudes), which the GPU "
                       "tests hold to the FP64 oracle within 1e-13 rel-L2 on this configuration's inputs")


def run_precision(args, world, rank, local, n=384):
    """Long-horizon precision study: wave25 at n^3 (384^3, the configuration's
    size; 192^3 with --workload precision192), 4320 steps, k = 10, 6 slabs,
    storage FP32, BF16, FR4 at 8/12/16/24 bits/value (both read-write levels
    and kappa), FP32 compute.  The formats run side by side with an FP64
    reference run, 100 steps at a time.  Every 100 steps: rel-L2, max-abs
    and the mean pointwise relative error on 100 sampled points per plane
    against the FP64 run over all 4320 steps, and against the FP32-storage
    run (a self-consistency check); Gpts/s per format."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import ricker
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    k, total, every = 10, 4320, 100
    T = n // 6
    kappa, src, dt = wave_inputs(n)
    w = (ricker(total, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float32)
    marks = list(range(every, total + 1, every))
    if total not in marks:
        marks.append(total)
    fmts = [("fp32", 16), ("bf16", 16), ("fr4", 8), ("fr4", 12), ("fr4", 16), ("fr4", 24)]
    plans, tms = {}, {}
    for fmt, rate in fmts:
        name = fmt_name(fmt, rate)
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format=fmt, rw_rate=rate, ro_format=fmt,
                        ro_rate=rate, slab_planes=T, profile=0)
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plans[name], tms[name] = plan, 0.0
    p64 = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp64 = torch.zeros_like(p64)
    k64 = torch.from_numpy(kappa.astype(np.float64)).cuda()
    w64 = w.astype(np.float64)
    errs = {name: [] for name in plans}
    self_errs = {name: [] for name in plans}
    done = 0
    for m in marks:
        ooc.ooc_wave25_steps_f64(p64, pp64, k64, m - done, src=src, w=w64, t=done)
        torch.cuda.synchronize()  # the FP64 run is not inside any format's timed calls
        fields = {}
        for name, plan in plans.items():
            e0, e1 = _cuda_events(torch)
            e0.record(plan.streams[0])
            plan.step(m - done)
            e1.record(plan.streams[2])
            e1.synchronize()
            tms[name] += e0.elapsed_time(e1)
            fields[name] = torch.from_numpy(plan.get_field(0, out=np.empty((n, n, n), dtype=np.float32))).cuda()
        torch.cuda.synchronize()
        for name, f in fields.items():
            e = field_errors(f, p64)
            errs[name].append([m, e["rel_l2"], e["max_abs"], e["mean_rel_sampled"]])
            se = field_errors(f, fields["fp32"])
            self_errs[name].append([m, se["rel_l2"], se["max_abs"]])
        del fields
        done = m
    speed = {name: n ** 3 * total / (tms[name] / 1e3) / 1e9 for name in plans}
    for plan in plans.values():
        plan.close()
    fault = ooc.ooc_take_device_fault()
    del p64, pp64, k64
    torch.cuda.empty_cache()
    if rank != 0:
        return 0
    line = {"workload": "precision" if n == 384 else f"precision{n}", "grid": [n, n, n], "steps": total, "k": k,
            "slab_planes": T, "nslab": -(-n // T), "reference": FP64_REFERENCE_NOTE,
            "errors_note": f"errors_every_100: [step, rel-L2, max-abs, mean relative error on 100 sampled points "
                           f"per plane] against the FP64 run, every {every} steps over all {total} steps",
            "self_consistency_note": "errors_vs_fp32_storage_every_100: the same pipeline with FP32 storage, "
                                     "not the FP64 run",
            "formats": {name: {"Gpts": speed[name], "errors_every_100": errs[name],
                               "errors_vs_fp32_storage_every_100": self_errs[name]} for name in plans},
            "device_fault": fault}
    print(json.dumps(line), flush=True)
    return 0


def run_wave1024_error(args, world, rank, local):
    """The 1024^3 wave configuration's accuracy run (Section VI-C): 2000 steps
    from rest with the Ricker source, k = 10, 4 GiB device budget; code 1
    (FP32 storage) and code 4 (read-write levels and kappa at FR4-16) side
    by side with an FP64 reference run, 100 steps at a time.  Every 100
    steps: rel-L2, max-abs and the sampled mean relative error of each code
    against the FP64 run; Gpts/s of each code over the run."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import ricker
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    n, k, total, every = 1024, 10, 2000, 100
    kappa, src, dt = wave_inputs(n)
    w = (ricker(total, dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float32)
    codes = {"code1_fp32": ("fp32", "fp32"), "code4_rw_ro_fr4-16": ("fr4", "fr4")}
    plans, tms = {}, {}
    for name, (rw, ro) in codes.items():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=k, rw_format=rw, rw_rate=16, ro_format=ro,
                        ro_rate=16, device_budget_bytes=4 << 30, profile=0)
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plans[name], tms[name] = plan, 0.0
    del zero
    p64 = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    pp64 = torch.zeros_like(p64)
    k64 = torch.from_numpy(kappa.astype(np.float64)).cuda()
    w64 = w.astype(np.float64)
    host = np.empty((n, n, n), dtype=np.float32)
    errs = {name: [] for name in plans}
    t_ref = 0.0
    done = 0
    for m in range(every, total + 1, every):
        e0, e1 = _cuda_events(torch)
        e0.record()
        ooc.ooc_wave25_steps_f64(p64, pp64, k64, m - done, src=src, w=w64, t=done)
        e1.record()
        e1.synchronize()
        t_ref += e0.elapsed_time(e1)
        for name, plan in plans.items():
            e0, e1 = _cuda_events(torch)
            e0.record(plan.streams[0])
            plan.step(m - done)
            e1.record(plan.streams[2])
            e1.synchronize()
            tms[name] += e0.elapsed_time(e1)
            f = torch.from_numpy(plan.get_field(0, out=host)).cuda()
            e = field_errors(f, p64)
            errs[name].append([m, e["rel_l2"], e["max_abs"], e["mean_rel_sampled"]])
            del f
        done = m
    for plan in plans.values():
        plan.close()
    fault = ooc.ooc_take_device_fault()
    del p64, pp64, k64
    torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"workload": "wave1024_error", "grid": [n, n, n], "steps": total, "k": k,
                          "device_budget_bytes": 4 << 30, "reference": FP64_REFERENCE_NOTE,
                          "fp64_reference_Gpts": n ** 3 * total / (t_ref / 1e3) / 1e9,
                          "errors_note": f"errors_every_100: [step, rel-L2, max-abs, mean relative error on 100 "
                                         f"sampled points per plane] against the FP64 run, every {every} steps",
                          "codes": {name: {"Gpts": n ** 3 * total / (tms[name] / 1e3) / 1e9,
                                           "errors_every_100": errs[name]} for name in plans},
                          "device_fault": fault}), flush=True)
    return 0


def run_adjoint512(args, world, rank, local):
    """Adjoint at 512^3: forward 1500 steps with FR4-16 checkpoints every 10
    steps in pinned host memory, backward replay + discrete adjoint, gradient
    w.r.t. kappa; checked against central differences of the misfit along four
    smooth random directions (GPU FP32 forward, FP64 misfit)."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import layered_velocity, ricker, smooth_random_field
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    n, N, every, rate = 512, 1500, 10, 16
    shape = (n, n, n)
    v_true = layered_velocity(shape, seed=3)
    dx = 10.0
    dt = 0.4 * dx / (v_true.max() * 1.05)
    c = dt / dx
    pert = np.clip(smooth_random_field(shape, 16.0, seed=13, dtype=np.float64), -1, 1)
    v = (v_true * (1.0 + 0.02 * pert)).astype(np.float32)
    src = (n // 2, n // 2, n // 2)
    w = (ricker(N, dt) * float((v_true[src[2], src[1], src[0]] * c) ** 2) * 1e3).astype(np.float32)
    rec = torch.tensor([(8 * n + y) * n + x for y in range(0, n, 8) for x in range(0, n, 8)], dtype=torch.int64,
                       device="cuda")
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    work = torch.empty(ooc.ooc_wave25_adjoint_work_bytes(shape, every, rate), dtype=torch.uint8, device="cuda")
    t_pin = time.perf_counter()
    h_ckpt = torch.empty(ooc.ooc_wave25_ckpt_bytes(shape, N, every, rate), dtype=torch.uint8, pin_memory=True)
    t_pin = time.perf_counter() - t_pin
    kap_true = ooc.ooc_kappa_from_velocity(torch.from_numpy(v_true.astype(np.float32)).cuda(), c)
    d = torch.empty((N, rec.numel()), device="cuda")
    ooc.ooc_wave25_forward_ckpt(kap_true, N, rec, d, every, rate, h_ckpt, work, streams, src=src, w=w)
    del kap_true
    kap = ooc.ooc_kappa_from_velocity(torch.from_numpy(v).cuda(), c)
    tr = torch.empty_like(d)
    e0, e1 = _cuda_events(torch)
    e0.record()
    ooc.ooc_wave25_forward_ckpt(kap, N, rec, tr, every, rate, h_ckpt, work, streams, src=src, w=w)
    e1.record()
    e1.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    res = (tr - d).contiguous()
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    e0, e1 = _cuda_events(torch)
    e0.record()
    ooc.ooc_wave25_backward_ckpt(kap, N, rec, res, every, rate, h_ckpt, g, work, streams, src=src, w=w)
    e1.record()
    e1.synchronize()
    ms_bwd = e0.elapsed_time(e1)

    def misfit(kk):
        t = torch.empty_like(d)
        ooc.ooc_wave25_forward_ckpt(kk, N, rec, t, every, rate, h_ckpt, work, streams, src=src, w=w)
        return 0.5 * float(((t.double() - d.double()) ** 2).sum())

    eps = 1e-3
    fds, ans = [], []
    for seed in (21, 22, 23, 24):  # four seeded smooth kappa-relative directions
        delta = torch.from_numpy(np.clip(smooth_random_field(shape, 8.0, seed=seed, dtype=np.float64), -1, 1)
                                 .astype(np.float32)).cuda() * kap
        fds.append((misfit(kap + eps * delta) - misfit(kap - eps * delta)) / (2 * eps))
        ans.append(float((g * delta.double()).sum()))
        del delta
    fd, an = fds[0], ans[0]
    rel = [abs(f - a) / abs(f) if f else None for f, a in zip(fds, ans)]
    if rank == 0:
        print(json.dumps({"workload": "adjoint512", "grid": list(shape), "steps": N, "ckpt_every": every,
                          "ckpt_rate": rate, "ckpt_bytes_pinned": h_ckpt.numel(), "pin_seconds": t_pin,
                          "ms_forward": ms_fwd, "ms_backward": ms_bwd,
                          "Gpts_forward": n ** 3 * N / (ms_fwd / 1e3) / 1e9,
                          "Gpts_backward": n ** 3 * N / (ms_bwd / 1e3) / 1e9,
                          "fd_directional": fd, "adjoint_directional": an,
                          "rel_diff": abs(fd - an) / abs(fd) if fd else None,
                          "fd_directions": fds, "adjoint_directions": ans, "rel_diff_directions": rel,
                          "fd_note": "central difference, eps 1e-3 of a smooth kappa-relative direction, GPU FP32 "
                                     "forward with FP64 misfit sums"}), flush=True)
    return 0


def fp64_window_kernels(ooc, torch, n=1024):
    """CUDA-event times of the FP64 path's kernels on one 56-plane window of
    n^2 planes (a smooth double field): FR4D encode and decode at 32 and 24
    bits per value, and one FP64 heat7 and wave25 step."""
    from synth import smooth_random_field
    shape = (56, n, n)
    d = torch.from_numpy(smooth_random_field(shape, 32.0, seed=2, dtype=np.float64)).cuda()
    dec = torch.empty_like(d)
    kern = {}
    for rate in (32, 24):
        w = torch.empty(ooc.ooc_compressed_bytes(n, n, 56, rate), dtype=torch.uint8, device="cuda")
        for name, fn in (("encode", lambda: ooc.ooc_compress64(d, rate, d_out=w)),
                         ("decode", lambda: ooc.ooc_decompress64(w, shape, rate, d_out=dec))):
            for _ in range(3):
                fn()
            e0, e1 = _cuda_events(torch)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                fn()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / 10
            kern[f"fr4d_{name}_R{rate}"] = {"us_per_launch": 1e3 * ms,
                                           "Gvalues_per_s": 56 * n * n / (ms / 1e3) / 1e9,
                                           "GBs": (8 + rate / 8) * 56 * n * n / (ms / 1e3) / 1e9}
    # the FP64 stencil kernels on the same window: heat7 and wave25 steps
    tmp = torch.empty_like(d)
    kap = torch.full_like(d, 0.05)
    for name, fn, per in (("heat7_f64", lambda: ooc.ooc_heat7_steps_f64(d, tmp, 2), 2),
                          ("wave25_f64", lambda: ooc.ooc_wave25_steps_f64(d, dec, kap, 2), 2)):
        fn()
        e0, e1 = _cuda_events(torch)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / (5 * per)
        kern[name] = {"us_per_step": 1e3 * ms, "Gpts_steps_per_s": 56 * n * n / (ms / 1e3) / 1e9}
    del d, dec, tmp, kap
    torch.cuda.empty_cache()
    return kern


def run_window56_fp64(args, world, rank, local):
    """The FP64 path's kernels on one 56-plane window of 1024^2 planes (the
    small ncu capture case of the fp64 workload)."""
    import torch

    import paper_2109_05410_gb300 as ooc
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    kern = fp64_window_kernels(ooc, torch)
    if rank == 0:
        print(json.dumps({"workload": "window56_fp64", "window": [56, 1024, 1024], "kernels": kern,
                          "device_fault": ooc.ooc_take_device_fault()}), flush=True)
    return 0


def run_fp64(args, world, rank, local):
    """FP64 fields, as the paper ran them (Section VI: double-precision
    fields stored at 32 and 24 of every 64 bits): heat7 and wave25 at 1024^3
    with FP64 compute, each with raw FP64 storage (the uncompressed
    pipeline, code 1) and FR4D at 32 and 24 bits per value (both read-write
    levels and kappa for the wave: code 4).  heat7: 2 GiB budget, k = 4, 32
    steps per call; wave25: 8 GiB budget (the FP32 wave's 4 GiB in doubles),
    k = 10, 20 steps per call, the layered velocity and the Ricker source of
    the wave1024 workload.  One untimed call, then timed calls.  Errors
    against the raw-FP64 pipeline on the central 64 planes (self-
    consistency; the FP64 oracle checks are GPU tests at smaller sizes).
    Also the FR4D kernels' CUDA-event times on one 56-plane window of 1024^2
    planes."""
    import torch

    import paper_2109_05410_gb300 as ooc
    from synth import ricker, smooth_random_field
    torch.cuda.set_device(local)
    ooc.build()
    ooc.lib()
    n = 1024
    reps = max(args.steps, 1)
    out = {"workload": "fp64", "grid": [n, n, n]}
    out["kernels_window56"] = fp64_window_kernels(ooc, torch, n)
    mid = slice(n // 2 - 32, n // 2 + 32)
    fmts = {"fp64": ("fp64", 64), "fr4d-32": ("fr4", 32), "fr4d-24": ("fr4", 24)}
    # heat7
    u0 = smooth_random_field((n, n, n), 32.0, seed=2, dtype=np.float64)
    heat = {}
    ref = None
    for name, (fmt, rate) in fmts.items():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="heat7", k=4, rw_format=fmt, rw_rate=rate,
                        device_budget_bytes=2 << 30, precision="fp64")
        plan.set_field(0, u0)
        plan.step(32)
        ms = timed_steps(torch, plan, 32, reps)
        t = sum(ms) / len(ms)
        got = plan.get_field(0)[mid].copy()
        heat[name] = {"Gpts": n ** 3 * 32 / (t / 1e3) / 1e9, "ms_per_call": t, "slab_planes": plan.info()["slab_planes"]}
        if name == "fp64":
            ref = got
        else:
            heat[name]["rel_l2_vs_fp64_storage"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        plan.close()
        del plan
        torch.cuda.empty_cache()
    del u0
    heat["speedup_fr4d32_vs_fp64"] = heat["fr4d-32"]["Gpts"] / heat["fp64"]["Gpts"]
    out["heat7"] = heat
    # wave25
    from synth import layered_velocity
    v = layered_velocity((n, n, n), seed=3)
    dt = 0.4 * 10.0 / float(v.max())
    kappa = (np.asarray(v, dtype=np.float64) * (dt / 10.0)) ** 2
    del v
    src = (n // 2, n // 2, n // 2)
    nsteps = 20
    w = (ricker(nsteps * (reps + 1), dt) * float(kappa[src[2], src[1], src[0]])).astype(np.float32)
    zero = np.zeros((n, n, n), dtype=np.float64)
    wave = {}
    ref = None
    for name, (fmt, rate) in fmts.items():
        plan = ooc.Plan(nx=n, ny=n, nz=n, stencil="wave25", k=10, rw_format=fmt, rw_rate=rate, ro_format=fmt,
                        ro_rate=rate, device_budget_bytes=8 << 30, precision="fp64")
        plan.set_field(0, zero)
        plan.set_field(1, zero)
        plan.set_field(2, kappa)
        plan.set_source(*src, w)
        plan.step(nsteps)
        ms = timed_steps(torch, plan, nsteps, reps)
        t = sum(ms) / len(ms)
        got = plan.get_field(0)[mid].copy()
        wave[name] = {"Gpts": n ** 3 * nsteps / (t / 1e3) / 1e9, "ms_per_call": t,
                      "slab_planes": plan.info()["slab_planes"]}
        if name == "fp64":
            ref = got
        else:
            wave[name]["rel_l2_vs_fp64_storage"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        plan.close()
        del plan
        torch.cuda.empty_cache()
    wave["speedup_fr4d32_vs_fp64"] = wave["fr4d-32"]["Gpts"] / wave["fp64"]["Gpts"]
    out["wave25"] = wave
    out["steps"] = reps
    out["error_note"] = ("rel-L2 of the central 64 planes against the same pipeline with raw FP64 storage "
                         "(self-consistency, not oracle error)")
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat1024",
                    choices=["heat1024", "kernels512", "window56", "wave1024", "wave1024_error", "precision",
                             "precision192", "adjoint512", "fp64", "window56_fp64"])
    args = ap.parse_args()
    world, rank, local = dist_init(args)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        runner = {"heat1024": run_gpu, "kernels512": run_kernels512, "window56": run_window56,
                  "wave1024": run_wave1024,
                  "precision": run_precision,
                  "precision192": lambda a, w, r, l: run_precision(a, w, r, l, n=192),
                  "wave1024_error": run_wave1024_error,
                  "adjoint512": run_adjoint512, "fp64": run_fp64,
                  "window56_fp64": run_window56_fp64}[args.workload]
        return runner(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
