"""CPU checks of bench.py's contract: the reference arm (the CPU oracle) at
N = 1 and under torchrun with two gloo ranks, and the multi-rank helpers
(barrier, max over ranks) with world size 2."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e")


def run(cmd, env=None, timeout=600):
    e = dict(os.environ)
    e.update(env or {})
    e["CUDA_VISIBLE_DEVICES"] = ""
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=e)


def json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_single():
    r = run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    line = lines[0]
    for k in REQUIRED:
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gpts/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_two_ranks_torchrun():
    r = run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
             "--master-addr", "127.0.0.1", "--master-port", "29517", "bench.py", "--impl", "reference",
             "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    bench.barrier(world)
    m = bench.max_over_ranks(world, float(10 * rank + 1))
    q.put((rank, m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, 29531, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 11.0), (1, 11.0)]
    assert all(p.exitcode == 0 for p in procs)


def test_overlap_summary_attributes_compute_idle_time():
    # Two slabs of a hand-made trace: the compute stream waits 1 ms for the
    # first H2D, 0.5 ms for the D2H before the second encode, and 0.1 ms for
    # nothing it can name; the compute stream is the busiest.
    sys.path.insert(0, ROOT)
    import bench
    tr = [
        {"kind": "h2d", "count": 1, "pass": 0, "slab": 0, "start_ms": 0.0, "end_ms": 1.0},
        {"kind": "decode", "count": 1, "pass": 0, "slab": 0, "start_ms": 1.0, "end_ms": 1.5},
        {"kind": "stencil", "count": 4, "pass": 0, "slab": 0, "start_ms": 1.6, "end_ms": 3.0},
        {"kind": "encode", "count": 1, "pass": 0, "slab": 0, "start_ms": 3.0, "end_ms": 3.5},
        {"kind": "d2h", "count": 1, "pass": 0, "slab": 0, "start_ms": 3.5, "end_ms": 6.5},
        {"kind": "h2d", "count": 1, "pass": 0, "slab": 1, "start_ms": 1.0, "end_ms": 2.0},
        {"kind": "decode", "count": 1, "pass": 0, "slab": 1, "start_ms": 3.5, "end_ms": 4.0},
        {"kind": "stencil", "count": 4, "pass": 0, "slab": 1, "start_ms": 4.0, "end_ms": 6.0},
        {"kind": "encode", "count": 1, "pass": 0, "slab": 1, "start_ms": 6.5, "end_ms": 7.0},
        {"kind": "d2h", "count": 1, "pass": 0, "slab": 1, "start_ms": 7.0, "end_ms": 8.0},
    ]
    o = bench.overlap_summary(tr)
    assert o["call_ms"] == pytest.approx(8.0)
    assert o["busy_ms"] == pytest.approx({"h2d": 2.0, "d2h": 4.0, "compute": 5.4})
    assert o["efficiency"] == pytest.approx(5.4 / 8.0)
    assert o["compute_idle_ms"] == pytest.approx({"waiting_h2d": 1.0, "waiting_d2h": 0.5, "other": 0.1})
    assert bench.overlap_summary([]) is None


def test_ncu_counters_follow_the_kernel_source(tmp_path, monkeypatch):
    # The bench ties its ncu DRAM and instruction counts to a hash of each
    # kernel's source file: comments and blank lines do not change it, code
    # does, and a changed source gives no counters (null traffic).
    sys.path.insert(0, ROOT)
    import bench
    d = tmp_path / "paper_2109_05410_gb300" / "csrc"
    d.mkdir(parents=True)
    names = sorted({n for c in bench.NCU_COUNTERS.values() for n in ([c["src"]] if isinstance(c["src"], str)
                                                                       else c["src"])})
    srcs = {n: open(os.path.join(ROOT, "paper_2109_05410_gb300", "csrc", n)).read() for n in names}

    def write(name, text):
        for n, t in srcs.items():
            (d / n).write_text(text if n == name else t)
        monkeypatch.setattr(bench, "ROOT", str(tmp_path))

    for kernel, c0 in bench.NCU_COUNTERS.items():
        first = c0["src"] if isinstance(c0["src"], str) else c0["src"][0]
        write(first, srcs[first])
        # counters taken on the current source
        c = dict(c0, sha=bench.source_sha(c0["src"]))
        monkeypatch.setitem(bench.NCU_COUNTERS, kernel, c)
        assert bench.ncu_counters(kernel) is c
        write(first, "// a new comment\n\n" + srcs[first].replace("namespace ooc {", "/* note */ namespace ooc {", 1))
        assert bench.ncu_counters(kernel) is c
        write(first, srcs[first].replace("namespace ooc {", "namespace ooc { constexpr int kChanged = 1;", 1))
        assert bench.ncu_counters(kernel) is None


def test_field_errors_match_the_oracle_metrics():
    # The bench computes its accuracy figures on the device; on CPU tensors
    # the same function must give the oracle's metrics (the same sampled
    # points, the same floor) on a field with values near zero.
    import numpy as np
    import torch

    import bench
    import oracle
    rng = np.random.default_rng(7)
    ref = rng.normal(size=(12, 10, 9))
    ref[3] *= 1e-6  # a plane below the floor
    got = (ref + 1e-5 * rng.normal(size=ref.shape)).astype(np.float32)
    want = oracle.error_metrics(got, ref)
    have = bench.field_errors(torch.from_numpy(got), torch.from_numpy(ref), zchunk=5)
    for key in ("rel_l2", "max_abs", "mean_rel_sampled"):
        assert abs(have[key] - want[key]) <= 1e-12 * abs(want[key]), key
    assert have["samples"] == want["samples"] and have["excluded"] == want["excluded"]
