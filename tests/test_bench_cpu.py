"""bench.py's host logic on the CPU: the reference arm's JSON line (the oracle
timed on the host cores), its multi-rank rule, the warm-up rule, the FP64
ALU roofline arithmetic and the workload description."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(args, env=None, timeout=600):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout, env=env)


def test_reference_arm_line():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "GLUPS" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["value"] > 0
    # the same workload description as the GPU arm
    want = bench.workload_config(bench.LEVELS, bench.M_PER_GPU, line["config"]["horizon"], "mixed")
    assert line["config"] == json.loads(json.dumps(want))
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = _run(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"], env=env, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_warmup_rule():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "2"], timeout=120)
    assert out.returncode != 0
    assert "warmup" in (out.stdout + out.stderr)


def test_fp64_alu_roofline():
    r = bench.fp64_alu(0.5)
    if bench.kernel_sha("fp64") != bench.FP64_ALU["sha"]:
        assert r is None  # counters taken on another kernel source are not reported
        return
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 2 * bench.sm_max_mhz() / 1e3)
    assert r["achieved"] == pytest.approx(0.5 * bench.FP64_ALU["pipe_inst_per_update"])
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # adds + multiplies + 2 x fused multiply-adds: between one and two FLOPs
    # per FP64-pipe instruction slot
    assert r["inst_per_cell_update"] * 0.5 < r["flop_per_cell_update"] < 2 * r["inst_per_cell_update"]


def test_workload_config():
    c = bench.workload_config(bench.LEVELS, 1000, "x", "mixed")
    assert c["l2"] == "inputs larger than L2 (lattice state 64 GB)"
    assert c["M_per_gpu"] == 1000 and c["levels"] == bench.LEVELS and c["precision"] == "mixed"
    small = bench.workload_config([(64, 32)], 1, "x", "fp64")
    assert small["l2"].startswith("inputs SMALLER than L2")
