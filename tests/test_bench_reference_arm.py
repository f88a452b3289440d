"""CPU checks of bench.py's reference arm (the FP64 oracle timed on the host cores): one JSON
line with the contract's keys on rank 0, nothing on the other ranks.  Small workloads only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"] + args,
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.strip()]


def _check_line(line, workload):
    j = json.loads(line)
    assert j["impl"] == "reference"
    assert j["value"] > 0 and j["ms_per_step"] == j["value"] and j["unit"] == "ms"
    assert j["higher_is_better"] is False and j["dtype"] == "f64" and j["data"] == "synthetic"
    assert j["config"]["workload"] == workload
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    return j


def test_reference_arm_headline_workload_small():
    lines = _bench(["--steps", "1", "--warmup", "0", "--n", "3000", "--d", "100", "--ref-rows", "1500"])
    assert len(lines) == 1
    j = _check_line(lines[0], "zipf_gmm_near_duplicates")
    assert "1500 of 3000 rows" in j["cpu_baseline"]["sample"]


def test_reference_arm_whole_workload_when_it_fits_the_budget():
    """Default: the whole workload every step (no extrapolation) when warm-up plus timed steps fit
    the time budget; past the budget, the largest row sample that fits."""
    lines = _bench(["--steps", "2", "--warmup", "1", "--n", "3000", "--d", "100"])
    j = _check_line(lines[0], "zipf_gmm_near_duplicates")
    assert "the full 3000 x 100 workload" in j["cpu_baseline"]["sample"]
    lines = _bench(["--steps", "2", "--warmup", "1", "--n", "3000", "--d", "100", "--ref-budget", "0.000001"])
    j = _check_line(lines[0], "zipf_gmm_near_duplicates")
    assert "of 3000 rows" in j["cpu_baseline"]["sample"]


def test_reference_arm_batched_workload_small():
    lines = _bench(["--workload", "kernel_blocks", "--batch", "24", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    j = _check_line(lines[0], "kernel_blocks")
    assert j["config"]["P"] == 24 and "24 of 24 kernel blocks" in j["cpu_baseline"]["sample"]


def test_reference_arm_fixed_rank_workload_small():
    lines = _bench(["--workload", "gmm_fixed_rank", "--n", "2000", "--d", "120", "--ref-rows", "1000",
                    "--block", "8", "--ranks", "10,20", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    j = _check_line(lines[0], "gmm_fixed_rank")
    assert [r["k"] for r in j["ranks"]] == [10, 20] and [r["k_out"] for r in j["ranks"]] == [10, 20]
    assert j["value"] == j["ranks"][0]["ms"]


def test_reference_arm_other_ranks_print_nothing():
    env = {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}
    assert _bench(["--steps", "1", "--warmup", "0", "--n", "2000", "--d", "50"], env) == []
    assert _bench(["--workload", "kernel_blocks", "--batch", "8", "--steps", "1", "--warmup", "0"], env) == []
